"""Parameter sets for BootMMPM bootstrapping (Alg. 1 of arXiv 2310.12441).

A *key set* fixes everything the evaluation keys depend on: the LWE dimension
n, the ring degree N, the ring modulus Q, the blind-rotation gadget (B, l_B)
and the key-switching gadget (B_KS, l_KS).  The key sizes do not depend on the
number m of polynomials in the test vector nor on the plaintext modulus t
(Section 5, items (1) and (2)), so one key set serves every job shape (m, t)
with the same N.  A *job shape* is (m, t); the input ciphertext modulus is
q' = 2*N*m (Algorithm 1, modulus switch), so Delta = q'/t.

Moduli: Q is prime with Q = 1 mod 2N (a negacyclic NTT of length N exists).
Above 2^32 we take the largest prime below 2^k of the form c 2^32 + 1: then
q Q mod 2^64 = q + ((q mod 2^32) c mod 2^32) 2^32, which saves multiplies in
every modular reduction of the NTT.  The toy modulus lies below 2^32 and is
the largest prime below 2^30 that is 1 mod 512.
"""
from __future__ import annotations

from dataclasses import dataclass, field


@dataclass(frozen=True)
class KeyParams:
    """Evaluation-key parameters (Algorithm 1 REQUIRE block)."""

    n: int            # LWE dimension of the input/output ciphertexts
    N: int            # ring degree of R_{N,Q} = Z_Q[x]/(x^N+1)
    Q: int            # prime ring modulus, Q = 1 mod 2N, Q < 2^62
    log2_B: int       # blind-rotation gadget base B = 2^log2_B
    l_B: int          # number of gadget digits, B^l_B >= Q
    log2_Bks: int     # key-switching base B_KS = 2^log2_Bks
    l_ks: int         # key-switching digits (approximate gadget, P = B_KS^l_ks)
    secret: str = "ternary"   # distribution of the LWE secret s: "binary" | "ternary"
    sigma: float = 3.2        # standard deviation of all fresh errors

    @property
    def B(self) -> int:
        return 1 << self.log2_B

    @property
    def Bks(self) -> int:
        return 1 << self.log2_Bks

    def validate(self) -> None:
        N, Q = self.N, self.Q
        if N & (N - 1) or N < 16:
            raise ValueError("N must be a power of two >= 16")
        if (Q - 1) % (2 * N):
            raise ValueError("Q must be 1 mod 2N")
        if Q >= 1 << 62:
            raise ValueError("Q must be below 2^62")
        if (1 << (self.log2_B * self.l_B)) < Q:
            raise ValueError("B^l_B must be >= Q")
        if self.log2_Bks * self.l_ks > 62:
            raise ValueError("B_KS^l_KS must stay below 2^63")


@dataclass(frozen=True)
class JobShape:
    """Per-ciphertext shape: m polynomials in the test vector, plaintext Z_t."""

    m: int
    t: int

    def q_prime(self, N: int) -> int:
        return 2 * N * self.m


@dataclass(frozen=True)
class Workload:
    name: str
    keys: KeyParams
    shape: JobShape
    count: int
    description: str = ""
    lut_mix: str = "random"   # "random" | "mixed" (random/identity 50/50)
    seed_base: int = 0
    extra: dict = field(default_factory=dict)


# Key sets -----------------------------------------------------------------
KEYS_TOY = KeyParams(n=64, N=256, Q=1073738753, log2_B=6, l_B=5,
                     log2_Bks=4, l_ks=7, secret="binary")
KEYS_N1024 = KeyParams(n=630, N=1024, Q=18014359854776321, log2_B=9, l_B=6,
                       log2_Bks=4, l_ks=7)
KEYS_N4096 = KeyParams(n=630, N=4096, Q=18014359854776321, log2_B=9, l_B=6,
                       log2_Bks=4, l_ks=7)
KEYS_N2048 = KeyParams(n=750, N=2048, Q=1152921092289986561, log2_B=10, l_B=6,
                       log2_Bks=4, l_ks=7)

# Plaintext-size sweep (Sec. 5 experiments): log n = 9, log Q = 54,
# log B = 15 (l_B = 4), ring degree 2^11 for every plaintext size; the
# single-polynomial (TFHE) layout needs N = 2^(log t + 6).  The paper's
# key-switching base 25 is read as 2^5 with 8 digits of the approximate gadget.
KEYS_SWEEP_N2048 = KeyParams(n=512, N=2048, Q=18014359854776321, log2_B=15, l_B=4,
                             log2_Bks=5, l_ks=8)
KEYS_SWEEP_N4096 = KeyParams(n=512, N=4096, Q=18014359854776321, log2_B=15, l_B=4,
                             log2_Bks=5, l_ks=8)

# Workloads ------------------------------------------------------------------
TOY = Workload("toy_n64_N256_m2_t32", KEYS_TOY, JobShape(m=2, t=32), 1,
               "plain bootstrap of 1 ciphertext", seed_base=1)
BATCH_N1024 = Workload("batch4096_n630_N1024_m4_t1024", KEYS_N1024,
                       JobShape(m=4, t=1024), 4096,
                       "4096 ciphertexts, one random LUT each", seed_base=2)
SINGLEPOLY_N4096 = Workload("batch4096_n630_N4096_m1_t1024", KEYS_N4096,
                            JobShape(m=1, t=1024), 4096,
                            "same inputs as the N=1024 batch, m=1 layout",
                            seed_base=2)
LARGE_N2048 = Workload("batch2048_n750_N2048_m8_t8192", KEYS_N2048,
                       JobShape(m=8, t=8192), 2048,
                       "2048 ciphertexts, random and identity LUTs 50/50",
                       lut_mix="mixed", seed_base=3)

# Uneven mix: six parameter sets over the two resident key sets.
UNEVEN_SETS = [
    ("S1", KEYS_N1024, JobShape(m=1, t=1 << 8)),
    ("S2", KEYS_N1024, JobShape(m=2, t=1 << 9)),
    ("S3", KEYS_N1024, JobShape(m=4, t=1 << 10)),
    ("S4", KEYS_N2048, JobShape(m=2, t=1 << 11)),
    ("S5", KEYS_N2048, JobShape(m=4, t=1 << 12)),
    ("S6", KEYS_N2048, JobShape(m=8, t=1 << 13)),
]

WORKLOADS = {w.name: w for w in (TOY, BATCH_N1024, SINGLEPOLY_N4096, LARGE_N2048)}

"""Seeded synthetic inputs shared by the CUDA path, the oracle, the tests and
the benchmark.

This module draws random numbers only.  It performs none of the method's
arithmetic: no encryption, no polynomial products, no key construction.
Every random quantity the method consumes (secrets, uniform masks, error
samples, messages, look-up tables) is drawn here and handed to both sides as
plain arrays, so the oracle and the library never need a shared generator.

Distributions (Algorithm 1 REQUIRE block and Section 2):
  * LWE secret s: uniform ternary {-1,0,1}^n ("binary": {0,1}^n);
  * RLWE secret z: uniform ternary coefficients;
  * masks: uniform in [0, modulus);
  * errors: a Gaussian of standard deviation sigma rounded to the nearest
    integer, tails cut at |e| <= 41 (about 12.8 sigma for sigma = 3.2);
  * messages: uniform in Z_t, or in [0, t/2) for identity-refresh tables;
  * look-up tables: negacyclic f: Z_t -> Z_t, f(k + t/2) = -f(k) mod t.

Stream separation: every quantity has its own numpy Generator seeded by
(seed, stream name), so two workloads that share a seed share the LWE secret
s of the same dimension n (this is how the N=1024/m=4 and the N=4096/m=1
layouts bootstrap the very same input ciphertexts).
"""
from __future__ import annotations

import zlib

import numpy as np

from .params import KeyParams

ERR_CUT = 41


def _rng(seed: int, stream: str) -> np.random.Generator:
    return np.random.default_rng([int(seed) & 0xFFFFFFFF, int(seed) >> 32,
                                  zlib.crc32(stream.encode())])


def gaussian_int8(rng: np.random.Generator, sigma: float, shape) -> np.ndarray:
    e = np.rint(rng.normal(0.0, sigma, size=shape))
    np.clip(e, -ERR_CUT, ERR_CUT, out=e)
    return e.astype(np.int8)


def uniform_mod(rng: np.random.Generator, modulus: int, shape) -> np.ndarray:
    return rng.integers(0, modulus, size=shape, dtype=np.uint64)


def ternary(rng: np.random.Generator, shape) -> np.ndarray:
    return rng.integers(-1, 2, size=shape, dtype=np.int8)


def lwe_secret(kp: KeyParams, seed: int) -> np.ndarray:
    rng = _rng(seed, f"lwe-secret-n{kp.n}")
    if kp.secret == "binary":
        return rng.integers(0, 2, size=kp.n, dtype=np.int8)
    return ternary(rng, kp.n)


def key_randomness(kp: KeyParams, seed: int, bsk_keys: int | None = None,
                   with_ksk: bool = True) -> dict:
    """All random draws of key generation.

    Shapes (C order):
      s        int8   [n]
      z        int8   [N]
      bsk_mask uint64 [K, 2, 2*l_B, N]   K = bsk_keys or n; uniform mod Q
      bsk_err  int8   [K, 2, 2*l_B, N]
      ksk_mask uint64 [N, l_ks, B_KS-1, n] uniform mod Q
      ksk_err  int8   [N, l_ks, B_KS-1]

    The k-th bootstrapping-key slice depends only on (seed, k), so asking for
    fewer keys (bsk_keys) returns a prefix of the full draw.
    """
    kp.validate()
    n, N, lB = kp.n, kp.N, kp.l_B
    K = n if bsk_keys is None else int(bsk_keys)
    out = {"s": lwe_secret(kp, seed),
           "z": ternary(_rng(seed, f"rlwe-secret-N{N}"), N)}
    # One generator per key index keeps prefixes stable.
    bm = np.empty((K, 2, 2 * lB, N), dtype=np.uint64)
    be = np.empty((K, 2, 2 * lB, N), dtype=np.int8)
    chunk = 64
    for k0 in range(0, K, chunk):
        k1 = min(K, k0 + chunk)
        rng = _rng(seed, f"bsk-N{N}-Q{kp.Q}-blk{k0 // chunk}")
        full_m = uniform_mod(rng, kp.Q, (chunk, 2, 2 * lB, N))
        full_e = gaussian_int8(rng, kp.sigma, (chunk, 2, 2 * lB, N))
        bm[k0:k1] = full_m[: k1 - k0]
        be[k0:k1] = full_e[: k1 - k0]
    out["bsk_mask"], out["bsk_err"] = bm, be
    if with_ksk:
        rng = _rng(seed, f"ksk-N{N}-n{n}-Q{kp.Q}")
        rows = (N, kp.l_ks, kp.Bks - 1)
        out["ksk_mask"] = uniform_mod(rng, kp.Q, rows + (n,))
        out["ksk_err"] = gaussian_int8(rng, kp.sigma, rows)
    return out


def messages(t: int, count: int, seed: int, half: np.ndarray | None = None) -> np.ndarray:
    """Uniform messages in Z_t; where half[i] is True, uniform in [0, t/2)."""
    rng = _rng(seed, f"messages-t{t}")
    msg = rng.integers(0, t, size=count, dtype=np.uint32)
    if half is not None:
        msg = np.where(half, msg % np.uint32(t // 2), msg).astype(np.uint32)
    return msg


def encryption_randomness(n: int, q_prime: int, sigma: float, count: int,
                          seed: int, prefix: int | None = None) -> dict:
    """Masks a in [0, q')^n and one error per ciphertext.

    prefix=K zeroes the masks a_{K+1..n}; such a ciphertext is still a valid
    encryption (under the first K secret coordinates) and lets a blind
    rotation be checked after its first K steps only.
    """
    rng = _rng(seed, f"enc-n{n}-q{q_prime}")
    mask = uniform_mod(rng, q_prime, (count, n))
    err = gaussian_int8(rng, sigma, count)
    if prefix is not None:
        mask[:, int(prefix):] = 0
    return {"mask": mask, "err": err}


def negacyclic_lut(rng: np.random.Generator, t: int) -> np.ndarray:
    """f(k) uniform for k < t/2 and f(k + t/2) = -f(k) mod t (Section 2, (7))."""
    lo = rng.integers(0, t, size=t // 2, dtype=np.int64)
    hi = (t - lo) % t
    return np.concatenate([lo, hi]).astype(np.uint32)


def identity_lut(t: int) -> np.ndarray:
    """Identity on [0, t/2), negacyclically extended (padding-bit refresh)."""
    lo = np.arange(t // 2, dtype=np.int64)
    return np.concatenate([lo, (t - lo) % t]).astype(np.uint32)


def luts(t: int, count: int, seed: int, mix: str = "random") -> tuple[np.ndarray, np.ndarray]:
    """count look-up tables of t entries and a flag 'identity' per table.

    mix="random": every table negacyclic-random; mix="mixed": even-indexed
    tables random, odd-indexed identity-refresh.
    """
    rng = _rng(seed, f"luts-t{t}")
    out = np.empty((count, t), dtype=np.uint32)
    ident = np.zeros(count, dtype=bool)
    idl = identity_lut(t)
    for i in range(count):
        if mix == "mixed" and i % 2 == 1:
            out[i] = idl
            ident[i] = True
        else:
            out[i] = negacyclic_lut(rng, t)
    return out, ident


def zipf_counts(total: int, n_sets: int, s: float, seed: int) -> np.ndarray:
    """Multinomial counts with P(rank k) proportional to k^-s."""
    rng = _rng(seed, "zipf")
    w = np.arange(1, n_sets + 1, dtype=np.float64) ** (-s)
    return rng.multinomial(total, w / w.sum())

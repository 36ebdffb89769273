"""CPU oracle for BootMMPM (arXiv 2310.12441, Algorithm 1) -- TEST INFRASTRUCTURE.

Only tests/, the smoke check of __graft_entry__ and the benchmark's CPU
baseline leg may import this package.  It is independent of the CUDA path:
it shares no code with it and imports nothing from the product package.

The arithmetic lives in bootmmpm_oracle.c (plain C, exact integers,
schoolbook negacyclic products).  This module marshals numpy arrays into it.

Parity pins (tests/test_oracle_*.py) tie every function here to what the
paper fixes: the MMPM group law and closed forms (Lemma 3, Example 1,
Lemma 6), the look-up property (Lemma 7), the exact error identities of the
external product (Eq. (error:grow)), of sample extraction (Eq.
(equ-sam-extr)) and of key switching (Eq. (equ-key-swi)), the FHEW/TFHE test
polynomial for m = 1, and end-to-end decryption of bootstrapped outputs.
"""
from __future__ import annotations

import ctypes as C

import numpy as np

from .build import build_oracle

_lib = None

u64p = C.POINTER(C.c_uint64)
u32p = C.POINTER(C.c_uint32)
i8p = C.POINTER(C.c_int8)


class _Params(C.Structure):
    _fields_ = [("n", C.c_uint32), ("N", C.c_uint32), ("log2_B", C.c_uint32),
                ("l_B", C.c_uint32), ("log2_Bks", C.c_uint32), ("l_ks", C.c_uint32),
                ("Q", C.c_uint64)]


def lib():
    global _lib
    if _lib is None:
        L = C.CDLL(build_oracle())
        L.orc_poly_mul.argtypes = [C.c_uint32, C.c_uint64, u64p, u64p, u64p]
        L.orc_mmpm_apply.argtypes = [C.c_uint32, C.c_uint32, C.c_uint64, C.c_uint64, u64p, u64p]
        L.orc_test_vector.argtypes = [C.c_uint32, C.c_uint32, C.c_uint32, C.c_uint64, u32p, u64p]
        L.orc_decompose.argtypes = [C.c_uint64, C.c_uint32, C.c_uint32, u64p]
        L.orc_external_product.argtypes = [C.POINTER(_Params), u64p, u64p, u64p, u64p, u64p]
        L.orc_cmux.argtypes = [C.POINTER(_Params), C.c_uint32, C.c_uint64, u64p, u64p, u64p, C.c_int]
        L.orc_blind_rotate.argtypes = [C.POINTER(_Params), C.c_uint32, C.c_uint32, u64p,
                                       C.c_uint32, u64p, u32p, u64p, C.c_int]
        L.orc_blind_rotate.restype = C.c_int
        L.orc_sample_extract.argtypes = [C.c_uint32, C.c_uint64, u64p, u64p, u64p]
        L.orc_ks_gadget.argtypes = [C.POINTER(_Params), C.c_uint32]
        L.orc_ks_gadget.restype = C.c_uint64
        L.orc_ks_digits.argtypes = [C.POINTER(_Params), C.c_uint64, u32p]
        L.orc_key_switch.argtypes = [C.POINTER(_Params), u64p, u64p, u64p]
        L.orc_keygen_bsk.argtypes = [C.POINTER(_Params), i8p, i8p, u64p, i8p, C.c_uint32,
                                     C.c_uint32, u64p]
        L.orc_keygen_ksk.argtypes = [C.POINTER(_Params), i8p, i8p, u64p, i8p, u64p]
        L.orc_encrypt.argtypes = [C.c_uint32, C.c_uint64, C.c_uint32, i8p, u32p, u64p, i8p,
                                  C.c_size_t, u64p]
        L.orc_lwe_phase.argtypes = [C.c_uint32, C.c_uint64, i8p, u64p]
        L.orc_lwe_phase.restype = C.c_uint64
        L.orc_decrypt.argtypes = [C.c_uint32, C.c_uint64, C.c_uint32, i8p, u64p, C.c_size_t, u32p]
        L.orc_rlwe_phase.argtypes = [C.c_uint32, C.c_uint64, i8p, u64p, u64p, u64p]
        L.orc_mod_switch.argtypes = [u64p, C.c_size_t, C.c_uint64, C.c_uint64, u64p]
        L.orc_two_round_tables.argtypes = [C.c_uint32, u32p, u32p, u32p]
        L.orc_bootstrap_arbitrary.argtypes = [C.POINTER(_Params), C.c_uint32, C.c_uint32, C.c_uint64,
                                              u64p, C.c_uint32, u64p, u64p, u32p, C.c_size_t, u64p]
        L.orc_bootstrap_arbitrary.restype = C.c_int
        L.orc_bootstrap.argtypes = [C.POINTER(_Params), C.c_uint32, C.c_uint32, u64p, C.c_uint32,
                                    u64p, u64p, u32p, C.c_size_t, u64p]
        L.orc_bootstrap.restype = C.c_int
        L.orc_mmpm_apply_gen.argtypes = [C.c_uint32, C.c_uint32, C.c_uint64, u32p, C.c_uint64, u64p, u64p]
        L.orc_mmpm_step_gen.argtypes = [C.c_uint32, C.c_uint32, C.c_uint64, u32p, u64p, u64p]
        L.orc_test_vector_gen.argtypes = [C.c_uint32, C.c_uint32, C.c_uint32, C.c_uint64, u32p, u32p, u64p]
        L.orc_blind_rotate_gen.argtypes = [C.POINTER(_Params), C.c_uint32, C.c_uint32, u32p, u64p,
                                           C.c_uint32, u64p, u32p, u64p, C.c_int]
        L.orc_blind_rotate_gen.restype = C.c_int
        L.orc_bootstrap_gen.argtypes = [C.POINTER(_Params), C.c_uint32, C.c_uint32, u32p, u64p,
                                        C.c_uint32, u64p, u64p, u32p, C.c_size_t, u64p]
        L.orc_bootstrap_gen.restype = C.c_int
        L.orc_philox4x32_10.argtypes = [u32p, u32p, u32p]
        L.orc_draw_uniform.argtypes = [C.c_uint64, C.c_uint32, C.c_uint32, C.c_uint64, C.c_uint64]
        L.orc_draw_uniform.restype = C.c_uint64
        L.orc_draw_ternary.argtypes = [C.c_uint64, C.c_uint32, C.c_uint32, C.c_uint64]
        L.orc_draw_ternary.restype = C.c_int
        L.orc_draw_binary.argtypes = [C.c_uint64, C.c_uint32, C.c_uint32, C.c_uint64]
        L.orc_draw_binary.restype = C.c_int
        L.orc_cdt.argtypes = [C.c_double, u64p]
        L.orc_draw_gaussian.argtypes = [C.c_uint64, C.c_uint32, C.c_uint32, C.c_uint64, u64p]
        L.orc_draw_gaussian.restype = C.c_int
        L.orc_seeded_lwe_secret.argtypes = [C.c_uint32, C.c_int, C.c_uint64, i8p]
        L.orc_seeded_rlwe_secret.argtypes = [C.c_uint32, C.c_uint64, i8p]
        L.orc_seeded_bsk_randomness.argtypes = [C.POINTER(_Params), C.c_double, C.c_uint64, C.c_uint32,
                                                u64p, i8p]
        L.orc_seeded_ksk_randomness.argtypes = [C.POINTER(_Params), C.c_double, C.c_uint64, u64p, i8p]
        L.orc_seeded_enc_randomness.argtypes = [C.c_uint32, C.c_uint64, C.c_double, C.c_uint64,
                                                C.c_size_t, u64p, i8p]
        _lib = L
    return _lib


def _p(a, dtype, ptr):
    a = np.ascontiguousarray(a, dtype=dtype)
    return a, a.ctypes.data_as(ptr)


def _params(kp) -> _Params:
    return _Params(kp.n, kp.N, kp.log2_B, kp.l_B, kp.log2_Bks, kp.l_ks, kp.Q)


# -- ring and group ---------------------------------------------------------

def poly_mul(N: int, Q: int, a, b) -> np.ndarray:
    a, pa = _p(a, np.uint64, u64p)
    b, pb = _p(b, np.uint64, u64p)
    out = np.empty(N, np.uint64)
    lib().orc_poly_mul(N, Q, pa, pb, out.ctypes.data_as(u64p))
    return out


def mmpm_apply(N: int, m: int, Q: int, c: int, vec) -> np.ndarray:
    """P(c) times an RLWE vector [m][2][N]."""
    vec, pv = _p(vec, np.uint64, u64p)
    out = np.empty((m, 2, N), np.uint64)
    lib().orc_mmpm_apply(N, m, Q, int(c), pv, out.ctypes.data_as(u64p))
    return out


def test_vector(N: int, m: int, t: int, Q: int, lut) -> np.ndarray:
    lut, pl = _p(lut, np.uint32, u32p)
    v = np.empty((m, N), np.uint64)
    lib().orc_test_vector(N, m, t, Q, pl, v.ctypes.data_as(u64p))
    return v


def decompose(x: int, log2_B: int, l_B: int) -> np.ndarray:
    d = np.empty(l_B, np.uint64)
    lib().orc_decompose(int(x), log2_B, l_B, d.ctypes.data_as(u64p))
    return d


# -- RLWE / RGSW --------------------------------------------------------------

def external_product(kp, a, b, C_rgsw):
    a, pa = _p(a, np.uint64, u64p)
    b, pb = _p(b, np.uint64, u64p)
    Cr, pc = _p(C_rgsw, np.uint64, u64p)
    oa = np.empty(kp.N, np.uint64)
    ob = np.empty(kp.N, np.uint64)
    prm = _params(kp)
    lib().orc_external_product(C.byref(prm), pa, pb, pc, oa.ctypes.data_as(u64p),
                               ob.ctypes.data_as(u64p))
    return oa, ob


def cmux(kp, m: int, ak: int, Cp, Cm, acc, parallel: bool = True) -> np.ndarray:
    acc = np.array(acc, dtype=np.uint64, copy=True, order="C")
    Cp, pp = _p(Cp, np.uint64, u64p)
    Cm, pm = _p(Cm, np.uint64, u64p)
    prm = _params(kp)
    lib().orc_cmux(C.byref(prm), m, int(ak), pp, pm, acc.ctypes.data_as(u64p), int(parallel))
    return acc


def blind_rotate(kp, m: int, t: int, bsk, ct, lut, parallel: bool = True) -> np.ndarray:
    bsk, pb = _p(bsk, np.uint64, u64p)
    ct, pc = _p(ct, np.uint64, u64p)
    lut, pl = _p(lut, np.uint32, u32p)
    acc = np.empty((m, 2, kp.N), np.uint64)
    prm = _params(kp)
    rc = lib().orc_blind_rotate(C.byref(prm), m, t, pb, bsk.shape[0], pc, pl,
                                acc.ctypes.data_as(u64p), int(parallel))
    if rc != 0:
        raise ValueError("ciphertext uses a bootstrapping key that was not provided")
    return acc


def sample_extract(N: int, Q: int, a, b) -> np.ndarray:
    a, pa = _p(a, np.uint64, u64p)
    b, pb = _p(b, np.uint64, u64p)
    out = np.empty(N + 1, np.uint64)
    lib().orc_sample_extract(N, Q, pa, pb, out.ctypes.data_as(u64p))
    return out


def ks_gadget(kp, j: int) -> int:
    prm = _params(kp)
    return int(lib().orc_ks_gadget(C.byref(prm), j))


def ks_digits(kp, a: int) -> np.ndarray:
    prm = _params(kp)
    d = np.empty(kp.l_ks, np.uint32)
    lib().orc_ks_digits(C.byref(prm), int(a), d.ctypes.data_as(u32p))
    return d


def key_switch(kp, lwe_N, ksk) -> np.ndarray:
    lwe_N, pl = _p(lwe_N, np.uint64, u64p)
    ksk, pk = _p(ksk, np.uint64, u64p)
    out = np.empty(kp.n + 1, np.uint64)
    prm = _params(kp)
    lib().orc_key_switch(C.byref(prm), pl, pk, out.ctypes.data_as(u64p))
    return out


# -- keys, encryption -------------------------------------------------------------

def keygen_bsk(kp, rnd: dict, k0: int = 0, k1: int | None = None) -> np.ndarray:
    """[k1-k0][2][2 l_B][2][N] coefficient-domain bootstrapping keys."""
    k1 = rnd["bsk_mask"].shape[0] if k1 is None else k1
    s, ps = _p(rnd["s"], np.int8, i8p)
    z, pz = _p(rnd["z"], np.int8, i8p)
    mk, pm = _p(rnd["bsk_mask"], np.uint64, u64p)
    er, pe = _p(rnd["bsk_err"], np.int8, i8p)
    out = np.empty((k1 - k0, 2, 2 * kp.l_B, 2, kp.N), np.uint64)
    prm = _params(kp)
    lib().orc_keygen_bsk(C.byref(prm), ps, pz, pm, pe, k0, k1, out.ctypes.data_as(u64p))
    return out


def keygen_ksk(kp, rnd: dict) -> np.ndarray:
    """[N][l_ks][B_ks-1][n+1] key-switching keys."""
    s, ps = _p(rnd["s"], np.int8, i8p)
    z, pz = _p(rnd["z"], np.int8, i8p)
    mk, pm = _p(rnd["ksk_mask"], np.uint64, u64p)
    er, pe = _p(rnd["ksk_err"], np.int8, i8p)
    out = np.empty((kp.N, kp.l_ks, kp.Bks - 1, kp.n + 1), np.uint64)
    prm = _params(kp)
    lib().orc_keygen_ksk(C.byref(prm), ps, pz, pm, pe, out.ctypes.data_as(u64p))
    return out


def encrypt(n: int, q: int, t: int, s, msg, mask, err) -> np.ndarray:
    s, ps = _p(s, np.int8, i8p)
    msg, pmsg = _p(msg, np.uint32, u32p)
    mask, pm = _p(mask, np.uint64, u64p)
    err, pe = _p(err, np.int8, i8p)
    count = msg.shape[0]
    ct = np.empty((count, n + 1), np.uint64)
    lib().orc_encrypt(n, q, t, ps, pmsg, pm, pe, count, ct.ctypes.data_as(u64p))
    return ct


def lwe_phase(n: int, q: int, s, ct) -> int:
    s, ps = _p(s, np.int8, i8p)
    ct, pc = _p(ct, np.uint64, u64p)
    return int(lib().orc_lwe_phase(n, q, ps, pc))


def decrypt(n: int, q: int, t: int, s, ct) -> np.ndarray:
    s, ps = _p(s, np.int8, i8p)
    ct, pc = _p(np.atleast_2d(ct), np.uint64, u64p)
    out = np.empty(ct.shape[0], np.uint32)
    lib().orc_decrypt(n, q, t, ps, pc, ct.shape[0], out.ctypes.data_as(u32p))
    return out


def rlwe_phase(N: int, Q: int, z, a, b) -> np.ndarray:
    z, pz = _p(z, np.int8, i8p)
    a, pa = _p(a, np.uint64, u64p)
    b, pb = _p(b, np.uint64, u64p)
    out = np.empty(N, np.uint64)
    lib().orc_rlwe_phase(N, Q, pz, pa, pb, out.ctypes.data_as(u64p))
    return out


def mod_switch(ct, q_from: int, q_to: int) -> np.ndarray:
    """Section 2 (9) on every word of ct (any shape)."""
    ct, pc = _p(ct, np.uint64, u64p)
    out = np.empty_like(ct)
    lib().orc_mod_switch(pc, ct.size, q_from, q_to, out.ctypes.data_as(u64p))
    return out


def bootstrap(kp, m: int, t: int, bsk, ksk, ct_in, luts) -> np.ndarray:
    """Algorithm 1 (modulus switches excluded) for count ciphertexts."""
    bsk, pb = _p(bsk, np.uint64, u64p)
    ksk, pk = _p(ksk, np.uint64, u64p)
    ct_in, pc = _p(np.atleast_2d(ct_in), np.uint64, u64p)
    luts, pl = _p(np.atleast_2d(luts), np.uint32, u32p)
    count = ct_in.shape[0]
    out = np.empty((count, kp.n + 1), np.uint64)
    prm = _params(kp)
    rc = lib().orc_bootstrap(C.byref(prm), m, t, pb, bsk.shape[0], pk, pc, pl, count,
                             out.ctypes.data_as(u64p))
    if rc != 0:
        raise ValueError("ciphertext uses a bootstrapping key that was not provided")
    return out


def two_round_tables(t: int, f) -> tuple[np.ndarray, np.ndarray]:
    """mp and the negacyclic extension F of f (both over Z_{2t})."""
    f, pf = _p(f, np.uint32, u32p)
    mp = np.empty(2 * t, np.uint32)
    F = np.empty(2 * t, np.uint32)
    lib().orc_two_round_tables(t, pf, mp.ctypes.data_as(u32p), F.ctypes.data_as(u32p))
    return mp, F


def bootstrap_arbitrary(kp, m: int, t: int, q: int, bsk, ksk, ct_in, f) -> np.ndarray:
    """Two-round bootstrap of any f: Z_t -> Z_t (one table of t entries per
    ciphertext); inputs and outputs in LWE_{n,q}, plaintext modulus 2t."""
    bsk, pb = _p(bsk, np.uint64, u64p)
    ksk, pk = _p(ksk, np.uint64, u64p)
    ct_in, pc = _p(np.atleast_2d(ct_in), np.uint64, u64p)
    f, pf = _p(np.atleast_2d(f), np.uint32, u32p)
    out = np.empty_like(ct_in)
    prm = _params(kp)
    rc = lib().orc_bootstrap_arbitrary(C.byref(prm), m, t, q, pb, bsk.shape[0], pk, pc, pf,
                                       ct_in.shape[0], out.ctypes.data_as(u64p))
    if rc != 0:
        raise ValueError("ciphertext uses a bootstrapping key that was not provided")
    return out


# -- general transitive generators (Theorem 1) ------------------------------------------

def mmpm_apply_gen(N: int, m: int, Q: int, u, c: int, vec) -> np.ndarray:
    """P(c) = A^c times an RLWE vector [m][2][N], A the generator of exponents
    u (Lemma 3's closed form)."""
    u, pu = _p(u, np.uint32, u32p)
    vec, pv = _p(vec, np.uint64, u64p)
    out = np.empty((m, 2, N), np.uint64)
    lib().orc_mmpm_apply_gen(N, m, Q, pu, int(c), pv, out.ctypes.data_as(u64p))
    return out


def mmpm_step_gen(N: int, m: int, Q: int, u, vec) -> np.ndarray:
    """One application of the generator A (no closed form involved)."""
    u, pu = _p(u, np.uint32, u32p)
    vec, pv = _p(vec, np.uint64, u64p)
    out = np.empty((m, 2, N), np.uint64)
    lib().orc_mmpm_step_gen(N, m, Q, pu, pv, out.ctypes.data_as(u64p))
    return out


def test_vector_gen(N: int, m: int, t: int, Q: int, u, lut) -> np.ndarray:
    u, pu = _p(u, np.uint32, u32p)
    lut, pl = _p(lut, np.uint32, u32p)
    v = np.empty((m, N), np.uint64)
    lib().orc_test_vector_gen(N, m, t, Q, pu, pl, v.ctypes.data_as(u64p))
    return v


def blind_rotate_gen(kp, m: int, t: int, u, bsk, ct, lut, parallel: bool = True) -> np.ndarray:
    u, pu = _p(u, np.uint32, u32p)
    bsk, pb = _p(bsk, np.uint64, u64p)
    ct, pc = _p(ct, np.uint64, u64p)
    lut, pl = _p(lut, np.uint32, u32p)
    acc = np.empty((m, 2, kp.N), np.uint64)
    prm = _params(kp)
    rc = lib().orc_blind_rotate_gen(C.byref(prm), m, t, pu, pb, bsk.shape[0], pc, pl,
                                    acc.ctypes.data_as(u64p), int(parallel))
    if rc != 0:
        raise ValueError("ciphertext uses a bootstrapping key that was not provided")
    return acc


def bootstrap_gen(kp, m: int, t: int, u, bsk, ksk, ct_in, luts) -> np.ndarray:
    """Algorithm 1 (modulus switches excluded) with generator exponents u
    ([count][m]) per ciphertext."""
    ct_in, pc = _p(np.atleast_2d(ct_in), np.uint64, u64p)
    count = ct_in.shape[0]
    u, pu = _p(np.broadcast_to(np.asarray(u, np.uint32).reshape(-1, m), (count, m)), np.uint32, u32p)
    bsk, pb = _p(bsk, np.uint64, u64p)
    ksk, pk = _p(ksk, np.uint64, u64p)
    luts, pl = _p(np.atleast_2d(luts), np.uint32, u32p)
    out = np.empty((count, kp.n + 1), np.uint64)
    prm = _params(kp)
    rc = lib().orc_bootstrap_gen(C.byref(prm), m, t, pu, pb, bsk.shape[0], pk, pc, pl, count,
                                 out.ctypes.data_as(u64p))
    if rc != 0:
        raise ValueError("ciphertext uses a bootstrapping key that was not provided")
    return out


# -- seeded randomness (Philox4x32-10 streams; see bootmmpm_oracle.c) ---------------

ERR_CUT = 41
KIND = {"lwe_secret": 1, "rlwe_secret": 2, "bsk_mask": 3, "bsk_err": 4, "ksk_mask": 5,
        "ksk_err": 6, "enc_mask": 7, "enc_err": 8}


def philox4x32_10(ctr, key) -> np.ndarray:
    c, pc = _p(ctr, np.uint32, u32p)
    k, pk = _p(key, np.uint32, u32p)
    out = np.empty(4, np.uint32)
    lib().orc_philox4x32_10(pc, pk, out.ctypes.data_as(u32p))
    return out


def draw_uniform(seed: int, kind: int, domain: int, i: int, modulus: int) -> int:
    return int(lib().orc_draw_uniform(seed, kind, domain, i, modulus))


def draw_ternary(seed: int, kind: int, domain: int, i: int) -> int:
    return int(lib().orc_draw_ternary(seed, kind, domain, i))


def draw_binary(seed: int, kind: int, domain: int, i: int) -> int:
    return int(lib().orc_draw_binary(seed, kind, domain, i))


def cdt(sigma: float) -> np.ndarray:
    T = np.empty(2 * ERR_CUT, np.uint64)
    lib().orc_cdt(sigma, T.ctypes.data_as(u64p))
    return T


def draw_gaussian(seed: int, kind: int, domain: int, i: int, T) -> int:
    T, pt = _p(T, np.uint64, u64p)
    return int(lib().orc_draw_gaussian(seed, kind, domain, i, pt))


def seeded_key_randomness(kp, seed: int, bsk_keys: int | None = None, with_ksk: bool = True) -> dict:
    """The randomness of key generation drawn from `seed` by the Philox stream
    layout (same shapes as the array-taking keygen functions read)."""
    n, N, lB = kp.n, kp.N, kp.l_B
    K = n if bsk_keys is None else int(bsk_keys)
    L = lib()
    s = np.empty(n, np.int8)
    L.orc_seeded_lwe_secret(n, int(kp.secret == "ternary"), seed, s.ctypes.data_as(i8p))
    z = np.empty(N, np.int8)
    L.orc_seeded_rlwe_secret(N, seed, z.ctypes.data_as(i8p))
    prm = _params(kp)
    bm = np.empty((K, 2, 2 * lB, N), np.uint64)
    be = np.empty((K, 2, 2 * lB, N), np.int8)
    L.orc_seeded_bsk_randomness(C.byref(prm), kp.sigma, seed, K, bm.ctypes.data_as(u64p),
                                be.ctypes.data_as(i8p))
    out = {"s": s, "z": z, "bsk_mask": bm, "bsk_err": be}
    if with_ksk:
        rows = (N, kp.l_ks, kp.Bks - 1)
        km = np.empty(rows + (n,), np.uint64)
        ke = np.empty(rows, np.int8)
        L.orc_seeded_ksk_randomness(C.byref(prm), kp.sigma, seed, km.ctypes.data_as(u64p),
                                    ke.ctypes.data_as(i8p))
        out["ksk_mask"], out["ksk_err"] = km, ke
    return out


def seeded_enc_randomness(n: int, q: int, sigma: float, count: int, seed: int) -> dict:
    """Encryption masks [count][n] in [0, q) and errors [count] from `seed`."""
    mask = np.empty((count, n), np.uint64)
    err = np.empty(count, np.int8)
    lib().orc_seeded_enc_randomness(n, q, sigma, seed, count, mask.ctypes.data_as(u64p),
                                    err.ctypes.data_as(i8p))
    return {"mask": mask, "err": err}


def encrypt_seeded(n: int, q: int, t: int, s, msg, sigma: float, seed: int) -> np.ndarray:
    """LWE_{n,q} encryption (Section 2, (8)) with masks and errors drawn from
    `seed`."""
    msg = np.ascontiguousarray(msg, np.uint32)
    r = seeded_enc_randomness(n, q, sigma, msg.shape[0], seed)
    return encrypt(n, q, t, s, msg, r["mask"], r["err"])

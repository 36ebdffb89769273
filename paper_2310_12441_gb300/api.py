"""Thin Python binding of libbootmmpm.so (include/bootmmpm.h).

Argument marshalling only: every step of the hot path runs in the library's
CUDA kernels.  Device buffers are torch tensors (int64 storage holds the
uint64 words bit for bit; int32 storage holds the uint32 table entries).
Loading fails loudly when the library cannot be built or found; there is no
CPU fallback.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

from . import build as _build
from .params import KeyParams
from . import synth

BM_OK = 0
STATUS = {0: "BM_OK", -1: "BM_EINVAL", -2: "BM_ENOTPRIME", -3: "BM_ENOMEM",
          -4: "BM_ENONNEGACYCLIC", -5: "BM_ETIMEDOUT", -6: "BM_ECUDA", -7: "BM_EBUSY",
          -8: "BM_EWORKSPACE"}

SYMBOLS = ["bm_keygen", "bm_free_secret_key", "bm_free_eval_key", "bm_eval_key_bytes",
           "bm_encrypt", "bm_decrypt", "bm_workspace_bytes", "bm_bootstrap_batch",
           "bm_host_staging_bytes", "bm_bootstrap_batch_host", "bm_blind_rotate",
           "bm_sample_extract", "bm_key_switch", "bm_poly_mul", "bm_workspace_status",
           "bm_modmul_peak", "bm_status_str", "bm_bootstrap_batch_noalloc",
           "bm_batch_create", "bm_batch_run", "bm_batch_free", "bm_mod_switch",
           "bm_arbitrary_workspace_bytes", "bm_bootstrap_arbitrary", "bm_secret_key_seeded",
           "bm_keygen_seeded", "bm_secret_key_get", "bm_encrypt_seeded", "bm_workspace_bytes_gen",
           "bm_bootstrap_batch_gen", "bm_kernel_shape_info", "bm_set_kernel_shape",
           "bm_get_kernel_shape"]

BATCH_PERSISTENT = 1
BATCH_GRAPH = 2
BATCH_ONE_BLOCK = 4

NOALLOC_SCRATCH_BYTES = 16 << 20


class BMError(RuntimeError):
    def __init__(self, code: int, what: str):
        super().__init__(f"{what}: {STATUS.get(code, code)}")
        self.code = code


class _KeyParams(C.Structure):
    _fields_ = [("n", C.c_uint32), ("N", C.c_uint32), ("log2_B", C.c_uint32),
                ("l_B", C.c_uint32), ("log2_Bks", C.c_uint32), ("l_ks", C.c_uint32),
                ("Q", C.c_uint64)]


class _KeyRandomness(C.Structure):
    _fields_ = [("s", C.c_void_p), ("z", C.c_void_p), ("bsk_mask", C.c_void_p),
                ("bsk_err", C.c_void_p), ("ksk_mask", C.c_void_p), ("ksk_err", C.c_void_p)]


JOB_DTYPE = np.dtype([("key", np.uint32), ("m", np.uint32), ("t", np.uint32),
                      ("reserved", np.uint32), ("in_off", np.uint64), ("lut_off", np.uint64),
                      ("out_off", np.uint64)])

_lib = None


def library_path() -> str:
    return _build.LIB


def load(build_if_needed: bool = True) -> C.CDLL:
    """Loads libbootmmpm.so (building it in-tree with nvcc when stale)."""
    global _lib
    if _lib is not None:
        return _lib
    if build_if_needed and not _build.up_to_date():
        _build.build()
    if not os.path.exists(_build.LIB):
        raise RuntimeError("libbootmmpm.so is missing: run __graft_entry__.build()")
    L = C.CDLL(_build.LIB)
    vp, sz, u32, i32 = C.c_void_p, C.c_size_t, C.c_uint32, C.c_int32
    L.bm_keygen.argtypes = [C.POINTER(_KeyParams), C.POINTER(_KeyRandomness), C.c_int,
                            C.POINTER(vp), C.POINTER(vp)]
    L.bm_keygen.restype = i32
    L.bm_free_secret_key.argtypes = [vp]
    L.bm_free_eval_key.argtypes = [vp]
    L.bm_eval_key_bytes.argtypes = [vp]
    L.bm_eval_key_bytes.restype = sz
    L.bm_encrypt.argtypes = [vp, C.c_uint64, u32, vp, vp, vp, sz, vp]
    L.bm_encrypt.restype = i32
    L.bm_decrypt.argtypes = [vp, C.c_uint64, u32, vp, sz, vp]
    L.bm_decrypt.restype = i32
    L.bm_workspace_bytes.argtypes = [vp, u32, vp, u32]
    L.bm_workspace_bytes.restype = sz
    L.bm_bootstrap_batch.argtypes = [vp, u32, vp, u32, vp, vp, vp, vp, sz, vp]
    L.bm_bootstrap_batch.restype = i32
    L.bm_host_staging_bytes.argtypes = [vp, u32, vp, u32]
    L.bm_host_staging_bytes.restype = sz
    L.bm_bootstrap_batch_host.argtypes = [vp, u32, vp, u32, vp, sz, vp, sz, vp, sz, vp, sz, vp]
    L.bm_bootstrap_batch_host.restype = i32
    L.bm_blind_rotate.argtypes = [vp, u32, vp, u32, u32, vp, vp, vp, vp, sz, vp]
    L.bm_blind_rotate.restype = i32
    L.bm_sample_extract.argtypes = [vp, vp, u32, vp, vp]
    L.bm_sample_extract.restype = i32
    L.bm_key_switch.argtypes = [vp, vp, u32, vp, vp]
    L.bm_key_switch.restype = i32
    L.bm_poly_mul.argtypes = [vp, vp, vp, u32, vp, vp]
    L.bm_poly_mul.restype = i32
    L.bm_workspace_status.argtypes = [vp, vp]
    L.bm_workspace_status.restype = i32
    L.bm_modmul_peak.argtypes = [C.c_int, u32, C.POINTER(C.c_double)]
    L.bm_modmul_peak.restype = i32
    L.bm_bootstrap_batch_noalloc.argtypes = [vp, u32, vp, u32, vp, vp, vp, vp, vp]
    L.bm_bootstrap_batch_noalloc.restype = i32
    L.bm_batch_create.argtypes = [vp, u32, vp, u32, vp, vp, vp, vp, sz, u32, C.POINTER(vp)]
    L.bm_batch_create.restype = i32
    L.bm_batch_run.argtypes = [vp, vp]
    L.bm_batch_run.restype = i32
    L.bm_batch_free.argtypes = [vp]
    L.bm_mod_switch.argtypes = [vp, vp, sz, C.c_uint64, C.c_uint64, vp]
    L.bm_mod_switch.restype = i32
    L.bm_arbitrary_workspace_bytes.argtypes = [vp, u32, u32, u32]
    L.bm_arbitrary_workspace_bytes.restype = sz
    L.bm_bootstrap_arbitrary.argtypes = [vp, u32, u32, C.c_uint64, vp, u32, vp, vp, vp, sz, vp]
    L.bm_bootstrap_arbitrary.restype = i32
    L.bm_secret_key_seeded.argtypes = [C.POINTER(_KeyParams), u32, C.c_uint64, C.POINTER(vp)]
    L.bm_secret_key_seeded.restype = i32
    L.bm_keygen_seeded.argtypes = [C.POINTER(_KeyParams), u32, C.c_double, C.c_uint64, C.c_int,
                                   C.POINTER(vp), C.POINTER(vp)]
    L.bm_keygen_seeded.restype = i32
    L.bm_secret_key_get.argtypes = [vp, vp, vp]
    L.bm_secret_key_get.restype = i32
    L.bm_encrypt_seeded.argtypes = [vp, C.c_uint64, u32, vp, sz, C.c_double, C.c_uint64, vp]
    L.bm_encrypt_seeded.restype = i32
    L.bm_workspace_bytes_gen.argtypes = [vp, u32, vp, u32, vp, vp]
    L.bm_workspace_bytes_gen.restype = sz
    L.bm_bootstrap_batch_gen.argtypes = [vp, u32, vp, u32, vp, vp, vp, vp, vp, vp, sz, vp]
    L.bm_bootstrap_batch_gen.restype = i32
    L.bm_kernel_shape_info.argtypes = [u32, u32, vp, vp, vp]
    L.bm_kernel_shape_info.restype = i32
    L.bm_set_kernel_shape.argtypes = [u32, u32]
    L.bm_set_kernel_shape.restype = i32
    L.bm_get_kernel_shape.argtypes = [u32, vp]
    L.bm_get_kernel_shape.restype = i32
    L.bm_status_str.argtypes = [i32]
    L.bm_status_str.restype = C.c_char_p
    _lib = L
    return L


def _check(code: int, what: str):
    if code != BM_OK:
        raise BMError(code, what)


def _ptr(t) -> int:
    """Raw address of a numpy array or torch tensor (contiguous)."""
    if isinstance(t, np.ndarray):
        assert t.flags.c_contiguous
        return t.ctypes.data
    assert t.is_contiguous()
    return t.data_ptr()


def _stream(stream) -> int | None:
    if stream is None:
        import torch
        return torch.cuda.current_stream().cuda_stream
    return stream if isinstance(stream, int) else stream.cuda_stream


class SecretKey:
    def __init__(self, handle, kp: KeyParams):
        self.handle, self.kp = handle, kp

    def __del__(self):
        if getattr(self, "handle", None) and _lib is not None:
            _lib.bm_free_secret_key(self.handle)
            self.handle = None


class EvalKey:
    def __init__(self, handle, kp: KeyParams, device: int):
        self.handle, self.kp, self.device = handle, kp, device

    @property
    def nbytes(self) -> int:
        return int(load().bm_eval_key_bytes(self.handle))

    def free(self):
        if getattr(self, "handle", None) and _lib is not None:
            _lib.bm_free_eval_key(self.handle)
            self.handle = None

    def __del__(self):
        self.free()


def bm_keygen(kp: KeyParams, rnd: dict, device: int = 0) -> tuple[SecretKey, EvalKey]:
    """Key generation from supplied randomness (see synth.key_randomness)."""
    L = load()
    prm = _kparams(kp)
    arrs = {k: np.ascontiguousarray(rnd[k]) for k in
            ("s", "z", "bsk_mask", "bsk_err", "ksk_mask", "ksk_err")}
    if arrs["bsk_mask"].shape[0] != kp.n:
        raise ValueError("bootstrapping-key randomness must cover all n coordinates")
    r = _KeyRandomness(*[_ptr(arrs[k]) for k in ("s", "z", "bsk_mask", "bsk_err",
                                                   "ksk_mask", "ksk_err")])
    sk, ek = C.c_void_p(), C.c_void_p()
    _check(L.bm_keygen(C.byref(prm), C.byref(r), device, C.byref(sk), C.byref(ek)), "bm_keygen")
    return SecretKey(sk.value, kp), EvalKey(ek.value, kp, device)


def keygen(kp: KeyParams, seed: int, device: int = 0) -> tuple[SecretKey, EvalKey]:
    """Key generation from caller-drawn randomness (synth's numpy streams)."""
    return bm_keygen(kp, synth.key_randomness(kp, seed), device)


SECRET_BINARY, SECRET_TERNARY = 0, 1


def _kparams(kp: KeyParams) -> _KeyParams:
    return _KeyParams(kp.n, kp.N, kp.log2_B, kp.l_B, kp.log2_Bks, kp.l_ks, kp.Q)


def _secret_kind(kp: KeyParams) -> int:
    return SECRET_TERNARY if kp.secret == "ternary" else SECRET_BINARY


def bm_secret_key_seeded(kp: KeyParams, seed: int) -> SecretKey:
    """The secret key (s, z) drawn from `seed` on the host (no device)."""
    prm = _kparams(kp)
    sk = C.c_void_p()
    _check(load().bm_secret_key_seeded(C.byref(prm), _secret_kind(kp), seed, C.byref(sk)),
           "bm_secret_key_seeded")
    return SecretKey(sk.value, kp)


def bm_keygen_seeded(kp: KeyParams, seed: int, device: int = 0) -> tuple[SecretKey, EvalKey]:
    """Secret and evaluation keys from `seed`, the evaluation key's masks and
    errors drawn on the device (keygen-from-seed)."""
    prm = _kparams(kp)
    sk, ek = C.c_void_p(), C.c_void_p()
    _check(load().bm_keygen_seeded(C.byref(prm), _secret_kind(kp), kp.sigma, seed, device, C.byref(sk),
                                   C.byref(ek)), "bm_keygen_seeded")
    return SecretKey(sk.value, kp), EvalKey(ek.value, kp, device)


def bm_secret_key_get(sk: SecretKey) -> tuple[np.ndarray, np.ndarray]:
    s = np.empty(sk.kp.n, np.int8)
    z = np.empty(sk.kp.N, np.int8)
    _check(load().bm_secret_key_get(sk.handle, _ptr(s), _ptr(z)), "bm_secret_key_get")
    return s, z


def bm_encrypt_seeded(sk: SecretKey, q: int, t: int, msg, seed: int, sigma: float | None = None) -> np.ndarray:
    msg = np.ascontiguousarray(msg, np.uint32)
    out = np.empty((msg.shape[0], sk.kp.n + 1), np.uint64)
    sg = sk.kp.sigma if sigma is None else sigma
    _check(load().bm_encrypt_seeded(sk.handle, q, t, _ptr(msg), msg.shape[0], sg, seed, _ptr(out)),
           "bm_encrypt_seeded")
    return out


def bm_encrypt(sk: SecretKey, q: int, t: int, msg, mask, err) -> np.ndarray:
    msg = np.ascontiguousarray(msg, np.uint32)
    mask = np.ascontiguousarray(mask, np.uint64)
    err = np.ascontiguousarray(err, np.int8)
    out = np.empty((msg.shape[0], sk.kp.n + 1), np.uint64)
    _check(load().bm_encrypt(sk.handle, q, t, _ptr(msg), _ptr(mask), _ptr(err), msg.shape[0],
                             _ptr(out)), "bm_encrypt")
    return out


def bm_decrypt(sk: SecretKey, q: int, t: int, ct) -> np.ndarray:
    ct = np.ascontiguousarray(np.atleast_2d(ct), np.uint64)
    out = np.empty(ct.shape[0], np.uint32)
    _check(load().bm_decrypt(sk.handle, q, t, _ptr(ct), ct.shape[0], _ptr(out)), "bm_decrypt")
    return out


def _keys(keys):
    keys = keys if isinstance(keys, (list, tuple)) else [keys]
    return (C.c_void_p * len(keys))(*[k.handle for k in keys]), len(keys)


def make_jobs(key_idx, m, t, in_off, lut_off, out_off) -> np.ndarray:
    cnt = max(np.size(x) for x in (key_idx, m, t, in_off, lut_off, out_off))
    jobs = np.zeros(cnt, JOB_DTYPE)
    jobs["key"], jobs["m"], jobs["t"] = key_idx, m, t
    jobs["in_off"], jobs["lut_off"], jobs["out_off"] = in_off, lut_off, out_off
    return jobs


def bm_workspace_bytes(keys, jobs: np.ndarray) -> int:
    karr, nk = _keys(keys)
    jobs = np.ascontiguousarray(jobs, JOB_DTYPE)
    return int(load().bm_workspace_bytes(karr, nk, _ptr(jobs), len(jobs)))


def bm_host_staging_bytes(keys, jobs: np.ndarray) -> int:
    karr, nk = _keys(keys)
    jobs = np.ascontiguousarray(jobs, JOB_DTYPE)
    return int(load().bm_host_staging_bytes(karr, nk, _ptr(jobs), len(jobs)))


def bm_bootstrap_batch(keys, jobs: np.ndarray, d_ct_in, d_lut, d_ct_out, d_ws, stream=None):
    karr, nk = _keys(keys)
    jobs = np.ascontiguousarray(jobs, JOB_DTYPE)
    _check(load().bm_bootstrap_batch(karr, nk, _ptr(jobs), len(jobs), _ptr(d_ct_in), _ptr(d_lut),
                                     _ptr(d_ct_out), _ptr(d_ws), d_ws.numel() * d_ws.element_size(),
                                     _stream(stream)), "bm_bootstrap_batch")


NUM_SHAPES = 5
SHAPE_DEFAULT = 0xFFFFFFFF


def kernel_shapes(N: int) -> dict:
    """{shape: (radix, threads, blocks per SM)} of the shapes that fit ring degree N."""
    out = {}
    for sh in range(NUM_SHAPES):
        r, t, b = C.c_uint32(), C.c_uint32(), C.c_uint32()
        if load().bm_kernel_shape_info(sh, N, C.byref(r), C.byref(t), C.byref(b)) == BM_OK:
            out[sh] = (r.value, t.value, b.value)
    return out


def set_kernel_shape(N: int, shape: int) -> None:
    _check(load().bm_set_kernel_shape(N, shape), "bm_set_kernel_shape")


def get_kernel_shape(N: int) -> int:
    v = C.c_uint32()
    _check(load().bm_get_kernel_shape(N, C.byref(v)), "bm_get_kernel_shape")
    return v.value


GEN_EXAMPLE1 = (1 << 64) - 1


def _gens(gens, gen_off):
    gens = np.ascontiguousarray(gens, np.uint32)
    gen_off = np.ascontiguousarray(gen_off, np.uint64)
    return gens, gen_off


def bm_workspace_bytes_gen(keys, jobs: np.ndarray, gens, gen_off) -> int:
    karr, nk = _keys(keys)
    jobs = np.ascontiguousarray(jobs, JOB_DTYPE)
    gens, gen_off = _gens(gens, gen_off)
    return int(load().bm_workspace_bytes_gen(karr, nk, _ptr(jobs), len(jobs), _ptr(gens), _ptr(gen_off)))


def bm_bootstrap_batch_gen(keys, jobs: np.ndarray, gens, gen_off, d_ct_in, d_lut, d_ct_out, d_ws, stream=None):
    """bm_bootstrap_batch with a transitive generator per job (Theorem 1):
    job i uses the exponents gens[gen_off[i]:gen_off[i] + m], or Example 1's
    P(1) where gen_off[i] == GEN_EXAMPLE1."""
    karr, nk = _keys(keys)
    jobs = np.ascontiguousarray(jobs, JOB_DTYPE)
    gens, gen_off = _gens(gens, gen_off)
    _check(load().bm_bootstrap_batch_gen(karr, nk, _ptr(jobs), len(jobs), _ptr(gens), _ptr(gen_off),
                                         _ptr(d_ct_in), _ptr(d_lut), _ptr(d_ct_out), _ptr(d_ws),
                                         d_ws.numel() * d_ws.element_size(), _stream(stream)),
           "bm_bootstrap_batch_gen")


def bm_bootstrap_batch_noalloc(keys, jobs: np.ndarray, d_ct_in, d_lut, d_ct_out, d_status=None,
                               stream=None):
    """bm_bootstrap_batch for callers that cannot allocate device memory: the
    scratch is a fixed array inside the library (NOALLOC_SCRATCH_BYTES), so no
    workspace is passed.  Calls that overlap on the GPU race on that array."""
    karr, nk = _keys(keys)
    jobs = np.ascontiguousarray(jobs, JOB_DTYPE)
    _check(load().bm_bootstrap_batch_noalloc(karr, nk, _ptr(jobs), len(jobs), _ptr(d_ct_in),
                                             _ptr(d_lut), _ptr(d_ct_out),
                                             None if d_status is None else _ptr(d_status),
                                             _stream(stream)), "bm_bootstrap_batch_noalloc")


class Batch:
    """A reusable batch (bm_batch_create): buffers stay bound until free()."""

    def __init__(self, keys, jobs: np.ndarray, d_ct_in, d_lut, d_ct_out, d_ws, flags: int = 0):
        karr, nk = _keys(keys)
        self._keys = keys          # keep the key handles alive
        self._bufs = (d_ct_in, d_lut, d_ct_out, d_ws)
        jobs = np.ascontiguousarray(jobs, JOB_DTYPE)
        h = C.c_void_p()
        _check(load().bm_batch_create(karr, nk, _ptr(jobs), len(jobs), _ptr(d_ct_in), _ptr(d_lut),
                                      _ptr(d_ct_out), _ptr(d_ws), d_ws.numel() * d_ws.element_size(),
                                      flags, C.byref(h)), "bm_batch_create")
        self.handle = h.value

    def run(self, stream=None):
        _check(load().bm_batch_run(self.handle, _stream(stream)), "bm_batch_run")

    def free(self):
        if getattr(self, "handle", None) and _lib is not None:
            _lib.bm_batch_free(self.handle)
            self.handle = None

    def __del__(self):
        self.free()


def bm_bootstrap_batch_host(keys, jobs: np.ndarray, h_ct_in, h_lut, h_ct_out, d_ws, stream=None):
    """h_* are host buffers (numpy arrays or pinned CPU tensors)."""
    karr, nk = _keys(keys)
    jobs = np.ascontiguousarray(jobs, JOB_DTYPE)

    def words(x):
        return x.size if isinstance(x, np.ndarray) else x.numel()
    _check(load().bm_bootstrap_batch_host(karr, nk, _ptr(jobs), len(jobs), _ptr(h_ct_in),
                                          words(h_ct_in), _ptr(h_lut), words(h_lut), _ptr(h_ct_out),
                                          words(h_ct_out), _ptr(d_ws),
                                          d_ws.numel() * d_ws.element_size(), _stream(stream)),
           "bm_bootstrap_batch_host")


def bm_blind_rotate(keys, jobs: np.ndarray, steps: int, d_ct_in, d_lut, d_acc_out, d_ws, stream=None):
    karr, nk = _keys(keys)
    jobs = np.ascontiguousarray(jobs, JOB_DTYPE)
    _check(load().bm_blind_rotate(karr, nk, _ptr(jobs), len(jobs), int(steps), _ptr(d_ct_in),
                                  _ptr(d_lut), _ptr(d_acc_out), _ptr(d_ws),
                                  d_ws.numel() * d_ws.element_size(), _stream(stream)),
           "bm_blind_rotate")


def bm_sample_extract(key: EvalKey, d_rlwe, count: int, d_out, stream=None):
    _check(load().bm_sample_extract(key.handle, _ptr(d_rlwe), count, _ptr(d_out), _stream(stream)),
           "bm_sample_extract")


def bm_key_switch(key: EvalKey, d_lwe_in, count: int, d_out, stream=None):
    _check(load().bm_key_switch(key.handle, _ptr(d_lwe_in), count, _ptr(d_out), _stream(stream)),
           "bm_key_switch")


def bm_poly_mul(key: EvalKey, d_a, d_b, count: int, d_out, stream=None):
    _check(load().bm_poly_mul(key.handle, _ptr(d_a), _ptr(d_b), count, _ptr(d_out), _stream(stream)),
           "bm_poly_mul")


def bm_mod_switch(d_in, d_out, q_from: int, q_to: int, stream=None):
    """Section 2 (9) on every word of d_in (device tensor) into d_out."""
    _check(load().bm_mod_switch(_ptr(d_in), _ptr(d_out), d_in.numel(), q_from, q_to, _stream(stream)),
           "bm_mod_switch")


def bm_arbitrary_workspace_bytes(key: EvalKey, m: int, t: int, count: int) -> int:
    return int(load().bm_arbitrary_workspace_bytes(key.handle, m, t, count))


def bm_bootstrap_arbitrary(key: EvalKey, m: int, t: int, q: int, d_f, count: int, d_ct_in, d_ct_out,
                           d_ws, stream=None):
    """Two-round bootstrap of any f: Z_t -> Z_t (tables d_f, t entries each)."""
    _check(load().bm_bootstrap_arbitrary(key.handle, m, t, q, _ptr(d_f), count, _ptr(d_ct_in),
                                         _ptr(d_ct_out), _ptr(d_ws), d_ws.numel() * d_ws.element_size(),
                                         _stream(stream)), "bm_bootstrap_arbitrary")


def bm_workspace_status(d_ws, stream=None) -> int:
    return int(load().bm_workspace_status(_ptr(d_ws), _stream(stream)))


def bm_modmul_peak(device: int = 0, iters: int = 1 << 14) -> float:
    r = C.c_double()
    _check(load().bm_modmul_peak(device, iters, C.byref(r)), "bm_modmul_peak")
    return r.value


# -- torch helpers -----------------------------------------------------------------

def to_device_u64(a: np.ndarray, device="cuda"):
    import torch
    return torch.from_numpy(np.ascontiguousarray(a, np.uint64).view(np.int64)).to(device)


def to_device_u32(a: np.ndarray, device="cuda"):
    import torch
    return torch.from_numpy(np.ascontiguousarray(a, np.uint32).view(np.int32)).to(device)


def from_device_u64(t) -> np.ndarray:
    return t.cpu().numpy().view(np.uint64)


def workspace(nbytes: int, device="cuda"):
    import torch
    return torch.zeros(max(int(nbytes), 256) + 256, dtype=torch.uint8, device=device)

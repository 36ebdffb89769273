"""Ring degree 8192: the single-polynomial layout of the plaintext-size sweep
at log t = 7 (Sec. 5, Table 1: N = 2^(log t + 6)), bit-exact with the oracle.

The key shape is the sweep's (log Q = 54, B = 2^15 x 4 digits, key-switching
base 2^5 x 8) with n = 16 LWE coefficients, so that the oracle's schoolbook
products stay affordable; ciphertexts whose masks are zero after two entries
make the oracle skip the other CMux steps (zero digits).  Every kernel shape
that holds a whole 8192-coefficient polynomial in one block is checked.
"""
import numpy as np
import pytest

from paper_2310_12441_gb300 import params as P
from paper_2310_12441_gb300 import synth

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

KP = P.KeyParams(n=16, N=8192, Q=P.KEYS_SWEEP_N2048.Q, log2_B=15, l_B=4, log2_Bks=5, l_ks=8)


@pytest.fixture(scope="module")
def api():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2310_12441_gb300 import api as A
    A.load()
    return A


@pytest.fixture(scope="module")
def keys(api, orc):
    rnd = synth.key_randomness(KP, 1013)
    sk, ek = api.bm_keygen(KP, rnd, 0)
    bsk = orc.keygen_bsk(KP, rnd, 0, 2)          # the keys of the first two CMux steps
    ksk = orc.keygen_ksk(KP, rnd)
    return rnd, sk, ek, bsk, ksk


def test_poly_mul_n8192_matches_schoolbook(api, orc, keys):
    _, _, ek, _, _ = keys
    rng = np.random.default_rng(8192)
    a = rng.integers(0, KP.Q, (2, KP.N), dtype=np.uint64)
    b = rng.integers(0, KP.Q, (2, KP.N), dtype=np.uint64)
    a[0] = 0; a[0, KP.N - 1] = 1               # x^(N-1) b: a negacyclic shift of every coefficient
    d_out = torch.zeros(2 * KP.N, dtype=torch.int64, device="cuda")
    api.bm_poly_mul(ek, api.to_device_u64(a), api.to_device_u64(b), 2, d_out)
    got = api.from_device_u64(d_out).reshape(2, KP.N)
    for i in range(2):
        assert np.array_equal(got[i], orc.poly_mul(KP.N, KP.Q, a[i], b[i])), i


@pytest.mark.parametrize("shape", [0, 1])
def test_bootstrap_n8192_single_polynomial_bit_exact(api, orc, keys, shape):
    """m = 1, t = 128 (q' = 2N = 16384, the Delta of the sweep's single-polynomial
    row): two prefix ciphertexts bootstrap to the oracle's exact words."""
    rnd, sk, ek, bsk, ksk = keys
    assert shape in api.kernel_shapes(KP.N)
    m, t, cnt = 1, 128, 2
    qp = 2 * KP.N * m
    msg = synth.messages(t, cnt, 3013)
    enc = synth.encryption_randomness(KP.n, qp, KP.sigma, cnt, 4013, prefix=2)
    ct = orc.encrypt(KP.n, qp, t, rnd["s"], msg, enc["mask"], enc["err"])
    luts, _ = synth.luts(t, cnt, 2013)
    jobs = api.make_jobs(0, m, t, np.arange(cnt) * (KP.n + 1), np.arange(cnt) * t, np.arange(cnt) * (KP.n + 1))
    d_in, d_lut = api.to_device_u64(ct.ravel()), api.to_device_u32(luts.ravel())
    d_out = torch.zeros(cnt * (KP.n + 1), dtype=torch.int64, device="cuda")
    ws = api.workspace(api.bm_workspace_bytes([ek], jobs))
    old = api.get_kernel_shape(KP.N)
    try:
        api.set_kernel_shape(KP.N, shape)
        api.bm_bootstrap_batch([ek], jobs, d_in, d_lut, d_out, ws)
        torch.cuda.synchronize()
    finally:
        api.set_kernel_shape(KP.N, old)
    assert api.bm_workspace_status(ws) == 0
    got = api.from_device_u64(d_out).reshape(cnt, KP.n + 1)
    assert np.array_equal(got, orc.bootstrap(KP, m, t, bsk, ksk, ct, luts))
    dec_in = orc.decrypt(KP.n, qp, t, rnd["s"], ct)
    assert np.array_equal(api.bm_decrypt(sk, KP.Q, t, got), luts[np.arange(cnt), dec_in])


def test_identity_two_rounds_n8192_full_length(api, keys):
    """The sweep's single-polynomial identity at log t = 7 (plaintext modulus
    2t = 256, q = 2N): every CMux step of both rounds, every output decrypts
    to its input."""
    rnd, sk, ek, _, _ = keys
    m, t, cnt = 1, 128, 64
    q = 2 * KP.N * m
    x = np.random.default_rng(7).integers(0, 2 * t, cnt).astype(np.uint32)
    enc = synth.encryption_randomness(KP.n, q, KP.sigma, cnt, 4113)
    ct = api.bm_encrypt(sk, q, 2 * t, x, enc["mask"], enc["err"])
    f = np.tile(np.arange(t, dtype=np.uint32), cnt)
    d_in = api.to_device_u64(ct.ravel())
    d_out = torch.zeros_like(d_in)
    ws = api.workspace(api.bm_arbitrary_workspace_bytes(ek, m, t, cnt))
    api.bm_bootstrap_arbitrary(ek, m, t, q, api.to_device_u32(f), cnt, d_in, d_out, ws)
    torch.cuda.synchronize()
    assert api.bm_workspace_status(ws) == 0
    out = api.from_device_u64(d_out).reshape(cnt, KP.n + 1)
    assert np.array_equal(api.bm_decrypt(sk, q, 2 * t, out), x % t)

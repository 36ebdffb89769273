"""Ring degrees above 8192 (the single-polynomial layout of the plaintext-size
sweep at log t >= 8, Sec. 5 Tables 1-2): two-pass transforms over global
memory and CMux steps as kernel sequences, bit-exact with the oracle.

Key shape of the sweep (log Q = 54, B = 2^15 x 4, key switching 2^5 x 8) at
N = 16384 with n = 16; a ciphertext whose mask is zero after its first entry
keeps the oracle's schoolbook products to one CMux step.
"""
import numpy as np
import pytest

from paper_2310_12441_gb300 import params as P
from paper_2310_12441_gb300 import synth

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

KP = P.KeyParams(n=16, N=16384, Q=P.KEYS_SWEEP_N2048.Q, log2_B=15, l_B=4, log2_Bks=5, l_ks=8)


@pytest.fixture(scope="module")
def api():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2310_12441_gb300 import api as A
    A.load()
    return A


@pytest.fixture(scope="module")
def keys(api, orc):
    rnd = synth.key_randomness(KP, 1016)
    sk, ek = api.bm_keygen(KP, rnd, 0)
    bsk = orc.keygen_bsk(KP, rnd, 0, 1)          # the key of the first CMux step
    ksk = orc.keygen_ksk(KP, rnd)
    return rnd, sk, ek, bsk, ksk


def test_poly_mul_n16384_matches_schoolbook(api, orc, keys):
    _, _, ek, _, _ = keys
    rng = np.random.default_rng(16384)
    a = rng.integers(0, KP.Q, (2, KP.N), dtype=np.uint64)
    b = rng.integers(0, KP.Q, (2, KP.N), dtype=np.uint64)
    a[0] = 0; a[0, 1] = 1                      # x b: a negacyclic shift
    d_out = torch.zeros(2 * KP.N, dtype=torch.int64, device="cuda")
    api.bm_poly_mul(ek, api.to_device_u64(a), api.to_device_u64(b), 2, d_out)
    got = api.from_device_u64(d_out).reshape(2, KP.N)
    for i in range(2):
        assert np.array_equal(got[i], orc.poly_mul(KP.N, KP.Q, a[i], b[i])), i


def test_no_kernel_shapes_above_8192(api):
    assert api.kernel_shapes(KP.N) == {}


def test_bootstrap_n16384_bit_exact(api, orc, keys):
    """m = 1, t = 256 (q' = 2N): two ciphertexts whose masks are zero after
    their first entry bootstrap to the oracle's exact words, and decrypt to
    f(Dec(input))."""
    rnd, sk, ek, bsk, ksk = keys
    m, t, cnt = 1, 256, 2
    qp = 2 * KP.N * m
    msg = synth.messages(t, cnt, 3016)
    enc = synth.encryption_randomness(KP.n, qp, KP.sigma, cnt, 4016, prefix=1)
    ct = orc.encrypt(KP.n, qp, t, rnd["s"], msg, enc["mask"], enc["err"])
    luts, _ = synth.luts(t, cnt, 2016)
    jobs = api.make_jobs(0, m, t, np.arange(cnt) * (KP.n + 1), np.arange(cnt) * t, np.arange(cnt) * (KP.n + 1))
    d_out = torch.zeros(cnt * (KP.n + 1), dtype=torch.int64, device="cuda")
    ws = api.workspace(api.bm_workspace_bytes([ek], jobs))
    api.bm_bootstrap_batch([ek], jobs, api.to_device_u64(ct.ravel()), api.to_device_u32(luts.ravel()), d_out, ws)
    torch.cuda.synchronize()
    assert api.bm_workspace_status(ws) == 0
    got = api.from_device_u64(d_out).reshape(cnt, KP.n + 1)
    assert np.array_equal(got, orc.bootstrap(KP, m, t, bsk, ksk, ct, luts))
    dec_in = orc.decrypt(KP.n, qp, t, rnd["s"], ct)
    assert np.array_equal(api.bm_decrypt(sk, KP.Q, t, got), luts[np.arange(cnt), dec_in])


def test_big_ring_needs_one_polynomial(api, keys):
    """Above 8192 only the single-polynomial layout (m = 1) is built."""
    _, _, ek, _, _ = keys
    jobs = api.make_jobs(0, 2, 256, [0], [0], [0])
    assert api.bm_workspace_bytes([ek], jobs) == 0


def test_identity_two_rounds_n16384_full_length(api, keys):
    """The sweep's single-polynomial identity at log t = 8 (plaintext modulus
    2t = 512, q = 2N): every CMux step of both rounds, every output decrypts
    to its input."""
    rnd, sk, ek, _, _ = keys
    m, t, cnt = 1, 256, 32
    q = 2 * KP.N * m
    x = np.random.default_rng(8).integers(0, 2 * t, cnt).astype(np.uint32)
    enc = synth.encryption_randomness(KP.n, q, KP.sigma, cnt, 4116)
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

"""Ring degrees 2^15 and 2^16 on the two-pass path (the plaintext-size
sweep's single-polynomial rows at log t = 9 and 10, Sec. 5 Tables 1-2).
Their row passes (2^15, 2^16) and column passes (2^16) have 8 stages, two
four-stage register chunks, where N = 2^14 has 7.

The oracle's schoolbook products are too slow at these sizes, so the ring
products are checked against the negacyclic product's definition: every
coefficient of x^e b (a signed rotation), and sampled coefficients of a
dense product, each summed exactly in Python integers.  The CMux steps are
checked by the full-length two-round identity, every output decrypted.
"""
import numpy as np
import pytest

from paper_2310_12441_gb300 import params as P
from paper_2310_12441_gb300 import synth

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

SIZES = (32768, 65536)


def kp_of(N):
    return P.KeyParams(n=16, N=N, Q=P.KEYS_SWEEP_N2048.Q, log2_B=15, l_B=4, log2_Bks=5, l_ks=8)


@pytest.fixture(scope="module")
def api():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2310_12441_gb300 import api as A
    A.load()
    return A


@pytest.fixture(scope="module", params=SIZES)
def keys(request, api):
    kp = kp_of(request.param)
    sk, ek = api.bm_keygen_seeded(kp, 1015 + request.param, 0)     # drawn on the device
    yield kp, sk, ek
    del ek
    torch.cuda.empty_cache()


def negacyclic_coeff(a, b, k, N, Q):
    """Coefficient k of a b mod (x^N + 1, Q), from the definition."""
    s = 0
    for i in range(N):
        j = k - i
        if j >= 0:
            s += int(a[i]) * int(b[j])
        else:
            s -= int(a[i]) * int(b[j + N])
    return s % Q


def test_poly_mul_monomial_and_sampled(api, keys):
    kp, _, ek = keys
    N, Q = kp.N, kp.Q
    rng = np.random.default_rng(N)
    a = rng.integers(0, Q, (2, N), dtype=np.uint64)
    b = rng.integers(0, Q, (2, N), dtype=np.uint64)
    e = 12345 % N
    a[0] = 0
    a[0, e] = 1                                  # x^e b
    d_out = torch.zeros(2 * N, dtype=torch.int64, device="cuda")
    api.bm_poly_mul(ek, api.to_device_u64(a), api.to_device_u64(b), 2, d_out)
    got = api.from_device_u64(d_out).reshape(2, N)
    # x^e b: coefficient j + e of b_j, negated where it wraps past x^N
    want = np.empty(N, np.uint64)
    bj = b[0].astype(object)
    for j in range(N):
        t = j + e
        want[t % N] = int(bj[j]) if t < N else (Q - int(bj[j])) % Q
    assert np.array_equal(got[0], want)
    for k in [0, 1, N // 2 - 1, N // 2, N - 2, N - 1] + list(rng.integers(0, N, 10)):
        assert int(got[1, k]) == negacyclic_coeff(a[1], b[1], int(k), N, Q), k


def test_identity_two_rounds_full_length(api, keys):
    """Every CMux step of both rounds at log t = log N - 6 (q = 2N): every
    output decrypts to its input."""
    kp, sk, ek = keys
    m, t, cnt = 1, kp.N // 64, 16
    q = 2 * kp.N * m
    x = np.random.default_rng(kp.N + 8).integers(0, 2 * t, cnt).astype(np.uint32)
    enc = synth.encryption_randomness(kp.n, q, kp.sigma, cnt, 4117)
    ct = api.bm_encrypt(sk, q, 2 * t, x, enc["mask"], enc["err"])
    f = np.tile(np.arange(t, dtype=np.uint32), cnt)
    d_in = api.to_device_u64(ct.ravel())
    d_out = torch.zeros_like(d_in)
    ws = api.workspace(api.bm_arbitrary_workspace_bytes(ek, m, t, cnt))
    api.bm_bootstrap_arbitrary(ek, m, t, q, api.to_device_u32(f), cnt, d_in, d_out, ws)
    torch.cuda.synchronize()
    assert api.bm_workspace_status(ws) == 0
    out = api.from_device_u64(d_out).reshape(cnt, kp.n + 1)
    assert np.array_equal(api.bm_decrypt(sk, q, 2 * t, out), x % t)

"""Other transitive generators (Theorem 1) on the GPU: bootstraps with a
generator per job are bit-exact with the oracle's (Lemma 3's P(c), the test
vector of Eq. (equ:test-gene)), and generators that are not transitive are
refused on the host."""
import numpy as np
import pytest

from paper_2310_12441_gb300 import params as P
from paper_2310_12441_gb300 import synth

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def api():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2310_12441_gb300 import api as A
    A.load()
    return A


def _odd_gens(rng, N, m, count):
    out = []
    while len(out) < count:
        u = rng.integers(0, 2 * N, m).astype(np.uint32)
        if int(u.sum()) % 2:
            out.append(u)
    return out


def _case(api, orc, kp, seed, m, t, count, prefix, example1_jobs=()):
    sk, ek = api.bm_keygen_seeded(kp, seed)
    rnd = orc.seeded_key_randomness(kp, seed, bsk_keys=prefix or kp.n)
    bsk, ksk = orc.keygen_bsk(kp, rnd), orc.keygen_ksk(kp, rnd)
    qp = 2 * kp.N * m
    msg = synth.messages(t, count, seed + 1)
    ct = api.bm_encrypt_seeded(sk, qp, t, msg, seed + 2)
    if prefix:
        ct[:, prefix:kp.n] = 0
    luts, _ = synth.luts(t, count, seed + 3)
    rng = np.random.default_rng(seed)
    u = np.stack(_odd_gens(rng, kp.N, m, count))
    for j in example1_jobs:
        u[j] = 0
        u[j, 0] = 1
    gens = u.ravel()
    gen_off = np.arange(count, dtype=np.uint64) * m
    if example1_jobs:
        gen_off[example1_jobs[0]] = api.GEN_EXAMPLE1     # by the sentinel, not by exponents
    W = kp.n + 1
    jobs = api.make_jobs(0, m, t, np.arange(count) * W, np.arange(count) * t, np.arange(count) * W)
    d_out = torch.zeros(count * W, dtype=torch.int64, device="cuda")
    ws = api.workspace(api.bm_workspace_bytes_gen([ek], jobs, gens, gen_off))
    api.bm_bootstrap_batch_gen([ek], jobs, gens, gen_off, api.to_device_u64(ct.ravel()),
                               api.to_device_u32(luts.ravel()), d_out, ws)
    torch.cuda.synchronize()
    assert api.bm_workspace_status(ws) == 0
    got = api.from_device_u64(d_out).reshape(count, W)
    want = orc.bootstrap_gen(kp, m, t, u, bsk, ksk, ct, luts)
    assert np.array_equal(got, want)
    dec_in = api.bm_decrypt(sk, qp, t, ct)
    assert np.array_equal(api.bm_decrypt(sk, kp.Q, t, got), luts[np.arange(count), dec_in])


def test_toy_generators_full_length_bit_exact(api, orc):
    """Toy set, all n = 64 steps, a different generator per job; jobs 0 and 1
    use Example 1's generator (by the sentinel and by its exponents)."""
    _case(api, orc, P.KEYS_TOY, 1001, 2, 32, 12, None, example1_jobs=(0, 1))


@pytest.mark.parametrize("kp,m,t", [(P.KEYS_N1024, 4, 1024), (P.KEYS_N2048, 8, 8192), (P.KEYS_N1024, 3, 768)],
                         ids=["n630_N1024_m4", "n750_N2048_m8", "n630_N1024_m3"])
def test_production_keys_generators_prefix_bit_exact(api, orc, kp, m, t):
    _case(api, orc, kp, 1200 + m, m, t, 4, 6)


def test_generators_that_are_not_transitive_are_refused(api):
    kp = P.KEYS_TOY
    sk, ek = api.bm_keygen_seeded(kp, 1001)
    jobs = api.make_jobs(0, 2, 32, 0, 0, 0)
    d = torch.zeros(kp.n + 1, dtype=torch.int64, device="cuda")
    dl = torch.zeros(32, dtype=torch.int32, device="cuda")
    ws = api.workspace(1 << 20)
    for u in ([2, 0], [1, 1], [512, 1]):          # even sum (Theorem 1), exponent >= 2N
        with pytest.raises(api.BMError) as e:
            api.bm_bootstrap_batch_gen([ek], jobs, np.array(u, np.uint32), np.zeros(1, np.uint64), d, dl, d, ws)
        assert e.value.code == -1

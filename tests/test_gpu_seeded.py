"""Keys generated on the GPU from a seed agree with the oracle's keys drawn
from the same seed (Algorithm 1 REQUIRE block): both sides implement the
same published generator (Philox4x32-10) and stream layout independently.
Compared through bootstrapped outputs, bit for bit (tolerance 0)."""
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


def _run(api, keys, jobs, ct, luts, out_words, flags=None):
    d_in = api.to_device_u64(np.ascontiguousarray(ct).ravel())
    d_lut = api.to_device_u32(np.ascontiguousarray(luts).ravel())
    d_out = torch.zeros(out_words, dtype=torch.int64, device="cuda")
    ws = api.workspace(api.bm_workspace_bytes(keys, jobs))
    if flags is None:
        api.bm_bootstrap_batch(keys, jobs, d_in, d_lut, d_out, ws)
    else:
        b = api.Batch(keys, jobs, d_in, d_lut, d_out, ws, flags)
        b.run()
        torch.cuda.synchronize()
        b.free()
    torch.cuda.synchronize()
    assert api.bm_workspace_status(ws) == 0
    return api.from_device_u64(d_out)


def _jobs(api, count, n, t, m):
    W = n + 1
    return api.make_jobs(0, m, t, np.arange(count) * W, np.arange(count) * t, np.arange(count) * W)


def test_seeded_keygen_toy_every_message_bit_exact(api, orc):
    """Toy set, all n = 64 CMux steps, every message of Z_32: device keys from
    the seed, oracle keys from the same seed, equal outputs."""
    kp, m, t = P.KEYS_TOY, 2, 32
    sk, ek = api.bm_keygen_seeded(kp, 1001)
    rnd = orc.seeded_key_randomness(kp, 1001)
    s, z = api.bm_secret_key_get(sk)
    assert np.array_equal(s, rnd["s"]) and np.array_equal(z, rnd["z"])
    bsk, ksk = orc.keygen_bsk(kp, rnd), orc.keygen_ksk(kp, rnd)
    qp = 2 * kp.N * m
    msg = np.arange(t, dtype=np.uint32)
    ct = api.bm_encrypt_seeded(sk, qp, t, msg, 4001)
    assert np.array_equal(ct, orc.encrypt_seeded(kp.n, qp, t, rnd["s"], msg, kp.sigma, 4001))
    luts, _ = synth.luts(t, t, 2001)
    got = _run(api, [ek], _jobs(api, t, kp.n, t, m), ct, luts, t * (kp.n + 1)).reshape(t, kp.n + 1)
    assert np.array_equal(got, orc.bootstrap(kp, m, t, bsk, ksk, ct, luts))


@pytest.mark.parametrize("kp,m,t", [(P.KEYS_N1024, 4, 1024), (P.KEYS_N2048, 8, 8192)],
                         ids=["n630_N1024", "n750_N2048"])
def test_device_draws_equal_the_oracle_streams(api, orc, kp, m, t):
    """Keys drawn on the device (bm_keygen_seeded) and keys built from the
    oracle's draws of the same streams (bm_keygen with those arrays) give the
    same bits for full-length bootstraps: every BSK and KSK word the device drew
    matches the oracle's stream."""
    seed = 77
    sk_d, ek_d = api.bm_keygen_seeded(kp, seed)
    rnd = orc.seeded_key_randomness(kp, seed)
    sk_a, ek_a = api.bm_keygen(kp, rnd)
    del rnd
    cnt = 32
    qp = 2 * kp.N * m
    msg = synth.messages(t, cnt, 61)
    ct = api.bm_encrypt_seeded(sk_d, qp, t, msg, 62)
    luts, _ = synth.luts(t, cnt, 63)
    jobs = _jobs(api, cnt, kp.n, t, m)
    a = _run(api, [ek_d], jobs, ct, luts, cnt * (kp.n + 1))
    b = _run(api, [ek_a], jobs, ct, luts, cnt * (kp.n + 1))
    assert np.array_equal(a, b)
    dec_in = api.bm_decrypt(sk_d, qp, t, ct)
    dec_out = api.bm_decrypt(sk_d, kp.Q, t, a.reshape(cnt, kp.n + 1))
    assert np.array_equal(dec_out, luts[np.arange(cnt), dec_in])


def test_seeded_keygen_rejects_bad_sigma(api):
    import ctypes as C
    L = api.load()
    kp = P.KEYS_TOY
    prm = api._kparams(kp)
    sk, ek = C.c_void_p(), C.c_void_p()
    for sigma in (0.0, 5.0):
        assert L.bm_keygen_seeded(C.byref(prm), 0, sigma, 1, 0, C.byref(sk), C.byref(ek)) == -1

"""The library's host-side seeded streams agree with the oracle's independent
implementation of the same generator (Philox4x32-10) and stream layout: the
secret key drawn from a seed, and LWE encryption with masks and errors drawn
from a seed (Section 2 (8)).  Host code only: no device is needed."""
import numpy as np
import pytest

from paper_2310_12441_gb300 import params as P
from paper_2310_12441_gb300 import synth


@pytest.fixture(scope="module")
def api():
    from paper_2310_12441_gb300 import api as A
    A.load()
    return A


@pytest.mark.parametrize("kp", [P.KEYS_TOY, P.KEYS_N1024, P.KEYS_N2048, P.KEYS_N4096],
                         ids=["toy", "n630_N1024", "n750_N2048", "n630_N4096"])
def test_secret_key_from_seed_equals_oracle(api, orc, kp):
    for seed in (1002, 2 ** 40 + 3):
        sk = api.bm_secret_key_seeded(kp, seed)
        s, z = api.bm_secret_key_get(sk)
        want = orc.seeded_key_randomness(kp, seed, bsk_keys=0, with_ksk=False)
        assert np.array_equal(s, want["s"]) and np.array_equal(z, want["z"])


@pytest.mark.parametrize("kp,m,t", [(P.KEYS_TOY, 2, 32), (P.KEYS_N1024, 4, 1024), (P.KEYS_N2048, 8, 8192)],
                         ids=["toy", "n630_N1024", "n750_N2048"])
def test_encryption_from_seed_equals_oracle(api, orc, kp, m, t):
    sk = api.bm_secret_key_seeded(kp, 7)
    s, _ = api.bm_secret_key_get(sk)
    qp = 2 * kp.N * m
    msg = synth.messages(t, 257, 12)
    got = api.bm_encrypt_seeded(sk, qp, t, msg, 4242)
    want = orc.encrypt_seeded(kp.n, qp, t, s, msg, kp.sigma, 4242)
    assert np.array_equal(got, want)
    assert np.array_equal(api.bm_decrypt(sk, qp, t, got), orc.decrypt(kp.n, qp, t, s, want))


def test_seeded_calls_reject_bad_arguments(api):
    kp = P.KEYS_TOY
    with pytest.raises(api.BMError):
        api.bm_secret_key_seeded(P.KeyParams(**{**kp.__dict__, "Q": kp.Q + 2}), 1)
    sk = api.bm_secret_key_seeded(kp, 1)
    for sigma in (0.0, -1.0, 4.5):
        with pytest.raises(api.BMError):
            api.bm_encrypt_seeded(sk, 1024, 32, np.zeros(2, np.uint32), 5, sigma=sigma)


def test_ring_degree_range_on_the_host(api, orc):
    """Key parameters are accepted up to ring degree 65536 (above 8192 the
    single-polynomial layout runs through two-pass transforms) and refused
    beyond; the secret key of a 65536-coefficient set still equals the
    oracle's draws."""
    kp = P.KeyParams(**{**P.KEYS_SWEEP_N2048.__dict__, "n": 16, "N": 65536})
    sk = api.bm_secret_key_seeded(kp, 5)
    s, z = api.bm_secret_key_get(sk)
    want = orc.seeded_key_randomness(kp, 5, bsk_keys=0, with_ksk=False)
    assert np.array_equal(s, want["s"]) and np.array_equal(z, want["z"])
    with pytest.raises(api.BMError):
        api.bm_secret_key_seeded(P.KeyParams(**{**kp.__dict__, "N": 131072}), 5)

"""Pins of the oracle's seeded randomness (keys and ciphertexts drawn from a
seed; Algorithm 1 REQUIRE block and Section 2 (8)).

The generator is Philox4x32-10 (Salmon, Moraes, Dror and Shaw, "Parallel
random numbers: as easy as 1, 2, 3", SC'11).  It is pinned by the published
known-answer vectors of that generator (Random123 distribution,
philox4x32 with 10 rounds).  Each derived distribution is pinned
statistically against its own definition: uniform residues, uniform ternary
and binary values, and the discrete Gaussian exp(-k^2 / (2 sigma^2)) / S.
The seeded keys are then pinned end to end by bootstrapping every toy
message.
"""
import math

import numpy as np
import pytest

from paper_2310_12441_gb300 import params as P
from paper_2310_12441_gb300 import synth

# Published known-answer vectors of Philox4x32-10: (counter, key, output).
PHILOX_KAT = [
    ((0x00000000, 0x00000000, 0x00000000, 0x00000000), (0x00000000, 0x00000000),
     (0x6627e8d5, 0xe169c58d, 0xbc57ac4c, 0x9b00dbd8)),
    ((0xffffffff, 0xffffffff, 0xffffffff, 0xffffffff), (0xffffffff, 0xffffffff),
     (0x408f276d, 0x41c83b0e, 0xa20bc7c6, 0x6d5451fd)),
    ((0x243f6a88, 0x85a308d3, 0x13198a2e, 0x03707344), (0xa4093822, 0x299f31d0),
     (0xd16cfe09, 0x94fdcceb, 0x5001e420, 0x24126ea1)),
]


def _chi2_ok(counts, expected, dof_extra=0):
    """Pearson chi-square against `expected`; accept unless p < 1e-5."""
    from scipy.stats import chi2
    counts = np.asarray(counts, float)
    expected = np.asarray(expected, float)
    stat = float(((counts - expected) ** 2 / expected).sum())
    dof = len(counts) - 1 - dof_extra
    return chi2.sf(stat, dof) > 1e-5, stat


@pytest.mark.parametrize("ctr,key,out", PHILOX_KAT)
def test_philox_known_answer_vectors(orc, ctr, key, out):
    assert tuple(int(x) for x in orc.philox4x32_10(ctr, key)) == out


def test_stream_layout_and_word_order(orc):
    """Element i of (seed, kind, domain) is the Philox block at counter
    (i mod 2^32, i >> 32, domain, kind) under key (seed mod 2^32, seed >> 32);
    a uniform residue reads the block as w0 + w1 2^32 + w2 2^64 + w3 2^96."""
    seed, kind, domain = 0x0123456789ABCDEF, 5, 2048
    for i in (0, 1, 77, (3 << 32) + 9):
        w = [int(x) for x in orc.philox4x32_10((i & 0xffffffff, i >> 32, domain, kind),
                                               (seed & 0xffffffff, seed >> 32))]
        assert orc.draw_uniform(seed, kind, domain, i, 1 << 32) == w[0]
        assert orc.draw_uniform(seed, kind, domain, i, 1 << 63) == w[0] + (w[1] << 32) - ((w[1] >> 31) << 63)
        U = w[0] | (w[1] << 32) | (w[2] << 64) | (w[3] << 96)
        Q = P.KEYS_N2048.Q
        assert orc.draw_uniform(seed, kind, domain, i, Q) == U % Q


@pytest.mark.parametrize("modulus", [P.KEYS_N2048.Q, 8192])
def test_uniform_residues(orc, modulus):
    r = orc.seeded_enc_randomness(1, modulus, 3.2, 200000, 11)["mask"][:, 0].astype(np.float64)
    assert r.max() < modulus
    bins = 64 if modulus > 8192 else 128
    counts = np.bincount((r * bins / modulus).astype(int), minlength=bins)
    ok, stat = _chi2_ok(counts, np.full(bins, len(r) / bins))
    assert ok, stat


def test_ternary_and_binary_frequencies(orc):
    kp_t = P.KEYS_N1024
    kp_b = P.KEYS_TOY
    tern, binr = [], []
    for seed in range(40):
        rnd = orc.seeded_key_randomness(kp_t, seed, bsk_keys=0, with_ksk=False)
        tern.append(rnd["s"])
        tern.append(rnd["z"])
        binr.append(orc.seeded_key_randomness(kp_b, seed, bsk_keys=0, with_ksk=False)["s"])
    tern = np.concatenate(tern).astype(int)
    binr = np.concatenate(binr).astype(int)
    assert set(np.unique(tern)) == {-1, 0, 1} and set(np.unique(binr)) == {0, 1}
    ok, stat = _chi2_ok(np.bincount(tern + 1), np.full(3, len(tern) / 3))
    assert ok, stat
    ok, stat = _chi2_ok(np.bincount(binr), np.full(2, len(binr) / 2))
    assert ok, stat


def test_cdt_is_monotone_and_symmetric(orc):
    T = orc.cdt(3.2).astype(object)
    assert all(T[j] <= T[j + 1] for j in range(len(T) - 1))
    # F_j + F_{2K-1-j} = 1 - rho(K-... ) up to rounding: the table is symmetric
    K = orc.ERR_CUT
    for j in range(K):
        s = T[j] + T[2 * K - 1 - j]
        assert abs(s - (1 << 64)) <= (1 << 14) or T[2 * K - 1 - j] == (1 << 64) - 1


@pytest.mark.parametrize("sigma", [3.2, 1.0])
def test_errors_follow_the_discrete_gaussian(orc, sigma):
    """Sampled errors against rho(k) = exp(-k^2/(2 sigma^2)) / S, computed here
    in Python directly from the definition (not through the table)."""
    cnt = 400000
    e = orc.seeded_enc_randomness(1, 1 << 20, sigma, cnt, 123)["err"].astype(int)
    K = orc.ERR_CUT
    rho = np.array([math.exp(-k * k / (2 * sigma * sigma)) for k in range(-K, K + 1)])
    pmf = rho / rho.sum()
    lim = int(math.ceil(4 * sigma))
    ks = np.arange(-lim, lim + 1)
    counts = [int((e == k).sum()) for k in ks] + [int((np.abs(e) > lim).sum())]
    expected = [cnt * pmf[k + K] for k in ks] + [cnt * (1 - pmf[K - lim:K + lim + 1].sum())]
    keep = np.array(expected) > 5
    counts = np.array(counts)[keep]
    expected = np.array(expected)[keep]
    expected *= counts.sum() / expected.sum()
    ok, stat = _chi2_ok(counts, expected)
    assert ok, stat
    assert abs(e.mean()) < 5 * sigma / math.sqrt(cnt)
    var = float((pmf * np.arange(-K, K + 1) ** 2).sum())
    assert abs(e.var() / var - 1) < 0.02


def test_key_streams_are_prefix_stable_and_separated(orc):
    """Counter-based streams: asking for fewer bootstrapping keys returns a
    prefix of the full draw; the two key sets of one seed and one n share s
    (so the N = 1024 and N = 4096 layouts bootstrap the same ciphertexts) but
    not z."""
    a = orc.seeded_key_randomness(P.KEYS_TOY, 5, bsk_keys=3, with_ksk=False)
    b = orc.seeded_key_randomness(P.KEYS_TOY, 5, bsk_keys=6, with_ksk=False)
    assert np.array_equal(a["bsk_mask"], b["bsk_mask"][:3])
    assert np.array_equal(a["bsk_err"], b["bsk_err"][:3])
    c = orc.seeded_key_randomness(P.KEYS_N1024, 5, bsk_keys=0, with_ksk=False)
    d = orc.seeded_key_randomness(P.KEYS_N4096, 5, bsk_keys=0, with_ksk=False)
    assert np.array_equal(c["s"], d["s"])
    assert not np.array_equal(c["z"], d["z"][:1024])
    e = orc.seeded_key_randomness(P.KEYS_TOY, 6, bsk_keys=3, with_ksk=False)
    assert not np.array_equal(a["bsk_mask"], e["bsk_mask"])


def test_seeded_encryption_phase(orc):
    kp = P.KEYS_N1024
    s = orc.seeded_key_randomness(kp, 7, bsk_keys=0, with_ksk=False)["s"]
    qp, t = 8192, 1024
    msg = synth.messages(t, 300, 9)
    ct = orc.encrypt_seeded(kp.n, qp, t, s, msg, 3.2, 77)
    err = orc.seeded_enc_randomness(kp.n, qp, 3.2, 300, 77)["err"].astype(int)
    assert np.abs(err).max() <= 41
    for i in range(300):
        assert orc.lwe_phase(kp.n, qp, s, ct[i]) == (int(msg[i]) * (qp // t) + err[i]) % qp


def test_seeded_toy_keys_bootstrap_every_message(orc):
    """Keys and ciphertexts of the toy set drawn from seeds: every message of
    Z_32 bootstraps to f(msg) (Definition 1)."""
    kp, m, t = P.KEYS_TOY, 2, 32
    rnd = orc.seeded_key_randomness(kp, 1001)
    bsk, ksk = orc.keygen_bsk(kp, rnd), orc.keygen_ksk(kp, rnd)
    qp = 2 * kp.N * m
    msg = np.arange(t, dtype=np.uint32)
    ct = orc.encrypt_seeded(kp.n, qp, t, rnd["s"], msg, kp.sigma, 4001)
    luts, _ = synth.luts(t, t, 2001)
    out = orc.bootstrap(kp, m, t, bsk, ksk, ct, luts)
    dec_in = orc.decrypt(kp.n, qp, t, rnd["s"], ct)
    assert np.array_equal(orc.decrypt(kp.n, kp.Q, t, rnd["s"], out), luts[np.arange(t), dec_in])

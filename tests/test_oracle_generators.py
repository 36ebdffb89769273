"""Pins of the oracle's general transitive generators (Section 3).

A generator is P(1) = A = (x^{u_i} delta_{tau(i), j}) with tau(i) = i - 1
mod m (the form (BP1:form) of Theorem 1).  The pins use what the paper fixes:
  * Lemma 3: the closed form of A^c equals c single applications of A;
  * Example 1: u = (1, 0, ..., 0) gives the P(c) of Eq. (ex1:BPc) and the
    test vector of Eq. (equ:test-use);
  * Lemma 4: ord(A) = m ord(x^{sum u}), with ord(x^s) = 2N / gcd(s, 2N);
  * Theorem 1: A acts transitively on the monic monomial indicator vectors
    (one orbit of size 2Nm) iff ord(x^{sum u}) = 2N, i.e. sum u odd;
  * Lemma 6: P(Nm) = -I for a transitive generator;
  * Lemma 7 / Example 2: the test vector of Eq. (equ:test-gene) has the
    look-up property for every phase;
  * Definition 1: bootstrapping with such a generator decrypts to f(msg).
"""
import math

import numpy as np
import pytest

from paper_2310_12441_gb300 import params as P
from paper_2310_12441_gb300 import synth

Q = 1073738753


def _gens(rng, N, m, odd=True, count=3):
    out = []
    while len(out) < count:
        u = rng.integers(0, 2 * N, m).astype(np.uint32)
        if (int(u.sum()) % 2 == 1) == odd:
            out.append(u)
    return out


def _random_vec(rng, N, m):
    return rng.integers(0, Q, (m, 2, N), dtype=np.uint64)


@pytest.mark.parametrize("N,m", [(8, 1), (8, 3), (4, 4), (16, 2)])
def test_closed_form_equals_repeated_application(orc, N, m):
    rng = np.random.default_rng(N * 10 + m)
    for u in _gens(rng, N, m, odd=True, count=2) + _gens(rng, N, m, odd=False, count=1):
        v = _random_vec(rng, N, m)
        step = v.copy()
        for c in range(2 * N * m + 3):
            assert np.array_equal(orc.mmpm_apply_gen(N, m, Q, u, c, v), step), (list(u), c)
            step = orc.mmpm_step_gen(N, m, Q, u, step)


@pytest.mark.parametrize("N,m", [(8, 1), (8, 3), (16, 4)])
def test_example1_generator_reduces_to_eq_ex1_bpc(orc, N, m):
    u = np.zeros(m, np.uint32)
    u[0] = 1
    rng = np.random.default_rng(m)
    v = _random_vec(rng, N, m)
    for c in range(2 * N * m):
        assert np.array_equal(orc.mmpm_apply_gen(N, m, Q, u, c, v), orc.mmpm_apply(N, m, Q, c, v))
    t = 2 * m
    lut = synth.negacyclic_lut(rng, t)
    assert np.array_equal(orc.test_vector_gen(N, m, t, Q, u, lut), orc.test_vector(N, m, t, Q, lut))


@pytest.mark.parametrize("N,m", [(8, 2), (8, 3), (4, 6)])
def test_order_is_m_times_order_of_x_to_the_sum(orc, N, m):
    """Lemma 4, found by searching the smallest l with A^l v = v for a
    generic v (distinct random coefficients, so A^l v = v iff A^l = I)."""
    rng = np.random.default_rng(7 * N + m)
    v = _random_vec(rng, N, m)
    for u in _gens(rng, N, m, True, 2) + _gens(rng, N, m, False, 3):
        s = int(u.sum())
        want = m * (2 * N // math.gcd(s, 2 * N))
        cur = orc.mmpm_step_gen(N, m, Q, u, v)
        l = 1
        while not np.array_equal(cur, v):
            cur = orc.mmpm_step_gen(N, m, Q, u, cur)
            l += 1
        assert l == want, (list(u), l, want)


@pytest.mark.parametrize("N,m", [(8, 2), (8, 3), (4, 5)])
def test_transitive_iff_sum_is_odd(orc, N, m):
    """Theorem 1: the orbit of e_0 under P(Z_{2Nm}) covers all 2Nm monic
    monomial indicator vectors x^i e_j iff sum u is odd."""
    rng = np.random.default_rng(3 * N + m)
    e0 = np.zeros((m, 2, N), np.uint64)
    e0[0, 1, 0] = 1
    for odd in (True, False):
        for u in _gens(rng, N, m, odd, 2):
            seen = set()
            for c in range(2 * N * m):
                r = orc.mmpm_apply_gen(N, m, Q, u, c, e0)
                nz = np.argwhere(r[:, 1, :] != 0)
                assert len(nz) == 1 and not r[:, 0, :].any()
                row, pos = (int(x) for x in nz[0])
                sign = 1 if int(r[row, 1, pos]) == 1 else -1
                assert int(r[row, 1, pos]) in (1, Q - 1)
                seen.add((row, pos if sign == 1 else pos + N))
            assert (len(seen) == 2 * N * m) == odd, (list(u), len(seen))
            if odd:
                v = _random_vec(rng, N, m)
                neg = orc.mmpm_apply_gen(N, m, Q, u, N * m, v)
                assert np.array_equal(neg, (Q - v) % Q)          # Lemma 6: P(Nm) = -I


@pytest.mark.parametrize("N,m,t", [(8, 2, 8), (8, 3, 12), (16, 4, 32)])
def test_lookup_property_of_the_general_test_vector(orc, N, m, t):
    """Lemma 7 with the test vector of Eq. (equ:test-gene): for every phase
    msg Delta + e with 2|e| <= Delta, the constant term of row 0 of
    P(phase)(0, v_0) decodes to f(msg)."""
    qp = 2 * N * m
    delta = qp // t
    rng = np.random.default_rng(N + m + t)
    dq = Q // t
    for u in _gens(rng, N, m, True, 2):
        lut = synth.negacyclic_lut(rng, t)
        v = orc.test_vector_gen(N, m, t, Q, u, lut)
        acc = np.zeros((m, 2, N), np.uint64)
        acc[:, 1, :] = v
        for msg in range(t):
            for e in range(-(delta // 2), (delta + 1) // 2):
                c = (msg * delta + e) % qp
                r = orc.mmpm_apply_gen(N, m, Q, u, c, acc)
                got = int(r[0, 1, 0])
                assert got in (int(lut[msg]) * dq % Q, (Q - int(lut[(msg + t // 2) % t]) * dq % Q) % Q)
                assert (got * t + Q // 2) // Q % t == lut[msg]


def test_general_generators_bootstrap_every_message(orc):
    """Toy keys, a different transitive generator per ciphertext: every
    message of Z_32 bootstraps to f(msg), and the Example 1 generator gives
    the bits of the standard oracle path."""
    kp, m, t = P.KEYS_TOY, 2, 32
    rnd = orc.seeded_key_randomness(kp, 1001)
    bsk, ksk = orc.keygen_bsk(kp, rnd), orc.keygen_ksk(kp, rnd)
    qp = 2 * kp.N * m
    msg = np.arange(t, dtype=np.uint32)
    ct = orc.encrypt_seeded(kp.n, qp, t, rnd["s"], msg, kp.sigma, 4002)
    luts, _ = synth.luts(t, t, 2002)
    rng = np.random.default_rng(5)
    u = np.stack(_gens(rng, kp.N, m, True, t))
    out = orc.bootstrap_gen(kp, m, t, u, bsk, ksk, ct, luts)
    dec_in = orc.decrypt(kp.n, qp, t, rnd["s"], ct)
    assert np.array_equal(orc.decrypt(kp.n, kp.Q, t, rnd["s"], out), luts[np.arange(t), dec_in])
    std = np.tile(np.array([1, 0], np.uint32), (2, 1))
    assert np.array_equal(orc.bootstrap_gen(kp, m, t, std, bsk, ksk, ct[:2], luts[:2]),
                          orc.bootstrap(kp, m, t, bsk, ksk, ct[:2], luts[:2]))

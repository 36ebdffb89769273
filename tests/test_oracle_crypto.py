"""Pins of the oracle's ciphertext-level functions: exact error identities,
decryption of fresh and bootstrapped ciphertexts, key-switching gadget.

The identities come from the paper: the phase of an external product
(Eq. (error:grow)), of sample extraction (Eq. (equ-sam-extr)) and of key
switching (Eq. (equ-key-swi)).  The keys' errors are known to the test (they
are inputs), so each identity is checked exactly, not statistically.
"""
import numpy as np
import pytest

from paper_2310_12441_gb300 import params as P
from paper_2310_12441_gb300 import synth


def _negacyclic_signed(a, b, N):
    """Exact integer product in Z[x]/(x^N+1) via numpy convolution."""
    full = np.convolve(np.array(a, dtype=object), np.array(b, dtype=object))
    out = [0] * N
    for k, c in enumerate(full):
        if k < N:
            out[k] += c
        else:
            out[k - N] -= c
    return out


def _centered(x, Q):
    x = int(x) % Q
    return x - Q if x > Q // 2 else x


SMALL = P.KeyParams(n=8, N=32, Q=1073738753, log2_B=6, l_B=5, log2_Bks=4, l_ks=7)


@pytest.fixture(scope="module")
def small_keys(orc):
    rnd = synth.key_randomness(SMALL, seed=99)
    return rnd, orc.keygen_bsk(SMALL, rnd), orc.keygen_ksk(SMALL, rnd)


def test_encrypt_decrypt_roundtrip(orc):
    kp = P.KEYS_N1024
    s = synth.lwe_secret(kp, 5)
    for m, t in [(4, 1024), (1, 256), (2, 512)]:
        qp = 2 * kp.N * m
        msg = synth.messages(t, 500, 7)
        enc = synth.encryption_randomness(kp.n, qp, kp.sigma, 500, 8)
        ct = orc.encrypt(kp.n, qp, t, s, msg, enc["mask"], enc["err"])
        delta = qp // t
        for i in range(500):
            ph = orc.lwe_phase(kp.n, qp, s, ct[i])
            assert ph == (int(msg[i]) * delta + int(enc["err"][i])) % qp
        ok = np.abs(enc["err"].astype(int)) * 2 < delta
        dec = orc.decrypt(kp.n, qp, t, s, ct)
        assert np.array_equal(dec[ok], msg[ok])


def test_bsk_rows_have_the_rgsw_phase(orc, small_keys):
    """Row j < l_B of RGSW_z(mu) has phase e_j - mu B^j z, row l_B + j has
    phase e_j + mu B^j (the convention under which g^{-1}(a,b) C encrypts
    mu * phase(a, b))."""
    rnd, bsk, _ = small_keys
    kp, N, Q = SMALL, SMALL.N, SMALL.Q
    z = rnd["z"].astype(int)
    for k in range(kp.n):
        for sgn in range(2):
            mu = max(int(rnd["s"][k]), 0) if sgn == 0 else max(-int(rnd["s"][k]), 0)
            for row in range(2 * kp.l_B):
                ph = orc.rlwe_phase(N, Q, rnd["z"], bsk[k, sgn, row, 0], bsk[k, sgn, row, 1])
                e = rnd["bsk_err"][k, sgn, row].astype(int)
                j = row % kp.l_B
                g = 1 << (kp.log2_B * j)
                expect = [int(x) for x in e]
                if mu and row < kp.l_B:
                    expect = [expect[c] - g * z[c] for c in range(N)]
                if mu and row >= kp.l_B:
                    expect[0] += g
                assert [int(x) for x in ph] == [x % Q for x in expect]


@pytest.mark.parametrize("mu_index", [0, 1])
def test_external_product_error_identity(orc, small_keys, mu_index):
    """Eq. (error:grow): phase(g^{-1}(v) C) = mu phase(v) + g^{-1}(v) e_C exactly."""
    rnd, bsk, _ = small_keys
    kp, N, Q = SMALL, SMALL.N, SMALL.Q
    # find a key whose plaintext is mu_index
    k, sgn = next((k, sg) for k in range(kp.n) for sg in range(2)
                  if (max(int(rnd["s"][k]), 0) if sg == 0 else max(-int(rnd["s"][k]), 0)) == mu_index)
    C = bsk[k, sgn]
    rng = np.random.default_rng(1)
    a = rng.integers(0, Q, N, dtype=np.uint64)
    b = rng.integers(0, Q, N, dtype=np.uint64)
    oa, ob = orc.external_product(kp, a, b, C)
    ph_out = orc.rlwe_phase(N, Q, rnd["z"], oa, ob)
    ph_in = orc.rlwe_phase(N, Q, rnd["z"], a, b)
    err = [0] * N
    for comp, src in enumerate((a, b)):
        for j in range(kp.l_B):
            dig = [(int(x) >> (kp.log2_B * j)) & (kp.B - 1) for x in src]
            e = rnd["bsk_err"][k, sgn, comp * kp.l_B + j].astype(int)
            prod = _negacyclic_signed(dig, e, N)
            err = [err[c] + prod[c] for c in range(N)]
    expect = [(mu_index * int(ph_in[c]) + err[c]) % Q for c in range(N)]
    assert [int(x) for x in ph_out] == expect


def test_sample_extract_phase(orc):
    """Eq. (equ-sam-extr): the LWE phase of the extracted sample under the
    coefficient vector of z equals the constant term of the RLWE phase."""
    N, Q = 64, 18014398509404161
    rng = np.random.default_rng(2)
    z = rng.integers(-1, 2, N, dtype=np.int8)
    for _ in range(5):
        a = rng.integers(0, Q, N, dtype=np.uint64)
        b = rng.integers(0, Q, N, dtype=np.uint64)
        lwe = orc.sample_extract(N, Q, a, b)
        assert orc.lwe_phase(N, Q, z, lwe) == int(orc.rlwe_phase(N, Q, z, a, b)[0])


def test_ks_gadget_and_digits(orc):
    """Approximate gadget: sum_j d_j g_j is within Q/(2P) + l_ks (B_ks-1)/2 of
    a, and every digit lies in [0, B_ks)."""
    for kp in (P.KEYS_TOY, P.KEYS_N1024, P.KEYS_N2048):
        g = [orc.ks_gadget(kp, j) for j in range(kp.l_ks)]
        Pw = 1 << (kp.log2_Bks * kp.l_ks)
        bound = kp.Q / (2 * Pw) + kp.l_ks * (kp.Bks - 1) / 2 + 1
        rng = np.random.default_rng(4)
        for a in list(rng.integers(0, kp.Q, 300, dtype=np.uint64)) + [0, kp.Q - 1, kp.Q // 2]:
            d = orc.ks_digits(kp, int(a))
            assert all(int(x) < kp.Bks for x in d)
            approx = sum(int(d[j]) * g[j] for j in range(kp.l_ks))
            diff = _centered(approx - int(a), kp.Q)
            assert abs(diff) <= bound


def test_ksk_rows_have_the_lwe_phase(orc, small_keys):
    rnd, _, ksk = small_keys
    kp, Q = SMALL, SMALL.Q
    for i in range(0, kp.N, 7):
        for j in range(kp.l_ks):
            g = orc.ks_gadget(kp, j)
            for v in range(1, kp.Bks):
                ph = orc.lwe_phase(kp.n, Q, rnd["s"], ksk[i, j, v - 1])
                assert ph == (v * int(rnd["z"][i]) * g + int(rnd["ksk_err"][i, j, v - 1])) % Q


def test_key_switch_error_identity(orc, small_keys):
    """Eq. (equ-key-swi): phase_s(out) = b - sum_ij (d_ij z_i g_j + e_ij), hence
    within sum_i |z_i| (Q/2P + l_ks (B_ks-1)/2) + N l_ks max|e| of phase_z(in)."""
    rnd, _, ksk = small_keys
    kp, N, Q = SMALL, SMALL.N, SMALL.Q
    rng = np.random.default_rng(9)
    g = [orc.ks_gadget(kp, j) for j in range(kp.l_ks)]
    for _ in range(5):
        lwe = rng.integers(0, Q, N + 1, dtype=np.uint64)
        out = orc.key_switch(kp, lwe, ksk)
        ph_out = orc.lwe_phase(kp.n, Q, rnd["s"], out)
        exact = int(lwe[N])
        for i in range(N):
            d = orc.ks_digits(kp, int(lwe[i]))
            for j in range(kp.l_ks):
                if d[j]:
                    exact -= int(d[j]) * int(rnd["z"][i]) * g[j] + int(rnd["ksk_err"][i, j, d[j] - 1])
        assert ph_out == exact % Q
        ph_in = orc.lwe_phase(N, Q, rnd["z"], lwe)
        Pw = 1 << (kp.log2_Bks * kp.l_ks)
        bound = (np.abs(rnd["z"]).sum() * (Q / (2 * Pw) + kp.l_ks * (kp.Bks - 1) / 2 + 1)
                 + N * kp.l_ks * 41)
        assert abs(_centered(ph_out - ph_in, Q)) <= bound


def test_cmux_selects_rotation(orc, small_keys):
    """Eq. (cmux:BP): for s_k in {1, 0, -1} the CMux output decrypts (row-wise
    RLWE phase) to P(-a s_k) applied to the input's phase, up to the key error
    term, whose size is at most 2 * 2 l_B N (B-1) max|e|."""
    rnd, bsk, _ = small_keys
    kp, N, Q = SMALL, SMALL.N, SMALL.Q
    m = 3
    rng = np.random.default_rng(12)
    acc = rng.integers(0, Q, (m, 2, N), dtype=np.uint64)
    bound = 2 * 2 * kp.l_B * N * (kp.B - 1) * 41
    seen = set()
    for k in range(kp.n):
        sk = int(rnd["s"][k])
        seen.add(sk)
        ak = int(rng.integers(0, 2 * N * m))
        out = orc.cmux(kp, m, ak, bsk[k, 0], bsk[k, 1], acc)
        ph_in = np.stack([orc.rlwe_phase(N, Q, rnd["z"], acc[i, 0], acc[i, 1]) for i in range(m)])
        ph_out = np.stack([orc.rlwe_phase(N, Q, rnd["z"], out[i, 0], out[i, 1]) for i in range(m)])
        ph_vec = np.zeros((m, 2, N), np.uint64)
        ph_vec[:, 1] = ph_in
        qp = 2 * N * m
        want = orc.mmpm_apply(N, m, Q, (-ak * sk) % qp, ph_vec)[:, 1]
        diff = [abs(_centered(int(x) - int(y), Q)) for x, y in zip(ph_out.ravel(), want.ravel())]
        assert max(diff) <= bound
    assert seen == {-1, 0, 1} or SMALL.secret == "binary"


def test_toy_bootstrap_all_messages(orc):
    """Definition 1 and Algorithm 1's ENSURE at the toy size: every message
    of Z_32 bootstraps to f(msg) under a random negacyclic table, and the
    output phase error is far inside Delta_Q / 2."""
    w = P.TOY
    kp, m, t = w.keys, w.shape.m, w.shape.t
    rnd = synth.key_randomness(kp, 1001)
    bsk = orc.keygen_bsk(kp, rnd)
    ksk = orc.keygen_ksk(kp, rnd)
    qp = 2 * kp.N * m
    msg = np.arange(t, dtype=np.uint32)
    enc = synth.encryption_randomness(kp.n, qp, kp.sigma, t, 4001)
    ct = orc.encrypt(kp.n, qp, t, rnd["s"], msg, enc["mask"], enc["err"])
    lut_tab, _ = synth.luts(t, 1, 2001)
    lut = np.repeat(lut_tab, t, axis=0)
    out = orc.bootstrap(kp, m, t, bsk, ksk, ct, lut)
    dec_in = orc.decrypt(kp.n, qp, t, rnd["s"], ct)
    dec_out = orc.decrypt(kp.n, kp.Q, t, rnd["s"], out)
    assert np.array_equal(dec_out, lut_tab[0][dec_in])
    dq = kp.Q // t
    for i in range(t):
        ph = orc.lwe_phase(kp.n, kp.Q, rnd["s"], out[i])
        e = _centered(ph - int(lut_tab[0][dec_in[i]]) * dq, kp.Q)
        assert abs(e) < dq // 64


def test_prefix_blind_rotation_skips_zero_steps(orc):
    """A ciphertext whose masks vanish after step K needs only the first K
    keys: steps with a_k = 0 apply P(0) = I and leave ACC unchanged."""
    kp = P.KEYS_TOY
    m, t = 2, 32
    rnd = synth.key_randomness(kp, 1001)
    bsk = orc.keygen_bsk(kp, rnd)
    qp = 2 * kp.N * m
    enc = synth.encryption_randomness(kp.n, qp, kp.sigma, 1, 4001, prefix=5)
    ct = orc.encrypt(kp.n, qp, t, rnd["s"], np.array([3], np.uint32), enc["mask"], enc["err"])
    lut = synth.luts(t, 1, 2001)[0][0]
    full = orc.blind_rotate(kp, m, t, bsk, ct[0], lut)
    part = orc.blind_rotate(kp, m, t, bsk[:5], ct[0], lut)
    assert np.array_equal(full, part)
    with pytest.raises(ValueError):
        orc.blind_rotate(kp, m, t, bsk[:4], ct[0], lut)


def test_mod_switch_identity_and_phase_bound(orc):
    """Section 2 (9): switching q -> q' rounds each word, so the phase moves
    to phase q'/q up to (|s|_1 + 1)/2 (one rounding of at most 1/2 per term)."""
    rng = np.random.default_rng(21)
    n, q = 64, 1 << 14
    s = rng.integers(-1, 2, n, dtype=np.int8)
    ct = rng.integers(0, q, (50, n + 1), dtype=np.uint64)
    assert np.array_equal(orc.mod_switch(ct, q, q), ct)
    bound = (np.abs(s.astype(int)).sum() + 1) / 2
    for qp in (1024, 4096, 1 << 13):
        sw = orc.mod_switch(ct, q, qp)
        assert int(sw.max()) < qp
        for i in range(len(ct)):
            ph = orc.lwe_phase(n, q, s, ct[i])
            ph2 = orc.lwe_phase(n, qp, s, sw[i])
            d = (ph2 - ph * qp / q) % qp
            d = d - qp if d > qp / 2 else d
            assert abs(d) <= bound + 1e-9


def test_mod_switch_keeps_messages(orc):
    kp = P.KEYS_TOY
    s = synth.lwe_secret(kp, 7)
    q, t, qp = 1 << 14, 8, 1024
    msg = synth.messages(t, 200, 9)
    enc = synth.encryption_randomness(kp.n, q, kp.sigma, 200, 10)
    ct = orc.encrypt(kp.n, q, t, s, msg, enc["mask"], enc["err"])
    assert np.array_equal(orc.decrypt(kp.n, qp, t, s, orc.mod_switch(ct, q, qp)), msg)


def test_two_round_tables(orc):
    """mp is negacyclic with sign(x) t = mp(x) + t/2 (Eqs. (rel:mp), (rel:sign));
    F is negacyclic over Z_{2t} and equals f(y mod t) on y in [-t/2, t/2)."""
    rng = np.random.default_rng(8)
    for t in (4, 8, 16, 32):
        T = 2 * t
        f = rng.integers(0, t, t).astype(np.uint32)
        mp, F = orc.two_round_tables(t, f)
        for x in range(T):
            xs = x if x < t else x - T                      # representative in [-t, t)
            sign = 0 if -t // 2 <= xs < t // 2 else 1
            assert (int(mp[x]) + t // 2) % T == sign * t
            assert int(mp[(x + t) % T]) == (T - int(mp[x])) % T
            assert int(F[(x + t) % T]) == (T - int(F[x])) % T
        for y in range(-t // 2, t // 2):
            assert int(F[y % T]) == int(f[y % t])


@pytest.mark.parametrize("fname", ["identity", "random", "constant"])
def test_two_round_bootstrap_any_function(orc, fname):
    """Section 4 (last part): with the two rounds every x in Z_{2t} (m = x mod t,
    any top bit) bootstraps to f(m) for f that need not be negacyclic."""
    kp = P.KEYS_TOY
    rnd = synth.key_randomness(kp, 1001)
    bsk = orc.keygen_bsk(kp, rnd)
    ksk = orc.keygen_ksk(kp, rnd)
    q, t, m = 1 << 14, 4, 2
    T = 2 * t
    f = {"identity": np.arange(t), "random": np.array([2, 3, 0, 3]),
         "constant": np.full(t, 1)}[fname].astype(np.uint32)
    x = np.arange(T, dtype=np.uint32)
    enc = synth.encryption_randomness(kp.n, q, kp.sigma, T, 78)
    ct = orc.encrypt(kp.n, q, T, rnd["s"], x, enc["mask"], enc["err"])
    tables = np.stack([f] * T) + np.arange(T)[:, None].astype(np.uint32) * 0
    out = orc.bootstrap_arbitrary(kp, m, t, q, bsk, ksk, ct, tables)
    assert np.array_equal(orc.decrypt(kp.n, q, T, rnd["s"], out), f[x % t])

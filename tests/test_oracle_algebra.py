"""Pins of the oracle's algebra against what the paper and the mathematics fix.

Nothing here re-types the oracle's formulas: each check goes through another
route (explicit matrices built from P(1), evaluation at the roots of x^N+1,
numpy's convolution, the paper's own closed forms and stated properties).
"""
import numpy as np
import pytest



def _negacyclic_np(a, b, Q):
    """Product in Z_Q[x]/(x^N+1) via numpy's full convolution, then folding."""
    N = len(a)
    full = np.convolve(np.array(a, dtype=object), np.array(b, dtype=object))
    out = [0] * N
    for k, c in enumerate(full):
        if k < N:
            out[k] += c
        else:
            out[k - N] -= c
    return np.array([x % Q for x in out], dtype=np.uint64)


def _root_2N(N, Q):
    """A primitive 2N-th root of unity mod Q (psi^N = -1)."""
    for g in range(2, Q):
        psi = pow(g, (Q - 1) // (2 * N), Q)
        if pow(psi, N, Q) == Q - 1:
            return psi
    raise AssertionError


@pytest.mark.parametrize("N", [8, 16, 32])
def test_poly_mul_evaluation_homomorphism(orc, N):
    """x^N + 1 splits over Z_Q into (x - psi^(2i+1)); a product in the ring is
    pinned by its values at these N points (Chinese remainder theorem)."""
    Q = 1073738753          # the toy modulus; 1 mod 512
    rng = np.random.default_rng(N)
    a = rng.integers(0, Q, N, dtype=np.uint64)
    b = rng.integers(0, Q, N, dtype=np.uint64)
    c = orc.poly_mul(N, Q, a, b)
    psi = _root_2N(N, Q)
    for i in range(N):
        x = pow(psi, 2 * i + 1, Q)
        ev = lambda p: sum(int(p[k]) * pow(x, k, Q) for k in range(N)) % Q
        assert ev(c) == ev(a) * ev(b) % Q


def test_poly_mul_matches_numpy_convolution(orc):
    rng = np.random.default_rng(1)
    for N in (16, 64):
        Q = 18014398509404161
        a = rng.integers(0, Q, N, dtype=np.uint64)
        b = rng.integers(0, Q, N, dtype=np.uint64)
        assert np.array_equal(orc.poly_mul(N, Q, a, b), _negacyclic_np(a, b, Q))


def test_poly_mul_x_to_the_N_is_minus_one(orc):
    N, Q = 32, 1073738753
    x1 = np.zeros(N, np.uint64); x1[1] = 1
    xN1 = np.zeros(N, np.uint64); xN1[N - 1] = 1
    r = orc.poly_mul(N, Q, x1, xN1)
    expect = np.zeros(N, np.uint64); expect[0] = Q - 1
    assert np.array_equal(r, expect)


# --- monic monomial permutation matrices -------------------------------------

class Mono:
    """A signed monomial +-x^e in Q[x]/(x^N+1), or zero."""

    def __init__(self, N, e=None, sign=1):
        self.N, self.e, self.sign = N, e, sign

    def __mul__(self, o):
        if self.e is None or o.e is None:
            return Mono(self.N)
        e, s = self.e + o.e, self.sign * o.sign
        while e >= self.N:
            e -= self.N
            s = -s
        return Mono(self.N, e, s)

    def __eq__(self, o):
        return (self.e is None and o.e is None) or (self.e == o.e and self.sign == o.sign)


def _P1(N, m):
    """P(1) of Eq. (ex:BP): x in the top-right corner, I_(m-1) below-left."""
    M = [[Mono(N) for _ in range(m)] for _ in range(m)]
    M[0][m - 1] = Mono(N, 1)
    for i in range(1, m):
        M[i][i - 1] = Mono(N, 0)
    return M


def _matmul(A, B, N):
    m = len(A)
    C = [[Mono(N) for _ in range(m)] for _ in range(m)]
    for i in range(m):
        for j in range(m):
            terms = [A[i][k] * B[k][j] for k in range(m)]
            nz = [t for t in terms if t.e is not None]
            assert len(nz) <= 1          # monomial permutation matrices stay so
            if nz:
                C[i][j] = nz[0]
    return C


def _identity(N, m):
    return [[Mono(N, 0) if i == j else Mono(N) for j in range(m)] for i in range(m)]


def _apply_explicit(M, vec, N, Q):
    """Matrix-vector product of a monomial matrix with an RLWE vector."""
    m = len(M)
    out = np.zeros_like(vec)
    for i in range(m):
        for j in range(m):
            t = M[i][j]
            if t.e is None:
                continue
            for comp in range(2):
                p = vec[j, comp]
                mono = np.zeros(N, np.uint64)
                mono[t.e] = 1 if t.sign > 0 else Q - 1
                out[i, comp] = _negacyclic_np(mono, p, Q)
    return out


@pytest.mark.parametrize("N,m", [(4, 1), (4, 3), (8, 2), (4, 4)])
def test_mmpm_action_equals_powers_of_P1(orc, N, m):
    """The closed-form action of P(c) (Eq. (ex1:BPc)) equals P(1)^c computed
    by explicit matrix products of (ex:BP), for every c in Z_{2Nm}."""
    Q = 7681
    rng = np.random.default_rng(N * 10 + m)
    vec = rng.integers(0, Q, (m, 2, N), dtype=np.uint64)
    P1 = _P1(N, m)
    Pc = _identity(N, m)
    for c in range(2 * N * m):
        assert np.array_equal(orc.mmpm_apply(N, m, Q, c, vec), _apply_explicit(Pc, vec, N, Q)), c
        Pc = _matmul(Pc, P1, N)
    # ord P(1) = 2Nm (Example 1, Lemma 4): P(1)^(2Nm) = I
    assert all(Pc[i][j] == _identity(N, m)[i][j] for i in range(m) for j in range(m))


@pytest.mark.parametrize("N,m", [(8, 3), (16, 4), (8, 1)])
def test_mmpm_group_law_order_and_special_elements(orc, N, m):
    Q = 7681
    qp = 2 * N * m
    rng = np.random.default_rng(7)
    vec = rng.integers(0, Q, (m, 2, N), dtype=np.uint64)
    # homomorphism P(u)P(v) = P(u+v mod 2Nm)
    for u, v in [(1, 2), (qp - 1, 1), (N * m, N * m), (5, qp - 3), (m, 3 * m + 1)]:
        left = orc.mmpm_apply(N, m, Q, u, orc.mmpm_apply(N, m, Q, v, vec))
        assert np.array_equal(left, orc.mmpm_apply(N, m, Q, (u + v) % qp, vec))
    # P(m) = x I (Example 1)
    xI = np.stack([np.stack([_negacyclic_np(np.eye(1, N, 1, dtype=np.uint64)[0], vec[i, c], Q)
                             for c in range(2)]) for i in range(m)])
    assert np.array_equal(orc.mmpm_apply(N, m, Q, m, vec), xI)
    # P(Nm) = -I (Lemma 6)
    assert np.array_equal(orc.mmpm_apply(N, m, Q, N * m, vec), (Q - vec) % Q)
    # no smaller power than 2Nm is the identity on a generic vector (order 2Nm)
    e0 = np.zeros((m, 2, N), np.uint64); e0[0, 1, 0] = 1
    seen = set()
    for c in range(qp):
        img = orc.mmpm_apply(N, m, Q, c, e0)
        seen.add(img.tobytes())
    # Theorem 1: P(1) is transitive on MMIV_m = {x^i e_j}: one orbit of 2Nm elements
    assert len(seen) == qp


# --- test vector and the look-up property ---------------------------------------

def _random_negacyclic(rng, t):
    lo = rng.integers(0, t, t // 2)
    return np.concatenate([lo, (t - lo) % t]).astype(np.uint32)


@pytest.mark.parametrize("N,m,t", [(16, 2, 8), (8, 4, 16), (32, 1, 16), (16, 3, 8), (256, 2, 32)])
def test_lookup_property(orc, N, m, t):
    """Lemma 7 / Eq. (equ:ex): for every phase u = msg*Delta + e with 2|e| < Delta
    (and the tie e = -Delta/2, read as msg), the constant term of the first row
    of P(u) (0, v_test) is f(msg) * floor(Q/t).  The entries of v_test are
    residues in Z_t scaled by floor(Q/t); a term that wraps around x^N comes
    back negated mod Q, i.e. as -f(msg + t/2) * floor(Q/t), which is
    f(msg) * floor(Q/t) + (Q mod t)."""
    Q = 1073738753
    qp = 2 * N * m
    if qp % t:
        pytest.skip("t must divide 2Nm")
    delta = qp // t
    rng = np.random.default_rng(N + m + t)
    lut = _random_negacyclic(rng, t)
    v = orc.test_vector(N, m, t, Q, lut)
    acc = np.zeros((m, 2, N), np.uint64)
    acc[:, 1, :] = v
    dq = Q // t
    for msg in range(t):
        for e in range(-(delta // 2), (delta + 1) // 2):
            u = (msg * delta + e) % qp
            r = orc.mmpm_apply(N, m, Q, u, acc)
            got = int(r[0, 1, 0])
            direct = int(lut[msg]) * dq % Q
            wrapped = (Q - int(lut[(msg + t // 2) % t]) * dq % Q) % Q
            assert got in (direct, wrapped), (msg, e)
            assert (got * t + Q // 2) // Q % t == lut[msg]
            assert not r[:, 0, :].any()


def test_test_vector_rows_follow_eq_ex(orc):
    """Eq. (equ:ex): row i of P(mu) v_test holds f'(mu - c*m - i) at x^c.  Here
    f'(w) is read off the test vector itself as the look-up result of P(w)."""
    N, m, t, Q = 8, 3, 8, 1073738753
    qp = 2 * N * m
    rng = np.random.default_rng(3)
    lut = _random_negacyclic(rng, t)
    acc = np.zeros((m, 2, N), np.uint64)
    acc[:, 1, :] = orc.test_vector(N, m, t, Q, lut)
    fprime = [int(orc.mmpm_apply(N, m, Q, w, acc)[0, 1, 0]) for w in range(qp)]
    for mu in range(qp):
        r = orc.mmpm_apply(N, m, Q, mu, acc)
        for i in range(m):
            for c in range(N):
                assert int(r[i, 1, c]) == fprime[(mu - c * m - i) % qp]


def test_m1_is_the_fhew_test_polynomial(orc):
    """For m = 1, v_test is the FHEW/TFHE test polynomial sum_i f'(i) x^(-i)
    (Eq. (test:FHEW)), f' the negacyclic extension that is f(msg) on the block
    msg*Delta + [-Delta/2, Delta/2)."""
    N, t, Q = 64, 16, 1073738753
    delta = 2 * N // t
    rng = np.random.default_rng(11)
    lut = _random_negacyclic(rng, t)
    fp = np.zeros(2 * N, dtype=np.int64)
    for msg in range(t):
        for e in range(-(delta // 2), delta - delta // 2):
            fp[(msg * delta + e) % (2 * N)] = lut[msg]
    dq = Q // t
    poly = [0] * N              # the test polynomial in R_{N,t}
    for i in range(N):          # f'(i) x^{-i} = -f'(i) x^{N-i} for i > 0
        if i == 0:
            poly[0] = (poly[0] + int(fp[i])) % t
        else:
            poly[N - i] = (poly[N - i] - int(fp[i])) % t
    v = orc.test_vector(N, 1, t, Q, lut)[0]   # scaled by floor(Q/t)
    assert [int(x) for x in v] == [c * dq % Q for c in poly]


def test_test_vector_is_negacyclic(orc):
    """v_(k+Nm) = -v_k (Section 3): P(Nm) v_test = -v_test, and the table's
    negacyclic symmetry f(k + t/2) = -f(k) shows up as a sign flip."""
    N, m, t, Q = 16, 4, 32, 1073738753
    rng = np.random.default_rng(5)
    lut = _random_negacyclic(rng, t)
    acc = np.zeros((m, 2, N), np.uint64)
    acc[:, 1, :] = orc.test_vector(N, m, t, Q, lut)
    half = orc.mmpm_apply(N, m, Q, N * m, acc)
    assert np.array_equal(half[:, 1], (Q - acc[:, 1]) % Q)


def test_decompose(orc):
    rng = np.random.default_rng(0)
    for log2_B, l_B, Q in [(6, 5, 1073738753), (9, 6, 18014398509404161), (10, 6, 1152921504606830593)]:
        for x in list(rng.integers(0, Q, 200, dtype=np.uint64)) + [0, Q - 1]:
            d = orc.decompose(int(x), log2_B, l_B)
            assert all(int(dj) < (1 << log2_B) for dj in d)
            assert sum(int(dj) << (log2_B * j) for j, dj in enumerate(d)) == int(x)


def test_workload_moduli():
    """Every modulus is prime, 1 mod 2N, within its bound; above 2^32 it is
    the largest such prime of the form c 2^32 + 1."""
    import sympy
    from paper_2310_12441_gb300 import params as P
    for kp, bits in [(P.KEYS_TOY, 30), (P.KEYS_N1024, 54), (P.KEYS_N4096, 54), (P.KEYS_N2048, 60)]:
        Q = kp.Q
        assert sympy.isprime(Q) and (Q - 1) % (2 * kp.N) == 0 and Q < 1 << bits
        kp.validate()
        if bits > 32:
            assert Q & 0xFFFFFFFF == 1
            c = Q >> 32
            for c2 in range(c + 1, ((1 << bits) - 1) >> 32):
                assert not sympy.isprime((c2 << 32) + 1)

/*
 * CPU oracle for BootMMPM (arXiv 2310.12441, Algorithm 1).
 *
 * TEST INFRASTRUCTURE ONLY.  Only the tests, the smoke check and the CPU
 * baseline leg of the benchmark may load this file's library.  The product
 * path never calls it, and it shares no code with the CUDA library.
 *
 * Plain, slow, obviously correct: exact integers (uint64 values, unsigned
 * __int128 accumulators), schoolbook negacyclic products (x^N = -1), no NTT,
 * no fusion.  Each function cites the passage of the paper it follows.  The
 * readings taken where the paper is silent or inconsistent are stated at the
 * function that takes them.
 *
 * Conventions shared with the paper:
 *  - LWE ciphertext (a_1..a_n, b) is stored as n+1 words, b last;
 *    phase = b - <a, s> (Section 2, (8)).
 *  - RLWE ciphertext (a, b), phase = b - a*z (Section 2, (12)).
 *  - RLWE vector of m rows: array [m][2][N], component 0 = a, 1 = b (Sec. 4).
 *  - RGSW ciphertext: [2*l_B][2][N]; row j < l_B is RLWE_z(0) + (mu*B^j, 0),
 *    row l_B + j is RLWE_z(0) + (0, mu*B^j).  The paper's RGSW phase
 *    C(1,-s)^T pairs the columns as (b, a) while its external product
 *    g^{-1}(a,b) C pairs them as (a, b); this layout is the one under which
 *    g^{-1}(a,b) C encrypts mu * phase(a,b) (Section 2, (14)).
 *  - Bootstrapping key: [n][2][2*l_B][2][N]; index 0 encrypts s_k+ =
 *    max(s_k, 0), index 1 encrypts s_k- = max(-s_k, 0) (Algorithm 1).
 *  - Key-switching key: [N][l_ks][B_ks - 1][n+1]; entry (i, j, v-1) is an
 *    LWE_{n,Q} encryption under s of v * z_i * g_j (Section 2, (11)).
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

typedef uint64_t u64;
typedef unsigned __int128 u128;

/* ------------------------------------------------------------------------ */
/* Modular helpers                                                          */
/* ------------------------------------------------------------------------ */

static u64 add_mod(u64 a, u64 b, u64 q) { u128 s = (u128)a + b; return (u64)(s % q); }
static u64 sub_mod(u64 a, u64 b, u64 q) { return a >= b ? a - b : (u64)((u128)a + q - b); }
static u64 neg_mod(u64 a, u64 q) { return a == 0 ? 0 : q - a; }
static u64 mul_mod(u64 a, u64 b, u64 q) { return (u64)(((u128)a * b) % q); }
static u64 from_signed(int64_t v, u64 q) {
    int64_t r = v % (int64_t)q;
    return r < 0 ? (u64)(r + (int64_t)q) : (u64)r;
}

/* ------------------------------------------------------------------------ */
/* Ring R_{N,Q} = Z_Q[x]/(x^N + 1)  (Section 2, (6))                        */
/* ------------------------------------------------------------------------ */

/* out = a * b in R_{N,Q} by the schoolbook rule: the coefficient of x^k
 * collects a_i b_j over i + j = k, and minus a_i b_j over i + j = k + N,
 * because x^N = -1. */
void orc_poly_mul(uint32_t N, u64 Q, const u64 *a, const u64 *b, u64 *out)
{
    u128 *pos = calloc(N, sizeof(u128)), *neg = calloc(N, sizeof(u128));
    for (uint32_t i = 0; i < N; i++) {
        for (uint32_t j = 0; j < N; j++) {
            u64 p = mul_mod(a[i], b[j], Q);
            if (i + j < N) pos[i + j] += p; else neg[i + j - N] += p;
        }
    }
    for (uint32_t k = 0; k < N; k++)
        out[k] = sub_mod((u64)(pos[k] % Q), (u64)(neg[k] % Q), Q);
    free(pos); free(neg);
}

/* out = x^e * p in R_{N,Q} for an integer exponent e (taken mod 2N): the
 * monomial x^(j+e) of p_j lands on x^((j+e) mod N) with sign -1 when
 * (j + e) mod 2N >= N. */
static void monomial_mul(uint32_t N, u64 Q, int64_t e, const u64 *p, u64 *out)
{
    int64_t twoN = 2 * (int64_t)N;
    int64_t ee = ((e % twoN) + twoN) % twoN;
    for (uint32_t j = 0; j < N; j++) {
        int64_t d = ((int64_t)j + ee) % twoN;
        if (d < (int64_t)N) out[d] = p[j];
        else out[d - N] = neg_mod(p[j], Q);
    }
}

/* ------------------------------------------------------------------------ */
/* Monic monomial permutation matrices (Section 3, Example 1)               */
/* ------------------------------------------------------------------------ */

/* out = P(c) * in for an RLWE vector in ([m][2][N]), c in Z_{2Nm}.
 * With c = a*m + b, a in [2N], b in [m], Eq. (ex1:BPc) gives the matrix
 *   P(c) = [[0, x^(a+1) I_b], [x^a I_(m-b), 0]],
 * so row i of the product is x^a * in_(i-b) for i >= b and
 * x^(a+1) * in_(i-b+m) for i < b.  (The printed Hadamard form (equ-hadam)
 * lists the rows in the opposite direction; the matrix and P(1) of
 * (ex:BP) agree with the rule used here.)  The product acts on both RLWE
 * components alike (Section 4). */
void orc_mmpm_apply(uint32_t N, uint32_t m, u64 Q, uint64_t c,
                    const u64 *in, u64 *out)
{
    uint64_t qp = 2ull * N * m;
    c %= qp;
    uint64_t a = c / m, b = c % m;
    for (uint32_t i = 0; i < m; i++) {
        uint32_t src = (i >= b) ? (uint32_t)(i - b) : (uint32_t)(i + m - b);
        int64_t e = (i >= b) ? (int64_t)a : (int64_t)a + 1;
        for (int comp = 0; comp < 2; comp++)
            monomial_mul(N, Q, e, in + ((size_t)src * 2 + comp) * N,
                         out + ((size_t)i * 2 + comp) * N);
    }
}

/* ------------------------------------------------------------------------ */
/* Test polynomial vector (Section 3, Example 2, Eq. (equ:test-use))        */
/* ------------------------------------------------------------------------ */

/* Negacyclic extension f' of f from Z_t to Z_{q'}, q' = 2Nm (Section 2, (7)):
 * f'(u) = f(round(u t / q') mod t) with round-half-up, i.e.
 * floor((u t + q'/2) / q').  The paper only requires f'(msg*Delta + e) =
 * f(msg) for 2|e| < Delta; round-half-up fixes the tie e = -Delta/2 and is
 * the same rule the decryption uses. */
static uint32_t f_ext(const uint32_t *lut, uint32_t t, uint64_t qp, uint64_t u)
{
    u128 num = (u128)(u % qp) * t + qp / 2;
    return lut[(uint32_t)((num / qp) % t)];
}

/* v[b][a] = f'(-(a*m + b) mod 2Nm) * floor(Q/t) mod Q, b in [m], a in [N]
 * (Eq. (equ:test-use) with the scaling of Algorithm 1's initial ACC).  An
 * entry -f is carried as the Z_t residue t - f before scaling. */
void orc_test_vector(uint32_t N, uint32_t m, uint32_t t, u64 Q,
                     const uint32_t *lut, u64 *v)
{
    uint64_t qp = 2ull * N * m;
    u64 dq = Q / t;
    for (uint32_t b = 0; b < m; b++)
        for (uint32_t a = 0; a < N; a++) {
            uint64_t idx = (uint64_t)a * m + b;
            uint64_t u = (qp - idx % qp) % qp;
            v[(size_t)b * N + a] = mul_mod(f_ext(lut, t, qp, u), dq, Q);
        }
}

/* ------------------------------------------------------------------------ */
/* Gadget decomposition (Section 2, (10))                                   */
/* ------------------------------------------------------------------------ */

/* Unsigned base-B digits of x in [0, Q): x = sum_{j<l_B} x_j B^j, x_j in [B].
 * (The paper lists x_0..x_{l_B}; l_B digits suffice because B^l_B >= Q.) */
void orc_decompose(u64 x, uint32_t log2_B, uint32_t l_B, u64 *digits)
{
    u64 B = 1ull << log2_B;
    for (uint32_t j = 0; j < l_B; j++) { digits[j] = x % B; x /= B; }
}

/* ------------------------------------------------------------------------ */
/* External product RLWE x RGSW (Section 2, (14); Section 4)                */
/* ------------------------------------------------------------------------ */

typedef struct {
    uint32_t n, N, log2_B, l_B, log2_Bks, l_ks;
    u64 Q;
} orc_params;

/* pos/neg += d * c negacyclically, d with small digits: the schoolbook rule
 * of orc_poly_mul with the products accumulated unreduced.  Zero digits are
 * skipped (they contribute nothing). */
static void mac_small(uint32_t N, const u64 *d, const u64 *c, u128 *pos, u128 *neg)
{
    for (uint32_t i = 0; i < N; i++) {
        u64 di = d[i];
        if (di == 0) continue;
        for (uint32_t j = 0; j < N - i; j++) pos[i + j] += (u128)di * c[j];
        for (uint32_t j = N - i; j < N; j++) neg[i + j - N] += (u128)di * c[j];
    }
}

/* Column col of g^{-1}(a, b) * C, with g^{-1}(a, b) = [g^{-1}(a) | g^{-1}(b)]
 * the 2*l_B digit polynomials and C the [2*l_B][2][N] RGSW matrix:
 * out = sum_j digit_j(a) * C[j][col] + digit_j(b) * C[l_B+j][col]. */
static void external_product_col(const orc_params *p, const u64 *a, const u64 *b,
                                 const u64 *C, int col, u64 *out)
{
    uint32_t N = p->N, lB = p->l_B;
    u64 *dig = malloc(sizeof(u64) * N);
    u128 *pos = calloc(N, sizeof(u128));
    u128 *neg = calloc(N, sizeof(u128));
    u64 *tmp = malloc(sizeof(u64) * lB);
    for (int comp = 0; comp < 2; comp++) {
        const u64 *src = comp == 0 ? a : b;
        for (uint32_t j = 0; j < lB; j++) {
            for (uint32_t i = 0; i < N; i++) {
                orc_decompose(src[i], p->log2_B, lB, tmp);
                dig[i] = tmp[j];
            }
            const u64 *row = C + (size_t)(comp * lB + j) * 2 * N;
            mac_small(N, dig, row + (size_t)col * N, pos, neg);
        }
    }
    for (uint32_t k = 0; k < N; k++)
        out[k] = sub_mod((u64)(pos[k] % p->Q), (u64)(neg[k] % p->Q), p->Q);
    free(dig); free(pos); free(neg); free(tmp);
}

/* (out_a, out_b) = g^{-1}(a, b) * C: both columns. */
void orc_external_product(const orc_params *p, const u64 *a, const u64 *b,
                          const u64 *C, u64 *out_a, u64 *out_b)
{
    external_product_col(p, a, b, C, 0, out_a);
    external_product_col(p, a, b, C, 1, out_b);
}

/* ------------------------------------------------------------------------ */
/* CMux over P (Section 4, Eq. (cmux:BP))                                   */
/* ------------------------------------------------------------------------ */

/* acc <- acc + g^{-1}(P(-a_k) acc - acc) C_k+ + g^{-1}(P(a_k) acc - acc) C_k-,
 * the RLWE-vector x RGSW products taken row by row.  ak in Z_{2Nm}.
 * Cp, Cm: [2*l_B][2][N].  'parallel' runs the 2*m independent row
 * products (and their two columns) in parallel. */
void orc_cmux(const orc_params *p, uint32_t m, uint64_t ak, const u64 *Cp,
              const u64 *Cm, u64 *acc, int parallel)
{
    uint32_t N = p->N;
    u64 Q = p->Q;
    uint64_t qp = 2ull * N * m;
    size_t vec = (size_t)m * 2 * N;
    u64 *rot = malloc(sizeof(u64) * vec * 2);   /* P(-a)acc, P(a)acc */
    u64 *diff = malloc(sizeof(u64) * vec * 2);
    u64 *prod = malloc(sizeof(u64) * vec * 2);
    orc_mmpm_apply(N, m, Q, (qp - ak % qp) % qp, acc, rot);
    orc_mmpm_apply(N, m, Q, ak % qp, acc, rot + vec);
    for (size_t i = 0; i < vec; i++) {
        diff[i] = sub_mod(rot[i], acc[i], Q);
        diff[vec + i] = sub_mod(rot[vec + i], acc[i], Q);
    }
    /* the 2m row products and their two output columns are independent */
    #pragma omp parallel for schedule(dynamic) if (parallel)
    for (int task = 0; task < (int)(4 * m); task++) {
        int col = task & 1, sgn = (task >> 1) / (int)m, r = (task >> 1) % (int)m;
        const u64 *d = diff + (size_t)sgn * vec + (size_t)r * 2 * N;
        u64 *o = prod + (size_t)sgn * vec + (size_t)r * 2 * N;
        external_product_col(p, d, d + N, sgn == 0 ? Cp : Cm, col, o + (size_t)col * N);
    }
    for (size_t i = 0; i < vec; i++)
        acc[i] = add_mod(add_mod(acc[i], prod[i], Q), prod[vec + i], Q);
    free(rot); free(diff); free(prod);
}

/* ------------------------------------------------------------------------ */
/* Blind rotation: Algorithm 1, phase accumulation                          */
/* ------------------------------------------------------------------------ */

/* acc ([m][2][N]) <- P(b) (0, v_test * floor(Q/t)), then for k = 1..n the
 * CMux of ct_k+, ct_k-.  ct: n+1 words in Z_{2Nm} (already modulus-switched).
 * bsk holds the first n_keys key pairs; the oracle requires a_k = 0 for
 * k >= n_keys: P(0) = I makes both differences zero, so such a step leaves
 * acc unchanged and needs no key.  Returns 0, or -1 on a missing key. */
int orc_blind_rotate(const orc_params *p, uint32_t m, uint32_t t,
                     const u64 *bsk, uint32_t n_keys, const uint64_t *ct,
                     const uint32_t *lut, u64 *acc, int parallel)
{
    uint32_t N = p->N, n = p->n, lB = p->l_B;
    u64 Q = p->Q;
    uint64_t qp = 2ull * N * m;
    size_t vec = (size_t)m * 2 * N;
    size_t rgsw = (size_t)2 * lB * 2 * N;
    u64 *v = malloc(sizeof(u64) * (size_t)m * N);
    u64 *init = calloc(vec, sizeof(u64));
    orc_test_vector(N, m, t, Q, lut, v);
    for (uint32_t r = 0; r < m; r++)
        memcpy(init + ((size_t)r * 2 + 1) * N, v + (size_t)r * N, sizeof(u64) * N);
    orc_mmpm_apply(N, m, Q, ct[n] % qp, init, acc);
    for (uint32_t k = 0; k < n; k++) {
        uint64_t ak = ct[k] % qp;
        if (k >= n_keys) {
            if (ak != 0) { free(v); free(init); return -1; }
            continue;
        }
        const u64 *Cp = bsk + (size_t)k * 2 * rgsw;
        orc_cmux(p, m, ak, Cp, Cp + rgsw, acc, parallel);
    }
    free(v); free(init);
    return 0;
}

/* ------------------------------------------------------------------------ */
/* Sample extraction (Section 2, (13), Eq. (equ-sam-extr))                  */
/* ------------------------------------------------------------------------ */

/* (a_0, -a_{N-1}, ..., -a_1, b_0) from the RLWE ciphertext (a, b). */
void orc_sample_extract(uint32_t N, u64 Q, const u64 *a, const u64 *b, u64 *lwe)
{
    lwe[0] = a[0];
    for (uint32_t i = 1; i < N; i++) lwe[i] = neg_mod(a[N - i], Q);
    lwe[N] = b[0];
}

/* ------------------------------------------------------------------------ */
/* Key switching (Section 2, (11), Eq. (equ-key-swi))                       */
/* ------------------------------------------------------------------------ */

/* Approximate gadget with P = B_ks^l_ks < Q: each a_i is first rounded to
 * a~_i = floor((a_i P + floor(Q/2)) / Q) mod P, then split into l_ks unsigned
 * base-B_ks digits d_ij; the gadget vector is g_j = floor((Q B_ks^j + P/2)/P),
 * so sum_j d_ij g_j ~ a_i.  The paper takes l_ks = ceil(log_Bks Q) digits of
 * a_i itself; with fewer digits this rounding keeps the key-switched phase
 * within Q/(2P) * |z|_1 of the exact one. */
u64 orc_ks_gadget(const orc_params *p, uint32_t j)
{
    u128 P = (u128)1 << (p->log2_Bks * p->l_ks);
    u128 num = (u128)p->Q << (p->log2_Bks * j);
    return (u64)((num + P / 2) / P);
}

void orc_ks_digits(const orc_params *p, u64 a, uint32_t *d)
{
    uint32_t sh = p->log2_Bks * p->l_ks;
    u128 P = (u128)1 << sh;
    u64 at = (u64)((((u128)a << sh) + p->Q / 2) / p->Q % P);
    for (uint32_t j = 0; j < p->l_ks; j++)
        d[j] = (uint32_t)((at >> (p->log2_Bks * j)) & ((1u << p->log2_Bks) - 1));
}

/* (a_out, b_out) = (0^n, b) - sum_{i<N, j<l_ks} ksk(i, j, d_ij) mod Q;
 * a zero digit selects nothing (ksk(i, j, 0) would encrypt 0). */
void orc_key_switch(const orc_params *p, const u64 *lwe_N, const u64 *ksk, u64 *out)
{
    uint32_t N = p->N, n = p->n, Bks = 1u << p->log2_Bks;
    u64 Q = p->Q;
    uint32_t *d = malloc(sizeof(uint32_t) * p->l_ks);
    for (uint32_t c = 0; c < n; c++) out[c] = 0;
    out[n] = lwe_N[N];
    for (uint32_t i = 0; i < N; i++) {
        orc_ks_digits(p, lwe_N[i], d);
        for (uint32_t j = 0; j < p->l_ks; j++) {
            if (d[j] == 0) continue;
            const u64 *row = ksk + (((size_t)i * p->l_ks + j) * (Bks - 1) + (d[j] - 1)) * (n + 1);
            for (uint32_t c = 0; c <= n; c++) out[c] = sub_mod(out[c], row[c], Q);
        }
    }
    free(d);
}

/* ------------------------------------------------------------------------ */
/* Key generation and LWE encryption (Section 2, (8), (11), (14))           */
/* ------------------------------------------------------------------------ */

/* acc = a * z for ternary z: the schoolbook sum of z_j x^j a over j. */
static void mul_ternary(uint32_t N, u64 Q, const u64 *a, const int8_t *z, u64 *out, u64 *tmp)
{
    for (uint32_t k = 0; k < N; k++) out[k] = 0;
    for (uint32_t j = 0; j < N; j++) {
        if (z[j] == 0) continue;
        monomial_mul(N, Q, (int64_t)j, a, tmp);
        for (uint32_t k = 0; k < N; k++)
            out[k] = z[j] > 0 ? add_mod(out[k], tmp[k], Q) : sub_mod(out[k], tmp[k], Q);
    }
}

/* Bootstrapping keys for k in [k0, k1): bsk_out[k - k0][sgn][row][col][N].
 * Row r of RGSW_z(mu): (a_r, a_r z + e_r) plus mu B^j on column 0 (r = j < l_B)
 * or column 1 (r = l_B + j).  mu = s_k+ (sgn 0) or s_k- (sgn 1).
 * mask/err index the full arrays [n][2][2 l_B][N]. */
void orc_keygen_bsk(const orc_params *p, const int8_t *s, const int8_t *z,
                    const u64 *mask, const int8_t *err, uint32_t k0, uint32_t k1,
                    u64 *bsk_out)
{
    uint32_t N = p->N, lB = p->l_B;
    u64 Q = p->Q;
    size_t rows = (size_t)(k1 - k0) * 2 * 2 * lB;
    #pragma omp parallel
    {
        u64 *tmp = malloc(sizeof(u64) * N);
        #pragma omp for schedule(dynamic)
        for (long rr = 0; rr < (long)rows; rr++) {
            size_t r = (size_t)rr;
            uint32_t row = r % (2 * lB);
            uint32_t sgn = (r / (2 * lB)) % 2;
            uint32_t k = k0 + (uint32_t)(r / (4 * lB));
            size_t src = (((size_t)k * 2 + sgn) * 2 * lB + row) * N;
            u64 *o = bsk_out + r * 2 * N;
            const u64 *a = mask + src;
            memcpy(o, a, sizeof(u64) * N);
            mul_ternary(N, Q, a, z, o + N, tmp);
            for (uint32_t c = 0; c < N; c++)
                o[N + c] = add_mod(o[N + c], from_signed(err[src + c], Q), Q);
            int sk = s[k];
            u64 mu = sgn == 0 ? (sk > 0 ? 1 : 0) : (sk < 0 ? 1 : 0);
            if (mu) {
                uint32_t j = row % lB;
                u64 g = (u64)(((u128)1 << (p->log2_B * j)) % Q);
                int col = row < lB ? 0 : 1;
                o[(size_t)col * N] = add_mod(o[(size_t)col * N], g, Q);
            }
        }
        free(tmp);
    }
}

/* Key-switching keys [N][l_ks][B_ks-1][n+1]: (a', <a', s> + e + v z_i g_j). */
void orc_keygen_ksk(const orc_params *p, const int8_t *s, const int8_t *z,
                    const u64 *mask, const int8_t *err, u64 *ksk_out)
{
    uint32_t N = p->N, n = p->n, Bks = 1u << p->log2_Bks;
    u64 Q = p->Q;
    size_t rows = (size_t)N * p->l_ks * (Bks - 1);
    #pragma omp parallel for schedule(static)
    for (long rr = 0; rr < (long)rows; rr++) {
        size_t r = (size_t)rr;
        uint32_t v = (uint32_t)(r % (Bks - 1)) + 1;
        uint32_t j = (uint32_t)((r / (Bks - 1)) % p->l_ks);
        uint32_t i = (uint32_t)(r / ((size_t)(Bks - 1) * p->l_ks));
        const u64 *a = mask + r * n;
        u64 *o = ksk_out + r * (n + 1);
        u64 b = from_signed(err[r], Q);
        for (uint32_t c = 0; c < n; c++) {
            o[c] = a[c];
            b = add_mod(b, mul_mod(a[c], from_signed(s[c], Q), Q), Q);
        }
        u64 msg = mul_mod(mul_mod(v, from_signed(z[i], Q), Q), orc_ks_gadget(p, j), Q);
        o[n] = add_mod(b, msg, Q);
    }
}

/* LWE_{n,q} encryption (Section 2, (8)): b = <a, s> + msg floor(q/t) + e mod q. */
void orc_encrypt(uint32_t n, u64 q, uint32_t t, const int8_t *s, const uint32_t *msg,
                 const u64 *mask, const int8_t *err, size_t count, u64 *ct)
{
    for (size_t i = 0; i < count; i++) {
        u64 *o = ct + i * (n + 1);
        u64 b = from_signed(err[i], q);
        for (uint32_t c = 0; c < n; c++) {
            o[c] = mask[i * n + c] % q;
            b = add_mod(b, mul_mod(o[c], from_signed(s[c], q), q), q);
        }
        o[n] = add_mod(b, mul_mod(msg[i] % t, q / t, q), q);
    }
}

/* phase(a, b) = b - <a, s> mod q. */
u64 orc_lwe_phase(uint32_t n, u64 q, const int8_t *s, const u64 *ct)
{
    u64 acc = ct[n] % q;
    for (uint32_t c = 0; c < n; c++)
        acc = sub_mod(acc, mul_mod(ct[c] % q, from_signed(s[c], q), q), q);
    return acc;
}

/* Decryption: round(phase * t / q) mod t, round half up (Section 2, (8)). */
void orc_decrypt(uint32_t n, u64 q, uint32_t t, const int8_t *s, const u64 *ct,
                 size_t count, uint32_t *msg)
{
    for (size_t i = 0; i < count; i++) {
        u64 ph = orc_lwe_phase(n, q, s, ct + i * (n + 1));
        msg[i] = (uint32_t)((((u128)ph * t + q / 2) / q) % t);
    }
}

/* RLWE phase b - a z, z ternary. */
void orc_rlwe_phase(uint32_t N, u64 Q, const int8_t *z, const u64 *a, const u64 *b, u64 *out)
{
    u64 *az = malloc(sizeof(u64) * N), *tmp = malloc(sizeof(u64) * N);
    mul_ternary(N, Q, a, z, az, tmp);
    for (uint32_t k = 0; k < N; k++) out[k] = sub_mod(b[k], az[k], Q);
    free(az); free(tmp);
}

/* ------------------------------------------------------------------------ */
/* Modulus switch (Section 2, (9)): x -> round(x q_to / q_from), rounding    */
/* half up, i.e. floor((x q_to + floor(q_from / 2)) / q_from) mod q_to,      */
/* applied to every word of the given ciphertexts.                           */
/* ------------------------------------------------------------------------ */
void orc_mod_switch(const u64 *in, size_t words, u64 q_from, u64 q_to, u64 *out)
{
    for (size_t i = 0; i < words; i++) {
        u128 x = (u128)(in[i] % q_from) * q_to + q_from / 2;
        out[i] = (u64)((x / q_from) % q_to);
    }
}

/* ------------------------------------------------------------------------ */
/* Algorithm 1 end to end (modulus switch q -> 2Nm is the identity here:    */
/* inputs are given in Z_{2Nm}; the final Q -> q switch is not applied).    */
/* ------------------------------------------------------------------------ */

/* ct_out = KeySwitch(SampleExtract(row 0 of the blind-rotated ACC)).
 * count ciphertexts, each with its own table of t entries; the batch runs
 * one ciphertext per thread, a single ciphertext parallel over rows. */
int orc_bootstrap(const orc_params *p, uint32_t m, uint32_t t, const u64 *bsk,
                  uint32_t n_keys, const u64 *ksk, const uint64_t *ct_in,
                  const uint32_t *luts, size_t count, u64 *ct_out)
{
    uint32_t N = p->N, n = p->n;
    int bad = 0;
    int inner = count == 1;
    #pragma omp parallel for schedule(dynamic) if (!inner) reduction(|:bad)
    for (long ii = 0; ii < (long)count; ii++) {
        size_t i = (size_t)ii;
        u64 *acc = malloc(sizeof(u64) * (size_t)m * 2 * N);
        u64 *lwe = malloc(sizeof(u64) * (N + 1));
        if (orc_blind_rotate(p, m, t, bsk, n_keys, ct_in + i * (n + 1),
                             luts + i * t, acc, inner) != 0)
            bad = 1;
        orc_sample_extract(N, p->Q, acc, acc + N, lwe);
        orc_key_switch(p, lwe, ksk, ct_out + i * (n + 1));
        free(acc); free(lwe);
    }
    return bad ? -1 : 0;
}

/* ------------------------------------------------------------------------ */
/* Arbitrary f: Z_t -> Z_t by two rounds (Section 4, last part): the input   */
/* encrypts m in [0, t) under plaintext modulus 2t; its unknown top bit is   */
/* extracted with the negacyclic mp (mp(x) = -t/2 on [-t/2, t/2), t/2 on     */
/* the rest of [-t, t)), using sign(x) t = mp(x) + t/2 (Eq. (rel:sign));     */
/* subtracting sign(x) t leaves y in [-t/2, t/2) with y = m mod t, and a    */
/* second bootstrap with the negacyclic extension F of f from [-t/2, t/2)    */
/* (F(y) = f(y mod t) there, F(y + t) = -F(y)) gives f(m).                   */
/* Inputs and outputs are LWE_{n,q}; bootstraps run at q' = 2Nm, plaintext   */
/* modulus 2t.                                                               */
/* ------------------------------------------------------------------------ */

/* Tables over Z_{2t}: mp[x] and F[y] (per job, from f's t entries). */
void orc_two_round_tables(uint32_t t, const uint32_t *f, uint32_t *mp, uint32_t *F)
{
    uint32_t T = 2 * t;
    for (uint32_t x = 0; x < T; x++) {
        /* x in [-t/2, t/2) mod 2t  <=>  x < t/2 or x >= 3t/2 */
        int lower = x < t / 2 || x >= 3 * t / 2;
        mp[x] = lower ? T - t / 2 : t / 2;
    }
    for (uint32_t y = 0; y < T; y++) {
        if (y < t / 2) F[y] = f[y] % T;
        else if (y >= 3 * t / 2) F[y] = f[y - t] % T;          /* y - 2t in [-t/2, 0): y mod t = y - t */
        else {                                                   /* F(y) = -F(y - t) */
            uint32_t z = (y + t) % T;                            /* (y - t) mod 2t: [0, t/2) or [3t/2, 2t) */
            uint32_t v = z < t / 2 ? f[z] : f[z - t];
            F[y] = (T - v % T) % T;
        }
    }
}

int orc_bootstrap_arbitrary(const orc_params *p, uint32_t m, uint32_t t, u64 q, const u64 *bsk,
                            uint32_t n_keys, const u64 *ksk, const u64 *ct_in, const uint32_t *f,
                            size_t count, u64 *ct_out)
{
    uint32_t n = p->n, T = 2 * t;
    u64 qp = 2ull * p->N * m;
    size_t W = (size_t)count * (n + 1);
    u64 *a = malloc(sizeof(u64) * W), *b = malloc(sizeof(u64) * W);
    uint32_t *mp = malloc(sizeof(uint32_t) * T * count), *F = malloc(sizeof(uint32_t) * T * count);
    for (size_t i = 0; i < count; i++)
        orc_two_round_tables(t, f + i * t, mp + i * T, F + i * T);
    int rc = 0;
    /* round 1: mp */
    orc_mod_switch(ct_in, W, q, qp, a);
    rc |= orc_bootstrap(p, m, T, bsk, n_keys, ksk, a, mp, count, b);
    orc_mod_switch(b, W, p->Q, q, b);
    /* y = x - (mp(x) + t/2) at modulus q, plaintext scale floor(q / 2t) */
    u64 half = (u64)(t / 2) * (q / T) % q;
    for (size_t i = 0; i < count; i++)
        for (uint32_t c = 0; c <= n; c++) {
            size_t k = i * (n + 1) + c;
            u64 v = sub_mod(ct_in[k] % q, b[k], q);
            a[k] = c == n ? sub_mod(v, half, q) : v;
        }
    /* round 2: F */
    orc_mod_switch(a, W, q, qp, a);
    rc |= orc_bootstrap(p, m, T, bsk, n_keys, ksk, a, F, count, b);
    orc_mod_switch(b, W, p->Q, q, ct_out);
    free(a); free(b); free(mp); free(F);
    return rc ? -1 : 0;
}

/* ------------------------------------------------------------------------ */
/* General transitive generators (Section 3: Theorem 1, Lemma 3, Lemma 4,   */
/* Example 2).                                                              */
/*                                                                          */
/* A generator is P(1) = A = (x^{u_i} delta_{tau(i), j}), tau(i) = i-1 mod m */
/* (the form (BP1:form): row 0 holds x^{u_0} in column m-1, row i >= 1      */
/* holds x^{u_i} in column i-1).  By Theorem 1 the group it generates acts  */
/* transitively on the monic monomial indicator vectors iff                 */
/* ord(x^{sum u}) = 2N, i.e. iff sum u is odd.  Example 1's P(1) is         */
/* u = (1, 0, ..., 0).                                                      */
/* ------------------------------------------------------------------------ */

/* E_c(i) = sum_{t in [c]} u_{(i - t) mod m}: the exponent of row i of A^c
 * (Lemma 3, Eq. (Al:res)), whose nonzero entry sits in column (i - c) mod m. */
static uint64_t gen_exponent(uint32_t m, const uint32_t *u, uint64_t c, uint32_t i)
{
    uint64_t S = 0;
    for (uint32_t k = 0; k < m; k++) S += u[k];
    uint64_t e = (c / m) * S;
    for (uint64_t t = 0; t < c % m; t++) e += u[(i + m - (uint32_t)t) % m];
    return e;
}

/* out = P(c) * in = A^c * in for an RLWE vector [m][2][N]: row i is
 * x^{E_c(i)} in_{(i - c) mod m} (Lemma 3). */
void orc_mmpm_apply_gen(uint32_t N, uint32_t m, u64 Q, const uint32_t *u, uint64_t c,
                        const u64 *in, u64 *out)
{
    for (uint32_t i = 0; i < m; i++) {
        uint32_t src = (uint32_t)((i + (uint64_t)m - c % m) % m);
        int64_t e = (int64_t)(gen_exponent(m, u, c, i) % (2ull * N));
        for (int comp = 0; comp < 2; comp++)
            monomial_mul(N, Q, e, in + ((size_t)src * 2 + comp) * N, out + ((size_t)i * 2 + comp) * N);
    }
}

/* One application of A: row i of the result is x^{u_i} in_{(i - 1) mod m}. */
void orc_mmpm_step_gen(uint32_t N, uint32_t m, u64 Q, const uint32_t *u, const u64 *in, u64 *out)
{
    for (uint32_t i = 0; i < m; i++)
        for (int comp = 0; comp < 2; comp++)
            monomial_mul(N, Q, (int64_t)u[i], in + ((size_t)((i + m - 1) % m) * 2 + comp) * N,
                         out + ((size_t)i * 2 + comp) * N);
}

/* Test vector of Eq. (equ:test-gene) scaled by floor(Q/t):
 *   v_0 = sum_{a in [N], b in [m]} f'(-(a m + b)) x^{a S + E_b(b)} e_b,
 * S = sum u, E_b(b) = u_b + ... + u_1 (the exponent of P(b) e_0, Eq.
 * (equ:basis-test-gene)); x^N = -1 folds every exponent into [N]. */
void orc_test_vector_gen(uint32_t N, uint32_t m, uint32_t t, u64 Q, const uint32_t *u,
                         const uint32_t *lut, u64 *v)
{
    uint64_t qp = 2ull * N * m;
    u64 dq = Q / t;
    uint64_t S = 0;
    for (uint32_t k = 0; k < m; k++) S += u[k];
    memset(v, 0, sizeof(u64) * (size_t)m * N);
    for (uint32_t b = 0; b < m; b++) {
        uint64_t Eb = gen_exponent(m, u, b, b);
        for (uint32_t a = 0; a < N; a++) {
            uint64_t idx = (uint64_t)a * m + b;
            uint64_t w = (qp - idx % qp) % qp;
            u64 val = mul_mod(f_ext(lut, t, qp, w), dq, Q);
            uint64_t e = ((uint64_t)a * S + Eb) % (2ull * N);
            size_t pos = (size_t)b * N + (e % N);
            v[pos] = e < N ? add_mod(v[pos], val, Q) : sub_mod(v[pos], val, Q);
        }
    }
}

/* acc <- acc + g^{-1}(P(-a_k) acc - acc) C_k+ + g^{-1}(P(a_k) acc - acc) C_k-
 * for the generator u (Eq. (cmux:BP)). */
static void cmux_gen(const orc_params *p, uint32_t m, const uint32_t *u, uint64_t ak, const u64 *Cp,
                     const u64 *Cm, u64 *acc, int parallel)
{
    uint32_t N = p->N;
    u64 Q = p->Q;
    uint64_t qp = 2ull * N * m;
    size_t vec = (size_t)m * 2 * N;
    u64 *rot = malloc(sizeof(u64) * vec * 2);
    u64 *diff = malloc(sizeof(u64) * vec * 2);
    u64 *prod = malloc(sizeof(u64) * vec * 2);
    orc_mmpm_apply_gen(N, m, Q, u, (qp - ak % qp) % qp, acc, rot);
    orc_mmpm_apply_gen(N, m, Q, u, ak % qp, acc, rot + vec);
    for (size_t i = 0; i < vec; i++) {
        diff[i] = sub_mod(rot[i], acc[i], Q);
        diff[vec + i] = sub_mod(rot[vec + i], acc[i], Q);
    }
    #pragma omp parallel for schedule(dynamic) if (parallel)
    for (int task = 0; task < (int)(4 * m); task++) {
        int col = task & 1, sgn = (task >> 1) / (int)m, r = (task >> 1) % (int)m;
        const u64 *d = diff + (size_t)sgn * vec + (size_t)r * 2 * N;
        u64 *o = prod + (size_t)sgn * vec + (size_t)r * 2 * N;
        external_product_col(p, d, d + N, sgn == 0 ? Cp : Cm, col, o + (size_t)col * N);
    }
    for (size_t i = 0; i < vec; i++)
        acc[i] = add_mod(add_mod(acc[i], prod[i], Q), prod[vec + i], Q);
    free(rot); free(diff); free(prod);
}

/* Algorithm 1's phase accumulation with the generator u: ACC = P(b)(0, v_0),
 * then the CMux of every step; same key and ciphertext conventions as
 * orc_blind_rotate. */
int orc_blind_rotate_gen(const orc_params *p, uint32_t m, uint32_t t, const uint32_t *u,
                         const u64 *bsk, uint32_t n_keys, const uint64_t *ct,
                         const uint32_t *lut, u64 *acc, int parallel)
{
    uint32_t N = p->N, n = p->n, lB = p->l_B;
    u64 Q = p->Q;
    uint64_t qp = 2ull * N * m;
    size_t vec = (size_t)m * 2 * N;
    size_t rgsw = (size_t)2 * lB * 2 * N;
    u64 *v = malloc(sizeof(u64) * (size_t)m * N);
    u64 *init = calloc(vec, sizeof(u64));
    orc_test_vector_gen(N, m, t, Q, u, lut, v);
    for (uint32_t r = 0; r < m; r++)
        memcpy(init + ((size_t)r * 2 + 1) * N, v + (size_t)r * N, sizeof(u64) * N);
    orc_mmpm_apply_gen(N, m, Q, u, ct[n] % qp, init, acc);
    for (uint32_t k = 0; k < n; k++) {
        uint64_t ak = ct[k] % qp;
        if (k >= n_keys) {
            if (ak != 0) { free(v); free(init); return -1; }
            continue;
        }
        const u64 *Cp = bsk + (size_t)k * 2 * rgsw;
        cmux_gen(p, m, u, ak, Cp, Cp + rgsw, acc, parallel);
    }
    free(v); free(init);
    return 0;
}

/* Algorithm 1 (modulus switches excluded) with a generator per ciphertext:
 * u holds count * m exponents, ciphertext i using u + i * m. */
int orc_bootstrap_gen(const orc_params *p, uint32_t m, uint32_t t, const uint32_t *u,
                      const u64 *bsk, uint32_t n_keys, const u64 *ksk, const uint64_t *ct_in,
                      const uint32_t *luts, size_t count, u64 *ct_out)
{
    uint32_t N = p->N, n = p->n;
    int bad = 0;
    int inner = count == 1;
    #pragma omp parallel for schedule(dynamic) if (!inner) reduction(|:bad)
    for (long ii = 0; ii < (long)count; ii++) {
        size_t i = (size_t)ii;
        u64 *acc = malloc(sizeof(u64) * (size_t)m * 2 * N);
        u64 *lwe = malloc(sizeof(u64) * (N + 1));
        if (orc_blind_rotate_gen(p, m, t, u + i * m, bsk, n_keys, ct_in + i * (n + 1),
                                 luts + i * t, acc, inner) != 0)
            bad = 1;
        orc_sample_extract(N, p->Q, acc, acc + N, lwe);
        orc_key_switch(p, lwe, ksk, ct_out + i * (n + 1));
        free(acc); free(lwe);
    }
    return bad ? -1 : 0;
}

/* ------------------------------------------------------------------------ */
/* Seeded randomness: keys and ciphertexts drawn from a seed                */
/* (Algorithm 1 REQUIRE block: s, z, the keys' masks and errors; Section 2, */
/* (8): encryption masks and errors).  The paper does not fix a generator;  */
/* this is the counter-based Philox4x32-10 of Salmon, Moraes, Dror and      */
/* Shaw, "Parallel random numbers: as easy as 1, 2, 3" (SC'11), written     */
/* here from that definition.  The CUDA library implements the same         */
/* published generator and stream layout independently.                    */
/*                                                                          */
/* Stream layout.  Every random quantity is one Philox block at             */
/*   counter = (i mod 2^32, i >> 32, domain, kind),                         */
/*   key     = (seed mod 2^32, seed >> 32),                                 */
/* where i is the quantity's element index:                                 */
/*   kind 1  LWE secret s_k,            i = k,                   domain 0   */
/*   kind 2  RLWE secret z_i,           i = i,                   domain N   */
/*   kind 3  bootstrapping-key mask,    i = ((k*2+sgn)*2l_B+row)*N + c, N   */
/*   kind 4  bootstrapping-key error,   same i,                  domain N   */
/*   kind 5  key-switching-key mask,    i = row*n + c,           domain N   */
/*   kind 6  key-switching-key error,   i = row,                 domain N   */
/*           (row = (i_N*l_ks + j)*(B_ks-1) + v-1)                          */
/*   kind 7  encryption mask,           i = ct*n + c,            domain 0   */
/*   kind 8  encryption error,          i = ct,                  domain 0   */
/* From the block (w0, w1, w2, w3):                                         */
/*   uniform mod M : (w0 + w1 2^32 + w2 2^64 + w3 2^96) mod M;              */
/*   ternary       : floor(3 w0 / 2^32) - 1;   binary: floor(2 w0 / 2^32);  */
/*   error         : the discrete Gaussian of parameter sigma (standard     */
/*                   deviation, reading R11) on [-41, 41] by inversion of   */
/*                   its cumulative table at r = w0 + w1 2^32 (orc_cdt).    */
/* ------------------------------------------------------------------------ */

#define ORC_ERR_CUT 41

/* Ten Philox rounds; the key is bumped by the Weyl constants before every
 * round but the first. */
void orc_philox4x32_10(const uint32_t ctr[4], const uint32_t key[2], uint32_t out[4])
{
    uint32_t c0 = ctr[0], c1 = ctr[1], c2 = ctr[2], c3 = ctr[3];
    uint32_t k0 = key[0], k1 = key[1];
    for (int r = 0; r < 10; r++) {
        if (r > 0) { k0 += 0x9E3779B9u; k1 += 0xBB67AE85u; }
        uint64_t p0 = (uint64_t)0xD2511F53u * c0;
        uint64_t p1 = (uint64_t)0xCD9E8D57u * c2;
        uint32_t n0 = (uint32_t)(p1 >> 32) ^ c1 ^ k0;
        uint32_t n1 = (uint32_t)p1;
        uint32_t n2 = (uint32_t)(p0 >> 32) ^ c3 ^ k1;
        uint32_t n3 = (uint32_t)p0;
        c0 = n0; c1 = n1; c2 = n2; c3 = n3;
    }
    out[0] = c0; out[1] = c1; out[2] = c2; out[3] = c3;
}

static void stream_block(uint64_t seed, uint32_t kind, uint32_t domain, uint64_t i, uint32_t w[4])
{
    uint32_t ctr[4] = {(uint32_t)i, (uint32_t)(i >> 32), domain, kind};
    uint32_t key[2] = {(uint32_t)seed, (uint32_t)(seed >> 32)};
    orc_philox4x32_10(ctr, key, w);
}

u64 orc_draw_uniform(uint64_t seed, uint32_t kind, uint32_t domain, uint64_t i, u64 modulus)
{
    uint32_t w[4];
    stream_block(seed, kind, domain, i, w);
    u128 U = (u128)w[0] | ((u128)w[1] << 32) | ((u128)w[2] << 64) | ((u128)w[3] << 96);
    return (u64)(U % modulus);
}

int orc_draw_ternary(uint64_t seed, uint32_t kind, uint32_t domain, uint64_t i)
{
    uint32_t w[4];
    stream_block(seed, kind, domain, i, w);
    return (int)(((uint64_t)w[0] * 3u) >> 32) - 1;
}

int orc_draw_binary(uint64_t seed, uint32_t kind, uint32_t domain, uint64_t i)
{
    uint32_t w[4];
    stream_block(seed, kind, domain, i, w);
    return (int)(w[0] >> 31);
}

/* Cumulative table of the discrete Gaussian rho(k) = exp(-k^2 / (2 sigma^2))
 * on k in [-41, 41]: F_j = (rho(-41) + ... + rho(-41 + j)) / S for j in
 * [0, 82), S the sum over all 83 points, both summed in double from -41
 * upward; T_j = floor(F_j 2^64), or 2^64 - 1 where F_j 2^64 >= 2^64 - 1. */
void orc_cdt(double sigma, u64 *T)
{
    double rho[2 * ORC_ERR_CUT + 1];
    double S = 0.0;
    double den = 2.0 * sigma * sigma;
    for (int k = -ORC_ERR_CUT; k <= ORC_ERR_CUT; k++) {
        double x = (double)(k * k) / den;
        rho[k + ORC_ERR_CUT] = exp(-x);
        S += rho[k + ORC_ERR_CUT];
    }
    double F = 0.0;
    for (int j = 0; j < 2 * ORC_ERR_CUT; j++) {
        F += rho[j];
        double v = ldexp(F / S, 64);
        T[j] = v >= 18446744073709551615.0 ? UINT64_MAX : (u64)v;
    }
}

/* Error sample: -41 plus the number of table entries at or below r. */
int orc_draw_gaussian(uint64_t seed, uint32_t kind, uint32_t domain, uint64_t i, const u64 *T)
{
    uint32_t w[4];
    stream_block(seed, kind, domain, i, w);
    u64 r = (u64)w[0] | ((u64)w[1] << 32);
    int e = -ORC_ERR_CUT;
    for (int j = 0; j < 2 * ORC_ERR_CUT; j++)
        if (r >= T[j]) e++;
    return e;
}

/* LWE secret s (kind 1): ternary, or binary when ternary == 0. */
void orc_seeded_lwe_secret(uint32_t n, int ternary, uint64_t seed, int8_t *s)
{
    for (uint32_t k = 0; k < n; k++)
        s[k] = (int8_t)(ternary ? orc_draw_ternary(seed, 1, 0, k) : orc_draw_binary(seed, 1, 0, k));
}

/* RLWE secret z (kind 2, domain N): ternary. */
void orc_seeded_rlwe_secret(uint32_t N, uint64_t seed, int8_t *z)
{
    for (uint32_t i = 0; i < N; i++) z[i] = (int8_t)orc_draw_ternary(seed, 2, N, i);
}

/* Masks and errors of the bootstrapping keys for k in [0, n_keys), laid out
 * as [n_keys][2][2 l_B][N] (the arrays orc_keygen_bsk reads). */
void orc_seeded_bsk_randomness(const orc_params *p, double sigma, uint64_t seed, uint32_t n_keys,
                               u64 *mask, int8_t *err)
{
    u64 T[2 * ORC_ERR_CUT];
    orc_cdt(sigma, T);
    size_t total = (size_t)n_keys * 2 * 2 * p->l_B * p->N;
    #pragma omp parallel for schedule(static)
    for (long ii = 0; ii < (long)total; ii++) {
        mask[ii] = orc_draw_uniform(seed, 3, p->N, (uint64_t)ii, p->Q);
        err[ii] = (int8_t)orc_draw_gaussian(seed, 4, p->N, (uint64_t)ii, T);
    }
}

/* Masks [rows][n] and errors [rows] of the key-switching keys, rows =
 * N l_ks (B_ks - 1) (the arrays orc_keygen_ksk reads). */
void orc_seeded_ksk_randomness(const orc_params *p, double sigma, uint64_t seed, u64 *mask, int8_t *err)
{
    u64 T[2 * ORC_ERR_CUT];
    orc_cdt(sigma, T);
    size_t rows = (size_t)p->N * p->l_ks * ((1u << p->log2_Bks) - 1);
    #pragma omp parallel for schedule(static)
    for (long rr = 0; rr < (long)rows; rr++) {
        for (uint32_t c = 0; c < p->n; c++)
            mask[(size_t)rr * p->n + c] = orc_draw_uniform(seed, 5, p->N, (uint64_t)rr * p->n + c, p->Q);
        err[rr] = (int8_t)orc_draw_gaussian(seed, 6, p->N, (uint64_t)rr, T);
    }
}

/* Encryption masks [count][n] in [0, q) and errors [count] (kinds 7, 8). */
void orc_seeded_enc_randomness(uint32_t n, u64 q, double sigma, uint64_t seed, size_t count,
                               u64 *mask, int8_t *err)
{
    u64 T[2 * ORC_ERR_CUT];
    orc_cdt(sigma, T);
    for (size_t i = 0; i < count; i++) {
        for (uint32_t c = 0; c < n; c++)
            mask[i * n + c] = orc_draw_uniform(seed, 7, 0, (uint64_t)i * n + c, q);
        err[i] = (int8_t)orc_draw_gaussian(seed, 8, 0, (uint64_t)i, T);
    }
}

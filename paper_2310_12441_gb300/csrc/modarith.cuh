// Modular arithmetic in Z_Q, Q < 2^61 prime, for sm_103a.
//
// Multiplication by a fixed operand uses Shoup's precomputed-quotient method
// (V. Shoup, NTL; analysed in D. Harvey, "Faster arithmetic for
// number-theoretic transforms", J. Symb. Comp. 2014): for w in [0, Q) and
// w' = floor(w 2^64 / Q), any a in [0, 2^64) gives
//     a w - floor(a w' / 2^64) Q  in [0, 2Q).
// Products of two variable operands are accumulated exactly in 128 bits
// (mad.lo.cc / madc.hi) and reduced once at the end.
#pragma once
#include <cstdint>

typedef uint64_t u64;
typedef uint32_t u32;

struct ModQ {
    u64 Q;
    u64 two_Q;
    u64 r64;      // 2^64 mod Q
    u64 r64_sh;   // floor(r64 * 2^64 / Q)
    u64 one_sh;   // floor(2^64 / Q): Shoup companion of w = 1
};

__device__ __forceinline__ u64 reduce_2q(u64 x, u64 Q) { return x >= Q ? x - Q : x; }

// a * w mod Q in [0, 2Q), Shoup.
__device__ __forceinline__ u64 mul_shoup_lazy(u64 a, u64 w, u64 wsh, u64 Q) {
    u64 q = __umul64hi(a, wsh);
    return a * w - q * Q;
}

// q * Q mod 2^64; when Q = c 2^32 + 1 (QLOW1), q Q = q + (q mod 2^32) c 2^32
// modulo 2^64, one 32-bit multiply.
template <bool QLOW1>
__device__ __forceinline__ u64 times_q(u64 q, u64 Q) {
    if constexpr (QLOW1) {
        return q + ((u64)((u32)q * (u32)(Q >> 32)) << 32);
    } else {
        return q * Q;
    }
}

// a * w mod Q by Shoup's method with the quotient taken from three of the
// four 32 x 32-bit partial products of a * w': dropping a_lo * w'_lo and the
// carries of the middle terms leaves an estimate at most 2 below
// floor(a w' / 2^64), so a w - q Q lies in [0, 4Q) (needs 4Q < 2^64).  No
// final correction; shoup3 adds one (result in [0, 2Q)).
template <bool QLOW1>
__device__ __forceinline__ u64 shoup3_lazy(u64 a, u64 w, u64 wsh, u64 Q) {
    const u32 a0 = (u32)a, a1 = (u32)(a >> 32);
    const u32 s0 = (u32)wsh, s1 = (u32)(wsh >> 32);
    const u64 q = (u64)a1 * s1 + __umulhi(a1, s0) + __umulhi(a0, s1);
    return a * w - times_q<QLOW1>(q, Q);
}

template <bool QLOW1>
__device__ __forceinline__ u64 shoup3(u64 a, u64 w, u64 wsh, u64 Q, u64 twoQ) {
    const u64 r = shoup3_lazy<QLOW1>(a, w, wsh, Q);
    return r >= twoQ ? r - twoQ : r;
}

__device__ __forceinline__ u64 mul_shoup(u64 a, u64 w, u64 wsh, u64 Q) {
    return reduce_2q(mul_shoup_lazy(a, w, wsh, Q), Q);
}

// 64-bit additions as single 64-bit integer instructions (sm_103a adds 64-bit
// words in one integer-ALU instruction; written out so that they stay off
// the multiplier pipe the modular products need).
__device__ __forceinline__ u64 add64c(u64 a, u64 b) {
    u64 r;
    asm("add.u64 %0, %1, %2;" : "=l"(r) : "l"(a), "l"(b));
    return r;
}

__device__ __forceinline__ u64 sub64c(u64 a, u64 b) {
    u64 r;
    asm("sub.u64 %0, %1, %2;" : "=l"(r) : "l"(a), "l"(b));
    return r;
}

// x >= c ? x - c : x, from the borrow of x - c.
__device__ __forceinline__ u64 csub64(u64 x, u64 c) {
    u64 r;
    asm("{\n\t.reg .u32 x0, x1, c0, c1, d0, d1, m;\n\t.reg .pred p;\n\t"
        "mov.b64 {x0, x1}, %1;\n\tmov.b64 {c0, c1}, %2;\n\t"
        "sub.cc.u32 d0, x0, c0;\n\tsubc.cc.u32 d1, x1, c1;\n\tsubc.u32 m, 0, 0;\n\t"
        "setp.eq.u32 p, m, 0;\n\t"
        "selp.b32 x0, d0, x0, p;\n\tselp.b32 x1, d1, x1, p;\n\t"
        "mov.b64 %0, {x0, x1};\n\t}"
        : "=l"(r) : "l"(x), "l"(c));
    return r;
}

__device__ __forceinline__ u64 add_mod(u64 a, u64 b, u64 Q) { return csub64(add64c(a, b), Q); }

// csub64 for x, c < 2^63: the sign of x - c decides (Q = c 2^32 + 1 keys have
// Q < 2^60, so every value their butterflies correct is below 8Q <= 2^63).
__device__ __forceinline__ u64 csub63(u64 x, u64 c) {
    u64 r;
    asm("{\n\t.reg .u32 x0, x1, c0, c1, d0, d1;\n\t.reg .pred p;\n\t"
        "mov.b64 {x0, x1}, %1;\n\tmov.b64 {c0, c1}, %2;\n\t"
        "sub.cc.u32 d0, x0, c0;\n\tsubc.u32 d1, x1, c1;\n\t"
        "setp.lt.s32 p, d1, 0;\n\t"
        "selp.b32 x0, x0, d0, p;\n\tselp.b32 x1, x1, d1, p;\n\t"
        "mov.b64 %0, {x0, x1};\n\t}"
        : "=l"(r) : "l"(x), "l"(c));
    return r;
}

// a - b mod Q for a, b in [0, Q): a - b, plus Q when a < b (a 64-bit
// compare and select; no borrow word, which would take a multiplier slot).
__device__ __forceinline__ u64 sub_mod(u64 a, u64 b, u64 Q) {
    u64 r;
    asm("{\n\t.reg .u64 d, q;\n\t.reg .pred p;\n\t"
        "setp.lo.u64 p, %1, %2;\n\tsub.u64 d, %1, %2;\n\tselp.b64 q, %3, 0, p;\n\tadd.u64 %0, d, q;\n\t}"
        : "=l"(r) : "l"(a), "l"(b), "l"(Q));
    return r;
}

// (hi:lo) += a * b, exact 128-bit accumulation.
__device__ __forceinline__ void mac128(u64 &lo, u64 &hi, u64 a, u64 b) {
    asm("mad.lo.cc.u64 %0, %2, %3, %0;\n\t"
        "madc.hi.u64 %1, %2, %3, %1;"
        : "+l"(lo), "+l"(hi)
        : "l"(a), "l"(b));
}

// (hi:lo) += a, exact 128-bit accumulation of a 64-bit value (64-bit
// add-with-carry on the integer ALU).
__device__ __forceinline__ void add128(u64 &lo, u64 &hi, u64 a) {
    asm("add.cc.u64 %0, %0, %2;\n\taddc.u64 %1, %1, 0;" : "+l"(lo), "+l"(hi) : "l"(a));
}

// (hi:lo) += v << sh for 0 < sh < 64.
__device__ __forceinline__ void add128_shl(u64 &lo, u64 &hi, u64 v, u32 sh) {
    const u64 vl = v << sh, vh = v >> (64 - sh);
    asm("add.cc.u64 %0, %0, %2;\n\taddc.u64 %1, %1, %3;" : "+l"(lo), "+l"(hi) : "l"(vl), "l"(vh));
}

// (hi 2^64 + lo) mod Q, any hi, lo < 2^64:  hi * (2^64 mod Q) + lo, each term
// Shoup-reduced into [0, 2Q), sum < 4Q < 2^63, then two conditional
// subtractions.
__device__ __forceinline__ u64 reduce128(u64 lo, u64 hi, const ModQ &m) {
    u64 x = mul_shoup_lazy(hi, m.r64, m.r64_sh, m.Q);
    u64 y = lo - __umul64hi(lo, m.one_sh) * m.Q;
    u64 s = x + y;
    if (s >= m.two_Q) s -= m.two_Q;
    if (s >= m.Q) s -= m.Q;
    return s;
}

// reduce128 with the cheaper quotients of Q = c 2^32 + 1 (QLOW1, so Q > 2^32
// and floor(2^64 / Q) < 2^32): hi * (2^64 mod Q) by the three-product Shoup
// ([0, 4Q)), lo by the quotient estimate floor((lo >> 32) floor(2^64/Q) / 2^32),
// at most 2 below floor(lo / Q) ([0, 3Q)); the sum is below 7Q < 2^64.
template <bool QLOW1>
__device__ __forceinline__ u64 reduce128q(u64 lo, u64 hi, const ModQ &m) {
    if constexpr (QLOW1) {
        const u64 Q = m.Q;
        const u64 x = shoup3_lazy<true>(hi, m.r64, m.r64_sh, Q);
        const u32 qe = __umulhi((u32)(lo >> 32), (u32)m.one_sh);
        u64 s = x + (lo - times_q<true>(qe, Q));
        s = csub63(s, 2 * m.two_Q);
        s = csub63(s, m.two_Q);
        s = csub63(s, Q);
        return s;
    } else {
        return reduce128(lo, hi, m);
    }
}

// Lazy forward (Cooley-Tukey) butterfly for Q = c 2^32 + 1: the seven
// products of the three-product Shoup quotient, the low word of Y W and q Q
// take the multiplier; the additions are single 64-bit ALU instructions:
//   q = y1 s1 + hi(y1 s0) + hi(y0 s1)           (Wsh = s1:s0, Y = y1:y0)
//   T = Y W - q Q  mod 2^64, in [0, 4Q)          (q Q = q + (q0 c) 2^32)
//   X <- X + T,  Y <- X + 4Q - T.
__device__ __forceinline__ void bfly_lazy_qlow1(u64 &X, u64 &Y, u64 W, u64 Wsh, u32 c, u64 fourQ) {
    asm("{\n\t"
        ".reg .u32 y0, y1, w0, w1, s0, s1, h1, h2, q0, q1, t0, t1, qc;\n\t"
        ".reg .u64 q, t, hw, h2w, qq, x;\n\t"
        "mov.b64 {y0, y1}, %1;\n\tmov.b64 {w0, w1}, %2;\n\tmov.b64 {s0, s1}, %3;\n\t"
        "mul.hi.u32 h1, y1, s0;\n\tmul.hi.u32 h2, y0, s1;\n\t"
        "mov.b64 hw, {h1, 0};\n\tmad.wide.u32 q, y1, s1, hw;\n\t"
        "mov.b64 h2w, {h2, 0};\n\tadd.u64 q, q, h2w;\n\t"
        "mov.b64 {q0, q1}, q;\n\t"
        "mul.wide.u32 t, y0, w0;\n\tmov.b64 {t0, t1}, t;\n\t"
        "mad.lo.u32 t1, y0, w1, t1;\n\tmad.lo.u32 t1, y1, w0, t1;\n\t"
        "mad.lo.u32 qc, q0, %4, q1;\n\t"
        "mov.b64 t, {t0, t1};\n\tmov.b64 qq, {q0, qc};\n\tsub.u64 t, t, qq;\n\t"
        "mov.b64 x, %0;\n\tadd.u64 %0, x, t;\n\tadd.u64 x, x, %5;\n\tsub.u64 %1, x, t;\n\t}"
        : "+l"(X), "+l"(Y)
        : "l"(W), "l"(Wsh), "r"(c), "l"(fourQ));
}

// Three-product Shoup product for Q = c 2^32 + 1 (see bfly_lazy_qlow1):
// Y W - q Q mod 2^64 in [0, 4Q).
__device__ __forceinline__ u64 shoup3_qlow1_lazy(u64 Y, u64 W, u64 Wsh, u32 c) {
    u64 T;
    asm("{\n\t"
        ".reg .u32 y0, y1, w0, w1, s0, s1, h1, h2, q0, q1, t0, t1, qc;\n\t"
        ".reg .u64 q, t, hw, h2w, qq;\n\t"
        "mov.b64 {y0, y1}, %1;\n\tmov.b64 {w0, w1}, %2;\n\tmov.b64 {s0, s1}, %3;\n\t"
        "mul.hi.u32 h1, y1, s0;\n\tmul.hi.u32 h2, y0, s1;\n\t"
        "mov.b64 hw, {h1, 0};\n\tmad.wide.u32 q, y1, s1, hw;\n\t"
        "mov.b64 h2w, {h2, 0};\n\tadd.u64 q, q, h2w;\n\t"
        "mov.b64 {q0, q1}, q;\n\t"
        "mul.wide.u32 t, y0, w0;\n\tmov.b64 {t0, t1}, t;\n\t"
        "mad.lo.u32 t1, y0, w1, t1;\n\tmad.lo.u32 t1, y1, w0, t1;\n\t"
        "mad.lo.u32 qc, q0, %4, q1;\n\t"
        "mov.b64 t, {t0, t1};\n\tmov.b64 qq, {q0, qc};\n\tsub.u64 %0, t, qq;\n\t}"
        : "=l"(T)
        : "l"(Y), "l"(W), "l"(Wsh), "r"(c));
    return T;
}

// Forward butterfly with one correction for Q = c 2^32 + 1 (Harvey's method
// with the invariant widened to [0, 8Q), which Q < 2^60 keeps below 2^63):
// X' = X mod 4Q in [0, 4Q), T = Y W mod Q in [0, 4Q) uncorrected;
// X <- X' + T, Y <- X' + 4Q - T, both in [0, 8Q).
__device__ __forceinline__ void bfly_ct_qlow1(u64 &X, u64 &Y, u64 W, u64 Wsh, u32 c, u64 fourQ) {
    const u64 Xr = csub63(X, fourQ);
    const u64 T = shoup3_qlow1_lazy(Y, W, Wsh, c);
    X = add64c(Xr, T);
    Y = sub64c(add64c(Xr, fourQ), T);
}

// Gentleman-Sande inverse butterfly with one correction, Q = c 2^32 + 1,
// values in [0, 4Q): U <- (U + V) mod 4Q, V <- (U - V + 4Q) W mod Q in
// [0, 4Q) uncorrected (the Shoup input stays below 8Q < 2^64).
__device__ __forceinline__ void bfly_gs_qlow1(u64 &U, u64 &V, u64 W, u64 Wsh, u32 c, u64 fourQ) {
    const u64 u = csub63(add64c(U, V), fourQ);
    V = shoup3_qlow1_lazy(sub64c(add64c(U, fourQ), V), W, Wsh, c);
    U = u;
}

// First forward stage on small digits (LAZY with SMALL0): y < 2^32, so W y is
// formed exactly, W y = w0 y + (w1 y) 2^32, and left unreduced:
// X <- X + W y, Y <- X - W y + qb (qb = Q B >= W y).
__device__ __forceinline__ void small_bfly(u64 &X, u64 &Y, u64 W, u64 qb) {
    asm("{\n\t.reg .u32 y0, w0, w1, t0, t1;\n\t.reg .u64 t, x;\n\t"
        "cvt.u32.u64 y0, %1;\n\tmov.b64 {w0, w1}, %2;\n\t"
        "mul.wide.u32 t, w0, y0;\n\tmov.b64 {t0, t1}, t;\n\t"
        "mad.lo.u32 t1, w1, y0, t1;\n\tmov.b64 t, {t0, t1};\n\t"
        "mov.b64 x, %0;\n\tadd.u64 %0, x, t;\n\tadd.u64 x, x, %3;\n\tsub.u64 %1, x, t;\n\t}"
        : "+l"(X), "+l"(Y)
        : "l"(W), "l"(qb));
}

// y W mod Q for a digit y < 2^32 and Q = c 2^32 + 1, in [0, 3Q): the Shoup
// quotient floor(y W' / 2^64) of W' = s1 2^32 + s0 is floor(y s1 / 2^32) or
// one more (y s0 / 2^64 < 1), so q = hi(y s1) leaves y W - q Q in [0, 3Q);
// q < 2^32, so q Q mod 2^64 = q + (q c mod 2^32) 2^32.
__device__ __forceinline__ u64 small_mul_qlow1(u64 y, u64 W, u64 Wsh, u32 c) {
    u64 T;
    asm("{\n\t.reg .u32 y0, w0, w1, s0, s1, q, t0, t1, qc;\n\t.reg .u64 t, qq;\n\t"
        "cvt.u32.u64 y0, %1;\n\t"
        "mov.b64 {w0, w1}, %2;\n\tmov.b64 {s0, s1}, %3;\n\t"
        "mul.hi.u32 q, y0, s1;\n\t"
        "mul.wide.u32 t, y0, w0;\n\tmov.b64 {t0, t1}, t;\n\t"
        "mad.lo.u32 t1, y0, w1, t1;\n\t"
        "mul.lo.u32 qc, q, %4;\n\t"
        "mov.b64 t, {t0, t1};\n\tmov.b64 qq, {q, qc};\n\tsub.u64 %0, t, qq;\n\t}"
        : "=l"(T) : "l"(y), "l"(W), "l"(Wsh), "r"(c));
    return T;
}

// v - qe Q with qe = floor((v >> 32) s / 2^32), s = floor(2^64 / Q) < 2^32,
// Q = c 2^32 + 1: qe is at most 2 below floor(v / Q), result in [0, 3Q).
__device__ __forceinline__ u64 reduce_est_qlow1(u64 v, u32 s, u32 c) {
    u64 r;
    asm("{\n\t.reg .u32 v0, v1, qe, qc;\n\t.reg .u64 qq;\n\t"
        "mov.b64 {v0, v1}, %1;\n\t"
        "mul.hi.u32 qe, v1, %2;\n\t"
        "mul.lo.u32 qc, qe, %3;\n\t"
        "mov.b64 qq, {qe, qc};\n\tsub.u64 %0, %1, qq;\n\t}"
        : "=l"(r) : "l"(v), "r"(s), "r"(c));
    return r;
}

// Gentleman-Sande inverse butterfly without corrections (Q = c 2^32 + 1):
// U <- U + V, V <- (U - V + q64) W mod Q in [0, 4Q), where q64 is a multiple
// of Q above every V.  Values below b grow to below max(2b, 4Q) per stage;
// the caller reduces them between radix-16 phases (see ntr::inv_from_smem).
__device__ __forceinline__ void bfly_gs_lazy_qlow1(u64 &U, u64 &V, u64 W, u64 Wsh, u32 c, u64 q64) {
    const u64 u = add64c(U, V);
    V = shoup3_qlow1_lazy(sub64c(add64c(U, q64), V), W, Wsh, c);
    U = u;
}

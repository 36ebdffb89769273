// Register-resident negacyclic NTT over Z_Q for batches of polynomials.
//
// Same transform as ntt.cuh (Cooley-Tukey forward with psi^bitrev twiddles,
// bit-reversed output; Gentleman-Sande inverse without the N^-1 factor), but
// each thread holds R = 2^RB coefficients of one polynomial in registers and
// performs up to RB butterfly stages on them (a radix-R phase); between
// phases the block exchanges values through shared memory.  A polynomial of
// N = 2^LOGN coefficients takes T = N/R threads and ceil(LOGN/RB) phases.
// The radix is a template parameter (R = 16 or 8): fewer values per thread
// need fewer registers, so more threads fit on an SM, at the price of more
// exchanges.
//
// Phase layouts: a thread of a phase whose RB-bit field sits at bits
// [F, F+RB) of the coefficient index holds the R indices that differ only
// in that field; its thread number l supplies the other bits (the bits below
// F first).  Forward phases take the fields from the top down
// (F = LOGN-RB, LOGN-2RB, ..., then 0), inverse phases from the bottom up
// (F = 0, RB, 2RB, ..., then LOGN-RB).  Stage s of the forward transform
// acts on index bit LOGN-1-s, stage s of the inverse on bit s; a butterfly
// group is the index shifted right past that bit.
//
// Butterflies are Harvey's lazy ones (D. Harvey, "Faster arithmetic for
// number-theoretic transforms", J. Symb. Comp. 2014): forward values stay in
// [0, 4Q), inverse values in [0, 2Q); twiddle products use the three-product
// Shoup quotient of modarith.cuh (with a one-multiply q Q when Q = c 2^32 + 1).
// Twiddles come as (w, w') pairs.
//
// Shared memory: every polynomial owns two regions of N words and the
// exchanges alternate between them (Swap): the store ending phase p goes to
// the region phase p-1 loaded from.  Index idx is stored at word
// idx ^ ((idx >> RB) & 15), which keeps every phase's accesses (and
// position-major accesses) free of bank conflicts for R = 8 and 16 (each
// half-warp touches 16 distinct words modulo 16).
//
// Synchronisation between phases: thread bit t of layout F carries index bit
// t (t < F) or t + RB (t >= F).  When no warp bit (t >= 5) changes its index
// bit between the storing and the loading layout (max(F, G) <= 5, or the
// polynomial fits in one warp), every warp reads back exactly the words it
// wrote, and __syncwarp() orders the exchange; then no other warp read those
// words in the previous phase either, so the store after next may reuse the
// region.  Otherwise the T threads of the polynomial meet at a named barrier
// (bar.sync 1 + polynomial, T).  The regions alternate across batches too:
// the multiply-accumulate of the previous batch reads the result region of
// every polynomial, which the second store of the next forward transform
// rewrites, so the caller orders those reads before that store (the
// before2 hook of fwd_to_smem).
#pragma once
#include "modarith.cuh"

namespace ntr {

template <int RB>
__device__ __forceinline__ u32 swz(u32 idx) { return idx ^ ((idx >> RB) & 15u); }

template <int RB, int F>
__device__ __forceinline__ u32 fidx(u32 l, u32 i) {
    return ((l >> F) << (F + RB)) | (i << F) | (l & ((1u << F) - 1u));
}

// The two shared regions of one polynomial; `next` is the one written next.
struct Swap {
    u64 *r0, *r1;
    int next;
    __device__ __forceinline__ u64 *take() {
        u64 *d = next ? r1 : r0;
        next ^= 1;
        return d;
    }
};

// Exchange between a phase storing in layout F and one loading in layout G
// stays within each warp (see the header).
template <int LOGN, int RB, int F, int G>
__host__ __device__ constexpr bool warp_local() {
    return LOGN - RB <= 5 || (F > G ? F : G) <= 5;
}

// Barrier of the T = 2^(LOGN-RB) threads of this thread's polynomial
// (T > 32; polynomial g = threadIdx.x / T uses barrier 1 + g).
template <int LOGN, int RB>
__device__ __forceinline__ void group_sync() {
    constexpr int T = 1 << (LOGN - RB);
    static_assert(T % 32 == 0, "whole warps per polynomial");
    asm volatile("bar.sync %0, %1;" ::"r"(1u + threadIdx.x / T), "n"(T) : "memory");
}

// Orders the exchange from layout F to layout G (BLOCK: a block barrier).
template <int LOGN, int RB, int F, int G, bool BLOCK = false>
__device__ __forceinline__ void phase_sync() {
    if constexpr (BLOCK) {
        __syncthreads();
    } else if constexpr (warp_local<LOGN, RB, F, G>()) {
        __syncwarp();
    } else {
        group_sync<LOGN, RB>();
    }
}

// Field start of forward phase t (t = 0 .. NPH-1) and of inverse phase t.
template <int LOGN, int RB>
__host__ __device__ constexpr int fwd_field(int t) {
    return t < (LOGN + RB - 1) / RB - 1 ? LOGN - RB * (t + 1) : 0;
}
template <int LOGN, int RB>
__host__ __device__ constexpr int inv_field(int t) {
    return t < (LOGN + RB - 1) / RB - 1 ? RB * t : LOGN - RB;
}

// Twiddle pair ti from a table in global memory, or in shared memory (SH).
template <bool SH = false>
__device__ __forceinline__ void twiddle(const u64 *__restrict__ tp, u32 ti, u64 &W, u64 &Wsh) {
    ulonglong2 v;
    if constexpr (SH) {
        v = reinterpret_cast<const ulonglong2 *>(tp)[ti];
    } else {
        v = __ldg(reinterpret_cast<const ulonglong2 *>(tp) + ti);
    }
    W = v.x;
    Wsh = v.y;
}

// Forward phase: NST stages starting at global stage S0, field [F, F+RB).
// LAZY: no per-stage corrections.  Products lie in [0, 4Q) and the sum and
// difference X + T, X - T + 4Q each grow the bound by 4Q, so inputs below Q
// leave the last stage below (1 + 4 LOGN) Q, which the caller guarantees
// fits in 64 bits.  Otherwise Harvey's [0, 4Q) invariant is kept, widened to
// [0, 8Q) with a single correction per butterfly when Q = c 2^32 + 1
// (bfly_ct_qlow1).
// SMALL0: the first stage's inputs are digits below B <= 2^32.  With
// Q = c 2^32 + 1 the product W Y takes the one-high-product quotient of
// small_mul_qlow1 ([0, 3Q)), and X + T, X - T + 4Q stay below B + 4Q (within
// both invariants).  Otherwise (LAZY only) W * Y is formed exactly (a
// 64 x 32-bit product) and left unreduced: X + W Y and X - W Y + Q B, both
// below B + Q B; the caller guarantees B + Q B + 4 Q (LOGN - 1) < 2^64.
template <int LOGN, int RB, int F, int S0, int NST, bool LAZY, bool SMALL0 = false, bool QLOW1 = false,
          bool TWS = false>
__device__ __forceinline__ void fwd_phase(u64 (&x)[1 << RB], u32 l, const u64 *__restrict__ twp, u64 Q,
                                          u64 twoQ, u64 qb = 0) {
    constexpr int R = 1 << RB;
    const u32 high = l >> F;
#pragma unroll
    for (int st = 0; st < NST; st++) {
        const int s = S0 + st;
        const int lb = LOGN - 1 - s - F;
#pragma unroll
        for (int i = 0; i < R; i++) {
            if (i & (1 << lb)) continue;
            const int i2 = i | (1 << lb);
            const u32 g = (high << (RB - 1 - lb)) | (u32)(i >> (lb + 1));
            u64 W, Wsh;
            if constexpr (TWS) {
                // shared table in the per-stage transposed order of
                // twiddle_slot(): the thread part of g runs fastest
                twiddle<true>(twp, (1u << s) + ((u32)(i >> (lb + 1)) << (LOGN - RB - F)) + high, W, Wsh);
            } else {
                twiddle<false>(twp, (1u << s) + g, W, Wsh);
            }
            if constexpr (SMALL0 && QLOW1 && S0 == 0) {
                if (st == 0) {
                    // digits below B <= 2^32: one high product for the quotient
                    const u64 X = x[i];
                    const u64 T = small_mul_qlow1(x[i2], W, Wsh, (u32)(Q >> 32));
                    x[i] = add64c(X, T);
                    x[i2] = sub64c(add64c(X, 2 * twoQ), T);
                    continue;
                }
            } else if constexpr (LAZY && SMALL0 && S0 == 0) {
                if (st == 0) {
                    small_bfly(x[i], x[i2], W, qb);
                    continue;
                }
            }
            if constexpr (LAZY && QLOW1) {
                bfly_lazy_qlow1(x[i], x[i2], W, Wsh, (u32)(Q >> 32), 2 * twoQ);
            } else if constexpr (LAZY) {
                const u64 X = x[i];
                const u64 T = shoup3_lazy<QLOW1>(x[i2], W, Wsh, Q);
                x[i] = X + T;
                x[i2] = X - T + 2 * twoQ;
            } else if constexpr (QLOW1) {
                bfly_ct_qlow1(x[i], x[i2], W, Wsh, (u32)(Q >> 32), 2 * twoQ);
            } else {
                u64 X = x[i];
                X = X >= twoQ ? X - twoQ : X;
                const u64 T = shoup3<QLOW1>(x[i2], W, Wsh, Q, twoQ);
                x[i] = X + T;
                x[i2] = X - T + twoQ;
            }
        }
    }
}

// Inverse phase: NST stages acting on bits SB, SB+1, ..., field [F, F+RB).
template <int LOGN, int RB, int F, int SB, int NST, bool QLOW1 = false, bool TWS = false, bool LZI = false>
__device__ __forceinline__ void inv_phase(u64 (&x)[1 << RB], u32 l, const u64 *__restrict__ itwp, u64 Q,
                                          u64 twoQ) {
    constexpr int R = 1 << RB;
    const u32 high = l >> F;
#pragma unroll
    for (int st = 0; st < NST; st++) {
        const int b = SB + st;
        const int lb = b - F;
#pragma unroll
        for (int i = 0; i < R; i++) {
            if (i & (1 << lb)) continue;
            const int i2 = i | (1 << lb);
            const u32 g = (high << (RB - 1 - lb)) | (u32)(i >> (lb + 1));
            u64 W, Wsh;
            if constexpr (TWS) {
                // shared table in the transposed order of inv_twiddle_slot()
                twiddle<true>(itwp, (1u << (LOGN - 1 - b)) + ((u32)(i >> (lb + 1)) << (LOGN - RB - F)) + high, W,
                              Wsh);
            } else {
                twiddle<false>(itwp, (1u << (LOGN - 1 - b)) + g, W, Wsh);
            }
            if constexpr (LZI) {
                bfly_gs_lazy_qlow1(x[i], x[i2], W, Wsh, (u32)(Q >> 32), Q << 6);
            } else if constexpr (QLOW1) {
                bfly_gs_qlow1(x[i], x[i2], W, Wsh, (u32)(Q >> 32), 2 * twoQ);
            } else {
                const u64 U = x[i], V = x[i2];
                u64 u = U + V;
                u = u >= twoQ ? u - twoQ : u;
                x[i] = u;
                x[i2] = shoup3<QLOW1>(U - V + twoQ, W, Wsh, Q, twoQ);
            }
        }
    }
}

// Index into the plain forward table (psi^bitrev(k) at k = 2^s + g) of slot
// `pos` of the transposed shared-memory copy read by fwd_phase<..., TWS>.
// Stage s sits in the phase whose field starts at F; there g = (high << a) | j
// with the thread part high = l >> F below 2^(LOGN-RB-F) and the register
// part j below 2^a, a = s - (LOGN-RB-F); slot 2^s + j 2^(LOGN-RB-F) + high
// holds it, so the threads of a warp read consecutive slots (no bank
// conflicts).
template <int LOGN, int RB>
__device__ __forceinline__ u32 twiddle_slot(u32 pos) {
    if (pos == 0) return 0;
    constexpr u32 NPH = (LOGN + RB - 1) / RB;
    const u32 s = 31 - __clz(pos);
    const u32 ph = s / RB;
    const u32 F = ph < NPH - 1 ? LOGN - RB - RB * ph : 0;
    const u32 sh = LOGN - RB - F;
    const u32 r = pos - (1u << s);
    const u32 j = r >> sh, high = r & ((1u << sh) - 1);
    return (1u << s) + ((high << (s - sh)) | j);
}

// The same for the inverse table (psi^-bitrev(k) at k = 2^s + g, used by the
// inverse stage on bit LOGN-1-s, which sits in the inverse phase with field F).
template <int LOGN, int RB>
__device__ __forceinline__ u32 inv_twiddle_slot(u32 pos) {
    if (pos == 0) return 0;
    constexpr u32 NPH = (LOGN + RB - 1) / RB;
    const u32 s = 31 - __clz(pos);
    const u32 q = (LOGN - 1 - s) / RB;
    const u32 F = q < NPH - 1 ? RB * q : LOGN - RB;
    const u32 sh = LOGN - RB - F;
    const u32 r = pos - (1u << s);
    const u32 j = r >> sh, high = r & ((1u << sh) - 1);
    return (1u << s) + ((high << (s - sh)) | j);
}

// Field accesses.  fidx(l, i) = fidx(l, 0) | (i << F) with disjoint bits, and
// the swizzle is linear over XOR on disjoint bits, so word
// swz(fidx(l, i)) = swz(fidx(l, 0)) ^ swz(i << F): one byte offset per thread
// XOR a compile-time constant per register (the address arithmetic stays on
// the integer ALU, off the multiplier the butterflies need).
template <int RB, int F>
__device__ __forceinline__ void store_field(const u64 (&x)[1 << RB], u64 *reg, u32 l) {
    char *b = reinterpret_cast<char *>(reg);
    const u32 sb = swz<RB>(fidx<RB, F>(l, 0)) << 3;
#pragma unroll
    for (int i = 0; i < (1 << RB); i++)
        *reinterpret_cast<u64 *>(b + (sb ^ (swz<RB>((u32)i << F) << 3))) = x[i];
}

template <int RB, int F>
__device__ __forceinline__ void load_field(u64 (&x)[1 << RB], const u64 *reg, u32 l) {
    const char *b = reinterpret_cast<const char *>(reg);
    const u32 sb = swz<RB>(fidx<RB, F>(l, 0)) << 3;
#pragma unroll
    for (int i = 0; i < (1 << RB); i++)
        x[i] = *reinterpret_cast<const u64 *>(b + (sb ^ (swz<RB>((u32)i << F) << 3)));
}

// Middle forward phases PH = 1 .. NPH-2 (field LOGN - RB (PH + 1)); `r` holds
// the previous phase's layout and its exchange has been ordered.  Returns the
// region holding the last middle phase's output.
template <int LOGN, int RB, int PH, bool LAZY, bool QLOW1, bool TWS, class Before2>
__device__ __forceinline__ u64 *fwd_middle(u64 (&x)[1 << RB], Swap &sw, u64 *r, u32 l, bool active,
                                           const u64 *__restrict__ twp, u64 Q, u64 twoQ, Before2 &before2) {
    constexpr int NPH = (LOGN + RB - 1) / RB;
    if constexpr (PH < NPH - 1) {
        constexpr int F = fwd_field<LOGN, RB>(PH), G = fwd_field<LOGN, RB>(PH + 1);
        if constexpr (PH == 1) before2();
        if (active) {
            load_field<RB, F>(x, r, l);
            fwd_phase<LOGN, RB, F, RB * PH, RB, LAZY, false, QLOW1, TWS>(x, l, twp, Q, twoQ);
        }
        u64 *r2 = sw.take();
        if (active) store_field<RB, F>(x, r2, l);
        phase_sync<LOGN, RB, F, G>();
        return fwd_middle<LOGN, RB, PH + 1, LAZY, QLOW1, TWS>(x, sw, r2, l, active, twp, Q, twoQ, before2);
    } else {
        return r;
    }
}

// Forward NTT.  On entry x holds indices l + T i (field [LOGN-RB, LOGN)) of
// this thread's polynomial, values below 4Q.  TWS: twp points to a copy of
// the twiddle pairs in shared memory.  Returns the region that holds
// the transform in bit-reversed positions, values in [0, Q), or with LAZY
// left for the multiply-accumulate (whose limbs are planned for it): below
// (1 + 4 LOGN) Q unreduced when QLOW1, else [0, 2Q) (swizzled); the caller
// must __syncthreads() before reading it.
// The regions alternate across transforms, so the second store of this
// transform goes to the region that held the previous transform's result.
// before2() runs in every thread before that store, between the first
// exchange and the second phase (where the thread holds no values in
// registers): the caller makes it wait until every reader of the previous
// results is done.  The first store goes to the other region, which only
// this polynomial's threads used last, before the caller's barrier that
// precedes its reads.
// Every thread of the block calls this (it contains barriers); threads with
// active == false (whole polynomials) only take part in the barriers.
template <int LOGN, int RB, bool LAZY, bool SMALL0, bool QLOW1, bool TWS, class Before2>
__device__ __forceinline__ u64 *fwd_to_smem(u64 (&x)[1 << RB], Swap &sw, u32 l, bool active,
                                            const u64 *__restrict__ twp, u64 Q, u64 one_sh, u64 qb,
                                            Before2 &&before2) {
    constexpr int R = 1 << RB;
    constexpr int NPH = (LOGN + RB - 1) / RB;
    static_assert(LOGN >= 8 && LOGN <= 13, "ring degree 256..8192");
    static_assert(RB == 3 || RB == 4, "radix 8 or 16");
    const u64 twoQ = 2 * Q;
    if (active) fwd_phase<LOGN, RB, LOGN - RB, 0, RB, LAZY, SMALL0, QLOW1, TWS>(x, l, twp, Q, twoQ, qb);
    u64 *r = sw.take();
    if (active) store_field<RB, LOGN - RB>(x, r, l);
    phase_sync<LOGN, RB, fwd_field<LOGN, RB>(0), fwd_field<LOGN, RB>(1)>();
    r = fwd_middle<LOGN, RB, 1, LAZY, QLOW1, TWS>(x, sw, r, l, active, twp, Q, twoQ, before2);
    if constexpr (NPH == 2) before2();
    if (active) {
        load_field<RB, 0>(x, r, l);
        fwd_phase<LOGN, RB, 0, RB * (NPH - 1), LOGN - RB * (NPH - 1), LAZY, false, QLOW1, TWS>(x, l, twp, Q, twoQ);
#pragma unroll
        for (int i = 0; i < R; i++) {
            u64 v = x[i];
            if constexpr (LAZY && QLOW1) {
                // left below (1 + 4 LOGN) Q for the multiply-accumulate
            } else if constexpr (LAZY) {
                v = v - __umul64hi(v, one_sh) * Q;     // Shoup with w = 1: [0, 2Q)
            } else if constexpr (QLOW1) {
                v = csub63(csub63(csub63(v, 2 * twoQ), twoQ), Q);     // [0, 8Q) -> [0, Q)
            } else {
                v = csub64(csub64(v, twoQ), Q);
            }
            x[i] = v;
        }
    }
    r = sw.take();
    if (active) store_field<RB, 0>(x, r, l);
    return r;
}

// Middle inverse phases QP = 1 .. NPH-2 (field RB QP).
template <int LOGN, int RB, int QP, bool QLOW1, bool TWS, bool LZI>
__device__ __forceinline__ u64 *inv_middle(u64 (&x)[1 << RB], Swap &sw, u64 *r, u32 l, bool active,
                                           const u64 *__restrict__ itwp, u64 Q, u64 twoQ, u64 one_sh) {
    constexpr int NPH = (LOGN + RB - 1) / RB;
    if constexpr (QP < NPH - 1) {
        constexpr int F = inv_field<LOGN, RB>(QP), G = inv_field<LOGN, RB>(QP + 1);
        if (active) {
            load_field<RB, F>(x, r, l);
            inv_phase<LOGN, RB, F, F, RB, QLOW1, TWS, LZI>(x, l, itwp, Q, twoQ);
            if constexpr (LZI) {
#pragma unroll
                for (int i = 0; i < (1 << RB); i++) x[i] = reduce_est_qlow1(x[i], (u32)one_sh, (u32)(Q >> 32));
            }
        }
        u64 *r2 = sw.take();
        if (active) store_field<RB, F>(x, r2, l);
        phase_sync<LOGN, RB, F, G>();
        return inv_middle<LOGN, RB, QP + 1, QLOW1, TWS, LZI>(x, sw, r2, l, active, itwp, Q, twoQ, one_sh);
    } else {
        return r;
    }
}

// Inverse NTT (without N^-1).  On entry region `in` holds the bit-reversed
// transform (swizzled, values below 2Q) and the block has passed a barrier
// since it was written; `in` must be the region sw wrote last, and no other
// polynomial's threads read this polynomial's regions until the caller's next
// block barrier.  On exit x holds natural-order coefficients l + T i, reduced
// to [0, Q).  With Q = c 2^32 + 1 the butterflies keep [0, 4Q) with one
// correction each (bfly_gs_qlow1), or with LZI (Q = c 2^32 + 1 and
// 128 Q < 2^64) none (bfly_gs_lazy_qlow1 with q64 = 64 Q).  A phase of four
// stages takes values below 3Q to below 48Q (3Q, 6Q, 12Q, 24Q, 48Q; inputs
// below Q reach 32Q; three stages stop at 24Q), so U - V + 64Q < 112Q < 2^64;
// between phases the values are brought back below 3Q by reduce_est_qlow1
// (one_sh = floor(2^64 / Q)).
template <int LOGN, int RB, bool QLOW1 = false, bool TWS = false, bool LZI = false>
__device__ __forceinline__ void inv_from_smem(u64 (&x)[1 << RB], const u64 *in, Swap &sw, u32 l, bool active,
                                              const u64 *__restrict__ itwp, u64 Q, u64 one_sh = 0) {
    constexpr int R = 1 << RB;
    constexpr int NPH = (LOGN + RB - 1) / RB;
    const u64 twoQ = 2 * Q;
    auto between = [&]() {
        if constexpr (LZI) {
#pragma unroll
            for (int i = 0; i < R; i++) x[i] = reduce_est_qlow1(x[i], (u32)one_sh, (u32)(Q >> 32));
        }
    };
    if (active) {
        load_field<RB, 0>(x, in, l);
        inv_phase<LOGN, RB, 0, 0, RB, QLOW1, TWS, LZI>(x, l, itwp, Q, twoQ);
        between();
    }
    u64 *r = sw.take();
    if (active) store_field<RB, 0>(x, r, l);
    phase_sync<LOGN, RB, inv_field<LOGN, RB>(0), inv_field<LOGN, RB>(1)>();
    r = inv_middle<LOGN, RB, 1, QLOW1, TWS, LZI>(x, sw, r, l, active, itwp, Q, twoQ, one_sh);
    if (active) {
        load_field<RB, LOGN - RB>(x, r, l);
        inv_phase<LOGN, RB, LOGN - RB, RB * (NPH - 1), LOGN - RB * (NPH - 1), QLOW1, TWS, LZI>(x, l, itwp, Q,
                                                                                             twoQ);
        between();
#pragma unroll
        for (int i = 0; i < R; i++)
            x[i] = (LZI || QLOW1) ? csub63(csub63(x[i], twoQ), Q) : csub64(x[i], Q);
    }
}

}  // namespace ntr

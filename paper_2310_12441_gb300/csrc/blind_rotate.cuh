// Blind rotation of BootMMPM (arXiv 2310.12441, Algorithm 1, phase
// accumulation) for one job per thread block; included by the kernels that
// launch it (one block per job, or a persistent block pulling jobs).
#pragma once
#include "common.cuh"
#include "ntt_reg.cuh"
#include <atomic>

// ---------------------------------------------------------------------------
// Device helpers
// ---------------------------------------------------------------------------

// Coefficient `c` of x^e * p in R_{N,Q}, e in [0, 2N).
__device__ __forceinline__ u64 rotated_coeff(const u64 *p, u32 c, u32 e, u32 N, u64 Q) {
    u32 j = c + 2 * N - e;
    if (j >= 2 * N) j -= 2 * N;
    if (j < N) return p[j];
    const u64 v = p[j - N];
    return v ? Q - v : 0;
}

__device__ __forceinline__ void set_status(u32 *status, bm_status code) {
    atomicCAS(status, 0u, (u32)(-code));
}

// Negacyclic table check: entries in [0, t) and f(k + t/2) = -f(k) mod t.
static __device__ bool lut_is_negacyclic(const u32 *__restrict__ lut, u32 t) {
    __shared__ int bad;
    if (threadIdx.x == 0) bad = 0;
    __syncthreads();
    for (u32 k = threadIdx.x; k < t / 2; k += blockDim.x) {
        const u32 a = lut[k], b = lut[k + t / 2];
        if (a >= t || b >= t || b != (t - a) % t) bad = 1;
    }
    __syncthreads();
    const bool ok = bad == 0;
    __syncthreads();
    return ok;
}

// ACC <- P(b) (0, v_test floor(Q/t)), v_test of Eq. (equ:test-use):
// row i, coefficient a of v_test is f'(-(a m + i) mod 2Nm), with the
// negacyclic extension f'(u) = f(floor((u t + Nm) / 2Nm) mod t).
static __device__ void acc_init(u64 *__restrict__ acc, const u32 *__restrict__ lut, u64 b, u32 m, u32 t,
                         u32 N, u64 Q) {
    const u64 qp = 2ull * N * m;
    const u64 dq = Q / t;
    const u32 ea = (u32)(b / m), bb = (u32)(b % m);
    for (u32 idx = threadIdx.x; idx < m * 2 * N; idx += blockDim.x) {
        const u32 c = idx % N;
        const u32 comp = (idx / N) & 1;
        const u32 i = idx / (2 * N);
        u64 val = 0;
        if (comp == 1) {
            const u32 src = i >= bb ? i - bb : i + m - bb;
            u32 e = i >= bb ? ea : ea + 1;
            if (e >= 2 * N) e -= 2 * N;
            u32 j = c + 2 * N - e;
            if (j >= 2 * N) j -= 2 * N;
            const bool neg = j >= N;
            if (neg) j -= N;
            const u64 w = ((u64)j * m + src) % qp;
            const u64 u = (qp - w) % qp;
            const u32 fi = (u32)(((u * t + qp / 2) / qp) % t);
            const u64 v = (u64)lut[fi] * dq;     // < t * floor(Q/t) <= Q
            val = neg ? (v ? Q - v : 0) : v;
        }
        acc[idx] = val;
    }
}

// ---------------------------------------------------------------------------
// Blind rotation kernel: one job per block of 512 threads.
//
// A CMux step handles the m rows one after another.  For row r the 4 l_B
// digit polynomials ("combos": sign x component x digit) are transformed P at
// a time (P = 512 / (N/16) polynomials per batch, each by N/16 threads holding
// 16 coefficients in registers).  The transforms land in shared memory; every
// thread then multiplies the positions it owns (q = tid + 512 j) with the key
// rows of the batch's combos and accumulates exactly in 128-bit registers, so
// the whole row needs a single reduction per position and column.  The
// reduced row sums go to the job's sum buffer; after the last row, the 2m
// sums are inverse-transformed (P per batch) and added to the rows of the
// next ACC buffer.
// ---------------------------------------------------------------------------
namespace brk {
// Block shape for a ring of 2^LOGN coefficients run by THREADS threads.
template <int LOGN, int THREADS>
struct Cfg {
    static constexpr int kThreads = THREADS;
    static constexpr int N = 1 << LOGN;
    static constexpr int T = N / 16;                               // threads per polynomial
    static constexpr int P = kThreads / T;                         // polynomials per batch
    static constexpr int PPT = N >= kThreads ? N / kThreads : 1;   // positions per thread
    static constexpr bool DSM = LOGN <= 11;                        // row differences in smem
    static constexpr size_t SMEM = 2ull * P * N * 8 + (DSM ? 4ull * N * 8 : 0);
};

// Blind rotation of one job by the whole block (all threads must call it).
// sm: C::SMEM bytes of shared memory.  Variant flags: see choose_variant().
template <int LOGN, int THREADS, bool LAZY, bool SMALL0, bool QLOW1>
__device__ __forceinline__ void br_job(const DevJob &J, u32 steps_limit, const u64 *__restrict__ ct_in,
                                       const u32 *__restrict__ luts, u64 *ws, u32 *status, u64 *sm) {
    using C = Cfg<LOGN, THREADS>;
    constexpr int N = C::N;
    const KeyDev *K = J.key;
    const u32 lbits = J.lbits;
    // a batch's C::P limb products must fit 64 bits, else fold after each one
    const bool fold_each = (unsigned __int128)C::P * ((2ull << lbits) - 1) * ((2ull << lbits) - 1) >=
                           ((unsigned __int128)1 << 64);
    const u32 m = J.m, t = J.t, lB = K->l_B, log2B = K->log2_B, n = K->n;
    const ModQ mq = K->mq;
    const u64 Q = mq.Q;
    const u64 qp = 2ull * N * m;
    const u64 Bmask = (1ull << log2B) - 1;
    const u64 *twp = K->twp, *itwp = K->itwp;
    const u32 tid = threadIdx.x;
    const size_t vec = (size_t)m * 2 * N;
    u64 *acc0 = ws + J.acc_off;
    u64 *acc1 = acc0 + vec;
    u64 *sums = acc1 + vec;
    const u64 *ct = ct_in + J.in_off;
    const u32 *lut = luts + J.lut_off;

    if (!lut_is_negacyclic(lut, t)) {
        if (tid == 0) set_status(status, BM_ENONNEGACYCLIC);
        for (u32 idx = tid; idx < 2 * vec; idx += blockDim.x) acc0[idx] = 0;
        return;
    }
    acc_init(acc0, lut, ct[n] % qp, m, t, N, Q);
    __syncthreads();

    const u32 p = tid / C::T;          // polynomial slot within a batch
    const u32 l = tid % C::T;          // thread within the polynomial
    ntr::Swap sw{sm + (size_t)p * N, sm + (size_t)(C::P + p) * N, 0};
    u64 *dbuf = sm + (size_t)2 * C::P * N;   // [4][N] row differences (DSM only)
    const u64 qb = Q << log2B;                 // Q * B, used when SMALL0
    const u64 lmask = (1ull << lbits) - 1;     // Karatsuba limb mask
    const u32 ncomb = 4 * lB;
    const size_t rgsw = (size_t)2 * lB * 2 * N;

    u64 *cur = acc0, *nxt = acc1;
    const u32 steps = steps_limit < n ? steps_limit : n;
    for (u32 k = 0; k < steps; k++) {
        const u64 ak = ct[k] % qp;
        const u64 *bsk_k = K->bsk + (size_t)k * 2 * rgsw;
        for (u32 r = 0; r < m; r++) {
            u64 lo[2][C::PPT], hi[2][C::PPT];
#pragma unroll
            for (int j = 0; j < C::PPT; j++) lo[0][j] = hi[0][j] = lo[1][j] = hi[1][j] = 0;
            if constexpr (C::DSM) {
                // D_(sign, comp) = P(c) ACC - ACC for row r, c = -a_k / a_k
                for (u32 w = tid; w < 4u * N; w += C::kThreads) {
                    const u32 pair = w / N, idx = w % N;
                    const u32 sgn = pair >> 1, comp = pair & 1;
                    const u64 cv = sgn == 0 ? (qp - ak) % qp : ak;
                    const u32 ea = (u32)(cv / m), bb = (u32)(cv % m);
                    const u32 src = r >= bb ? r - bb : r + m - bb;
                    u32 e = r >= bb ? ea : ea + 1;
                    if (e >= 2 * N) e -= 2 * N;
                    const u64 *srow = cur + ((size_t)src * 2 + comp) * N;
                    const u64 *orow = cur + ((size_t)r * 2 + comp) * N;
                    dbuf[w] = sub_mod(rotated_coeff(srow, idx, e, N, Q), orow[idx], Q);
                }
                __syncthreads();
            }
            for (u32 c0 = 0; c0 < ncomb; c0 += C::P) {
                // --- this thread's digit polynomial, transformed into shared memory
                const u32 c = c0 + p;
                const bool active = c < ncomb;
                u64 x[16];
                if (active && C::DSM) {
                    const u32 pair = c / lB, sh = (c % lB) * log2B;
                    const u64 *dp = dbuf + (size_t)pair * N;
#pragma unroll
                    for (int i = 0; i < 16; i++) x[i] = (dp[l + C::T * i] >> sh) & Bmask;
                } else if (active) {
                    const u32 sgn = c / (2 * lB), comp = (c / lB) & 1, d = c % lB;
                    const u64 cv = sgn == 0 ? (qp - ak) % qp : ak;
                    const u32 ea = (u32)(cv / m), bb = (u32)(cv % m);
                    const u32 src = r >= bb ? r - bb : r + m - bb;
                    u32 e = r >= bb ? ea : ea + 1;
                    if (e >= 2 * N) e -= 2 * N;
                    const u64 *srow = cur + ((size_t)src * 2 + comp) * N;
                    const u64 *orow = cur + ((size_t)r * 2 + comp) * N;
                    const u32 sh = d * log2B;
#pragma unroll
                    for (int i = 0; i < 16; i++) {
                        const u32 idx = l + C::T * i;
                        const u64 D = sub_mod(rotated_coeff(srow, idx, e, N, Q), orow[idx], Q);
                        x[i] = (D >> sh) & Bmask;
                    }
                }
                u64 *out = ntr::fwd_to_smem<LOGN, LAZY, SMALL0, QLOW1>(x, sw, l, active, twp, Q, mq.one_sh, qb);
                // regions of the other polynomials of the batch sit at stride N
                const u64 *slots = out - (size_t)p * N;
                __syncthreads();
                // --- multiply-accumulate against the key rows of the batch's combos
                // (combo c = (sign, component, digit) is key row c of the step).
                // Karatsuba on half-width limbs x = x1 2^lbits + x0: the limb
                // products x1 b1, x0 b0 and (x0 + x1)(b0 + b1) are summed over
                // the batch in 64-bit registers, then folded into the 128-bit
                // row sums as hi 2^(2 lbits) + (mid - hi - lo) 2^lbits + lo.
                const u64 *bsk_c0 = bsk_k + (size_t)c0 * 2 * N;
                const u32 nc = ncomb - c0 < (u32)C::P ? ncomb - c0 : (u32)C::P;
                auto fold = [&](int j, u64 (&kh)[2], u64 (&kl)[2], u64 (&km)[2]) {
#pragma unroll
                    for (int col = 0; col < 2; col++) {
                        add128(lo[col][j], hi[col][j], kl[col]);
                        add128_shl(lo[col][j], hi[col][j], km[col] - kh[col] - kl[col], lbits);
                        add128_shl(lo[col][j], hi[col][j], kh[col], 2 * lbits);
                        kh[col] = kl[col] = km[col] = 0;
                    }
                };
                auto kara = [&](u64 xv, u64 bv, u64 &kh, u64 &kl, u64 &km) {
                    const u32 x0 = (u32)(xv & lmask), x1 = (u32)(xv >> lbits);
                    const u32 b0 = (u32)(bv & lmask), b1 = (u32)(bv >> lbits);
                    kh += (u64)x1 * b1;
                    kl += (u64)x0 * b0;
                    km += (u64)(x0 + x1) * (b0 + b1);
                };
                if (nc == (u32)C::P && !fold_each) {
                    // full batch: every key word of a position is requested first
#pragma unroll
                    for (int j = 0; j < C::PPT; j++) {
                        const u32 q = tid + C::kThreads * j;
                        if (q < (u32)N) {
                            const u32 sq = ntr::swz(q);
                            u64 bv[C::P][2];
#pragma unroll
                            for (int cc = 0; cc < C::P; cc++) {
                                bv[cc][0] = __ldg(bsk_c0 + (size_t)cc * 2 * N + q);
                                bv[cc][1] = __ldg(bsk_c0 + (size_t)cc * 2 * N + N + q);
                            }
                            u64 kh[2] = {0, 0}, kl[2] = {0, 0}, km[2] = {0, 0};
#pragma unroll
                            for (int cc = 0; cc < C::P; cc++) {
                                const u64 xv = slots[(size_t)cc * N + sq];
                                kara(xv, bv[cc][0], kh[0], kl[0], km[0]);
                                kara(xv, bv[cc][1], kh[1], kl[1], km[1]);
                            }
                            fold(j, kh, kl, km);
                        }
                    }
                } else {
                    for (int j = 0; j < C::PPT; j++) {
                        const u32 q = tid + C::kThreads * j;
                        if (q < (u32)N) {
                            const u32 sq = ntr::swz(q);
                            u64 kh[2] = {0, 0}, kl[2] = {0, 0}, km[2] = {0, 0};
                            for (u32 cc = 0; cc < nc; cc++) {
                                const u64 xv = slots[(size_t)cc * N + sq];
                                const u64 *brow = bsk_c0 + (size_t)cc * 2 * N + q;
                                kara(xv, __ldg(brow), kh[0], kl[0], km[0]);
                                kara(xv, __ldg(brow + N), kh[1], kl[1], km[1]);
                                if (fold_each) fold(j, kh, kl, km);
                            }
                            fold(j, kh, kl, km);
                        }
                    }
                }
            }
            // --- reduced row sums (NTT domain) to the sum buffer
#pragma unroll
            for (int j = 0; j < C::PPT; j++) {
                const u32 q = tid + C::kThreads * j;
                if (q < (u32)N) {
                    sums[((size_t)r * 2) * N + q] = reduce128(lo[0][j], hi[0][j], mq);
                    sums[((size_t)r * 2 + 1) * N + q] = reduce128(lo[1][j], hi[1][j], mq);
                }
            }
        }
        __syncthreads();
        // --- inverse transforms of the 2m row sums, ACC update
        for (u32 u0 = 0; u0 < 2 * m; u0 += C::P) {
            const u32 u = u0 + p;
            const bool active = u < 2 * m;
            u64 x[16];
            u64 *in = sw.take();
            if (active) {
                const u64 *sp = sums + (size_t)u * N;
#pragma unroll
                for (int i = 0; i < 16; i++) {
                    const u32 idx = l + C::T * i;
                    in[ntr::swz(idx)] = sp[idx];
                }
            }
            __syncthreads();
            ntr::inv_from_smem<LOGN, QLOW1>(x, in, sw, l, active, itwp, Q);
            if (active) {
                const size_t base = (size_t)u * N;
#pragma unroll
                for (int i = 0; i < 16; i++) {
                    const size_t o = base + l + C::T * i;
                    nxt[o] = add_mod(cur[o], x[i], Q);
                }
            }
        }
        __syncthreads();
        u64 *tmp = cur;
        cur = nxt;
        nxt = tmp;
    }
}

}  // namespace brk

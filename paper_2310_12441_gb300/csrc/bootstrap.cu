// Blind rotation, sample extraction and key switching of BootMMPM
// (arXiv 2310.12441, Algorithm 1) and the C-ABI entry points that launch them.
//
// One thread block runs one job.  Its RLWE-vector accumulator ACC
// ([m][2][N] words, Section 4) lives in two global buffers of the
// workspace (read the old one, write the new one, swap), which stay in L2.
// Per CMux step k (Eq. (cmux:BP)) and per row r the block
//   1. forms D = P(c) ACC - ACC for row r, c = -a_k (sign +) and c = a_k
//      (sign -), reading the source row and monomial of Eq. (ex1:BPc);
//   2. splits each component of D into l_B unsigned base-B digit polynomials
//      (Section 2 item (10)) and transforms them (negacyclic NTT);
//   3. multiplies them with the NTT-domain key rows of ct_k+ / ct_k- and
//      sums all 2 x 2 l_B products per output column in exact 128-bit
//      registers (Section 2 item (14), summed over both CMux terms);
//   4. reduces, inverse-transforms (N^-1 is folded into the key) and adds
//      the result to row r of ACC.
#include <cstring>
#include <mutex>
#include <vector>

#include "common.cuh"
#include "ntt.cuh"
#include "ntt_reg.cuh"

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
__device__ bool lut_is_negacyclic(const u32 *__restrict__ lut, u32 t) {
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
__device__ void acc_init(u64 *__restrict__ acc, const u32 *__restrict__ lut, u64 b, u32 m, u32 t,
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
// Up to N = 1024 two blocks of 256 threads share an SM (two jobs whose
// barriers and memory phases overlap each other's arithmetic); larger rings
// use one block of 512 threads.
template <int LOGN>
struct Cfg {
    static constexpr int kThreads = LOGN <= 10 ? 256 : 512;
    static constexpr int kBlocksPerSM = 512 / kThreads;
    static constexpr int N = 1 << LOGN;
    static constexpr int T = N / 16;                               // threads per polynomial
    static constexpr int P = kThreads / T;                         // polynomials per batch
    static constexpr int PPT = N >= kThreads ? N / kThreads : 1;   // positions per thread
    static constexpr bool DSM = LOGN <= 11;                        // row differences in smem
    static constexpr size_t SMEM = 2ull * P * N * 8 + (DSM ? 4ull * N * 8 : 0);
};
}  // namespace brk

template <int LOGN, bool LAZY, bool SMALL0, bool QLOW1>
__global__ void __launch_bounds__(brk::Cfg<LOGN>::kThreads, brk::Cfg<LOGN>::kBlocksPerSM)
    k_blind_rotate(const DevJob *__restrict__ jobs, u32 steps_limit, const u64 *__restrict__ ct_in,
                   const u32 *__restrict__ luts, u64 *ws, u32 *status, u32 lbits, bool fold_each) {
    using C = brk::Cfg<LOGN>;
    constexpr int N = C::N;
    extern __shared__ u64 sm[];
    const DevJob J = jobs[blockIdx.x];
    const KeyDev *K = J.key;
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

// ---------------------------------------------------------------------------
// Sample extraction + key switching
// ---------------------------------------------------------------------------

// a~ = floor((a P + floor(Q/2)) / Q) mod P, exact: the Shoup-style quotient
// estimate floor(a P' / 2^64), P' = floor(P 2^64 / Q), is at most 2 below the
// true quotient; the remainder fits in 64 bits and fixes it.
__device__ __forceinline__ u64 ks_round(u64 a, const KeyDev &K) {
    const u32 sh = K.log2_Bks * K.l_ks;
    const u64 Q = K.mq.Q;
    u64 q = __umul64hi(a, K.ks_pq);
    u64 r = (a << sh) + Q / 2 - q * Q;
    for (int it = 0; it < 3 && r >= Q; it++) { r -= Q; q++; }
    return q & ((1ull << sh) - 1);
}

// out = (0^n, b) - sum_{i,j} KSK(i, j, d_ij) for the LWE_{N,Q} sample given
// by get_a(i) (i < N) and b.  Threads own output columns; digits of all N
// coefficients are precomputed into shared memory (one byte each).
template <typename GetA>
__device__ void key_switch_block(const KeyDev &K, GetA get_a, u64 b, u64 *__restrict__ out) {
    extern __shared__ unsigned char dsm[];
    const u32 N = K.N, n = K.n, lks = K.l_ks, B1 = (1u << K.log2_Bks) - 1;
    for (u32 i = threadIdx.x; i < N; i += blockDim.x) {
        const u64 at = ks_round(get_a(i), K);
        for (u32 j = 0; j < lks; j++) dsm[i * lks + j] = (unsigned char)((at >> (K.log2_Bks * j)) & B1);
    }
    __syncthreads();
    constexpr int CPT = 8;   // columns per thread (n + 1 <= 8 * blockDim)
    u64 lo[CPT], hi[CPT];
#pragma unroll
    for (int q = 0; q < CPT; q++) lo[q] = hi[q] = 0;
    const size_t rowlen = n + 1;
    for (u32 i = 0; i < N; i++) {
        for (u32 j = 0; j < lks; j++) {
            const u32 d = dsm[i * lks + j];
            if (!d) continue;
            const u64 *row = K.ksk + (((size_t)i * lks + j) * B1 + (d - 1)) * rowlen;
#pragma unroll
            for (int q = 0; q < CPT; q++) {
                const u32 c = threadIdx.x + q * blockDim.x;
                if (c <= n) add128(lo[q], hi[q], __ldg(row + c));
            }
        }
    }
    const u64 Q = K.mq.Q;
#pragma unroll
    for (int q = 0; q < CPT; q++) {
        const u32 c = threadIdx.x + q * blockDim.x;
        if (c <= n) {
            const u64 sum = reduce128(lo[q], hi[q], K.mq);
            out[c] = sub_mod(c == n ? b : 0, sum, Q);
        }
    }
}

// Row 0 of the final ACC -> LWE_{N,Q} (Eq. (equ-sam-extr)) -> key switch.
__global__ void k_extract_keyswitch(const DevJob *__restrict__ jobs, u32 steps_limit,
                                    const u64 *__restrict__ ws, u64 *__restrict__ ct_out) {
    const DevJob J = jobs[blockIdx.x];
    const KeyDev &K = *J.key;
    const u32 N = K.N;
    const u32 steps = steps_limit < K.n ? steps_limit : K.n;
    const u64 *acc = ws + J.acc_off + ((steps & 1) ? (size_t)J.m * 2 * N : 0);
    const u64 Q = K.mq.Q;
    auto get_a = [&](u32 i) -> u64 {
        if (i == 0) return acc[0];
        const u64 v = acc[N - i];
        return v ? Q - v : 0;
    };
    key_switch_block(K, get_a, acc[N], ct_out + J.out_off);
}

__global__ void k_key_switch(const KeyDev *Kp, const u64 *__restrict__ lwe_in, u64 *__restrict__ out) {
    const KeyDev &K = *Kp;
    const u64 *in = lwe_in + (size_t)blockIdx.x * (K.N + 1);
    auto get_a = [&](u32 i) -> u64 { return in[i]; };
    key_switch_block(K, get_a, in[K.N], out + (size_t)blockIdx.x * (K.n + 1));
}

__global__ void k_sample_extract(const KeyDev *Kp, const u64 *__restrict__ rlwe, u64 *__restrict__ lwe) {
    const KeyDev &K = *Kp;
    const u32 N = K.N;
    const u64 Q = K.mq.Q;
    const u64 *a = rlwe + (size_t)blockIdx.x * 2 * N;
    u64 *o = lwe + (size_t)blockIdx.x * (N + 1);
    for (u32 i = threadIdx.x; i < N; i += blockDim.x) {
        const u64 v = i == 0 ? a[0] : a[N - i];
        o[i] = (i == 0 || v == 0) ? v : Q - v;
    }
    if (threadIdx.x == 0) o[N] = a[N];
}

__global__ void k_copy_acc(const DevJob *__restrict__ jobs, u32 steps_limit, const u64 *__restrict__ ws,
                           u64 *__restrict__ out) {
    const DevJob J = jobs[blockIdx.x];
    const u32 N = J.N;
    const u32 steps = steps_limit < J.n ? steps_limit : J.n;
    const size_t words = (size_t)J.m * 2 * N;
    const u64 *acc = ws + J.acc_off + ((steps & 1) ? words : 0);
    for (size_t i = threadIdx.x; i < words; i += blockDim.x) out[J.out_off + i] = acc[i];
}

// Negacyclic products through the NTT: one pair per block.
__global__ void k_poly_mul(const KeyDev *Kp, const u64 *__restrict__ a, const u64 *__restrict__ b,
                           u64 *__restrict__ out) {
    extern __shared__ u64 sm[];
    const KeyDev &K = *Kp;
    const u32 N = K.N;
    const u64 Q = K.mq.Q;
    const size_t off = (size_t)blockIdx.x * N;
    for (u32 i = threadIdx.x; i < N; i += blockDim.x) {
        sm[i] = a[off + i] % Q;
        sm[N + i] = b[off + i] % Q;
    }
    __syncthreads();
    cta_ntt_fwd(sm, 2, K.logN, K.tw, K.twsh, Q);
    for (u32 i = threadIdx.x; i < N; i += blockDim.x) {
        u64 lo = 0, hi = 0;
        mac128(lo, hi, sm[i], sm[N + i]);
        sm[i] = mul_shoup(reduce128(lo, hi, K.mq), K.ninv, K.ninv_sh, Q);
    }
    __syncthreads();
    cta_ntt_inv(sm, 1, K.logN, K.itw, K.itwsh, Q);
    for (u32 i = threadIdx.x; i < N; i += blockDim.x) out[off + i] = sm[i];
}

// Throughput probe: independent Shoup multiplication chains per thread.
__global__ void k_modmul_probe(u64 *out, u32 iters, u64 Q, u64 w, u64 wsh) {
    u64 x0 = threadIdx.x + 1, x1 = x0 + 7, x2 = x0 + 13, x3 = x0 + 29;
    u64 x4 = x0 + 31, x5 = x0 + 37, x6 = x0 + 41, x7 = x0 + 43;
    for (u32 i = 0; i < iters; i++) {
        x0 = mul_shoup_lazy(x0, w, wsh, Q);
        x1 = mul_shoup_lazy(x1, w, wsh, Q);
        x2 = mul_shoup_lazy(x2, w, wsh, Q);
        x3 = mul_shoup_lazy(x3, w, wsh, Q);
        x4 = mul_shoup_lazy(x4, w, wsh, Q);
        x5 = mul_shoup_lazy(x5, w, wsh, Q);
        x6 = mul_shoup_lazy(x6, w, wsh, Q);
        x7 = mul_shoup_lazy(x7, w, wsh, Q);
    }
    out[blockIdx.x * blockDim.x + threadIdx.x] = x0 ^ x1 ^ x2 ^ x3 ^ x4 ^ x5 ^ x6 ^ x7;
}

// ---------------------------------------------------------------------------
// Host side
// ---------------------------------------------------------------------------

namespace {

size_t align_up(size_t x, size_t a) { return (x + a - 1) / a * a; }

struct Plan {
    size_t jobs_off, acc_off_bytes, total;
    std::vector<DevJob> dj;
};

bm_status validate_jobs(const bm_eval_key *const *keys, uint32_t n_keys, const bm_job *jobs,
                        uint32_t count, int *device) {
    if (!keys || n_keys == 0 || (!jobs && count)) return BM_EINVAL;
    for (uint32_t i = 0; i < n_keys; i++)
        if (!keys[i]) return BM_EINVAL;
    *device = keys[0]->device;
    for (uint32_t i = 0; i < n_keys; i++)
        if (keys[i]->device != *device) return BM_EINVAL;
    for (uint32_t i = 0; i < count; i++) {
        const bm_job &j = jobs[i];
        if (j.key >= n_keys || j.reserved) return BM_EINVAL;
        const bm_eval_key *k = keys[j.key];
        if (j.m < 1 || j.m > BM_MAX_M) return BM_EINVAL;
        if (j.t < 2 || (j.t & 1) || (u64)j.t > 2ull * k->p.N * j.m) return BM_EINVAL;
    }
    return BM_OK;
}

bm_status make_plan(const bm_eval_key *const *keys, const bm_job *jobs, uint32_t count, Plan &pl) {
    pl.jobs_off = BM_WS_HEADER;
    size_t off = align_up(pl.jobs_off + sizeof(DevJob) * (size_t)count, 256);
    pl.acc_off_bytes = off;
    pl.dj.resize(count);
    size_t acc_words = 0;
    for (uint32_t i = 0; i < count; i++) {
        const bm_eval_key *k = keys[jobs[i].key];
        DevJob &d = pl.dj[i];
        d.key = k->d_view;
        d.m = jobs[i].m;
        d.t = jobs[i].t;
        d.N = k->p.N;
        d.n = k->p.n;
        d.in_off = jobs[i].in_off;
        d.lut_off = jobs[i].lut_off;
        d.out_off = jobs[i].out_off;
        d.acc_off = acc_words;
        acc_words += 3ull * 2 * jobs[i].m * k->p.N;
    }
    pl.total = off + acc_words * 8;
    return BM_OK;
}

template <int LOGN, bool LAZY, bool SMALL0, bool QLOW1>
bm_status launch_br_v(const DevJob *d_jobs, uint32_t first, uint32_t cnt, u32 steps, const uint64_t *ct_in,
                      const uint32_t *lut, u64 *ws_acc, u32 *status, u32 lbits, bool fold_each,
                      cudaStream_t st) {
    using C = brk::Cfg<LOGN>;
    const size_t smem = C::SMEM;
    auto kern = k_blind_rotate<LOGN, LAZY, SMALL0, QLOW1>;
    BM_CUDA_TRY(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    kern<<<cnt, C::kThreads, smem, st>>>(d_jobs + first, steps, ct_in, lut, ws_acc, status, lbits, fold_each);
    BM_CUDA_TRY(cudaGetLastError());
    return BM_OK;
}

// Variant choice for one key set:
//  - the correction-free forward transform needs (1 + 4 log2 N) Q < 2^64, its
//    exact first stage B + Q B + 4 Q (log2 N - 1) < 2^64;
//  - Q = c 2^32 + 1 selects the one-multiply q Q;
//  - the Karatsuba limbs have lbits = ceil(bits(Q - 1) / 2) bits; a batch's P
//    limb products fit 64 bits when P (2^(lbits+1) - 1)^2 < 2^64, otherwise
//    they are folded after every combo.
template <int LOGN>
bm_status launch_br(const DevJob *d_jobs, uint32_t first, uint32_t cnt, u32 steps, const uint64_t *ct_in,
                    const uint32_t *lut, u64 *ws_acc, u32 *status, u64 Q, u32 log2B, cudaStream_t st) {
    typedef unsigned __int128 u128;
    using C = brk::Cfg<LOGN>;
    const u128 lim = (u128)1 << 64;
    const bool lazy = (u128)(1 + 4 * LOGN) * Q < lim;
    const u128 B = (u128)1 << log2B;
    const bool small0 = lazy && log2B <= 31 && B + (u128)Q * B + (u128)4 * Q * (LOGN - 1) < lim;
    const bool qlow1 = (Q & 0xffffffffull) == 1;
    u32 qbits = 0;
    while (qbits < 64 && ((Q - 1) >> qbits)) qbits++;
    const u32 lbits = (qbits + 1) / 2;
    const u128 limb = ((u128)1 << (lbits + 1)) - 1;
    const bool fold_each = (u128)C::P * limb * limb >= lim;
#define BM_LAUNCH(LZ, S0, QL) \
    return launch_br_v<LOGN, LZ, S0, QL>(d_jobs, first, cnt, steps, ct_in, lut, ws_acc, status, lbits, fold_each, st)
    if (small0 && qlow1) BM_LAUNCH(true, true, true);
    if (small0) BM_LAUNCH(true, true, false);
    if (qlow1) BM_LAUNCH(false, false, true);
    BM_LAUNCH(false, false, false);
#undef BM_LAUNCH
}

// Launches blind rotation for every job; jobs are grouped by ring degree
// (one launch per run of equal N in job order).
bm_status run_blind_rotation(const bm_eval_key *const *keys, const bm_job *jobs, uint32_t count,
                             u32 steps, const Plan &pl, const uint64_t *d_ct_in, const uint32_t *d_lut,
                             char *ws, cudaStream_t st) {
    const DevJob *d_jobs = (const DevJob *)(ws + pl.jobs_off);
    u64 *ws_acc = (u64 *)(ws + pl.acc_off_bytes);
    u32 *status = (u32 *)ws;
    uint32_t i = 0;
    while (i < count) {
        const bm_eval_key *k = keys[jobs[i].key];
        const u32 N = k->p.N;
        uint32_t j = i + 1;
        const u64 Q = k->p.Q;
        const u32 log2B = k->p.log2_B;
        while (j < count && keys[jobs[j].key]->p.N == N && keys[jobs[j].key]->p.Q == Q &&
               keys[jobs[j].key]->p.log2_B == log2B)
            j++;
        bm_status s = BM_OK;
        switch (N) {
            case 256: s = launch_br<8>(d_jobs, i, j - i, steps, d_ct_in, d_lut, ws_acc, status, Q, log2B, st); break;
            case 512: s = launch_br<9>(d_jobs, i, j - i, steps, d_ct_in, d_lut, ws_acc, status, Q, log2B, st); break;
            case 1024: s = launch_br<10>(d_jobs, i, j - i, steps, d_ct_in, d_lut, ws_acc, status, Q, log2B, st); break;
            case 2048: s = launch_br<11>(d_jobs, i, j - i, steps, d_ct_in, d_lut, ws_acc, status, Q, log2B, st); break;
            case 4096: s = launch_br<12>(d_jobs, i, j - i, steps, d_ct_in, d_lut, ws_acc, status, Q, log2B, st); break;
            default: return BM_EINVAL;
        }
        if (s != BM_OK) return s;
        i = j;
    }
    return BM_OK;
}

bm_status upload_plan(const Plan &pl, char *ws, cudaStream_t st) {
    if (!pl.dj.empty())
        BM_CUDA_TRY(cudaMemcpyAsync(ws + pl.jobs_off, pl.dj.data(), sizeof(DevJob) * pl.dj.size(),
                                    cudaMemcpyHostToDevice, st));
    return BM_OK;
}

struct DeviceGuard {
    int prev = -1;
    explicit DeviceGuard(int dev) {
        cudaGetDevice(&prev);
        if (prev != dev) cudaSetDevice(dev);
    }
    ~DeviceGuard() {
        int cur = -1;
        cudaGetDevice(&cur);
        if (prev >= 0 && cur != prev) cudaSetDevice(prev);
    }
};

}  // namespace

extern "C" size_t bm_workspace_bytes(const bm_eval_key *const *keys, uint32_t n_keys, const bm_job *jobs,
                                     uint32_t count) {
    int dev = 0;
    if (validate_jobs(keys, n_keys, jobs, count, &dev) != BM_OK) return 0;
    Plan pl;
    make_plan(keys, jobs, count, pl);
    return pl.total;
}

static bm_status bootstrap_impl(const bm_eval_key *const *keys, uint32_t n_keys, const bm_job *jobs,
                                uint32_t count, u32 steps, bool do_ks, const uint64_t *d_ct_in,
                                const uint32_t *d_lut, uint64_t *d_out, void *d_ws, size_t ws_bytes,
                                void *stream) {
    int dev = 0;
    bm_status s = validate_jobs(keys, n_keys, jobs, count, &dev);
    if (s != BM_OK) return s;
    if (!d_ws || ((uintptr_t)d_ws & 255)) return BM_EINVAL;
    if (count && (!d_ct_in || !d_lut || !d_out)) return BM_EINVAL;
    Plan pl;
    make_plan(keys, jobs, count, pl);
    if (ws_bytes < pl.total) return BM_EWORKSPACE;
    if (count == 0) return BM_OK;
    DeviceGuard g(dev);
    cudaStream_t st = (cudaStream_t)stream;
    char *ws = (char *)d_ws;
    if ((s = upload_plan(pl, ws, st)) != BM_OK) return s;
    if ((s = run_blind_rotation(keys, jobs, count, steps, pl, d_ct_in, d_lut, ws, st)) != BM_OK) return s;
    const DevJob *d_jobs = (const DevJob *)(ws + pl.jobs_off);
    const u64 *ws_acc = (const u64 *)(ws + pl.acc_off_bytes);
    if (do_ks) {
        u32 maxN = 0, maxn = 0, maxlks = 0;
        for (uint32_t i = 0; i < n_keys; i++) {
            maxN = keys[i]->p.N > maxN ? keys[i]->p.N : maxN;
            maxn = keys[i]->p.n > maxn ? keys[i]->p.n : maxn;
            maxlks = keys[i]->p.l_ks > maxlks ? keys[i]->p.l_ks : maxlks;
        }
        const u32 threads = (maxn + 1 + 7) / 8 < 128 ? 128 : ((maxn + 1 + 7) / 8 + 31) / 32 * 32;
        const size_t smem = (size_t)maxN * maxlks;
        k_extract_keyswitch<<<count, threads, smem, st>>>(d_jobs, steps, ws_acc, d_out);
    } else {
        k_copy_acc<<<count, 256, 0, st>>>(d_jobs, steps, ws_acc, d_out);
    }
    BM_CUDA_TRY(cudaGetLastError());
    return BM_OK;
}

extern "C" bm_status bm_bootstrap_batch(const bm_eval_key *const *keys, uint32_t n_keys, const bm_job *jobs,
                                        uint32_t count, const uint64_t *d_ct_in, const uint32_t *d_lut,
                                        uint64_t *d_ct_out, void *d_ws, size_t ws_bytes, void *stream) {
    return bootstrap_impl(keys, n_keys, jobs, count, 0xffffffffu, true, d_ct_in, d_lut, d_ct_out, d_ws,
                          ws_bytes, stream);
}

extern "C" bm_status bm_blind_rotate(const bm_eval_key *const *keys, uint32_t n_keys, const bm_job *jobs,
                                     uint32_t count, uint32_t steps, const uint64_t *d_ct_in,
                                     const uint32_t *d_lut, uint64_t *d_acc_out, void *d_ws, size_t ws_bytes,
                                     void *stream) {
    return bootstrap_impl(keys, n_keys, jobs, count, steps, false, d_ct_in, d_lut, d_acc_out, d_ws,
                          ws_bytes, stream);
}

extern "C" size_t bm_host_staging_bytes(const bm_eval_key *const *keys, uint32_t n_keys, const bm_job *jobs,
                                        uint32_t count) {
    int dev = 0;
    if (validate_jobs(keys, n_keys, jobs, count, &dev) != BM_OK) return 0;
    size_t in_w = 0, lut_w = 0, out_w = 0;
    for (uint32_t i = 0; i < count; i++) {
        const bm_eval_key *k = keys[jobs[i].key];
        in_w = jobs[i].in_off + k->p.n + 1 > in_w ? jobs[i].in_off + k->p.n + 1 : in_w;
        lut_w = jobs[i].lut_off + jobs[i].t > lut_w ? jobs[i].lut_off + jobs[i].t : lut_w;
        out_w = jobs[i].out_off + k->p.n + 1 > out_w ? jobs[i].out_off + k->p.n + 1 : out_w;
    }
    return align_up(in_w * 8, 256) + align_up(lut_w * 4, 256) + align_up(out_w * 8, 256);
}

extern "C" bm_status bm_bootstrap_batch_host(const bm_eval_key *const *keys, uint32_t n_keys,
                                             const bm_job *jobs, uint32_t count, const uint64_t *h_ct_in,
                                             size_t ct_in_words, const uint32_t *h_lut, size_t lut_words,
                                             uint64_t *h_ct_out, size_t ct_out_words, void *d_ws,
                                             size_t ws_bytes, void *stream) {
    int dev = 0;
    bm_status s = validate_jobs(keys, n_keys, jobs, count, &dev);
    if (s != BM_OK) return s;
    if (!h_ct_in || !h_lut || !h_ct_out || !d_ws) return BM_EINVAL;
    for (uint32_t i = 0; i < count; i++) {
        const bm_eval_key *k = keys[jobs[i].key];
        if (jobs[i].in_off + k->p.n + 1 > ct_in_words || jobs[i].lut_off + jobs[i].t > lut_words ||
            jobs[i].out_off + k->p.n + 1 > ct_out_words)
            return BM_EINVAL;
    }
    const size_t need = bm_workspace_bytes(keys, n_keys, jobs, count);
    const size_t stage = bm_host_staging_bytes(keys, n_keys, jobs, count);
    if (ws_bytes < need + stage) return BM_EWORKSPACE;
    DeviceGuard g(dev);
    cudaStream_t st = (cudaStream_t)stream;
    char *base = (char *)d_ws + align_up(need, 256);
    uint64_t *d_in = (uint64_t *)base;
    uint32_t *d_lut = (uint32_t *)(base + align_up(ct_in_words * 8, 256));
    uint64_t *d_out = (uint64_t *)((char *)d_lut + align_up(lut_words * 4, 256));
    if ((char *)d_out + ct_out_words * 8 > (char *)d_ws + ws_bytes) return BM_EWORKSPACE;
    BM_CUDA_TRY(cudaMemcpyAsync(d_in, h_ct_in, ct_in_words * 8, cudaMemcpyHostToDevice, st));
    BM_CUDA_TRY(cudaMemcpyAsync(d_lut, h_lut, lut_words * 4, cudaMemcpyHostToDevice, st));
    s = bm_bootstrap_batch(keys, n_keys, jobs, count, d_in, d_lut, d_out, d_ws, need, stream);
    if (s != BM_OK) return s;
    BM_CUDA_TRY(cudaMemcpyAsync(h_ct_out, d_out, ct_out_words * 8, cudaMemcpyDeviceToHost, st));
    BM_CUDA_TRY(cudaStreamSynchronize(st));
    return BM_OK;
}

extern "C" bm_status bm_sample_extract(const bm_eval_key *key, const uint64_t *d_rlwe, uint32_t count,
                                       uint64_t *d_lwe_out, void *stream) {
    if (!key || (count && (!d_rlwe || !d_lwe_out))) return BM_EINVAL;
    if (!count) return BM_OK;
    DeviceGuard g(key->device);
    k_sample_extract<<<count, 256, 0, (cudaStream_t)stream>>>(key->d_view, d_rlwe, d_lwe_out);
    BM_CUDA_TRY(cudaGetLastError());
    return BM_OK;
}

extern "C" bm_status bm_key_switch(const bm_eval_key *key, const uint64_t *d_lwe_in, uint32_t count,
                                   uint64_t *d_out, void *stream) {
    if (!key || (count && (!d_lwe_in || !d_out))) return BM_EINVAL;
    if (!count) return BM_OK;
    DeviceGuard g(key->device);
    const u32 n = key->p.n;
    const u32 threads = (n + 1 + 7) / 8 < 128 ? 128 : ((n + 1 + 7) / 8 + 31) / 32 * 32;
    const size_t smem = (size_t)key->p.N * key->p.l_ks;
    k_key_switch<<<count, threads, smem, (cudaStream_t)stream>>>(key->d_view, d_lwe_in, d_out);
    BM_CUDA_TRY(cudaGetLastError());
    return BM_OK;
}

extern "C" bm_status bm_poly_mul(const bm_eval_key *key, const uint64_t *d_a, const uint64_t *d_b,
                                 uint32_t count, uint64_t *d_out, void *stream) {
    if (!key || (count && (!d_a || !d_b || !d_out))) return BM_EINVAL;
    if (!count) return BM_OK;
    DeviceGuard g(key->device);
    const u32 N = key->p.N;
    const size_t smem = 2 * (size_t)N * 8;
    BM_CUDA_TRY(cudaFuncSetAttribute(k_poly_mul, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    k_poly_mul<<<count, N / 2 < 512 ? N / 2 : 512, smem, (cudaStream_t)stream>>>(key->d_view, d_a, d_b, d_out);
    BM_CUDA_TRY(cudaGetLastError());
    return BM_OK;
}

extern "C" bm_status bm_workspace_status(void *d_ws, void *stream) {
    if (!d_ws) return BM_EINVAL;
    u32 v = 0;
    BM_CUDA_TRY(cudaMemcpyAsync(&v, d_ws, 4, cudaMemcpyDeviceToHost, (cudaStream_t)stream));
    BM_CUDA_TRY(cudaStreamSynchronize((cudaStream_t)stream));
    BM_CUDA_TRY(cudaMemsetAsync(d_ws, 0, 4, (cudaStream_t)stream));
    BM_CUDA_TRY(cudaStreamSynchronize((cudaStream_t)stream));
    return -(bm_status)v;
}

extern "C" bm_status bm_modmul_peak(int device, uint32_t iters, double *rate) {
    if (!rate || iters == 0) return BM_EINVAL;
    DeviceGuard g(device);
    int sms = 0;
    BM_CUDA_TRY(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, device));
    const u32 blocks = (u32)sms * 8, threads = 256;
    u64 *d_out = nullptr;
    BM_CUDA_TRY(cudaMalloc(&d_out, (size_t)blocks * threads * 8));
    const u64 Q = 18014398509404161ull, w = 123456789012345ull;
    const u64 wsh = (u64)(((unsigned __int128)w << 64) / Q);
    cudaEvent_t e0, e1;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    k_modmul_probe<<<blocks, threads>>>(d_out, iters / 8 + 1, Q, w, wsh);   // warm-up
    cudaEventRecord(e0);
    k_modmul_probe<<<blocks, threads>>>(d_out, iters, Q, w, wsh);
    cudaEventRecord(e1);
    cudaError_t err = cudaEventSynchronize(e1);
    float ms = 0;
    cudaEventElapsedTime(&ms, e0, e1);
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    cudaFree(d_out);
    if (err != cudaSuccess) return BM_ECUDA;
    *rate = (double)blocks * threads * 8.0 * iters / (ms * 1e-3);
    return BM_OK;
}

// ---------------------------------------------------------------------------
// Bootstrapping without any device allocation.
//
// Some callers cannot allocate device memory when they want to bootstrap:
// code embedded in a host application whose memory pool already holds the
// GPU's memory, serving loops where a cudaMalloc or cudaFree would stall
// the whole device, and components that must keep their device footprint
// fixed after start-up.  For them, the job table, status word and
// accumulators of a batch live in one fixed array compiled into this
// library instead of a caller-supplied workspace.
// ---------------------------------------------------------------------------

static __device__ __align__(256) unsigned char g_noalloc_scratch[BM_NOALLOC_SCRATCH_BYTES];

namespace {
constexpr int kMaxDevices = 64;
std::mutex g_noalloc_mu;
void *g_noalloc_ptr[kMaxDevices];   // device address of the array, per device

__global__ void k_noalloc_status(const u32 *word, int32_t *out) {
    if (threadIdx.x == 0 && blockIdx.x == 0) *out = -(int32_t)(*word);
}
}  // namespace

extern "C" bm_status bm_bootstrap_batch_noalloc(const bm_eval_key *const *keys, uint32_t n_keys,
                                                const bm_job *jobs, uint32_t count,
                                                const uint64_t *d_ct_in, const uint32_t *d_lut,
                                                uint64_t *d_ct_out, int32_t *d_status, void *stream) {
    int dev = 0;
    bm_status s = validate_jobs(keys, n_keys, jobs, count, &dev);
    if (s != BM_OK) return s;
    if (dev < 0 || dev >= kMaxDevices) return BM_EINVAL;
    Plan pl;
    make_plan(keys, jobs, count, pl);
    if (pl.total > BM_NOALLOC_SCRATCH_BYTES) {
        fprintf(stderr, "bootmmpm: batch needs %zu bytes of scratch, more than the %u built in\n",
                pl.total, (unsigned)BM_NOALLOC_SCRATCH_BYTES);
        return BM_EWORKSPACE;
    }
    DeviceGuard g(dev);
    void *scratch = nullptr;
    {
        // Host code sees only a stand-in for the array; its device address is
        // looked up once per device, with that device current.
        std::lock_guard<std::mutex> lk(g_noalloc_mu);
        if (!g_noalloc_ptr[dev]) {
            void *p = nullptr;
            cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
            if (e != cudaSuccess || !p) {
                fprintf(stderr, "bootmmpm: cudaGetSymbolAddress failed: %s\n", cudaGetErrorString(e));
                return BM_ECUDA;
            }
            g_noalloc_ptr[dev] = p;
        }
        scratch = g_noalloc_ptr[dev];
    }
    cudaStream_t st = (cudaStream_t)stream;
    // The array keeps the previous call's contents: the status word must
    // start at zero (job table and accumulators are fully rewritten).
    BM_CUDA_TRY(cudaMemsetAsync(scratch, 0, BM_WS_HEADER, st));
    s = bootstrap_impl(keys, n_keys, jobs, count, 0xffffffffu, true, d_ct_in, d_lut, d_ct_out, scratch,
                       BM_NOALLOC_SCRATCH_BYTES, stream);
    if (s != BM_OK) return s;
    if (d_status) {
        k_noalloc_status<<<1, 32, 0, st>>>((const u32 *)scratch, d_status);
        BM_CUDA_TRY(cudaGetLastError());
    }
    return BM_OK;
}

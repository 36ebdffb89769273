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

// Load of an accumulator word.  Rows written by other blocks of a cluster are
// read at L2 (ld.global.cg), never from this SM's L1.
__device__ __forceinline__ u64 acc_load(const u64 *p, bool l2) { return l2 ? __ldcg(p) : *p; }

// Coefficient `c` of x^e * p in R_{N,Q}, e in [0, 2N).
__device__ __forceinline__ u64 rotated_coeff(const u64 *p, u32 c, u32 e, u32 N, u64 Q, bool l2 = false) {
    u32 j = c + 2 * N - e;
    if (j >= 2 * N) j -= 2 * N;
    if (j < N) return acc_load(p + j, l2);
    const u64 v = acc_load(p + j - N, l2);
    return v ? Q - v : 0;
}

// Rank of this block in its thread-block cluster and the cluster's size (0
// and 1 for a launch without clusters).
__device__ __forceinline__ u32 cluster_rank() {
    u32 r;
    asm volatile("mov.u32 %0, %%cluster_ctarank;" : "=r"(r));
    return r;
}
__device__ __forceinline__ u32 cluster_size() {
    u32 r;
    asm volatile("mov.u32 %0, %%cluster_nctarank;" : "=r"(r));
    return r;
}

// Barrier over every thread of every block of the cluster; writes before it
// (global memory included) are visible to all of them after it.  Every
// block arrives once per CMux step, so no block can wait for one that has
// left: the blocks of a cluster run the same job and the same step count.
__device__ __forceinline__ void cluster_sync() {
    asm volatile("barrier.cluster.arrive.release.aligned;\n\tbarrier.cluster.wait.acquire.aligned;" ::: "memory");
}

__device__ __forceinline__ void set_status(u32 *status, bm_status code) {
    atomicCAS(status, 0u, (u32)(-code));
}

// Shared-memory mbarrier (arrive/wait split barrier of the block's threads).
__device__ __forceinline__ u32 smem_u32(const void *p) { return (u32)__cvta_generic_to_shared(p); }
__device__ __forceinline__ void mbar_init(u64 *bar, u32 count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}
// Arrival (release: this thread's earlier shared-memory reads are ordered
// before any access that a waiter makes after its wait).
__device__ __forceinline__ void mbar_arrive(u64 *bar) {
    asm volatile("{\n\t.reg .b64 st;\n\tmbarrier.arrive.shared::cta.b64 st, [%0];\n\t}" ::"r"(smem_u32(bar))
                 : "memory");
}
// Waits (acquire) for the completion of the phase with this parity.  Bounded:
// after 2^24 polls (each may suspend the thread for a while) it sets
// BM_ETIMEDOUT in the status word and returns, so a missing arrival can
// never hang the GPU (every thread of the block arrives once per phase, so
// this does not happen in a correct launch).
__device__ __forceinline__ void mbar_wait(u64 *bar, u32 parity, u32 *status) {
    const u32 a = smem_u32(bar);
    for (u32 it = 0; it < (1u << 24); it++) {
        u32 ok;
        asm volatile("{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
                     "selp.u32 %0, 1, 0, p;\n\t}"
                     : "=r"(ok)
                     : "r"(a), "r"(parity)
                     : "memory");
        if (ok) return;
    }
    set_status(status, BM_ETIMEDOUT);
}

// The key words of one combo at one position, both columns, in one 16-byte
// load (read-only for the kernel's lifetime): w0 holds the low limbs of
// columns 0 and 1 (as two 32-bit halves), w1 their high limbs.
__device__ __forceinline__ void key_load2(const u64 *p, u64 &w0, u64 &w1) {
    const ulonglong2 v = __ldg(reinterpret_cast<const ulonglong2 *>(p));
    w0 = v.x;
    w1 = v.y;
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

// Row i of P(c) = A^c (Lemma 3, Eq. (Al:res)): its source row (i - c) mod m
// and monomial exponent E_c(i) mod 2N, c = a m + b.
//  - gS == 0, the generator of Example 1: E_c(i) = a + [i < b] (Eq. (ex1:BPc));
//  - otherwise a generator A = (x^{u_i} delta_{i-1 mod m, j}) of Theorem 1 with
//    S = sum u = gS and pre[k] = u_0 + ... + u_{k-1} (all mod 2N):
//    E_c(i) = a S + sum_{t in [b]} u_{(i - t) mod m}.
// (mmpm_row_ab takes a = c / m and b = c mod m, which the rows of one CMux
// step share; 2N is a power of two.)
__device__ __forceinline__ void mmpm_row_ab(u32 a, u32 b, u32 i, u32 m, u32 twoN, u32 gS, const u32 *pre,
                                            u32 &src, u32 &e) {
    src = i >= b ? i - b : i + m - b;
    if (!gS) {
        e = i >= b ? a : a + 1;
        if (e >= twoN) e -= twoN;
        return;
    }
    u32 w = 0;
    if (b != 0) w = b <= i + 1 ? pre[i + 1] + twoN - pre[i + 1 - b] : pre[i + 1] + pre[m] + twoN - pre[m + i + 1 - b];
    e = (u32)(((u64)a * gS + w) & (twoN - 1));
}
__device__ __forceinline__ void mmpm_row(u32 c, u32 i, u32 m, u32 twoN, u32 gS, const u32 *pre, u32 &src,
                                         u32 &e) {
    mmpm_row_ab(c / m, c % m, i, m, twoN, gS, pre, src, e);
}

// ACC <- P(b) (0, v_test floor(Q/t)) with the negacyclic extension
// f'(u) = f(floor((u t + Nm) / 2Nm) mod t).
//  - Generator of Example 1, v_test of Eq. (equ:test-use): coefficient j of
//    row s is f'(-(j m + s) mod 2Nm).
//  - General generator, v_test of Eq. (equ:test-gene): the term
//    f'(-(a m + s)) x^{a S + E_s} of row s (a in [N], E_s = u_1 + ... + u_s)
//    lands on coefficient j = (a S + E_s) mod N, negated when
//    (a S + E_s) mod 2N >= N; so coefficient j holds the term
//    a = (j - E_s) S^-1 mod N.
// Rows i with i mod rows_step == row0 only (the rows of one block of a cluster).
static __device__ void acc_init(u64 *__restrict__ acc, const u32 *__restrict__ lut, u64 b, u32 m, u32 t,
                                u32 N, u64 Q, u32 gS, u32 gSinv, const u32 *pre, u32 row0 = 0,
                                u32 rows_step = 1) {
    const u64 qp = 2ull * N * m;
    const u64 dq = Q / t;
    const u32 twoN = 2 * N;
    for (u32 idx = threadIdx.x; idx < m * 2 * N; idx += blockDim.x) {
        const u32 c = idx % N;
        const u32 comp = (idx / N) & 1;
        const u32 i = idx / (2 * N);
        if (i % rows_step != row0) continue;
        u64 val = 0;
        if (comp == 1) {
            u32 src, e;
            mmpm_row((u32)(b % qp), i, m, twoN, gS, pre, src, e);
            u32 j = c + twoN - e;
            if (j >= twoN) j -= twoN;
            bool neg = j >= N;
            if (neg) j -= N;
            u32 a = j;
            if (gS) {
                const u32 Es = pre[src + 1] + twoN - pre[1];          // u_1 + ... + u_s (mod 2N)
                a = (u32)(((u64)((j + twoN - Es % twoN) % N) * gSinv) % N);
                if (((u64)a * gS + Es) % twoN >= N) neg = !neg;
            }
            const u64 w = ((u64)a * m + src) % qp;
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
// Shared memory of one block (see Cfg): two exchange regions per polynomial
// of a batch, the row differences when they fit, the forward twiddle pairs.
// With `blocks` blocks per SM each block plans within its share of the SM
// (226 KB for one block, 112 KB each for two).
__host__ __device__ constexpr size_t smem_budget(int blocks) { return blocks > 1 ? 112 * 1024 : 226 * 1024; }
__host__ __device__ constexpr size_t smem_dbudget(int blocks) { return blocks > 1 ? 96 * 1024 : 200 * 1024; }
__host__ __device__ constexpr size_t smem_regions(int logn, int threads, int rb) {
    return 2ull * (threads / ((1 << logn) >> rb)) * (1ull << logn) * 8;
}
__host__ __device__ constexpr size_t smem_dbytes(int logn, int threads, int rb, int blocks = 1) {
    return smem_regions(logn, threads, rb) + 4ull * (1ull << logn) * 8 <= smem_dbudget(blocks)
               ? 4ull * (1ull << logn) * 8
           : smem_regions(logn, threads, rb) + (1ull << logn) * 8 <= smem_dbudget(blocks) ? (1ull << logn) * 8
                                                                                          : 0;
}
__host__ __device__ constexpr size_t smem_twbytes(int logn, int threads, int rb, int blocks = 1) {
    return smem_regions(logn, threads, rb) + smem_dbytes(logn, threads, rb, blocks) + 16ull * (1ull << logn) <=
                   smem_budget(blocks)
               ? 16ull * (1ull << logn)
               : 0;
}
__host__ __device__ constexpr size_t smem_bytes(int logn, int threads, int rb, int blocks = 1) {
    return smem_regions(logn, threads, rb) + smem_dbytes(logn, threads, rb, blocks) +
           smem_twbytes(logn, threads, rb, blocks);
}

// Block shape for a ring of 2^LOGN coefficients run by THREADS threads,
// each holding 2^RB coefficients of a polynomial in the transforms, BLK
// blocks per SM.
template <int LOGN, int THREADS, int RB = 4, int BLK = 1>
struct Cfg {
    static constexpr int kThreads = THREADS;
    static constexpr int N = 1 << LOGN;
    static constexpr int R = 1 << RB;                              // coefficients per thread
    static constexpr int T = N / R;                                // threads per polynomial
    static constexpr int P = kThreads / T;                         // polynomials per batch
    static constexpr int PPT = N >= kThreads ? N / kThreads : 1;   // positions per thread
    // rows per batch (every key word the multiply-accumulate loads would serve G
    // rows; G = 2 measured 17% slower on GB300: the extra accumulators cost more
    // registers than the halved key loads save)
    static constexpr int G = 1;
    static constexpr int CPB = P / G;                              // combos per batch
    // key words a thread holds at once in the multiply-accumulate (fewer
    // where a 1024-thread block leaves 64 registers per thread)
    static constexpr int KC = kThreads >= 1024 && CPB > 4 ? 4 : CPB;
    // Row sums per position: exact 128-bit registers, reduced once per row;
    // with 8 or more positions per thread (N = 8192) they stay in the job's
    // sum buffer instead (L2), reduced mod Q and updated by their owner
    // after every batch (128-bit sums of 8 positions in registers spilled
    // kilobytes per thread).
    static constexpr bool RED = PPT >= 8;
    static constexpr int PPTR = RED ? 1 : PPT;                    // positions of the register sums
    static constexpr size_t REGIONS = 2ull * P * N * 8;            // two regions per polynomial
    static constexpr bool DSM = REGIONS + 4ull * G * N * 8 <= smem_dbudget(BLK);   // row differences in smem
    // otherwise (N >= 4096, or 2048 with two blocks per SM) the difference of
    // one (sign, component) pair, built before the batches of its digits
    static constexpr bool DPAIR = !DSM && REGIONS + N * 8ull <= smem_dbudget(BLK);
    static constexpr size_t DBYTES = DSM ? 4ull * G * N * 8 : DPAIR ? N * 8ull : 0;
    // forward twiddle pairs in shared memory when they fit, else read
    // through L1 from the key's table
    static constexpr size_t TWBYTES = smem_twbytes(LOGN, THREADS, RB, BLK);
    static constexpr bool TWSM = TWBYTES != 0;
    static constexpr size_t SMEM = REGIONS + DBYTES + TWBYTES;
    static_assert(G != 1 || SMEM == smem_bytes(LOGN, THREADS, RB, BLK), "smem_bytes mirrors Cfg");
    static_assert(P >= 1 && P * T == THREADS, "whole polynomials per batch");
    static_assert(T <= 32 || P <= 15, "a named barrier per polynomial (ids 1..15)");
    static_assert(SMEM <= 227 * 1024 - 1024, "shared memory per block");
};

// Blind rotation of one job by the whole block (all threads must call it).
// sm: C::SMEM bytes of shared memory.  Variant flags: see choose_variant().
// Launched in thread-block clusters of S blocks per job, block s of the
// cluster takes the rows r = s mod S: the rows of a step only read the
// previous accumulator, so they are independent, and one cluster barrier per
// step orders the accumulator updates (rows S times fewer per block, so the
// job's latency drops by up to S; the work is the same).
//
// A CMux step handles the m rows G at a time.  For a group of rows, the
// 4 l_B digit polynomials per row ("combos": sign x component x digit) are
// transformed P at a time, CPB combos of every row of the group per batch
// (each polynomial by N/16 threads holding 16 coefficients in registers).
// The transforms land in shared memory; every thread then multiplies the
// positions it owns (q = tid + THREADS j) with the key rows of the batch's
// combos (Karatsuba on half-width limbs, exact 128-bit row sums), so the
// whole row needs a single reduction per position and column.  The reduced
// row sums go to the job's sum buffer; after the last row the 2m sums are
// inverse-transformed (P per batch) and added to the rows of the next ACC
// buffer.
template <int LOGN, int THREADS, int RB, bool LAZY, bool SMALL0, bool QLOW1, int BLK = 1>
__device__ __forceinline__ void br_job(const DevJob &J, u32 steps_limit, const u64 *__restrict__ ct_in,
                                       const u32 *__restrict__ luts, u64 *ws, u32 *status, u64 *sm) {
    using C = Cfg<LOGN, THREADS, RB, BLK>;
    constexpr int R = C::R;
    constexpr int N = C::N, G = C::G, CPB = C::CPB;
    const KeyDev *K = J.key;
    // (keys of the Q = c 2^32 + 1 kernels have 30-bit limbs: choose_variant)
    const u32 lbits = QLOW1 ? 30u : J.lbits;
    const bool fold_each = J.fold_each != 0;
    const u32 m = J.m, t = J.t, lB = K->l_B, log2B = K->log2_B, n = K->n;
    const ModQ mq = K->mq;
    const u64 Q = mq.Q;
    const u32 qp = 2u * N * m;                 // 2Nm < 2^20
    const u32 Bmask = (u32)((1ull << log2B) - 1);   // digits fit 32 bits (log2 B <= 32)
    const u64 *twp = K->twp, *itwp = K->itwp;
    const u32 tid = threadIdx.x;
    const size_t vec = (size_t)m * 2 * N;
    u64 *acc0 = ws + J.acc_off;
    u64 *acc1 = acc0 + vec;
    u64 *sums = acc1 + vec;
    const u64 *ct = ct_in + J.in_off;
    const u32 *lut = luts + J.lut_off;

    // row split over the blocks of a cluster (1 block: all rows)
    const u32 crank = cluster_rank(), csize = cluster_size();
    const bool split = csize > 1;
    if (!lut_is_negacyclic(lut, t)) {
        // every block of the cluster sees the same table and leaves here
        if (tid == 0 && crank == 0) set_status(status, BM_ENONNEGACYCLIC);
        for (u32 idx = tid; idx < 2 * vec; idx += blockDim.x)
            if ((idx / (2 * N)) % m % csize == crank) acc0[idx] = 0;
        return;
    }
    const u32 *gpre = J.gS ? status + J.gpre : nullptr;
    // Split barrier between a batch's multiply-accumulate and the next
    // transform's second store.  Every thread arrives once after the
    // barrier below (completing phase 0, as if a multiply-accumulate had
    // preceded the first batch) and once after each multiply-accumulate, and
    // waits once per batch, on the parity of the phase its previous arrival
    // belongs to; the block barrier before each multiply-accumulate keeps
    // every thread within one phase of the others.
    __shared__ __align__(8) u64 mac_bar_word;
    u64 *const mac_bar = &mac_bar_word;
    if (tid == 0) mbar_init(mac_bar, blockDim.x);
    u32 mac_parity = 0;
    acc_init(acc0, lut, ct[n] % qp, m, t, N, Q, J.gS, J.gSinv, gpre, crank, csize);
    // forward twiddle pairs to shared memory (read by every transform), in
    // the transposed order of ntr::twiddle_slot
    u64 *tws = sm + (C::REGIONS + C::DBYTES) / 8;
    for (u32 pos = tid; C::TWSM && pos < (u32)N; pos += C::kThreads) {
        const u32 src = ntr::twiddle_slot<LOGN, RB>(pos);
        tws[2 * pos] = __ldg(twp + 2 * src);
        tws[2 * pos + 1] = __ldg(twp + 2 * src + 1);
    }
    // combo c = (pair, digit) as pair | (digit log2 B) << 8, so the batches
    // find their digit without dividing by the runtime l_B
    __shared__ u32 ctab[4 * BM_MAX_L_B];
    if (tid < 4 * lB) ctab[tid] = (tid / lB) | (((tid % lB) * log2B) << 8);
    if (split) cluster_sync(); else __syncthreads();
    mbar_arrive(mac_bar);

    const u32 p = tid / C::T;          // polynomial slot within a batch
    const u32 l = tid % C::T;          // thread within the polynomial
    const u32 pc = p / G, pg = p % G;  // its combo within the batch and row within the group
    ntr::Swap sw{sm + (size_t)p * N, sm + (size_t)(C::P + p) * N, 0};
    u64 *dbuf = sm + (size_t)2 * C::P * N;     // [G][4][N] row differences (DSM), or one pair's [N] (DPAIR)
    const u64 qb = Q << log2B;                 // Q * B, for the exact small first stage (LAZY, not QLOW1)
    const u64 lmask = (1ull << lbits) - 1;     // Karatsuba limb mask
    const u32 ncomb = 4 * lB;
    const size_t rgsw = (size_t)2 * lB * 2 * N;

    // Limb products of a transform value xv with the key words of the two
    // columns: x1 b1, x0 b0 and (x0 + x1)(b0 + b1) accumulate with
    // mad.wide.u32 (one multiplier instruction each, the addition included).
    // xv's limbs are split once (funnel shift: lbits <= 31 and xv <
    // 2^(lbits + 32)) for both columns.  The key stores per position the low
    // limbs of both columns in w0 and their high limbs in w1 (32-bit halves),
    // so one 64-bit addition w0 + w1 forms both columns' limb sums b0 + b1
    // (each below 2^32: no carry crosses the halves).
    const u32 lmask32 = (u32)lmask;
    auto kara2 = [&](u64 xv, u64 w0, u64 w1, u64 (&kh)[2], u64 (&kl)[2], u64 (&km)[2]) {
        if constexpr (QLOW1) {
            asm("{\n\t.reg .u32 v0, v1, x0, x1, xs, a0, a1, as, c0, c1, cs;\n\t.reg .u64 s;\n\t"
                "mov.b64 {v0, v1}, %6;\n\t"
                "shf.r.clamp.b32 x1, v0, v1, 30;\n\t"
                "and.b32 x0, v0, 1073741823;\n\t"
                "add.u32 xs, x0, x1;\n\t"
                "mov.b64 {a0, c0}, %7;\n\t"
                "mov.b64 {a1, c1}, %8;\n\t"
                "add.u64 s, %7, %8;\n\t"
                "mov.b64 {as, cs}, s;\n\t"
                "mad.wide.u32 %0, x1, a1, %0;\n\t"
                "mad.wide.u32 %1, x0, a0, %1;\n\t"
                "mad.wide.u32 %2, xs, as, %2;\n\t"
                "mad.wide.u32 %3, x1, c1, %3;\n\t"
                "mad.wide.u32 %4, x0, c0, %4;\n\t"
                "mad.wide.u32 %5, xs, cs, %5;\n\t}"
                : "+l"(kh[0]), "+l"(kl[0]), "+l"(km[0]), "+l"(kh[1]), "+l"(kl[1]), "+l"(km[1])
                : "l"(xv), "l"(w0), "l"(w1));
            return;
        }
        asm("{\n\t.reg .u32 v0, v1, x0, x1, xs, a0, a1, as, c0, c1, cs;\n\t.reg .u64 s;\n\t"
            "mov.b64 {v0, v1}, %6;\n\t"
            "shf.r.clamp.b32 x1, v0, v1, %9;\n\t"
            "and.b32 x0, v0, %10;\n\t"
            "add.u32 xs, x0, x1;\n\t"
            "mov.b64 {a0, c0}, %7;\n\t"
            "mov.b64 {a1, c1}, %8;\n\t"
            "add.u64 s, %7, %8;\n\t"
            "mov.b64 {as, cs}, s;\n\t"
            "mad.wide.u32 %0, x1, a1, %0;\n\t"
            "mad.wide.u32 %1, x0, a0, %1;\n\t"
            "mad.wide.u32 %2, xs, as, %2;\n\t"
            "mad.wide.u32 %3, x1, c1, %3;\n\t"
            "mad.wide.u32 %4, x0, c0, %4;\n\t"
            "mad.wide.u32 %5, xs, cs, %5;\n\t}"
            : "+l"(kh[0]), "+l"(kl[0]), "+l"(km[0]), "+l"(kh[1]), "+l"(kl[1]), "+l"(km[1])
            : "l"(xv), "l"(w0), "l"(w1), "r"(lbits), "r"(lmask32));
    };

    // one pair's difference in shared memory serves batches that each take
    // digits of a single pair (CPB divides l_B; G = 1)
    const bool dpair = C::DPAIR && G == 1 && lB % CPB == 0;
    u64 *cur = acc0, *nxt = acc1;
    const u32 steps = steps_limit < n ? steps_limit : n;
    for (u32 k = 0; k < steps; k++) {
        // a_k mod q' (q' = 2Nm is a power of two for power-of-two m); the
        // rows of the step share c = -a_k, a_k and their quotients by m
        const u64 ctk = ct[k];
        const u32 ak = (qp & (qp - 1)) == 0 ? (u32)ctk & (qp - 1) : (u32)(ctk % qp);
        u32 ca[2], cb[2];
#pragma unroll
        for (int sg = 0; sg < 2; sg++) {
            const u32 cv = sg == 0 ? (ak ? qp - ak : 0u) : ak;
            ca[sg] = cv / m;
            cb[sg] = cv - ca[sg] * m;
        }
        const u64 *bsk_k = K->bsk + (size_t)k * 2 * rgsw;
        for (u32 r0 = crank * G; r0 < m; r0 += G * csize) {
            u64 lo[G][2][C::PPTR], hi[G][2][C::PPTR];
#pragma unroll
            for (int g = 0; g < G; g++)
#pragma unroll
                for (int j = 0; j < C::PPTR; j++) lo[g][0][j] = hi[g][0][j] = lo[g][1][j] = hi[g][1][j] = 0;
            if constexpr (C::RED) {
                // this thread's row sums start at zero in the sum buffer
#pragma unroll
                for (int g = 0; g < G; g++)
#pragma unroll
                    for (int j = 0; j < C::PPT; j++) {
                        const u32 q = tid + C::kThreads * j;
                        if (r0 + g < m && q < (u32)N) {
                            sums[((size_t)(r0 + g) * 2) * N + q] = 0;
                            sums[((size_t)(r0 + g) * 2 + 1) * N + q] = 0;
                        }
                    }
            }
            // source row and monomial exponent of P(c) for rows r0 + g,
            // c = -a_k (sign 0) and c = a_k (sign 1), Eq. (ex1:BPc)
            u32 rsrc[G][2], rexp[G][2];
#pragma unroll
            for (int g = 0; g < G; g++)
#pragma unroll
                for (int sg = 0; sg < 2; sg++) {
                    const u32 r = r0 + g;
                    mmpm_row_ab(ca[sg], cb[sg], r < m ? r : 0, m, 2 * N, J.gS, gpre, rsrc[g][sg], rexp[g][sg]);
                }
            // D_(row, sign, comp) = P(c) ACC - ACC into drow: coefficient idx of
            // x^e src is src[idx - e] for idx >= e, else -src[idx - e + N]
            // (e < N; for e >= N the two cases swap sign)
            auto build_d = [&](u32 g, u32 pair, u64 *drow) {
                const u32 r = r0 + g;
                const u32 sgn = pair >> 1, comp = pair & 1;
                const u64 *srow = cur + (rsrc[g][sgn] * 2 + comp) * (u32)N;
                const u64 *orow = cur + (r * 2 + comp) * (u32)N;
                const u32 e = rexp[g][sgn];
                const bool flip = e >= (u32)N;
                const u32 es = flip ? e - N : e;
                // this thread's loads of the row issued together, four
                // coefficients at a time
                constexpr int ITER = (N + C::kThreads - 1) / C::kThreads;
                constexpr int CH = ITER < 4 ? ITER : 4;
#pragma unroll
                for (int i0 = 0; i0 < ITER; i0 += CH) {
                    u64 v[CH], o[CH];
#pragma unroll
                    for (int it = 0; it < CH; it++) {
                        const u32 idx = tid + (i0 + it) * C::kThreads;
                        if (idx < (u32)N) {
                            const bool wrap = idx < es;
                            v[it] = acc_load(srow + (wrap ? idx + N - es : idx - es), split);
                            o[it] = acc_load(orow + idx, split);
                        }
                    }
#pragma unroll
                    for (int it = 0; it < CH; it++) {
                        const u32 idx = tid + (i0 + it) * C::kThreads;
                        if (idx < (u32)N) {
                            const bool wrap = idx < es;
                            const u64 sv = (wrap != flip) ? sub_mod(0, v[it], Q) : v[it];
                            drow[idx] = sub_mod(sv, o[it], Q);
                        }
                    }
                }
            };
            if constexpr (C::DSM) {
                // all four differences of the row (G = 1): per coefficient the
                // four rotated source words and the row's own two words are
                // requested together, one L2 round trip for the row
                static_assert(G == 1, "one row per group");
                constexpr int ITER = (N + C::kThreads - 1) / C::kThreads;
                const u64 *srow[4], *orow[2];
                u32 es[4];
                bool flip[4];
#pragma unroll
                for (int pair = 0; pair < 4; pair++) {
                    const u32 sgn = pair >> 1, comp = pair & 1;
                    srow[pair] = cur + (rsrc[0][sgn] * 2 + comp) * (u32)N;
                    const u32 e = rexp[0][sgn];
                    flip[pair] = e >= (u32)N;
                    es[pair] = flip[pair] ? e - N : e;
                }
                orow[0] = cur + (r0 * 2) * (u32)N;
                orow[1] = cur + (r0 * 2 + 1) * (u32)N;
#pragma unroll
                for (int it = 0; it < ITER; it++) {
                    const u32 idx = tid + it * C::kThreads;
                    if (idx < (u32)N) {
                        u64 v[4], o[2];
#pragma unroll
                        for (int pair = 0; pair < 4; pair++) {
                            const bool wrap = idx < es[pair];
                            v[pair] = acc_load(srow[pair] + (wrap ? idx + N - es[pair] : idx - es[pair]), split);
                        }
                        o[0] = acc_load(orow[0] + idx, split);
                        o[1] = acc_load(orow[1] + idx, split);
#pragma unroll
                        for (int pair = 0; pair < 4; pair++) {
                            const bool wrap = idx < es[pair];
                            const u64 sv = (wrap != flip[pair]) ? sub_mod(0, v[pair], Q) : v[pair];
                            dbuf[pair * N + idx] = sub_mod(sv, o[pair & 1], Q);
                        }
                    }
                }
                __syncthreads();
            }
            for (u32 c0 = 0; c0 < ncomb; c0 += CPB) {
                if constexpr (C::DPAIR) {
                    // the first batch of a (sign, component) pair builds its
                    // difference; every thread read the previous pair's before
                    // the previous batch's barrier preceding its
                    // multiply-accumulate
                    const u32 b0 = ctab[c0];
                    if (dpair && (b0 >> 8) == 0) {
                        build_d(0, b0 & 255u, dbuf);
                        __syncthreads();
                    }
                }
                // --- this thread's digit polynomial, transformed into shared memory
                const u32 c = c0 + pc, r = r0 + pg;
                const bool active = pc < (u32)CPB && c < ncomb && r < m;
                u64 x[R];
                const u32 ce = ctab[c < ncomb ? c : 0u];
                const u32 pair = ce & 255u, sh = ce >> 8;
                if (active) {
                    if (C::DSM || dpair) {
                        const u64 *dp = dbuf + (C::DSM ? ((size_t)pg * 4 + pair) * N : 0);
#pragma unroll
                        for (int i = 0; i < R; i++) x[i] = (u32)(dp[l + C::T * i] >> sh) & Bmask;
                    } else {
                        const u32 sgn = pair >> 1, comp = pair & 1;
                        const u64 *srow = cur + ((size_t)rsrc[pg][sgn] * 2 + comp) * N;
                        const u64 *orow = cur + ((size_t)r * 2 + comp) * N;
#pragma unroll
                        for (int i = 0; i < R; i++) {
                            const u32 idx = l + C::T * i;
                            const u64 D = sub_mod(rotated_coeff(srow, idx, rexp[pg][sgn], N, Q, split),
                                                  acc_load(orow + idx, split), Q);
                            x[i] = (u32)(D >> sh) & Bmask;
                        }
                    }
                }
                // The second store of the transform rewrites the region every
                // thread read in the previous batch's multiply-accumulate: wait
                // for all of the block's arrivals after those reads (a split
                // barrier, so a thread that has finished its multiply-accumulate
                // goes on with this batch's digits and first transform phase).
                auto wait_mac = [&]() {
                    mbar_wait(mac_bar, mac_parity, status);
                    mac_parity ^= 1u;
                };
                u64 *out = ntr::fwd_to_smem<LOGN, RB, LAZY, SMALL0, QLOW1, C::TWSM>(x, sw, l, active,
                                                                                    C::TWSM ? tws : twp, Q,
                                                                                    mq.one_sh, qb, wait_mac);
                // regions of the other polynomials of the batch sit at stride N;
                // polynomial cc G + g holds combo c0 + cc of row r0 + g
                const u64 *slots = out - (size_t)p * N;
                // --- multiply-accumulate against the key rows of the batch's combos
                // (combo c = (sign, component, digit) is key row c of the step).
                // Limb products x1 b1, x0 b0 and (x0 + x1)(b0 + b1) are summed over
                // the batch in 64-bit registers, then folded into the 128-bit row
                // sums as hi 2^(2 lbits) + (mid - hi - lo) 2^lbits + lo.
                const u64 *bsk_c0 = bsk_k + (size_t)c0 * 2 * N;
                const u32 nc = ncomb - c0 < (u32)CPB ? ncomb - c0 : (u32)CPB;
                const bool full = nc == (u32)CPB && !fold_each;
                // The next position's key words for the first PRE combos (all of a
                // batch of at most 4, half of a larger one) are loaded while the
                // current position is multiplied.
                // (not at 64 registers per thread, 1024 threads per SM: the extra words
                // spilled and measured 4% slower at N = 2048 and 4096)
                constexpr bool PIPE = C::PPT > 1 && (int)C::kThreads * C::PPT == N && C::kThreads * BLK < 1024;
                constexpr int PRE = CPB <= 4 ? CPB : CPB / 2;
                u64 bnext[PIPE ? PRE : 1][2];
                // (Requesting the first key words before the barrier below, to
                // overlap their latency with the wait, measured slower with 1024
                // threads: the held words spilled.)
                __syncthreads();
                if constexpr (PIPE) {
                    if (full) {
#pragma unroll
                        for (int cc = 0; cc < PRE; cc++) {
                            key_load2(bsk_c0 + (size_t)cc * 2 * N + 2 * tid, bnext[cc][0], bnext[cc][1]);
                        }
                    }
                }
#pragma unroll
                for (int j = 0; j < C::PPT; j++) {
                    const u32 q = tid + C::kThreads * j;
                    if (q < (u32)N) {
                        const u32 sq = ntr::swz<RB>(q);
                        u64 kh[G][2], kl[G][2], km[G][2];
#pragma unroll
                        for (int g = 0; g < G; g++) kh[g][0] = kl[g][0] = km[g][0] = kh[g][1] = kl[g][1] = km[g][1] = 0;
                        auto fold = [&]() {
#pragma unroll
                            for (int g = 0; g < G; g++)
#pragma unroll
                                for (int col = 0; col < 2; col++) {
                                    if constexpr (C::RED) {
                                        u64 *sp = sums + ((size_t)(r0 + g) * 2 + col) * N + q;
                                        u64 l0 = *sp, h0 = 0;
                                        add128(l0, h0, kl[g][col]);
                                        add128_shl(l0, h0, km[g][col] - kh[g][col] - kl[g][col], lbits);
                                        add128_shl(l0, h0, kh[g][col], 2 * lbits);
                                        *sp = reduce128q<QLOW1>(l0, h0, mq);
                                    } else {
                                        add128(lo[g][col][j], hi[g][col][j], kl[g][col]);
                                        add128_shl(lo[g][col][j], hi[g][col][j], km[g][col] - kh[g][col] - kl[g][col],
                                                   lbits);
                                        add128_shl(lo[g][col][j], hi[g][col][j], kh[g][col], 2 * lbits);
                                    }
                                    kh[g][col] = kl[g][col] = km[g][col] = 0;
                                }
                        };
                        if (full) {
                            // full batch: the position's key words are requested first
                            u64 bv[CPB][2];
                            if constexpr (PIPE) {
#pragma unroll
                                for (int cc = 0; cc < PRE; cc++) {
                                    bv[cc][0] = bnext[cc][0];
                                    bv[cc][1] = bnext[cc][1];
                                }
#pragma unroll
                                for (int cc = PRE; cc < CPB; cc++) {
                                    key_load2(bsk_c0 + (size_t)cc * 2 * N + 2 * q, bv[cc][0], bv[cc][1]);
                                }
                                if (j + 1 < C::PPT) {
#pragma unroll
                                    for (int cc = 0; cc < PRE; cc++) {
                                        key_load2(bsk_c0 + (size_t)cc * 2 * N + 2 * (q + C::kThreads), bnext[cc][0],
                                                  bnext[cc][1]);
                                    }
                                }
                            } else if constexpr (C::KC < CPB) {
                                // KC combos' key words at a time (register budget)
#pragma unroll
                                for (int k0 = 0; k0 < CPB; k0 += C::KC) {
                                    u64 kv[C::KC][2];
#pragma unroll
                                    for (int cc = 0; cc < C::KC; cc++) {
                                        key_load2(bsk_c0 + (size_t)(k0 + cc) * 2 * N + 2 * q, kv[cc][0], kv[cc][1]);
                                    }
#pragma unroll
                                    for (int cc = 0; cc < C::KC; cc++)
#pragma unroll
                                        for (int g = 0; g < G; g++) {
                                            if (G == 1 || r0 + g < m) {
                                                const u64 xv = slots[(size_t)((k0 + cc) * G + g) * N + sq];
                                                kara2(xv, kv[cc][0], kv[cc][1], kh[g], kl[g], km[g]);
                                            }
                                        }
                                }
                            } else {
#pragma unroll
                                for (int cc = 0; cc < CPB; cc++) {
                                    key_load2(bsk_c0 + (size_t)cc * 2 * N + 2 * q, bv[cc][0], bv[cc][1]);
                                }
                            }
                            if constexpr (PIPE || C::KC == CPB) {
#pragma unroll
                            for (int cc = 0; cc < CPB; cc++)
#pragma unroll
                                for (int g = 0; g < G; g++) {
                                    if (G == 1 || r0 + g < m) {
                                        const u64 xv = slots[(size_t)(cc * G + g) * N + sq];
                                        kara2(xv, bv[cc][0], bv[cc][1], kh[g], kl[g], km[g]);
                                    }
                                }
                            }
                        } else {
                            for (u32 cc = 0; cc < nc; cc++) {
                                u64 b0, b1;
                                key_load2(bsk_c0 + (size_t)cc * 2 * N + 2 * q, b0, b1);
#pragma unroll
                                for (int g = 0; g < G; g++) {
                                    if (G == 1 || r0 + g < m) {
                                        const u64 xv = slots[(size_t)(cc * G + g) * N + sq];
                                        kara2(xv, b0, b1, kh[g], kl[g], km[g]);
                                    }
                                }
                                if (fold_each) fold();
                            }
                        }
                        fold();
                    }
                }
                // this thread's reads of the batch's results are done
                mbar_arrive(mac_bar);
            }
            // --- reduced row sums (NTT domain) to the sum buffer
#pragma unroll
            for (int g = 0; g < G; g++) {
                const u32 r = r0 + g;
                if (G == 1 || r < m) {
#pragma unroll
                    for (int j = 0; j < C::PPT; j++) {
                        const u32 q = tid + C::kThreads * j;
                        if (q < (u32)N) {
                            if constexpr (!C::RED) {     // (RED: already there)
                                sums[((size_t)r * 2) * N + q] = reduce128q<QLOW1>(lo[g][0][j], hi[g][0][j], mq);
                                sums[((size_t)r * 2 + 1) * N + q] = reduce128q<QLOW1>(lo[g][1][j], hi[g][1][j], mq);
                            }
                        }
                    }
                }
            }
        }
        __syncthreads();
        // inverse twiddle pairs into the row-difference buffer, free until the
        // next step (transposed order of ntr::inv_twiddle_slot)
        const u64 *itw_use = itwp;
        if constexpr (C::DSM) {
            for (u32 pos = tid; pos < (u32)N; pos += C::kThreads) {
                const u32 src = ntr::inv_twiddle_slot<LOGN, RB>(pos);
                dbuf[2 * pos] = __ldg(itwp + 2 * src);
                dbuf[2 * pos + 1] = __ldg(itwp + 2 * src + 1);
            }
            itw_use = dbuf;
        }
        // --- inverse transforms of this block's 2 mr row sums (rows crank +
        // csize i), ACC update
        const u32 mr = crank < m ? (m - 1 - crank) / csize + 1 : 0;
        for (u32 u0 = 0; u0 < 2 * mr; u0 += C::P) {
            const u32 ui = u0 + p;
            const bool active = ui < 2 * mr;
            const u32 u = 2 * (crank + csize * (ui >> 1)) + (ui & 1);
            u64 x[R];
            u64 *in = sw.take();
            if (active) {
                const u64 *sp = sums + (size_t)u * N;
#pragma unroll
                for (int i = 0; i < R; i++) x[i] = sp[l + C::T * i];
                ntr::store_field<RB, LOGN - RB>(x, in, l);    // index l + T i
            }
            __syncthreads();
            ntr::inv_from_smem<LOGN, RB, QLOW1, C::DSM, LAZY && QLOW1>(x, in, sw, l, active, itw_use, Q, mq.one_sh);
            if (active) {
                const size_t base = (size_t)u * N;
#pragma unroll
                for (int i = 0; i < R; i++) {
                    const size_t o = base + l + C::T * i;
                    nxt[o] = add_mod(cur[o], x[i], Q);
                }
            }
        }
        if (split) cluster_sync(); else __syncthreads();
        u64 *tmp = cur;
        cur = nxt;
        nxt = tmp;
    }
}

}  // namespace brk

// Ring degrees above 8192: the single-polynomial layout of the plaintext-size
// sweep at log t >= 8 (Sec. 5, Tables 1-2, N = 2^(log t + 6)), m = 1.
//
// A polynomial of 8N bytes no longer fits one thread block's shared memory,
// so its transforms run in two passes over global memory and the CMux steps
// of a launch run as a sequence of kernels (digits, column pass, row pass,
// multiply-accumulate, inverse row and column passes, accumulator update).
// The transform is the one of ntt.cuh: Cooley-Tukey with psi^bitrev twiddles
// in place (bit-reversed output), Gentleman-Sande inverse without N^-1.
// With N = N1 N2, forward stages 0 .. log N1 - 1 pair elements of the columns
// {c + N2 t : t < N1} (stage s, group t >> (log N1 - s): the same twiddle for
// every column); stages log N1 + s', s' < log N2, pair elements of the rows
// [r N2, (r + 1) N2) (group (r << s') + (o >> (log N2 - s')), twiddle index
// ((N1 + r) << s') + (o >> (log N2 - s'))).  The inverse runs the row pass
// first, then the column pass, each stage backwards.  Each pass keeps
// 2^4 values per thread in registers for four stages at a time (one
// shared-memory exchange and barrier per four stages).  For Q = c 2^32 + 1
// the butterflies are lazy (forward values below 8Q, inverse below 4Q, brought
// into [0, Q) where a transform ends); other moduli correct every butterfly.
#include "blind_rotate.cuh"

namespace bign {

constexpr u32 TC = 16;     // columns per block of the column pass
constexpr u32 TR = 32;     // rows per block of the row pass
constexpr u32 NT = 256;    // threads per block (three blocks per SM: at most 80 registers)

// Threads per block of a column pass: the work items of its four-stage
// chunk, TC 2^(log N1 - 4) (128 at N1 = 128), at most NT.
inline u32 col_threads(u32 l1) { return (TC << (l1 - 4)) < NT ? NT / 2 : NT; }

// Polynomial p of launch row y: a flat array of polynomials, or the
// digit / sum buffers of job y (after the job's three [2][N] accumulator
// buffers: ACC ping-pong, row sums; then 4 l_B digit polynomials).
struct LocFlat {
    u64 *base;
    const KeyDev *key;
    u32 per;
    __device__ u64 *poly(u32 y, u32 p) const { return base + ((size_t)y * per + p) * key->N; }
    __device__ const KeyDev &k(u32) const { return *key; }
    __device__ u32 count(u32) const { return per; }
};
struct LocJobs {
    const DevJob *jobs;
    u64 *ws;
    u32 sel;    // 0: digit polynomials, 1: the two row sums
    __device__ u64 *poly(u32 y, u32 p) const {
        const DevJob &J = jobs[y];
        const size_t vec = (size_t)2 * J.N;
        return ws + J.acc_off + (sel == 0 ? 3 * vec : 2 * vec) + (size_t)p * J.N;
    }
    __device__ const KeyDev &k(u32 y) const { return *jobs[y].key; }
    __device__ u32 count(u32 y) const { return sel == 0 ? 4 * jobs[y].key->l_B : 2; }
};

__device__ __forceinline__ void split_log(u32 logN, u32 &l1, u32 &l2) {
    l1 = logN / 2;
    l2 = logN - l1;
}

// ---- Arithmetic of the passes.  For Q = c 2^32 + 1 < 2^60 (QL) the
// butterflies are the lazy ones of modarith.cuh: forward values in [0, 8Q),
// inverse values in [0, 4Q), brought into [0, Q) where a transform ends;
// for other moduli every butterfly corrects into [0, Q).
__device__ __forceinline__ bool qlow1_of(u64 Q) { return (Q & 0xffffffffull) == 1 && Q < (1ull << 60); }

template <bool QL>
struct Arith {
    u64 Q, fourQ;
    u32 c;
    __device__ explicit Arith(u64 q) : Q(q), fourQ(4 * q), c((u32)(q >> 32)) {}
    __device__ __forceinline__ void fwd(u64 &X, u64 &Y, u64 W, u64 Wsh) const {
        if constexpr (QL) {
            bfly_ct_qlow1(X, Y, W, Wsh, c, fourQ);
        } else {
            const u64 U = X, V = mul_shoup(Y, W, Wsh, Q);
            X = add_mod(U, V, Q);
            Y = sub_mod(U, V, Q);
        }
    }
    __device__ __forceinline__ void inv(u64 &X, u64 &Y, u64 W, u64 Wsh) const {
        if constexpr (QL) {
            bfly_gs_qlow1(X, Y, W, Wsh, c, fourQ);
        } else {
            const u64 U = X, V = Y;
            X = add_mod(U, V, Q);
            Y = mul_shoup(U + Q - V, W, Wsh, Q);
        }
    }
    // forward butterfly of the first stage on digits X, Y < 2^32 (QL): Y W
    // by the one-quotient product (below 3Q), both outputs below 4Q + X
    __device__ __forceinline__ void fwd_small(u64 &X, u64 &Y, u64 W, u64 Wsh) const {
        if constexpr (QL) {
            const u64 T = small_mul_qlow1(Y, W, Wsh, c), x = X;
            X = add64c(x, T);
            Y = sub64c(add64c(x, fourQ), T);
        } else {
            fwd(X, Y, W, Wsh);
        }
    }
    // the last forward stage's value (below 8Q) into [0, Q)
    __device__ __forceinline__ u64 fwd_final(u64 x) const {
        if constexpr (QL) return csub63(csub63(csub63(x, fourQ), 2 * Q), Q);
        else return x;
    }
    // the last inverse stage's value (below 4Q) into [0, Q)
    __device__ __forceinline__ u64 inv_final(u64 x) const {
        if constexpr (QL) return csub63(csub63(x, 2 * Q), Q);
        else return x;
    }
};

// Row tiles in shared memory: element e of row q at q qs + e + (e >> 4), one
// pad word per 16 (qs = N2 + N2 / 16), so that the later stages' strided
// accesses fall on distinct banks.  Column tiles: element e of column q at
// q + TC e.
__device__ __forceinline__ u32 row_stride(u32 N2) { return N2 + N2 / 16; }
__device__ __forceinline__ u32 row_at(u32 q, u32 qs, u32 e) { return q * qs + e + (e >> 4); }

// Stage s0 + r of a register chunk (see pass_chunk), r a constant so that
// every index into x is one.  SM0: stage 0 of a forward transform of digits.
template <int R, int r, bool INV, bool QL, bool SM0>
__device__ __forceinline__ void chunk_stage(u64 (&x)[1 << R], const u64 *__restrict__ tp, u32 tb, u32 s0, u32 G,
                                            const Arith<QL> &A) {
    constexpr u32 h = 1u << (R - 1 - r);
#pragma unroll
    for (u32 gi = 0; gi < (1u << r); gi++) {
        const ulonglong2 W = __ldg(reinterpret_cast<const ulonglong2 *>(tp) + ((tb << (s0 + r)) + (G << r) + gi));
#pragma unroll
        for (u32 j = 0; j < h; j++) {
            if constexpr (INV) A.inv(x[gi * 2 * h + j], x[gi * 2 * h + j + h], W.x, W.y);
            else if constexpr (SM0 && r == 0) A.fwd_small(x[gi * 2 * h + j], x[gi * 2 * h + j + h], W.x, W.y);
            else A.fwd(x[gi * 2 * h + j], x[gi * 2 * h + j + h], W.x, W.y);
        }
    }
}

// The chunk's stages in order: r = 0 .. R - 1 forward, R - 1 .. 0 inverse.
template <int R, int k, bool INV, bool QL, bool SM0>
__device__ __forceinline__ void chunk_stages(u64 (&x)[1 << R], const u64 *__restrict__ tp, u32 tb, u32 s0, u32 G,
                                             const Arith<QL> &A) {
    if constexpr (k < R) {
        chunk_stage<R, INV ? R - 1 - k : k, INV, QL, SM0>(x, tp, tb, s0, G, A);
        chunk_stages<R, k + 1, INV, QL, SM0>(x, tp, tb, s0, G, A);
    }
}

// Stages s0 .. s0 + R - 1 (forward) or s0 + R - 1 .. s0 (inverse) of the
// length-2^l transforms of nseq sequences, 2^R values per work item in
// registers.  Item (q, G, J), G < 2^s0, J < 2^(l - s0 - R), holds the
// elements G 2^(l - s0) + J + i 2^(l - s0 - R), i < 2^R, of sequence q; at
// stage s0 + r it pairs i with i + 2^(R - 1 - r) under twiddle
// ((tb0 + (q & qmask)) << (s0 + r)) + (G << r) + (i >> (R - r)), which is
// the twiddle of the stage's group in the whole transform (columns: tb0 = 1,
// qmask = 0; rows: tb0 = N1 + first row, qmask = rows per polynomial - 1).
// ROW: J varies fastest across threads, then G, then the row; columns: the
// column varies fastest.  ld(q, e) and st(q, e, v) fetch and put element e
// of sequence q (the shared-memory tile, or global memory for the first and
// last chunk of a pass).  NTH threads per block; SM0: the chunk starts at
// stage 0 of a forward transform of digits below 2^32.
template <int R, bool INV, bool ROW, bool QL, u32 NTH, bool SM0, class Ld, class St>
__device__ __forceinline__ void pass_chunk(u32 l, u32 s0, u32 nseq, u32 tb0, u32 qmask, const u64 *__restrict__ tp,
                                           const Arith<QL> &A, Ld &ld, St &st) {
    constexpr u32 V = 1u << R;
    const u32 lJ = l - s0 - R, items = nseq << (l - R);
    for (u32 w = threadIdx.x; w < items; w += NTH) {
        u32 q, G, J;
        if constexpr (ROW) {
            J = w & ((1u << lJ) - 1);
            G = (w >> lJ) & ((1u << s0) - 1);
            q = w >> (l - R);
        } else {
            q = w & (TC - 1);
            J = (w >> 4) & ((1u << lJ) - 1);
            G = (w >> 4) >> lJ;
        }
        const u32 e0 = (G << (l - s0)) + J;
        u64 x[V];
#pragma unroll
        for (u32 i = 0; i < V; i++) x[i] = ld(q, e0 + (i << lJ));
        chunk_stages<R, 0, INV, QL, SM0>(x, tp, tb0 + (q & qmask), s0, G, A);
#pragma unroll
        for (u32 i = 0; i < V; i++) st(q, e0 + (i << lJ), x[i]);
    }
}

// The stages of one pass.  The ring degrees of this path (2^14 .. 2^16) give
// passes of 7 or 8 stages: two register chunks, stages 0-3 and 4 .. l - 1
// (the inverse takes them in the other order), one barrier between them.
// The first chunk takes its values through ld_first, the second puts them
// through st_last; in between they sit in the tile sm (row tiles of stride
// qs).  The caller synchronises before sm is reused.  NTH threads per
// block; SM0: a forward transform of digits below 2^32.
template <bool INV, bool ROW, bool QL, u32 NTH = NT, bool SM0 = false, class Ld, class St>
__device__ __forceinline__ void pass_stages(u64 *sm, u32 l, u32 nseq, u32 qs, u32 tb0, u32 qmask,
                                            const u64 *__restrict__ tp, const Arith<QL> &A, Ld &&ld_first,
                                            St &&st_last) {
    auto ld_sm = [&](u32 q, u32 e) { return ROW ? sm[row_at(q, qs, e)] : sm[q + TC * e]; };
    auto st_sm = [&](u32 q, u32 e, u64 v) {
        if constexpr (ROW) sm[row_at(q, qs, e)] = v;
        else sm[q + TC * e] = v;
    };
    if constexpr (!INV) {
        pass_chunk<4, INV, ROW, QL, NTH, SM0>(l, 0, nseq, tb0, qmask, tp, A, ld_first, st_sm);
        __syncthreads();
        if (l == 8) pass_chunk<4, INV, ROW, QL, NTH, false>(l, 4, nseq, tb0, qmask, tp, A, ld_sm, st_last);
        else pass_chunk<3, INV, ROW, QL, NTH, false>(l, 4, nseq, tb0, qmask, tp, A, ld_sm, st_last);
    } else {
        if (l == 8) pass_chunk<4, INV, ROW, QL, NTH, false>(l, 4, nseq, tb0, qmask, tp, A, ld_first, st_sm);
        else pass_chunk<3, INV, ROW, QL, NTH, false>(l, 4, nseq, tb0, qmask, tp, A, ld_first, st_sm);
        __syncthreads();
        pass_chunk<4, INV, ROW, QL, NTH, false>(l, 0, nseq, tb0, qmask, tp, A, ld_sm, st_last);
    }
}

// Column pass of TC columns from c0 of polynomial a, in place.  smem: N1 TC
// words.  The forward pass leaves its values lazy (the row pass continues
// them); the inverse pass ends the transform.
template <bool INV, bool QL, u32 NTH>
__device__ void cols_body(u64 *sm, u64 *a, u32 c0, u32 l1, u32 N2, const KeyDev &K) {
    const Arith<QL> A(K.mq.Q);
    u64 *col = a + c0;
    pass_stages<INV, false, QL, NTH>(
        sm, l1, TC, 0, 1, 0, INV ? K.itwp : K.twp, A, [&](u32 q, u32 e) { return col[q + (size_t)N2 * e]; },
        [&](u32 q, u32 e, u64 v) { col[q + (size_t)N2 * e] = INV ? A.inv_final(v) : v; });
}

// Row pass of rows [r0, r0 + TR) of polynomial a (a at row r0), in place.
// smem: TR (N2 + N2 / 16) words.  The forward pass ends the transform; the
// inverse one leaves its values lazy for the column pass.
template <bool INV, bool QL>
__device__ void rows_body(u64 *sm, u64 *a, u32 r0, u32 l1, u32 l2, const KeyDev &K) {
    const Arith<QL> A(K.mq.Q);
    const u32 N2 = 1u << l2;
    pass_stages<INV, true, QL>(
        sm, l2, TR, row_stride(N2), (1u << l1) + r0, TR - 1, INV ? K.itwp : K.twp, A,
        [&](u32 q, u32 e) { return a[(size_t)q * N2 + e]; },
        [&](u32 q, u32 e, u64 v) { a[(size_t)q * N2 + e] = INV ? v : A.fwd_final(v); });
}

// Column pass: block (x = p * (N2 / TC) + chunk, y) transforms columns
// [chunk TC, (chunk + 1) TC) of polynomial p of row y.
template <bool INV, class Loc, u32 NTH>
__global__ void __launch_bounds__(NTH, 3 * NT / NTH) k_cols(Loc loc, u32 per) {
    extern __shared__ u64 sm[];
    const KeyDev &K = loc.k(blockIdx.y);
    u32 l1, l2;
    split_log(K.logN, l1, l2);
    const u32 N2 = 1u << l2, chunks = N2 / TC;
    const u32 p = blockIdx.x / chunks, c0 = (blockIdx.x % chunks) * TC;
    if (p >= per || p >= loc.count(blockIdx.y)) return;
    u64 *a = loc.poly(blockIdx.y, p);
    if (qlow1_of(K.mq.Q)) cols_body<INV, true, NTH>(sm, a, c0, l1, N2, K);
    else cols_body<INV, false, NTH>(sm, a, c0, l1, N2, K);
}

// Row pass: block (x = p * (N1 / TR) + chunk, y) transforms rows
// [chunk TR, (chunk + 1) TR) of polynomial p of row y.
template <bool INV, class Loc>
__global__ void __launch_bounds__(NT, 3) k_rows(Loc loc, u32 per) {
    extern __shared__ u64 sm[];
    const KeyDev &K = loc.k(blockIdx.y);
    u32 l1, l2;
    split_log(K.logN, l1, l2);
    const u32 N1 = 1u << l1, N2 = 1u << l2, chunks = N1 / TR;
    const u32 p = blockIdx.x / chunks, r0 = (blockIdx.x % chunks) * TR;
    if (p >= per || p >= loc.count(blockIdx.y)) return;
    u64 *a = loc.poly(blockIdx.y, p) + (size_t)r0 * N2;
    if (qlow1_of(K.mq.Q)) rows_body<INV, true>(sm, a, r0, l1, l2, K);
    else rows_body<INV, false>(sm, a, r0, l1, l2, K);
}

// Dynamic shared memory of a kernel, with the largest shared-memory carveout
// (several blocks of these kernels share an SM).
template <class F>
bm_status smem_attrs(F *kernel, size_t bytes) {
    BM_CUDA_TRY(cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes));
    BM_CUDA_TRY(cudaFuncSetAttribute(kernel, cudaFuncAttributePreferredSharedMemoryCarveout,
                                     (int)cudaSharedmemCarveoutMaxShared));
    return BM_OK;
}

// The row pass alone (the step's inverse starts with it).
template <class Loc>
bm_status transform_rows(Loc loc, u32 rows, u32 per, u32 N, bool inverse, cudaStream_t st) {
    u32 logN = 0;
    while ((1u << logN) < N) logN++;
    const u32 l1 = logN / 2, l2 = logN - l1, N1 = 1u << l1, N2 = 1u << l2;
    if (l1 < 7 || l2 > 8) return BM_EINVAL;     // passes of 7 or 8 stages (pass_stages)
    const size_t smr = (size_t)TR * (N2 + N2 / 16) * 8;
    auto kr = inverse ? k_rows<true, Loc> : k_rows<false, Loc>;
    bm_status s0 = smem_attrs(kr, smr);
    if (s0 != BM_OK) return s0;
    kr<<<dim3(per * (N1 / TR), rows), NT, smr, st>>>(loc, per);
    BM_CUDA_TRY(cudaGetLastError());
    return BM_OK;
}

template <class Loc>
bm_status transform(Loc loc, u32 rows, u32 per, u32 N, bool inverse, cudaStream_t st) {
    u32 logN = 0;
    while ((1u << logN) < N) logN++;
    const u32 l1 = logN / 2, l2 = logN - l1, N1 = 1u << l1, N2 = 1u << l2;
    if (l1 < 7 || l2 > 8) return BM_EINVAL;     // passes of 7 or 8 stages (pass_stages)
    const size_t smc = (size_t)N1 * TC * 8, smr = (size_t)TR * (N2 + N2 / 16) * 8;
    const u32 nc = col_threads(l1);
    auto kc = nc == NT ? (inverse ? k_cols<true, Loc, NT> : k_cols<false, Loc, NT>)
                       : (inverse ? k_cols<true, Loc, NT / 2> : k_cols<false, Loc, NT / 2>);
    auto kr = inverse ? k_rows<true, Loc> : k_rows<false, Loc>;
    bm_status s0 = smem_attrs(kc, smc);
    if (s0 == BM_OK) s0 = smem_attrs(kr, smr);
    if (s0 != BM_OK) return s0;
    const dim3 gc(per * (N2 / TC), rows), gr(per * (N1 / TR), rows);
    if (!inverse) {
        kc<<<gc, nc, smc, st>>>(loc, per);
        kr<<<gr, NT, smr, st>>>(loc, per);
    } else {
        kr<<<gr, NT, smr, st>>>(loc, per);
        kc<<<gc, nc, smc, st>>>(loc, per);
    }
    BM_CUDA_TRY(cudaGetLastError());
    return BM_OK;
}

// ACC <- P(b) (0, v_test floor(Q/t)) (blind_rotate.cuh: acc_init), or zero
// and BM_ENONNEGACYCLIC for a table that is not negacyclic.
__global__ void k_init(const DevJob *__restrict__ jobs, const u64 *__restrict__ ct_in,
                       const u32 *__restrict__ luts, u64 *ws, u32 *status) {
    const DevJob &J = jobs[blockIdx.x];
    const KeyDev &K = *J.key;
    u64 *acc0 = ws + J.acc_off;
    const u32 *lut = luts + J.lut_off;
    if (!lut_is_negacyclic(lut, J.t)) {
        if (threadIdx.x == 0) set_status(status, BM_ENONNEGACYCLIC);
        for (u32 i = threadIdx.x; i < 4 * J.N; i += blockDim.x) acc0[i] = 0;
        return;
    }
    const u32 *gpre = J.gS ? status + J.gpre : nullptr;
    const u32 qp = 2u * J.N * J.m;
    acc_init(acc0, lut, ct_in[J.in_off + K.n] % qp, 1, J.t, J.N, K.mq.Q, J.gS, J.gSinv, gpre);
}

// ---- Step kernels: digits fused into the forward column pass, the
// multiply-accumulate into the forward row pass, the accumulator update into
// the inverse column pass (three passes over the digit polynomials per step
// where separate kernels made six).

// Digits + forward column pass of step k: block (x = pair (N2 / TC) + chunk,
// y = job) builds the difference of (sign, component) pair `pair` on its TC
// columns, then for every digit transforms the digit columns (stages
// 0 .. log N1 - 1) into the job's digit polynomial pair l_B + d.  smem:
// 2 N1 TC words (the difference, the digit tile).
template <bool QL, u32 NTH>
__device__ void digits_cols_body(u64 *sm, const DevJob &J, const KeyDev &K, const u64 *__restrict__ ct_in, u64 *ws,
                                 u32 k, const u32 *status) {
    const Arith<QL> A(K.mq.Q);
    u32 l1, l2;
    split_log(K.logN, l1, l2);
    const u32 N = J.N, N1 = 1u << l1, N2 = 1u << l2, chunks = N2 / TC;
    const u32 pair = blockIdx.x / chunks, c0 = (blockIdx.x % chunks) * TC;
    const u32 lB = K.l_B, log2B = K.log2_B;
    const u64 Q = K.mq.Q, Bmask = (1ull << log2B) - 1;
    const size_t vec = (size_t)2 * N;
    const u64 *cur = ws + J.acc_off + ((k & 1) ? vec : 0);
    u64 *X = ws + J.acc_off + 3 * vec;
    const u32 qp = 2u * N;
    const u32 ak = (u32)(ct_in[J.in_off + k] % qp);
    const u32 *gpre = J.gS ? status + J.gpre : nullptr;
    const u32 sgn = pair >> 1, comp = pair & 1;
    u32 src, e;
    mmpm_row(sgn == 0 ? (ak ? qp - ak : 0u) : ak, 0, 1, 2 * N, J.gS, gpre, src, e);
    const u64 *row = cur + (size_t)comp * N;
    u64 *Dt = sm, *tile = sm + N1 * TC;
    for (u32 x = threadIdx.x; x < N1 * TC; x += NTH) {
        const u32 i = c0 + x % TC + N2 * (x / TC);
        Dt[x] = sub_mod(rotated_coeff(row, i, e, N, Q), row[i], Q);
    }
    for (u32 d = 0; d < lB; d++) {
        __syncthreads();     // the difference is complete; the previous digit is out of the tile
        const u32 sh = d * log2B;
        u64 *a = X + (size_t)(pair * lB + d) * N + c0;
        pass_stages<false, false, QL, NTH, true>(
            tile, l1, TC, 0, 1, 0, K.twp, A, [&](u32 q, u32 e) { return (Dt[q + TC * e] >> sh) & Bmask; },
            [&](u32 q, u32 e, u64 v) { a[q + (size_t)N2 * e] = v; });
    }
}

template <u32 NTH>
__global__ void __launch_bounds__(NTH, 3 * NT / NTH) k_digits_cols(const DevJob *__restrict__ jobs, const u64 *__restrict__ ct_in,
                                                    u64 *ws, u32 k, const u32 *status) {
    extern __shared__ u64 sm[];
    const DevJob &J = jobs[blockIdx.y];
    const KeyDev &K = *J.key;
    if (k >= K.n) return;
    if (qlow1_of(K.mq.Q)) digits_cols_body<true, NTH>(sm, J, K, ct_in, ws, k, status);
    else digits_cols_body<false, NTH>(sm, J, K, ct_in, ws, k, status);
}

// Forward row pass of all 4 l_B digit polynomials on rows [r0, r0 + trm)
// (trm a power of two), then the multiply-accumulate of those positions
// against the key rows of step k (exact 128-bit sums, reduced) into the
// job's row sums.  The transform outputs enter the sums unreduced: below 8Q
// (QL, Q < 2^60) times key words below Q, 4 l_B <= 32 of them stay below
// 2^128.  Block (x = row chunk, y = job); smem: 4 l_B trm (N2 + N2 / 16)
// words.
template <bool QL>
__device__ void rows_mac_body(u64 *sm, const DevJob &J, const KeyDev &K, u64 *ws, u32 k, u32 trm) {
    const Arith<QL> A(K.mq.Q);
    u32 l1, l2;
    split_log(K.logN, l1, l2);
    const u32 N = J.N, N1 = 1u << l1, N2 = 1u << l2, qs = row_stride(N2);
    const u32 r0 = blockIdx.x * trm, nc = 4 * K.l_B, lb = K.lbits, w = trm * N2;
    const size_t vec = (size_t)2 * N;
    const u64 *X = ws + J.acc_off + 3 * vec;
    u64 *sums = ws + J.acc_off + 2 * vec;
    // row q = c trm + rr of the tile is row r0 + rr of digit polynomial c
    const u32 ltrm = __ffs(trm) - 1;
    const u64 *Xr = X + (size_t)r0 * N2;
    pass_stages<false, true, QL>(
        sm, l2, nc * trm, qs, N1 + r0, trm - 1, K.twp, A,
        [&](u32 q, u32 e) { return Xr[(size_t)(q >> ltrm) * N + ((q & (trm - 1)) << l2) + e]; },
        [&](u32 q, u32 e, u64 v) { sm[row_at(q, qs, e)] = v; });
    __syncthreads();
    const u64 *bk = K.bsk + (size_t)k * 2 * (2 * K.l_B * 2 * N);
    for (u32 pos = threadIdx.x; pos < w; pos += NT) {
        const size_t i = (size_t)r0 * N2 + pos;
        const u32 rr = pos >> l2, o = pos & (N2 - 1);
        u64 lo0 = 0, hi0 = 0, lo1 = 0, hi1 = 0;
        for (u32 c = 0; c < nc; c += 4) {      // nc = 4 l_B: four combos' loads in flight
            ulonglong2 wv[4];
            u64 x[4];
#pragma unroll
            for (u32 u = 0; u < 4; u++) {
                wv[u] = __ldg(reinterpret_cast<const ulonglong2 *>(bk + (size_t)(c + u) * 2 * N + 2 * i));
                x[u] = sm[row_at((c + u) * trm + rr, qs, o)];
            }
#pragma unroll
            for (u32 u = 0; u < 4; u++) {
                mac128(lo0, hi0, x[u], (wv[u].x & 0xffffffffull) + ((wv[u].y & 0xffffffffull) << lb));
                mac128(lo1, hi1, x[u], (wv[u].x >> 32) + ((wv[u].y >> 32) << lb));
            }
        }
        sums[i] = reduce128(lo0, hi0, K.mq);
        sums[N + i] = reduce128(lo1, hi1, K.mq);
    }
}

__global__ void __launch_bounds__(NT, 3) k_rows_mac(const DevJob *__restrict__ jobs, u64 *ws, u32 k, u32 trm) {
    extern __shared__ u64 sm[];
    const DevJob &J = jobs[blockIdx.y];
    const KeyDev &K = *J.key;
    if (k >= K.n) return;
    if (qlow1_of(K.mq.Q)) rows_mac_body<true>(sm, J, K, ws, k, trm);
    else rows_mac_body<false>(sm, J, K, ws, k, trm);
}

// Inverse column pass of the two row sums (stages log N1 - 1 .. 0) fused
// with the accumulator update of step k.  Block (x = comp (N2 / TC) +
// chunk, y = job); smem N1 TC words.
template <bool QL, u32 NTH>
__device__ void cols_inv_update_body(u64 *sm, const DevJob &J, const KeyDev &K, u64 *ws, u32 k) {
    const Arith<QL> A(K.mq.Q);
    u32 l1, l2;
    split_log(K.logN, l1, l2);
    const u32 N = J.N, N2 = 1u << l2, chunks = N2 / TC;
    const u32 comp = blockIdx.x / chunks, c0 = (blockIdx.x % chunks) * TC;
    const u64 Q = K.mq.Q;
    const size_t vec = (size_t)2 * N;
    const u64 *cur = ws + J.acc_off + ((k & 1) ? vec : 0) + (size_t)comp * N;
    u64 *nxt = ws + J.acc_off + ((k & 1) ? 0 : vec) + (size_t)comp * N;
    const u64 *a = ws + J.acc_off + 2 * vec + (size_t)comp * N;
    pass_stages<true, false, QL, NTH>(
        sm, l1, TC, 0, 1, 0, K.itwp, A, [&](u32 q, u32 e) { return a[c0 + q + (size_t)N2 * e]; },
        [&](u32 q, u32 e, u64 v) {
            const size_t i = c0 + q + (size_t)N2 * e;
            nxt[i] = add_mod(cur[i], A.inv_final(v), Q);
        });
}

template <u32 NTH>
__global__ void __launch_bounds__(NTH, 3 * NT / NTH) k_cols_inv_update(const DevJob *__restrict__ jobs, u64 *ws, u32 k) {
    extern __shared__ u64 sm[];
    const DevJob &J = jobs[blockIdx.y];
    const KeyDev &K = *J.key;
    if (k >= K.n) return;
    if (qlow1_of(K.mq.Q)) cols_inv_update_body<true, NTH>(sm, J, K, ws, k);
    else cols_inv_update_body<false, NTH>(sm, J, K, ws, k);
}

// RGSW row finish of key generation (the formula of keygen.cu, elementwise):
// a (mask) and e (error) rows already transformed.
__global__ void k_bsk_finish(const u64 *__restrict__ a, const u64 *__restrict__ e, const int8_t *__restrict__ s,
                             const u64 *__restrict__ zhat, u64 *__restrict__ bsk, const KeyDev *Kp, size_t row0) {
    const KeyDev &K = *Kp;
    const u32 N = K.N, lB = K.l_B;
    const u64 Q = K.mq.Q;
    const size_t r = blockIdx.y, row_id = row0 + r;
    const u32 row = (u32)(row_id % (2 * lB));
    const u32 sgn = (u32)((row_id / (2 * lB)) % 2);
    const int sk = s[row_id / (4 * lB)];
    const bool mu = sgn == 0 ? sk > 0 : sk < 0;
    u64 g = 0;
    if (mu) {
        u64 gg = 1 % Q;
        for (u32 d = 0; d < row % lB; d++) {
            u64 lo = 0, hi = 0;
            mac128(lo, hi, gg, 1ull << K.log2_B);
            gg = reduce128(lo, hi, K.mq);
        }
        g = gg;
    }
    const u64 g0 = row < lB ? g : 0, g1 = row < lB ? 0 : g;
    const u64 lmask = (1ull << K.lbits) - 1;
    u64 *o = bsk + row_id * 2 * N;
    for (u32 i = blockIdx.x * blockDim.x + threadIdx.x; i < N; i += gridDim.x * blockDim.x) {
        const u64 ah = a[r * N + i], eh = e[r * N + i];
        u64 lo = 0, hi = 0;
        mac128(lo, hi, ah, zhat[i]);
        add128(lo, hi, eh);
        add128(lo, hi, g1);
        const u64 c1 = reduce128(lo, hi, K.mq);
        const u64 c0 = add_mod(ah, g0, Q);
        const u64 w0 = mul_shoup(c0, K.ninv, K.ninv_sh, Q), w1 = mul_shoup(c1, K.ninv, K.ninv_sh, Q);
        o[2 * i] = (w0 & lmask) | ((w1 & lmask) << 32);
        o[2 * i + 1] = (w0 >> K.lbits) | ((w1 >> K.lbits) << 32);
    }
}

__global__ void k_pointwise(u64 *a, const u64 *__restrict__ b, size_t words, const KeyDev *Kp) {
    const KeyDev &K = *Kp;
    for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < words; i += (size_t)gridDim.x * blockDim.x) {
        u64 lo = 0, hi = 0;
        mac128(lo, hi, a[i], b[i]);
        a[i] = mul_shoup(reduce128(lo, hi, K.mq), K.ninv, K.ninv_sh, K.mq.Q);
    }
}

__global__ void k_reduce_copy(u64 *dst, const u64 *__restrict__ src, size_t words, u64 Q) {
    for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < words; i += (size_t)gridDim.x * blockDim.x)
        dst[i] = src[i] % Q;
}

}  // namespace bign

size_t bm_big_extra_words(u32 N, u32 l_B) { return N > BM_MAX_N_BLOCK ? (size_t)4 * l_B * N : 0; }

// Forward or inverse transform of `count` contiguous polynomials of key K.
bm_status bm_big_ntt(u64 *polys, uint32_t count, const KeyDev *d_key, u32 N, bool inverse, cudaStream_t st) {
    if (!count) return BM_OK;
    return bign::transform(bign::LocFlat{polys, d_key, count}, 1, count, N, inverse, st);
}

// BSK rows [row0, row0 + rows) from their transformed masks and errors.
bm_status bm_big_bsk_finish(const u64 *a, const u64 *e, const int8_t *d_s, const u64 *d_zhat, u64 *d_bsk,
                            const KeyDev *d_key, u32 N, size_t row0, uint32_t rows, cudaStream_t st) {
    const dim3 grid((N + 255) / 256 < 64 ? (N + 255) / 256 : 64, rows);
    bign::k_bsk_finish<<<grid, 256, 0, st>>>(a, e, d_s, d_zhat, d_bsk, d_key, row0);
    BM_CUDA_TRY(cudaGetLastError());
    return BM_OK;
}

// Negacyclic products a b (count pairs of N words, any values below 2^64)
// through the two-pass transform; scratch: count N words.
bm_status bm_big_poly_mul(const u64 *a, const u64 *b, uint32_t count, u64 *out, u64 *scratch, const KeyDev *d_key,
                          u64 Q, u32 N, cudaStream_t st) {
    const size_t words = (size_t)count * N;
    const unsigned blocks = (unsigned)((words + 255) / 256 < 4096 ? (words + 255) / 256 : 4096);
    bign::k_reduce_copy<<<blocks, 256, 0, st>>>(out, a, words, Q);
    bign::k_reduce_copy<<<blocks, 256, 0, st>>>(scratch, b, words, Q);
    BM_CUDA_TRY(cudaGetLastError());
    bm_status s;
    if ((s = bm_big_ntt(out, count, d_key, N, false, st)) != BM_OK) return s;
    if ((s = bm_big_ntt(scratch, count, d_key, N, false, st)) != BM_OK) return s;
    bign::k_pointwise<<<blocks, 256, 0, st>>>(out, scratch, words, d_key);
    BM_CUDA_TRY(cudaGetLastError());
    return bm_big_ntt(out, count, d_key, N, true, st);
}

// Blind rotation of jobs [0, cnt) of `jobs` (device table; ring degree N
// above 8192, m = 1): CMux steps 0 .. steps - 1 of every job (fewer for jobs
// whose key has fewer), the final ACC where the one-block kernels leave it.
bm_status bm_launch_br_big(u32 N, const DevJob *jobs, uint32_t cnt, u32 steps, const uint64_t *ct_in,
                           const uint32_t *lut, u64 *ws_acc, u32 *status, cudaStream_t st) {
    if (!cnt) return BM_OK;
    bign::k_init<<<cnt, 1024, 0, st>>>(jobs, ct_in, lut, ws_acc, status);
    BM_CUDA_TRY(cudaGetLastError());
    u32 logN = 0;
    while ((1u << logN) < N) logN++;
    const u32 l1 = logN / 2, l2 = logN - l1, N1 = 1u << l1, N2 = 1u << l2;
    // rows per block of the row pass + multiply-accumulate: the digit rows of
    // every combo a key can have (4 BM_MAX_L_B), 64 KB of values (68 KB with
    // the row padding)
    const u32 ncmax = 4 * BM_MAX_L_B;
    u32 trm = 1;
    while (2 * trm * ncmax * N2 <= 8192 && 2 * trm <= N1) trm *= 2;     // a power of two
    const size_t sm_dc = (size_t)2 * N1 * bign::TC * 8, sm_rm = (size_t)ncmax * trm * (N2 + N2 / 16) * 8,
                 sm_ci = (size_t)N1 * bign::TC * 8;
    if (l1 < 7 || l2 > 8) return BM_EINVAL;     // passes of 7 or 8 stages (pass_stages)
    bm_status s0;
    const u32 nc = bign::col_threads(l1);
    auto kdc = nc == bign::NT ? bign::k_digits_cols<bign::NT> : bign::k_digits_cols<bign::NT / 2>;
    auto kci = nc == bign::NT ? bign::k_cols_inv_update<bign::NT> : bign::k_cols_inv_update<bign::NT / 2>;
    if ((s0 = bign::smem_attrs(kdc, sm_dc)) != BM_OK) return s0;
    if ((s0 = bign::smem_attrs(bign::k_rows_mac, sm_rm)) != BM_OK) return s0;
    if ((s0 = bign::smem_attrs(kci, sm_ci)) != BM_OK) return s0;
    const dim3 g_dc(4 * (N2 / bign::TC), cnt), g_rm(N1 / trm, cnt), g_ci(2 * (N2 / bign::TC), cnt);
    for (u32 k = 0; k < steps; k++) {
        kdc<<<g_dc, nc, sm_dc, st>>>(jobs, ct_in, ws_acc, k, status);
        bign::k_rows_mac<<<g_rm, bign::NT, sm_rm, st>>>(jobs, ws_acc, k, trm);
        BM_CUDA_TRY(cudaGetLastError());
        // inverse: row pass of the two sums, then the column pass with the update
        bm_status s = bign::transform_rows(bign::LocJobs{jobs, ws_acc, 1}, cnt, 2, N, true, st);
        if (s != BM_OK) return s;
        kci<<<g_ci, nc, sm_ci, st>>>(jobs, ws_acc, k);
        BM_CUDA_TRY(cudaGetLastError());
    }
    return BM_OK;
}

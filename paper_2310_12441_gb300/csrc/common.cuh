// Internal types shared by the translation units of libbootmmpm.
#pragma once
#include <cuda_runtime.h>
#include <cstdint>
#include <cstdio>

#include "modarith.cuh"
#include "../../include/bootmmpm.h"

#define BM_MAX_L_B 8
#define BM_MAX_M 1024   // q' = 2Nm <= 2^23 (u32 arithmetic on exponents)
#define BM_MAX_N_BLOCK 8192   // largest ring degree of the one-block kernels
#define BM_MAX_N 65536        // largest ring degree (above BM_MAX_N_BLOCK: big.cu, m = 1)
#define BM_MAX_QP (1u << 23)

// Device-resident description of one evaluation key set.  One copy lives in
// device memory (owned by the bm_eval_key) so jobs can point at it.
struct KeyDev {
    const u64 *bsk;    // [n][2][2 l_B][N][2], NTT domain, scaled by N^-1 (limbs, see lbits)
    const u64 *ksk;    // [N][l_ks][B_ks - 1][n + 1]
    const u64 *tw;     // forward twiddles psi^bitrev(k), k in [0, N)
    const u64 *twsh;   // their Shoup companions
    const u64 *itw;    // inverse twiddles psi^-bitrev(k)
    const u64 *itwsh;
    const u64 *twp;    // forward (twiddle, companion) pairs, 16-byte aligned
    const u64 *itwp;   // inverse pairs
    ModQ mq;
    u64 ninv, ninv_sh; // N^-1 mod Q and companion
    u64 ks_pq;         // floor(P 2^64 / Q), P = B_ks^l_ks
    u32 n, N, logN, log2_B, l_B, log2_Bks, l_ks;
    u32 lbits;         // BSK words b (column 0) and b' (column 1) of a position are stored as
                       // (b mod 2^lbits) | (b' mod 2^lbits) 2^32, (b >> lbits) | (b' >> lbits) 2^32
};

// One job as the kernels see it.
struct DevJob {
    const KeyDev *key;
    u32 m, t, N, n;
    u64 in_off, lut_off, out_off;
    u64 acc_off;       // element offset of the job's three [m][2][N] buffers in the
                       // workspace: ACC ping-pong and the per-step row sums
    u32 variant;       // arithmetic variant of the key's modulus (BR_V_* flags)
    u32 lbits;         // Karatsuba limb width (see limb_plan on the host)
    u32 fold_each;     // 1: a batch's limb products may exceed 64 bits, fold per combo
    u32 gS;            // generator: 0 for P(1) of Example 1, else S = sum u mod 2N (odd)
    u32 gSinv;         // S^-1 mod 2N
    u32 pad;
    u64 gpre;          // u32 offset from the workspace start of the prefix sums
                       // pre[k] = (u_0 + ... + u_{k-1}) mod 2N, k in [0, m] (gS != 0)
};

// Arithmetic variants of the blind rotation, chosen per key set on the host.
#define BR_V_QLOW1 1u   // Q = c 2^32 + 1: one-multiply q Q
#define BR_V_LAZY 2u    // correction-free forward NTT with an exact first stage

// Arithmetic variant of a key set (BR_V_* flags):
//  - BR_V_QLOW1: Q = c 2^32 + 1 < 2^60;
//  - BR_V_LAZY: the correction-free forward transform.  With Q = c 2^32 + 1
//    it needs (1 + 4 log2 N) Q < 2^62 (its outputs go unreduced into the
//    multiply-accumulate, whose limbs then stay at most 31 bits) and the
//    correction-free inverse 128 Q < 2^64; otherwise (1 + 4 log2 N) Q < 2^64
//    and the exact first stage B + Q B + 4 Q (log2 N - 1) < 2^64 with B < 2^32.
inline u32 choose_variant(const bm_key_params &p) {
    typedef unsigned __int128 u128;
    u32 logN = 0;
    while ((1u << logN) < p.N) logN++;
    const u128 lim = (u128)1 << 64, Q = p.Q, B = (u128)1 << p.log2_B;
    u32 v = 0;
    // (Q < 2^60 keeps every value the Q = c 2^32 + 1 butterflies correct below 2^63)
    bool qlow1 = (p.Q & 0xffffffffull) == 1 && p.Q < (1ull << 60);
    // the Q = c 2^32 + 1 kernels also fix the multiply-accumulate's limbs at
    // 30 bits (limb_plan: the transform outputs' bound below 2^60, above 2^58)
    const bool lazy1 = (1 + 4 * (u128)logN) * Q < ((u128)1 << 62) && 128 * Q < lim;
    const u128 xmax1 = lazy1 ? (1 + 4 * (u128)logN) * Q : Q;
    if (qlow1 && !(xmax1 - 1 >= ((u128)1 << 58) && xmax1 - 1 < ((u128)1 << 60))) qlow1 = false;
    if (qlow1) {
        if (lazy1) v |= BR_V_LAZY;
        v |= BR_V_QLOW1;
    } else if ((1 + 4 * (u128)logN) * Q < lim && p.log2_B <= 31 && B + Q * B + 4 * Q * (logN - 1) < lim &&
               128 * Q < lim) {
        v |= BR_V_LAZY;
    }
    return v;
}

// Karatsuba limbs of the multiply-accumulate (blind_rotate.cuh): a transform
// value x < xmax and a key word b < Q are split at `lbits` bits, and the
// products x1 b1, x0 b0, (x0 + x1)(b0 + b1) of a batch of CPB combos are
// summed in 64-bit registers.  xmax is where the forward transform leaves
// its outputs (ntr::fwd_to_smem): (1 + 4 log2 N) Q (lazy, Q = c 2^32 + 1,
// unreduced), 2Q (lazy), Q.  lbits = ceil(bits(xmax - 1) / 2); fold_each when
// CPB times the largest middle product could reach 2^64 (then each combo is
// folded at once).  The key stores every BSK word b pre-split as
// (b mod 2^lbits) | (b >> lbits) 2^32.
inline void limb_plan(const bm_key_params &p, u32 variant, u32 &lbits, u32 &fold_each) {
    typedef unsigned __int128 u128;
    u32 logN = 0;
    while ((1u << logN) < p.N) logN++;
    const u128 xmax = (variant & BR_V_LAZY) ? ((variant & BR_V_QLOW1) ? (1 + 4 * (u128)logN) : 2) * (u128)p.Q
                                            : (u128)p.Q;
    u32 bits = 0;
    while (bits < 66 && ((xmax - 1) >> bits)) bits++;
    lbits = (bits + 1) / 2;
    const u128 lim = (u128)1 << lbits;
    const u128 sx = (lim - 1) + ((xmax - 1) >> lbits), sb = (lim - 1) + ((u128)(p.Q - 1) >> lbits);
    const u32 cpb = 512u / (p.N / 16u);     // the largest CPB of any kernel shape
    // (the variant rules keep xmax and Q below 2^62, so the limb sums sx and
    // sb stay below 2^32)
    fold_each = (u128)cpb * sx * sb >= ((u128)1 << 64);
}

// Workspace header: [0] status word, [1 + c] job counter of persistent class c.
#define BM_WS_COUNTER_WORD 1
#define BM_MAX_CLASSES 15

// Host-side evaluation key.
struct bm_eval_key {
    int device;
    bm_key_params p;
    u32 logN;
    KeyDev host_view;  // same fields as the device copy (pointers are device pointers)
    KeyDev *d_view;
    u64 *d_bsk, *d_ksk, *d_tables;
    size_t bytes;
};

struct bm_secret_key {
    bm_key_params p;
    int8_t *s;
    int8_t *z;
};

#define BM_CUDA_TRY(call)                                                   \
    do {                                                                    \
        cudaError_t e_ = (call);                                            \
        if (e_ != cudaSuccess) {                                            \
            fprintf(stderr, "bootmmpm: %s failed: %s (%s:%d)\n", #call,     \
                    cudaGetErrorString(e_), __FILE__, __LINE__);            \
            return BM_ECUDA;                                                \
        }                                                                   \
    } while (0)

// Workspace header: the device status word sits at offset 0.
#define BM_WS_HEADER 256

// Persistent blind rotation of one class of jobs (same ring degree 1024..4096
// and arithmetic variant; persistent.cu): one block per SM pulls the class's
// jobs from `counter` (a word of the workspace header).  dry: only set the
// kernel's attributes (before a stream capture).
bm_status bm_launch_persistent_class(u32 N, u32 variant, u32 shape, const DevJob *d_jobs, uint32_t count,
                                     uint32_t steps, const uint64_t *ct_in, const uint32_t *lut, u64 *ws_acc,
                                     u32 *status, u32 *counter, int device, bool dry, cudaStream_t st);

// Blind-rotation launches per ring degree (br_n*.cu): jobs [0, cnt) of
// `jobs`, all of ring degree N and arithmetic variant `variant`, with kernel
// shape `shape` (br_launch.cuh); dry: only set the kernel's attributes.
#define BM_NUM_SHAPES 5
bm_status bm_launch_br_small(u32 N, u32 variant, u32 shape, const DevJob *jobs, uint32_t cnt, u32 mmax,
                             u32 max_cluster, u32 steps, const uint64_t *ct_in, const uint32_t *lut, u64 *ws_acc,
                             u32 *status, cudaStream_t st, bool dry);
bm_status bm_launch_br_n1024(u32 variant, u32 shape, const DevJob *jobs, uint32_t cnt, u32 mmax, u32 max_cluster,
                             u32 steps, const uint64_t *ct_in, const uint32_t *lut, u64 *ws_acc, u32 *status,
                             cudaStream_t st, bool dry);
bm_status bm_launch_br_n2048(u32 variant, u32 shape, const DevJob *jobs, uint32_t cnt, u32 mmax, u32 max_cluster,
                             u32 steps, const uint64_t *ct_in, const uint32_t *lut, u64 *ws_acc, u32 *status,
                             cudaStream_t st, bool dry);
bm_status bm_launch_br_n4096(u32 variant, u32 shape, const DevJob *jobs, uint32_t cnt, u32 mmax, u32 max_cluster,
                             u32 steps, const uint64_t *ct_in, const uint32_t *lut, u64 *ws_acc, u32 *status,
                             cudaStream_t st, bool dry);
bm_status bm_launch_br_n8192(u32 variant, u32 shape, const DevJob *jobs, uint32_t cnt, u32 mmax, u32 max_cluster,
                             u32 steps, const uint64_t *ct_in, const uint32_t *lut, u64 *ws_acc, u32 *status,
                             cudaStream_t st, bool dry);

// Ring degrees above BM_MAX_N_BLOCK (big.cu): two-pass transforms in global
// memory, CMux steps as kernel sequences.  Jobs of such degrees have m = 1 and
// 4 l_B N more workspace words (their digit polynomials).
size_t bm_big_extra_words(u32 N, u32 l_B);
bm_status bm_big_ntt(u64 *polys, uint32_t count, const KeyDev *d_key, u32 N, bool inverse, cudaStream_t st);
bm_status bm_big_bsk_finish(const u64 *a, const u64 *e, const int8_t *d_s, const u64 *d_zhat, u64 *d_bsk,
                            const KeyDev *d_key, u32 N, size_t row0, uint32_t rows, cudaStream_t st);
bm_status bm_big_poly_mul(const u64 *a, const u64 *b, uint32_t count, u64 *out, u64 *scratch, const KeyDev *d_key,
                          u64 Q, u32 N, cudaStream_t st);
bm_status bm_launch_br_big(u32 N, const DevJob *jobs, uint32_t cnt, u32 steps, const uint64_t *ct_in,
                           const uint32_t *lut, u64 *ws_acc, u32 *status, cudaStream_t st);

// Host helpers (keygen.cu)
bm_status bm_check_key_params(const bm_key_params *p);
u64 host_mulmod(u64 a, u64 b, u64 Q);

// Persistent blind rotation for uneven batches: one kernel per class of jobs
// that share a ring degree and an arithmetic variant, one block of 512
// threads per SM pulling the class's jobs (longest first) from a counter in
// the workspace header until none are left.
//
// A single kernel switching over every (ring degree, variant) path would
// inline a dozen copies of the rotation into one register allocation: it
// spilled about 9.6 KB per thread.  Per class, the kernel spills at most a
// few bytes.  The host launches the classes concurrently (forked streams,
// longest class first), so the blocks of a later class take over each SM as
// the earlier class runs out of jobs.
#include "br_launch.cuh"

namespace {

// Persistent shapes: those of one block per SM (0: radix 16 x 512 threads,
// 1: radix 8 x 1024 threads, 4: radix 8 x 512 threads).
__host__ __device__ constexpr bool persistent_shape(int logn, int sh) {
    return br_shape(sh).blocks == 1 && br_shape_fits(logn, sh);
}

template <int LOGN, u32 V, int SH>
__global__ void __launch_bounds__(br_shape(SH).threads, 1)
    k_blind_rotate_persistent(const DevJob *__restrict__ jobs, u32 count, u32 steps,
                              const u64 *__restrict__ ct_in, const u32 *__restrict__ luts, u64 *ws,
                              u32 *status, u32 *counter) {
    extern __shared__ __align__(16) u64 sm[];
    constexpr bool lazy = (V & BR_V_LAZY) != 0, q1 = (V & BR_V_QLOW1) != 0;
    // two slots: thread 0 fetches the next index into one while every thread
    // reads the current one from the other; the barrier that ends each job
    // orders the fetch before the read
    __shared__ u32 s_next[2];
    if (threadIdx.x == 0) s_next[0] = atomicAdd(counter, 1u);
    __syncthreads();
    u32 slot = 0;
#pragma unroll 1
    for (;;) {
        const u32 idx = s_next[slot];
        if (idx >= count) break;
        if (threadIdx.x == 0) s_next[slot ^ 1] = atomicAdd(counter, 1u);
        brk::br_job<LOGN, br_shape(SH).threads, br_shape(SH).rb, lazy, lazy || q1, q1, br_shape(SH).blocks>(
            jobs[idx], steps, ct_in, luts, ws, status, sm);
        __syncthreads();
        slot ^= 1;
    }
}

template <int LOGN, u32 V, int SH>
bm_status launch_class(const DevJob *d_jobs, uint32_t count, uint32_t steps, const uint64_t *ct_in,
                       const uint32_t *lut, u64 *ws_acc, u32 *status, u32 *counter, int sms, bool dry,
                       cudaStream_t st) {
    using C = brk::Cfg<LOGN, br_shape(SH).threads, br_shape(SH).rb, br_shape(SH).blocks>;
    auto kern = k_blind_rotate_persistent<LOGN, V, SH>;
    static std::atomic<uint64_t> attr_done{0};
    bm_status s = ensure_smem(kern, C::SMEM, attr_done);
    if (s != BM_OK) return s;
    if (dry) return BM_OK;
    const u32 grid = (u32)sms < count ? (u32)sms : count;
    BM_CUDA_TRY(cudaMemsetAsync(counter, 0, sizeof(u32), st));
    kern<<<grid, C::kThreads, C::SMEM, st>>>(d_jobs, count, steps, (const u64 *)ct_in, lut, ws_acc, status, counter);
    BM_CUDA_TRY(cudaGetLastError());
    return BM_OK;
}

// Shapes other than 0 for the variants of Q = c 2^32 + 1 only (as the
// grouped launches).
template <int LOGN, u32 V>
bm_status launch_class_shape(u32 shape, const DevJob *d_jobs, uint32_t count, uint32_t steps, const uint64_t *ct_in,
                             const uint32_t *lut, u64 *ws_acc, u32 *status, u32 *counter, int sms, bool dry,
                             cudaStream_t st) {
    if constexpr ((V & BR_V_QLOW1) && persistent_shape(LOGN, 1))
        if (shape == 1)
            return launch_class<LOGN, V, 1>(d_jobs, count, steps, ct_in, lut, ws_acc, status, counter, sms, dry, st);
    if constexpr ((V & BR_V_QLOW1) && persistent_shape(LOGN, 4))
        if (shape == 4)
            return launch_class<LOGN, V, 4>(d_jobs, count, steps, ct_in, lut, ws_acc, status, counter, sms, dry, st);
    return launch_class<LOGN, V, 0>(d_jobs, count, steps, ct_in, lut, ws_acc, status, counter, sms, dry, st);
}

template <int LOGN>
bm_status launch_variant(u32 variant, u32 shape, const DevJob *d_jobs, uint32_t count, uint32_t steps,
                         const uint64_t *ct_in, const uint32_t *lut, u64 *ws_acc, u32 *status, u32 *counter, int sms,
                         bool dry, cudaStream_t st) {
    switch (variant) {
        case BR_V_LAZY | BR_V_QLOW1:
            return launch_class_shape<LOGN, BR_V_LAZY | BR_V_QLOW1>(shape, d_jobs, count, steps, ct_in, lut, ws_acc,
                                                                   status, counter, sms, dry, st);
        case BR_V_LAZY:
            return launch_class_shape<LOGN, BR_V_LAZY>(shape, d_jobs, count, steps, ct_in, lut, ws_acc, status,
                                                       counter, sms, dry, st);
        case BR_V_QLOW1:
            return launch_class_shape<LOGN, BR_V_QLOW1>(shape, d_jobs, count, steps, ct_in, lut, ws_acc, status,
                                                        counter, sms, dry, st);
        default:
            return launch_class_shape<LOGN, 0>(shape, d_jobs, count, steps, ct_in, lut, ws_acc, status, counter, sms,
                                               dry, st);
    }
}

}  // namespace

// Ring degrees 1024..4096 only; the host routes other degrees elsewhere.
// dry: only set the kernel's shared-memory limit (before a stream capture).
bm_status bm_launch_persistent_class(u32 N, u32 variant, u32 shape, const DevJob *d_jobs, uint32_t count,
                                     uint32_t steps, const uint64_t *ct_in, const uint32_t *lut, u64 *ws_acc,
                                     u32 *status, u32 *counter, int device, bool dry, cudaStream_t st) {
    int sms = 0;
    BM_CUDA_TRY(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, device));
    switch (N) {
        case 1024:
            return launch_variant<10>(variant, shape, d_jobs, count, steps, ct_in, lut, ws_acc, status, counter, sms,
                                      dry, st);
        case 2048:
            return launch_variant<11>(variant, shape, d_jobs, count, steps, ct_in, lut, ws_acc, status, counter, sms,
                                      dry, st);
        case 4096:
            return launch_variant<12>(variant, shape, d_jobs, count, steps, ct_in, lut, ws_acc, status, counter, sms,
                                      dry, st);
        default: return BM_EINVAL;
    }
}

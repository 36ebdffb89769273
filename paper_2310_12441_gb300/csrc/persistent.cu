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
#include "blind_rotate.cuh"

namespace {

constexpr int kPThreads = 512;

template <int LOGN, u32 V>
__global__ void __launch_bounds__(kPThreads, 1)
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
        brk::br_job<LOGN, kPThreads, lazy, lazy, q1>(jobs[idx], steps, ct_in, luts, ws, status, sm);
        __syncthreads();
        slot ^= 1;
    }
}

template <int LOGN, u32 V>
bm_status launch_class(const DevJob *d_jobs, uint32_t count, uint32_t steps, const uint64_t *ct_in,
                       const uint32_t *lut, u64 *ws_acc, u32 *status, u32 *counter, int sms, bool dry,
                       cudaStream_t st) {
    constexpr size_t smem = brk::Cfg<LOGN, kPThreads>::SMEM;
    auto kern = k_blind_rotate_persistent<LOGN, V>;
    static std::atomic<uint64_t> attr_done{0};
    int dev = 0;
    BM_CUDA_TRY(cudaGetDevice(&dev));
    const uint64_t bit = 1ull << (dev & 63);
    if (!(attr_done.load() & bit)) {
        BM_CUDA_TRY(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
        attr_done.fetch_or(bit);
    }
    if (dry) return BM_OK;
    const u32 grid = (u32)sms < count ? (u32)sms : count;
    BM_CUDA_TRY(cudaMemsetAsync(counter, 0, sizeof(u32), st));
    kern<<<grid, kPThreads, smem, st>>>(d_jobs, count, steps, (const u64 *)ct_in, lut, ws_acc, status, counter);
    BM_CUDA_TRY(cudaGetLastError());
    return BM_OK;
}

template <int LOGN>
bm_status launch_variant(u32 variant, const DevJob *d_jobs, uint32_t count, uint32_t steps, const uint64_t *ct_in,
                         const uint32_t *lut, u64 *ws_acc, u32 *status, u32 *counter, int sms, bool dry,
                         cudaStream_t st) {
    switch (variant) {
        case BR_V_LAZY | BR_V_QLOW1:
            return launch_class<LOGN, BR_V_LAZY | BR_V_QLOW1>(d_jobs, count, steps, ct_in, lut, ws_acc, status,
                                                             counter, sms, dry, st);
        case BR_V_LAZY:
            return launch_class<LOGN, BR_V_LAZY>(d_jobs, count, steps, ct_in, lut, ws_acc, status, counter, sms,
                                                 dry, st);
        case BR_V_QLOW1:
            return launch_class<LOGN, BR_V_QLOW1>(d_jobs, count, steps, ct_in, lut, ws_acc, status, counter, sms,
                                                  dry, st);
        default:
            return launch_class<LOGN, 0>(d_jobs, count, steps, ct_in, lut, ws_acc, status, counter, sms, dry, st);
    }
}

}  // namespace

// Ring degrees 1024..4096 only; the host routes other degrees elsewhere.
// dry: only set the kernel's shared-memory limit (before a stream capture).
bm_status bm_launch_persistent_class(u32 N, u32 variant, const DevJob *d_jobs, uint32_t count, uint32_t steps,
                                     const uint64_t *ct_in, const uint32_t *lut, u64 *ws_acc, u32 *status,
                                     u32 *counter, int device, bool dry, cudaStream_t st) {
    int sms = 0;
    BM_CUDA_TRY(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, device));
    switch (N) {
        case 1024: return launch_variant<10>(variant, d_jobs, count, steps, ct_in, lut, ws_acc, status, counter, sms, dry, st);
        case 2048: return launch_variant<11>(variant, d_jobs, count, steps, ct_in, lut, ws_acc, status, counter, sms, dry, st);
        case 4096: return launch_variant<12>(variant, d_jobs, count, steps, ct_in, lut, ws_acc, status, counter, sms, dry, st);
        default: return BM_EINVAL;
    }
}

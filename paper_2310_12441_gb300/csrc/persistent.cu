// Persistent blind rotation: one block of 512 threads per SM pulls jobs of
// any ring degree and key set from a counter until none are left, so an
// uneven batch (several parameter sets, skewed counts) runs as one launch.
// The host lists the longest jobs first.
#include "blind_rotate.cuh"

namespace {

constexpr int kPThreads = 512;

template <int LOGN, u32 V>
__device__ __forceinline__ void run(const DevJob &J, u32 steps, const u64 *ct_in, const u32 *luts, u64 *ws,
                                    u32 *status, u64 *sm) {
    constexpr bool lazy = (V & BR_V_LAZY) != 0, q1 = (V & BR_V_QLOW1) != 0;
    brk::br_job<LOGN, kPThreads, lazy, lazy, q1>(J, steps, ct_in, luts, ws, status, sm);
}

template <int LOGN>
__device__ __forceinline__ void dispatch_variant(const DevJob &J, u32 steps, const u64 *ct_in,
                                                 const u32 *luts, u64 *ws, u32 *status, u64 *sm) {
    switch (J.variant) {
        case BR_V_LAZY | BR_V_QLOW1: run<LOGN, BR_V_LAZY | BR_V_QLOW1>(J, steps, ct_in, luts, ws, status, sm); break;
        case BR_V_LAZY: run<LOGN, BR_V_LAZY>(J, steps, ct_in, luts, ws, status, sm); break;
        case BR_V_QLOW1: run<LOGN, BR_V_QLOW1>(J, steps, ct_in, luts, ws, status, sm); break;
        default: run<LOGN, 0>(J, steps, ct_in, luts, ws, status, sm); break;
    }
}

__global__ void __launch_bounds__(kPThreads, 1)
    k_blind_rotate_persistent(const DevJob *__restrict__ jobs, u32 count, u32 steps,
                              const u64 *__restrict__ ct_in, const u32 *__restrict__ luts, u64 *ws,
                              u32 *status, u32 *counter) {
    extern __shared__ __align__(16) u64 sm[];
    __shared__ u32 s_next;
    for (;;) {
        if (threadIdx.x == 0) s_next = atomicAdd(counter, 1u);
        __syncthreads();
        const u32 idx = s_next;
        __syncthreads();
        if (idx >= count) break;
        const DevJob J = jobs[idx];
        switch (J.N) {
            case 1024: dispatch_variant<10>(J, steps, ct_in, luts, ws, status, sm); break;
            case 2048: dispatch_variant<11>(J, steps, ct_in, luts, ws, status, sm); break;
            case 4096: dispatch_variant<12>(J, steps, ct_in, luts, ws, status, sm); break;
            default: if (threadIdx.x == 0) atomicCAS(status, 0u, (u32)(-BM_EINVAL)); break;
        }
        __syncthreads();
    }
}

constexpr size_t kSmem = brk::Cfg<11, kPThreads>::SMEM > brk::Cfg<10, kPThreads>::SMEM
                             ? (brk::Cfg<11, kPThreads>::SMEM > brk::Cfg<12, kPThreads>::SMEM
                                    ? brk::Cfg<11, kPThreads>::SMEM
                                    : brk::Cfg<12, kPThreads>::SMEM)
                             : brk::Cfg<10, kPThreads>::SMEM;

}  // namespace

size_t bm_persistent_smem() { return kSmem; }

// Sets the kernel's shared-memory limit once per device (before any capture).
bm_status bm_prepare_persistent_br(int device) {
    static std::atomic<uint64_t> attr_done{0};
    const uint64_t bit = 1ull << (device & 63);
    if (!(attr_done.load() & bit)) {
        BM_CUDA_TRY(cudaFuncSetAttribute(k_blind_rotate_persistent, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)kSmem));
        attr_done.fetch_or(bit);
    }
    return BM_OK;
}

// Ring degrees 1024..4096 only; the host routes other degrees elsewhere.
bm_status bm_launch_persistent_br(const DevJob *d_jobs, uint32_t count, uint32_t steps, const uint64_t *ct_in,
                                  const uint32_t *lut, u64 *ws_acc, u32 *status, u32 *counter, int device,
                                  cudaStream_t st) {
    bm_status s = bm_prepare_persistent_br(device);
    if (s != BM_OK) return s;
    int sms = 0;
    BM_CUDA_TRY(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, device));
    const u32 grid = (u32)sms < count ? (u32)sms : count;
    BM_CUDA_TRY(cudaMemsetAsync(counter, 0, sizeof(u32), st));
    k_blind_rotate_persistent<<<grid, kPThreads, kSmem, st>>>(d_jobs, count, steps, (const u64 *)ct_in, lut,
                                                               ws_acc, status, counter);
    BM_CUDA_TRY(cudaGetLastError());
    return BM_OK;
}

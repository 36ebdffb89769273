// Launch of the blind-rotation kernel (one job per block, or per cluster of
// blocks in latency mode) for every arithmetic variant and kernel shape.
// Included by one translation unit per ring degree (br_n*.cu), so that the
// instances compile in parallel.
#pragma once
#include <atomic>
#include <mutex>
#include <vector>

#include "blind_rotate.cuh"

// Kernel shapes (the autotuner's candidates): 2^rb coefficients per thread in
// the transforms, threads per block, blocks resident per SM.  A shape fits a
// ring degree when whole polynomials fill a batch and the blocks' shared
// memory fits an SM.
struct BrShape {
    int rb, threads, blocks;
};
__host__ __device__ constexpr BrShape br_shape(int sh) {
    return sh == 1 ? BrShape{3, 1024, 1}
         : sh == 2 ? BrShape{4, 256, 2}
         : sh == 3 ? BrShape{3, 512, 2}
         : sh == 4 ? BrShape{3, 512, 1}
                   : BrShape{4, 512, 1};
}
__host__ __device__ constexpr bool br_shape_fits(int logn, int sh) {
    const BrShape b = br_shape(sh);
    const int T = (1 << logn) >> b.rb;
    if (b.threads % T != 0 || b.threads < T) return false;
    const size_t smem = brk::smem_bytes(logn, b.threads, b.rb, b.blocks);
    return smem <= 226 * 1024 && (smem + 1024) * b.blocks <= 228 * 1024;
}

template <int LOGN, int SH, bool LAZY, bool SMALL0, bool QLOW1>
__global__ void __launch_bounds__(br_shape(SH).threads, br_shape(SH).blocks)
    k_blind_rotate(const DevJob *__restrict__ jobs, u32 steps_limit, const u64 *__restrict__ ct_in,
                   const u32 *__restrict__ luts, u64 *ws, u32 *status) {
    extern __shared__ __align__(16) u64 sm[];
    // a cluster of blocks shares one job (rows split); plain launches: 1 block
    brk::br_job<LOGN, br_shape(SH).threads, br_shape(SH).rb, LAZY, SMALL0, QLOW1, br_shape(SH).blocks>(
        jobs[blockIdx.x / cluster_size()], steps_limit, ct_in, luts, ws, status, sm);
}

// Sets the dynamic shared-memory limit of a kernel once per device.
template <typename K>
bm_status ensure_smem(K kern, size_t smem, std::atomic<uint64_t> &done) {
    int dev = 0;
    BM_CUDA_TRY(cudaGetDevice(&dev));
    const uint64_t bit = 1ull << (dev & 63);
    if (!(done.load() & bit)) {
        BM_CUDA_TRY(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
        done.fetch_or(bit);
    }
    return BM_OK;
}

// Blocks per job (thread-block cluster size, rows split) for a launch of
// `cnt` jobs of at most `mmax` rows: the smallest S in {1, 2, 4, 8}, S <=
// min(mmax, max_cluster), that minimises waves(S) x ceil(mmax / S), where
// waves(S) = ceil(cnt / clusters resident at once).  A full batch keeps one
// block per job; a batch of fewer jobs than SMs spreads each job's rows over
// a cluster, cutting its latency by up to S.
template <typename K>
u32 pick_cluster(K kern, u32 threads, size_t smem, u32 cnt, u32 mmax, u32 max_cluster) {
    struct Occ { const void *k; u32 s; int dev; int slots; };
    static std::mutex mu;
    static std::vector<Occ> cache;
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return 1;
    auto slots = [&](u32 S) -> int {
        std::lock_guard<std::mutex> lk(mu);
        for (const Occ &o : cache)
            if (o.k == (const void *)kern && o.s == S && o.dev == dev) return o.slots;
        int n = 0;
        cudaLaunchConfig_t cfg = {};
        cfg.gridDim = dim3(S);
        cfg.blockDim = dim3(threads);
        cfg.dynamicSmemBytes = smem;
        cudaLaunchAttribute at[1];
        at[0].id = cudaLaunchAttributeClusterDimension;
        at[0].val.clusterDim.x = S;
        at[0].val.clusterDim.y = 1;
        at[0].val.clusterDim.z = 1;
        cfg.attrs = at;
        cfg.numAttrs = 1;
        if (cudaOccupancyMaxActiveClusters(&n, kern, &cfg) != cudaSuccess) {
            cudaGetLastError();
            n = 0;
        }
        cache.push_back({(const void *)kern, S, dev, n});
        return n;
    };
    u32 best = 1;
    const int s1 = slots(1);
    if (s1 <= 0) return 1;
    u64 best_cost = (u64)((cnt + s1 - 1) / s1) * mmax;
    for (u32 S = 2; S <= 8 && S <= max_cluster && S <= mmax; S *= 2) {
        const int sl = slots(S);
        if (sl <= 0) break;
        const u64 cost = (u64)((cnt + sl - 1) / sl) * ((mmax + S - 1) / S);
        if (cost < best_cost) {
            best_cost = cost;
            best = S;
        }
    }
    return best;
}

// dry: only set the kernel's attributes and occupancy (done before a
// CUDA-graph capture).
template <int LOGN, int SH, bool LAZY, bool SMALL0, bool QLOW1>
bm_status launch_br_v(const DevJob *jobs, uint32_t cnt, u32 mmax, u32 max_cluster, u32 steps,
                      const uint64_t *ct_in, const uint32_t *lut, u64 *ws_acc, u32 *status, cudaStream_t st,
                      bool dry) {
    using C = brk::Cfg<LOGN, br_shape(SH).threads, br_shape(SH).rb, br_shape(SH).blocks>;
    static std::atomic<uint64_t> attr_done{0};
    auto kern = k_blind_rotate<LOGN, SH, LAZY, SMALL0, QLOW1>;
    bm_status s = ensure_smem(kern, C::SMEM, attr_done);
    if (s != BM_OK) return s;
    const u32 S = max_cluster > 1 ? pick_cluster(kern, C::kThreads, C::SMEM, cnt, mmax, max_cluster) : 1;
    if (dry) return BM_OK;
    if (S == 1) {
        kern<<<cnt, C::kThreads, C::SMEM, st>>>(jobs, steps, ct_in, lut, ws_acc, status);
    } else {
        cudaLaunchConfig_t cfg = {};
        cfg.gridDim = dim3(cnt * S);
        cfg.blockDim = dim3(C::kThreads);
        cfg.dynamicSmemBytes = C::SMEM;
        cfg.stream = st;
        cudaLaunchAttribute at[1];
        at[0].id = cudaLaunchAttributeClusterDimension;
        at[0].val.clusterDim.x = S;
        at[0].val.clusterDim.y = 1;
        at[0].val.clusterDim.z = 1;
        cfg.attrs = at;
        cfg.numAttrs = 1;
        BM_CUDA_TRY(cudaLaunchKernelEx(&cfg, kern, jobs, steps, ct_in, lut, ws_acc, status));
    }
    BM_CUDA_TRY(cudaGetLastError());
    return BM_OK;
}

// Every fitting shape for the variants of moduli Q = c 2^32 + 1 (the
// production key sets); shape 0 alone otherwise.  A shape that does not
// fit (or is not compiled for the variant) falls back to shape 0.
template <int LOGN, bool LAZY, bool SMALL0, bool QLOW1>
bm_status launch_shape(u32 shape, const DevJob *jobs, uint32_t cnt, u32 mmax, u32 max_cluster, u32 steps,
                       const uint64_t *ct_in, const uint32_t *lut, u64 *ws_acc, u32 *status, cudaStream_t st,
                       bool dry) {
#define BM_SHAPE(SH)                                                                                           \
    if constexpr (QLOW1 && br_shape_fits(LOGN, SH))                                                            \
        if (shape == SH)                                                                                       \
            return launch_br_v<LOGN, SH, LAZY, SMALL0, QLOW1>(jobs, cnt, mmax, max_cluster, steps, ct_in, lut, \
                                                              ws_acc, status, st, dry);
    if constexpr (LOGN >= 10) {
        BM_SHAPE(1)
        BM_SHAPE(2)
        BM_SHAPE(3)
        BM_SHAPE(4)
    }
#undef BM_SHAPE
    return launch_br_v<LOGN, 0, LAZY, SMALL0, QLOW1>(jobs, cnt, mmax, max_cluster, steps, ct_in, lut, ws_acc,
                                                     status, st, dry);
}

template <int LOGN>
bm_status launch_br(u32 variant, u32 shape, const DevJob *jobs, uint32_t cnt, u32 mmax, u32 max_cluster, u32 steps,
                    const uint64_t *ct_in, const uint32_t *lut, u64 *ws_acc, u32 *status, cudaStream_t st,
                    bool dry) {
#define BM_LAUNCH(LZ, S0, QL) \
    return launch_shape<LOGN, LZ, S0, QL>(shape, jobs, cnt, mmax, max_cluster, steps, ct_in, lut, ws_acc, status, st, dry)
    switch (variant) {
        case BR_V_LAZY | BR_V_QLOW1: BM_LAUNCH(true, true, true);
        case BR_V_LAZY: BM_LAUNCH(true, true, false);
        case BR_V_QLOW1: BM_LAUNCH(false, true, true);
        default: BM_LAUNCH(false, false, false);
    }
#undef BM_LAUNCH
}

// The shape a launch of this variant actually uses for a requested shape.
inline u32 br_effective_shape(int logn, u32 variant, u32 shape) {
    if (shape == 0 || logn < 10 || !(variant & BR_V_QLOW1) || shape >= 5 || !br_shape_fits(logn, (int)shape)) return 0;
    return shape;
}

// Blind-rotation launches for ring degrees 256 and 512 (every variant; one
// kernel shape).
#include "br_launch.cuh"

bm_status bm_launch_br_small(u32 N, u32 variant, u32 shape, const DevJob *jobs, uint32_t cnt, u32 mmax,
                             u32 max_cluster, u32 steps, const uint64_t *ct_in, const uint32_t *lut, u64 *ws_acc,
                             u32 *status, cudaStream_t st, bool dry) {
    if (N == 256)
        return launch_br<8>(variant, shape, jobs, cnt, mmax, max_cluster, steps, ct_in, lut, ws_acc, status, st, dry);
    if (N == 512)
        return launch_br<9>(variant, shape, jobs, cnt, mmax, max_cluster, steps, ct_in, lut, ws_acc, status, st, dry);
    return BM_EINVAL;
}

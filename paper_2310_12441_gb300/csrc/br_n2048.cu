// Blind-rotation launches for ring degree 2048 (every variant and kernel shape).
#include "br_launch.cuh"

bm_status bm_launch_br_n2048(u32 variant, u32 shape, const DevJob *jobs, uint32_t cnt, u32 mmax, u32 max_cluster,
                           u32 steps, const uint64_t *ct_in, const uint32_t *lut, u64 *ws_acc, u32 *status,
                           cudaStream_t st, bool dry) {
    return launch_br<11>(variant, shape, jobs, cnt, mmax, max_cluster, steps, ct_in, lut, ws_acc, status, st, dry);
}

// Blind-rotation launches for ring degree 8192 (every variant; the kernel
// shapes that hold a whole polynomial in one block: radix 8 with 1024
// threads, radix 16 with 512).
#include "br_launch.cuh"

bm_status bm_launch_br_n8192(u32 variant, u32 shape, const DevJob *jobs, uint32_t cnt, u32 mmax, u32 max_cluster,
                             u32 steps, const uint64_t *ct_in, const uint32_t *lut, u64 *ws_acc, u32 *status,
                             cudaStream_t st, bool dry) {
    return launch_br<13>(variant, shape, jobs, cnt, mmax, max_cluster, steps, ct_in, lut, ws_acc, status, st, dry);
}

// Batched persistent lens kernel, precision class 1 (0 = FP64, 1 = double-float).
#include "batch.cuh"

namespace flints {
int batch_max_wpb() {
    const size_t per = batch_warp_smem<0>() > batch_warp_smem<1>() ? batch_warp_smem<0>() : batch_warp_smem<1>();
    const int fit = (int)(device_smem_optin() / per);
    return fit < 1 ? 1 : (fit > 8 ? 8 : fit);
}
cudaError_t batch_prepare_p1(int wpb, int *max_blocks_per_sm) { return batch_prepare<1>(wpb, max_blocks_per_sm); }
cudaError_t batch_launch_p1(const BatchHeader *hdr, const BatchJob *jobs, unsigned long long *next_tile, int wpb,
                             int blocks, cudaStream_t st) {
    return batch_launch<1>(hdr, jobs, next_tile, wpb, blocks, st);
}
}  // namespace flints

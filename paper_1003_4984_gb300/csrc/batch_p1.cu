// Batched persistent lens kernels of precision class 1 (0 = FP64, 1 = double-float),
// one per spin (0, 2) and stencil size (16, 24, 32, 48).
#include "batch.cuh"

namespace flints {
cudaError_t batch_prepare_p1(int c, int wpb, int *max_blocks_per_sm) {
    return batch_prepare_cls<1>(c, wpb, max_blocks_per_sm);
}
cudaError_t batch_launch_p1(int c, const BatchHeader *hdr, const BatchJob *jobs, unsigned long long *next_tile,
                             int wpb, int blocks, cudaStream_t st) {
    return batch_launch_cls<1>(c, hdr, jobs, next_tile, wpb, blocks, st);
}
int batch_fit_wpb_p1(int c) { return batch_fit_wpb_cls<1>(c); }
}  // namespace flints

// Job table of the batched persistent launch (shared by the host API and the kernel).
#pragma once
#include "common.cuh"

namespace flints {

struct BatchJob {
    LensArgs a;
    int R_rings, K, spin, precision;
    int64_t tile_begin, ntiles;
};

// Job classes: 8 * precision + 4 * (spin == 2) + index of K in {16, 24, 32, 48};
// each class runs in its own persistent kernel, specialised (shared memory,
// registers) for its stencil size.
constexpr int BATCH_CLASSES = 16;
__host__ __device__ constexpr int batch_k_index(int K) { return K == 16 ? 0 : (K == 24 ? 1 : (K == 32 ? 2 : 3)); }

struct BatchHeader {
    int njobs[BATCH_CLASSES];       // per class
    int job_offset[BATCH_CLASSES];  // index of the class's first job in the job array
    int64_t total_tiles[BATCH_CLASSES];
    int tile_pts;
    int pad;
};

}  // namespace flints

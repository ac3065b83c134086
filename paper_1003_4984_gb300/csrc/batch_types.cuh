// Job table of the batched persistent launch (shared by the host API and the kernel).
#pragma once
#include "common.cuh"

namespace flints {

struct BatchJob {
    LensArgs a;
    int R_rings, K, spin, precision;
    int64_t tile_begin, ntiles;
};

struct BatchHeader {
    int njobs[2];         // per precision class (0 = FP64, 1 = mixed)
    int job_offset[2];    // index of the class's first job in the job array
    int64_t total_tiles[2];
    int tile_pts;
    int pad;
};

}  // namespace flints

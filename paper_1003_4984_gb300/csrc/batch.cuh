// Persistent batched lens launch: many target ranges of different plans
// (Nside, K, spin) in one launch per class (precision, spin, K), each kernel
// specialised like the single-range kernel (its own shared-memory slice and
// register budget; the launches of empty classes exit at once).  Warps take tiles from a
// device work queue (one atomic per tile) in the order the host staged them
// (costliest jobs first), find the tile's job by binary search over the jobs'
// first tiles and run the same per-tile code as the single-range kernel.
// There is no inter-block waiting: a warp that finds the queue empty exits.
// Plan calls of spin 0 and 2 launch the same class kernels with a one-job table
// (api.cu), the code that measured fastest for single ranges as well.
#pragma once
#include "batch_types.cuh"
#include "lens.cuh"

namespace flints {

template <int MIXED, int SPIN, int K>
__global__ void __launch_bounds__(256, 2) batch_kernel(const BatchHeader *__restrict__ hdr,
                                                      const BatchJob *__restrict__ jobs,
                                                      unsigned long long *next_tile) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    constexpr int CLS = 8 * MIXED + (SPIN == 2 ? 4 : 0) + batch_k_index(K);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    unsigned char *wbase = smem_raw + (size_t)warp * warp_smem_bytes<K, SPIN, MIXED>();
    const int nj = hdr->njobs[CLS];
    const int64_t total = hdr->total_tiles[CLS];
    const int tile_pts = hdr->tile_pts;
    const BatchJob *J = jobs + hdr->job_offset[CLS];
    if (nj <= 0) return;
    Counters ctr;
    for (;;) {
        unsigned long long t = 0;
        if (lane == 0) t = atomicAdd(next_tile + CLS, 1ull);
        t = __shfl_sync(FULL, t, 0);
        if ((int64_t)t >= total) break;
        int lo = 0, hi = nj - 1;
        while (lo < hi) {
            const int mid = (lo + hi + 1) >> 1;
            if (J[mid].tile_begin <= (int64_t)t) lo = mid;
            else hi = mid - 1;
        }
        const LensArgs a = J[lo].a;
        process_tile<K, SPIN, MIXED>(a, J[lo].R_rings, (int64_t)t - J[lo].tile_begin, tile_pts, wbase, lane, ctr);
        flush_counters(ctr, a.counters, lane);
        __syncwarp();
    }
}

// warps per block that fit in the opt-in shared memory for a class
template <int MIXED, int SPIN, int K>
int batch_fit_wpb();

// The kernel's dynamic shared-memory limit is a property of the kernel function,
// shared by every batch object and plan that launches it: it is always set to the
// largest block that fits, so a launch with fewer warps per block never finds it
// lowered by another caller; the occupancy is queried for the requested shape.
template <int MIXED, int SPIN, int K>
cudaError_t batch_prepare(int wpb, int *max_blocks_per_sm) {
    const size_t smem = (size_t)wpb * warp_smem_bytes<K, SPIN, MIXED>();
    const size_t smem_max = (size_t)batch_fit_wpb<MIXED, SPIN, K>() * warp_smem_bytes<K, SPIN, MIXED>();
    auto kern = batch_kernel<MIXED, SPIN, K>;
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)(smem > smem_max ? smem : smem_max));
    if (e != cudaSuccess) return e;
    return cudaOccupancyMaxActiveBlocksPerMultiprocessor(max_blocks_per_sm, kern, wpb * 32, smem);
}

template <int MIXED, int SPIN, int K>
cudaError_t batch_launch(const BatchHeader *hdr, const BatchJob *jobs, unsigned long long *next_tile, int wpb,
                         int blocks, cudaStream_t st) {
    const size_t smem = (size_t)wpb * warp_smem_bytes<K, SPIN, MIXED>();
    batch_kernel<MIXED, SPIN, K><<<blocks, wpb * 32, smem, st>>>(hdr, jobs, next_tile);
    return cudaGetLastError();
}

template <int MIXED, int SPIN, int K>
int batch_fit_wpb() {
    const int fit = (int)(device_smem_optin() / warp_smem_bytes<K, SPIN, MIXED>());
    return fit < 1 ? 1 : (fit > 8 ? 8 : fit);
}

// dispatch over the class index within a precision: 4 * (spin == 2) + K index
#define FLINTS_BATCH_CASES(F, ...)              \
    switch (c & 7) {                            \
        case 0: return F<MIXED, 0, 16>(__VA_ARGS__); \
        case 1: return F<MIXED, 0, 24>(__VA_ARGS__); \
        case 2: return F<MIXED, 0, 32>(__VA_ARGS__); \
        case 3: return F<MIXED, 0, 48>(__VA_ARGS__); \
        case 4: return F<MIXED, 2, 16>(__VA_ARGS__); \
        case 5: return F<MIXED, 2, 24>(__VA_ARGS__); \
        case 6: return F<MIXED, 2, 32>(__VA_ARGS__); \
        default: return F<MIXED, 2, 48>(__VA_ARGS__); \
    }
template <int MIXED>
cudaError_t batch_prepare_cls(int c, int wpb, int *mx) {
    FLINTS_BATCH_CASES(batch_prepare, wpb, mx)
}
template <int MIXED>
cudaError_t batch_launch_cls(int c, const BatchHeader *hdr, const BatchJob *jobs, unsigned long long *next_tile,
                             int wpb, int blocks, cudaStream_t st) {
    FLINTS_BATCH_CASES(batch_launch, hdr, jobs, next_tile, wpb, blocks, st)
}
template <int MIXED>
int batch_fit_wpb_cls(int c) {
    FLINTS_BATCH_CASES(batch_fit_wpb)
}
#undef FLINTS_BATCH_CASES

}  // namespace flints

// Persistent batched lens launch: many target ranges of different plans
// (Nside, K, spin) in one launch per precision.  Warps take tiles from a
// device work queue (one atomic per tile) in the order the host staged them
// (costliest jobs first), find the tile's job by binary search over the jobs'
// first tiles and run the same per-tile code as the single-range kernel.
// There is no inter-block waiting: a warp that finds the queue empty exits.
#pragma once
#include "batch_types.cuh"
#include "lens.cuh"

namespace flints {

template <int MIXED>
constexpr size_t batch_warp_smem() {
    // the largest per-warp slice over the supported (K, spin) classes
    return warp_smem_bytes<48, 2, MIXED>();
}

template <int MIXED>
__global__ void __launch_bounds__(256, 1) batch_kernel(const BatchHeader *__restrict__ hdr,
                                                      const BatchJob *__restrict__ jobs,
                                                      unsigned long long *next_tile) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    unsigned char *wbase = smem_raw + (size_t)warp * batch_warp_smem<MIXED>();
    const int nj = hdr->njobs[MIXED];
    const int64_t total = hdr->total_tiles[MIXED];
    const int tile_pts = hdr->tile_pts;
    const BatchJob *J = jobs + hdr->job_offset[MIXED];
    if (nj <= 0) return;
    Counters ctr;
    for (;;) {
        unsigned long long t = 0;
        if (lane == 0) t = atomicAdd(next_tile + MIXED, 1ull);
        t = __shfl_sync(FULL, t, 0);
        if ((int64_t)t >= total) break;
        int lo = 0, hi = nj - 1;
        while (lo < hi) {
            const int mid = (lo + hi + 1) >> 1;
            if (J[mid].tile_begin <= (int64_t)t) lo = mid;
            else hi = mid - 1;
        }
        const LensArgs a = J[lo].a;
        const int R = J[lo].R_rings, K = J[lo].K, spin = J[lo].spin;
        const int64_t lt = (int64_t)t - J[lo].tile_begin;
        if (spin == 0) {
            if (K == 16) process_tile<16, 0, MIXED>(a, R, lt, tile_pts, wbase, lane, ctr);
            else if (K == 24) process_tile<24, 0, MIXED>(a, R, lt, tile_pts, wbase, lane, ctr);
            else if (K == 32) process_tile<32, 0, MIXED>(a, R, lt, tile_pts, wbase, lane, ctr);
            else process_tile<48, 0, MIXED>(a, R, lt, tile_pts, wbase, lane, ctr);
        } else {
            if (K == 16) process_tile<16, 2, MIXED>(a, R, lt, tile_pts, wbase, lane, ctr);
            else if (K == 24) process_tile<24, 2, MIXED>(a, R, lt, tile_pts, wbase, lane, ctr);
            else if (K == 32) process_tile<32, 2, MIXED>(a, R, lt, tile_pts, wbase, lane, ctr);
            else process_tile<48, 2, MIXED>(a, R, lt, tile_pts, wbase, lane, ctr);
        }
        flush_counters(ctr, a.counters, lane);
        __syncwarp();
    }
}

template <int MIXED>
cudaError_t batch_prepare(int wpb, int *max_blocks_per_sm) {
    const size_t smem = (size_t)wpb * batch_warp_smem<MIXED>();
    cudaError_t e = cudaFuncSetAttribute(batch_kernel<MIXED>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    return cudaOccupancyMaxActiveBlocksPerMultiprocessor(max_blocks_per_sm, batch_kernel<MIXED>, wpb * 32, smem);
}

template <int MIXED>
cudaError_t batch_launch(const BatchHeader *hdr, const BatchJob *jobs, unsigned long long *next_tile, int wpb,
                         int blocks, cudaStream_t st) {
    const size_t smem = (size_t)wpb * batch_warp_smem<MIXED>();
    batch_kernel<MIXED><<<blocks, wpb * 32, smem, st>>>(hdr, jobs, next_tile);
    return cudaGetLastError();
}

}  // namespace flints

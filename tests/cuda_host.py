"""Run the library's CUDA sources on the host (test helper): a CUDA-runtime
stand-in and a thread-block emulator, so that the host API of a .cu file and
the kernels it launches run unchanged on the CPU.

* Kernel launches ``k<<<grid, block, smem, stream>>>(args)`` become
  host_launch(grid, block, smem, [&] { k(args); }): the blocks run one after
  another, each on ``block`` host threads (a pool kept for the launch).
  Threads of a block run freely between barriers: __syncthreads waits for the
  block's threads, warp intrinsics (shuffles, ballots, reductions, __syncwarp)
  for the 32 threads of the warp, so a missing barrier shows as a wrong
  result instead of being hidden by lock-step execution.  A thread that
  returns from the kernel leaves both barriers.
* ``__shared__`` variables are function statics (one copy, shared by the
  block's threads; blocks run one at a time); dynamic shared memory is one
  static buffer.
* Device memory is host memory: cudaMalloc is an aligned allocation, copies
  and sets are memcpy and memset, streams are synchronous; cuFFT's batched
  one-dimensional transforms are direct sums (small sizes only).
* Device math not in the C library: sincospi, sinpif (sin/cos of pi x), bit
  casts; the rounding intrinsics and rsqrt(f) come from host_compile.SHIM.
"""
from __future__ import annotations

import os
import re

from tests import host_compile as hc

RUNTIME = r"""
#include <algorithm>
#include <atomic>
#include <cstddef>
#include <map>
#include <mutex>
#include <thread>
#include <type_traits>
#include <math.h>
typedef int cudaError_t;
enum { cudaSuccess = 0, cudaErrorInvalidValue = 1, cudaErrorMemoryAllocation = 2, cudaErrorInvalidConfiguration = 9,
       cudaErrorUnknown = 999 };
typedef void *cudaStream_t;
enum cudaMemcpyKind { cudaMemcpyHostToHost, cudaMemcpyHostToDevice, cudaMemcpyDeviceToHost, cudaMemcpyDeviceToDevice,
                      cudaMemcpyDefault };
enum cudaFuncAttribute { cudaFuncAttributeMaxDynamicSharedMemorySize };
enum cudaDeviceAttr { cudaDevAttrMultiProcessorCount, cudaDevAttrMaxSharedMemoryPerBlockOptin };
#ifdef FLINTS_HOST_SANITIZE
// exact sizes (so that the address sanitizer sees an access past the end) and
// contents that are not zero (device memory is not cleared)
static inline cudaError_t host_alloc_raw(void **p, size_t n) {
    if (posix_memalign(p, 256, n ? n : 1)) return cudaErrorMemoryAllocation;
    std::memset(*p, 0xff, n ? n : 1);
    return cudaSuccess;
}
#else
static inline cudaError_t host_alloc_raw(void **p, size_t n) {
    *p = std::aligned_alloc(256, (n + 255) / 256 * 256 + 256);
    return *p ? cudaSuccess : cudaErrorMemoryAllocation;
}
#endif
// ledger of live device allocations (bytes as requested), for the drivers' checks
static std::mutex g_dev_mutex;
static std::map<void *, size_t> g_dev_allocs;
static size_t g_dev_live = 0, g_dev_alloc_calls = 0;
static inline cudaError_t cudaMalloc(void **p, size_t n) {
    const cudaError_t e = host_alloc_raw(p, n);
    if (e == cudaSuccess) {
        std::lock_guard<std::mutex> lk(g_dev_mutex);
        g_dev_allocs[*p] = n;
        g_dev_live += n;
        ++g_dev_alloc_calls;
    }
    return e;
}
template <class T> static inline cudaError_t cudaMalloc(T **p, size_t n) { return cudaMalloc((void **)p, n); }
static inline cudaError_t cudaFree(void *p) {
    if (p) {
        std::lock_guard<std::mutex> lk(g_dev_mutex);
        auto it = g_dev_allocs.find(p);
        if (it != g_dev_allocs.end()) {
            g_dev_live -= it->second;
            g_dev_allocs.erase(it);
        }
    }
    std::free(p);
    return cudaSuccess;
}
enum { cudaHostAllocDefault = 0 };
static inline cudaError_t cudaHostAlloc(void **p, size_t n, unsigned) { return host_alloc_raw(p, n); }
static inline cudaError_t cudaFreeHost(void *p) { std::free(p); return cudaSuccess; }
static inline cudaError_t cudaGetSymbolAddress(void **p, const void *sym) { *p = const_cast<void *>(sym); return cudaSuccess; }
static inline cudaError_t cudaMemcpyAsync(void *d, const void *s, size_t n, cudaMemcpyKind, cudaStream_t = 0) {
    std::memmove(d, s, n);
    return cudaSuccess;
}
static inline cudaError_t cudaMemcpy(void *d, const void *s, size_t n, cudaMemcpyKind k) { return cudaMemcpyAsync(d, s, n, k); }
static inline cudaError_t cudaMemsetAsync(void *d, int v, size_t n, cudaStream_t = 0) {
    std::memset(d, v, n);
    return cudaSuccess;
}
static inline cudaError_t cudaStreamSynchronize(cudaStream_t) { return cudaSuccess; }
static inline cudaError_t cudaDeviceSynchronize() { return cudaSuccess; }
static inline cudaError_t cudaGetDevice(int *d) { *d = 0; return cudaSuccess; }
static inline cudaError_t cudaSetDevice(int) { return cudaSuccess; }
static inline cudaError_t cudaGetLastError() { return cudaSuccess; }
static inline const char *cudaGetErrorString(cudaError_t) { return "host stand-in"; }
template <class F> static inline cudaError_t cudaFuncSetAttribute(F, cudaFuncAttribute, int) { return cudaSuccess; }
static inline cudaError_t cudaDeviceGetAttribute(int *v, cudaDeviceAttr a, int) {
    *v = a == cudaDevAttrMultiProcessorCount ? 152 : 232448;
    return cudaSuccess;
}
template <class F> static inline cudaError_t cudaOccupancyMaxActiveBlocksPerMultiprocessor(int *n, F, int, size_t) {
    *n = 2;
    return cudaSuccess;
}

// ------------------------------------------------------------ blocks and warps
struct dim3 {
    unsigned x = 1, y = 1, z = 1;
    dim3(unsigned a = 1, unsigned b = 1, unsigned c = 1) : x(a), y(b), z(c) {}
};
static thread_local dim3 threadIdx, blockIdx;
static dim3 blockDim, gridDim;
#ifdef FLINTS_HOST_SANITIZE
static unsigned char *g_dyn_smem = nullptr;  // per launch: exactly the requested bytes, not cleared
#else
static unsigned char g_dyn_smem[256 * 1024] __attribute__((aligned(256)));
#endif

// a barrier of a changing number of threads: arrive() waits for the others, leave()
// removes the caller (a thread that returned from the kernel)
struct HostBarrier {
    std::mutex m;
    int count = 0, expected = 0;
    std::atomic<unsigned> gen{0};
    void reset(int n) { count = 0; expected = n; }
    void arrive(bool leave = false) {
        unsigned g;
        {
            std::lock_guard<std::mutex> lk(m);
            g = gen.load();
            if (leave) --expected;
            else ++count;
            if (count >= expected) {
                count = 0;
                gen.store(g + 1);
                gen.notify_all();
                return;
            }
        }
        if (!leave) {
            for (int spin = 0; spin < 64 && gen.load() == g; ++spin) std::this_thread::yield();
            while (gen.load() == g) gen.wait(g);  // sleep until the last thread arrives
        }
    }
};
static HostBarrier g_block_bar, g_warp_bar_of[32];
static uint64_t g_warp_slot_of[32][32];
static thread_local int t_lane = 0, t_warp = 0;

template <class T> static inline uint64_t to_word(T v) {
    static_assert(sizeof(T) <= 8, "one word per lane");
    uint64_t b = 0;
    std::memcpy(&b, &v, sizeof(T));
    return b;
}
template <class T> static inline T from_word(uint64_t b) {
    T v;
    std::memcpy(&v, &b, sizeof(T));
    return v;
}
static inline void __syncwarp(unsigned = 0xffffffffu) { g_warp_bar_of[t_warp].arrive(); }
static inline void __syncthreads() { g_block_bar.arrive(); }
template <class T> static inline T __shfl_sync(unsigned, T v, int src) {
    g_warp_slot_of[t_warp][t_lane] = to_word(v);
    __syncwarp();
    const uint64_t r = g_warp_slot_of[t_warp][src & 31];
    __syncwarp();
    return from_word<T>(r);
}
template <class T> static inline T __shfl_xor_sync(unsigned m, T v, int x) { return __shfl_sync(m, v, t_lane ^ x); }
template <class T> static inline T __shfl_up_sync(unsigned m, T v, int d) {
    return __shfl_sync(m, v, t_lane >= d ? t_lane - d : t_lane);
}
template <class T> static inline T __shfl_down_sync(unsigned m, T v, int d) {
    return __shfl_sync(m, v, t_lane + d < 32 ? t_lane + d : t_lane);
}
static inline unsigned __ballot_sync(unsigned, int pred) {
    g_warp_slot_of[t_warp][t_lane] = pred != 0;
    __syncwarp();
    unsigned m = 0;
    for (int l = 0; l < 32; ++l) m |= (unsigned)(g_warp_slot_of[t_warp][l] & 1u) << l;
    __syncwarp();
    return m;
}
static inline int __any_sync(unsigned m, int pred) { return __ballot_sync(m, pred) != 0; }
static inline int __all_sync(unsigned m, int pred) { return __ballot_sync(m, pred) == 0xffffffffu; }
static inline unsigned __reduce_add_sync(unsigned, unsigned v) {
    g_warp_slot_of[t_warp][t_lane] = v;
    __syncwarp();
    uint64_t s = 0;
    for (int l = 0; l < 32; ++l) s += g_warp_slot_of[t_warp][l];
    __syncwarp();
    return (unsigned)s;
}
static inline int __popc(unsigned x) { return __builtin_popcount(x); }
static inline int __clz(unsigned x) { return x ? __builtin_clz(x) : 32; }
static std::mutex g_atomic_mutex;
template <class T> static inline T atomicAdd(T *p, T v) {
    std::lock_guard<std::mutex> lk(g_atomic_mutex);
    T o = *p;
    *p += v;
    return o;
}
template <class T> static inline T atomicMax(T *p, T v) {
    std::lock_guard<std::mutex> lk(g_atomic_mutex);
    T o = *p;
    if (v > o) *p = v;
    return o;
}

template <class F> static cudaError_t host_launch(dim3 grid, dim3 block, size_t smem, F body) {
    const unsigned nthr = block.x * block.y * block.z;
#ifdef FLINTS_HOST_SANITIZE
    if (smem > 256 * 1024) return cudaErrorInvalidValue;
    void *dyn = nullptr;
    if (posix_memalign(&dyn, 256, smem ? smem : 1)) return cudaErrorMemoryAllocation;
    std::memset(dyn, 0xff, smem ? smem : 1);
    g_dyn_smem = static_cast<unsigned char *>(dyn);
#else
    if (smem > sizeof g_dyn_smem) return cudaErrorInvalidValue;
#endif
    blockDim = block;
    gridDim = grid;
    HostBarrier start, end;
    start.reset(nthr);
    end.reset(nthr);
    std::vector<std::thread> pool;
    for (unsigned t = 0; t < nthr; ++t)
        pool.emplace_back([&, t] {
            threadIdx = dim3(t % block.x, (t / block.x) % block.y, t / (block.x * block.y));
            t_lane = t & 31;
            t_warp = t >> 5;
            for (unsigned b = 0; b < grid.x * grid.y * grid.z; ++b) {
                if (t == 0) {  // between two full barriers: nobody uses the block's barriers
                    g_block_bar.reset(nthr);
                    for (unsigned w = 0; w < (nthr + 31) / 32; ++w) g_warp_bar_of[w].reset(std::min(32u, nthr - 32 * w));
                }
                start.arrive();
                blockIdx = dim3(b % grid.x, (b / grid.x) % grid.y, b / (grid.x * grid.y));
                body();
                g_warp_bar_of[t_warp].arrive(true);  // this thread has returned from the kernel
                g_block_bar.arrive(true);
                end.arrive();
            }
        });
    for (auto &th : pool) th.join();
#ifdef FLINTS_HOST_SANITIZE
    std::free(dyn);
    g_dyn_smem = nullptr;
#endif
    return cudaSuccess;
}
// lgamma without glibc's write of the global sign (signgam): the device function has
// no global state, and the emulated threads call it at once
static inline double flints_host_lgamma(double x) { int s; return lgamma_r(x, &s); }
#define lgamma flints_host_lgamma
static inline void sincospi(double x, double *s, double *c) { *s = std::sin(M_PI * x); *c = std::cos(M_PI * x); }
static inline float sinpif(float x) { return (float)std::sin(M_PI * (double)x); }
static inline double __longlong_as_double(long long v) { double d; std::memcpy(&d, &v, 8); return d; }
static inline long long __double_as_longlong(double d) { long long v; std::memcpy(&v, &d, 8); return v; }
static inline float __uint2float_rn(unsigned v) { return (float)v; }
struct double2 { double x, y; };
struct float2 { float x, y; };
struct float4 { float x, y, z, w; };
static inline double2 make_double2(double x, double y) { return {x, y}; }
static inline float2 make_float2(float x, float y) { return {x, y}; }
static inline float4 make_float4(float x, float y, float z, float w) { return {x, y, z, w}; }
template <class T> static inline T __ldg(const T *p) { return *p; }
using std::floor; using std::fabs; using std::fmax; using std::isfinite; using std::atan2; using std::min; using std::max;

// cuFFT stand-in: one-dimensional batched transforms by direct summation (the
// sizes of the small skies tested), unnormalised like cuFFT; Z2D takes the
// n/2 + 1 non-negative frequencies of a Hermitian spectrum
typedef int cufftHandle;
typedef int cufftResult;
enum { CUFFT_SUCCESS = 0, CUFFT_INVALID_PLAN = 1 };
typedef double2 cufftDoubleComplex;
typedef double cufftDoubleReal;
typedef enum { CUFFT_Z2Z = 0x69, CUFFT_Z2D = 0x6c, CUFFT_D2Z = 0x6a } cufftType;
#define CUFFT_FORWARD -1
#define CUFFT_INVERSE 1
struct HostFftPlan {
    int n = 0, batch = 0;
    long long idist = 0, odist = 0;
    cufftType type = CUFFT_Z2Z;
};
static std::vector<HostFftPlan> g_fft_plans;
static inline cufftResult cufftCreate(cufftHandle *h) {
    g_fft_plans.emplace_back();
    *h = (int)g_fft_plans.size() - 1;
    return CUFFT_SUCCESS;
}
static inline cufftResult cufftSetAutoAllocation(cufftHandle, int) { return CUFFT_SUCCESS; }
static inline cufftResult cufftMakePlanMany(cufftHandle h, int rank, int *n, int *, int, int idist, int *, int,
                                            int odist, cufftType type, int batch, size_t *ws) {
    if (rank != 1) return CUFFT_INVALID_PLAN;
    g_fft_plans[h] = HostFftPlan{n[0], batch, idist, odist, type};
    *ws = 0;
    return CUFFT_SUCCESS;
}
static inline cufftResult cufftGetSize(cufftHandle, size_t *ws) { *ws = 0; return CUFFT_SUCCESS; }
static inline cufftResult cufftSetWorkArea(cufftHandle, void *) { return CUFFT_SUCCESS; }
static inline cufftResult cufftSetStream(cufftHandle, cudaStream_t) { return CUFFT_SUCCESS; }
static inline cufftResult cufftDestroy(cufftHandle) { return CUFFT_SUCCESS; }
static inline void host_dft(const double2 *in, double2 *out, int n, int sign, bool hermitian_in) {
    std::vector<double2> x(n), y(n);
    for (int k = 0; k < n; ++k) {
        if (!hermitian_in) x[k] = in[k];
        else if (k <= n / 2) x[k] = in[k];
        else x[k] = double2{in[n - k].x, -in[n - k].y};
    }
    for (int j = 0; j < n; ++j) {
        long double re = 0, im = 0;
        for (int k = 0; k < n; ++k) {
            const long long q = ((long long)j * k) % n;
            const long double ang = (long double)sign * 2.0L * 3.14159265358979323846264338327950288L * q / n;
            const long double c = cosl(ang), s = sinl(ang);
            re += x[k].x * c - x[k].y * s;
            im += x[k].x * s + x[k].y * c;
        }
        y[j] = double2{(double)re, (double)im};
    }
    for (int j = 0; j < n; ++j) out[j] = y[j];
}
static inline cufftResult cufftExecZ2Z(cufftHandle h, cufftDoubleComplex *in, cufftDoubleComplex *out, int dir) {
    const HostFftPlan &p = g_fft_plans[h];
    for (int b = 0; b < p.batch; ++b) host_dft(in + b * p.idist, out + b * p.odist, p.n, dir, false);
    return CUFFT_SUCCESS;
}
static inline cufftResult cufftExecZ2D(cufftHandle h, cufftDoubleComplex *in, cufftDoubleReal *out) {
    const HostFftPlan &p = g_fft_plans[h];
    std::vector<double2> y(p.n);
    for (int b = 0; b < p.batch; ++b) {
        host_dft(in + b * p.idist, y.data(), p.n, +1, true);
        for (int j = 0; j < p.n; ++j) out[b * p.odist + j] = y[j].x;
    }
    return CUFFT_SUCCESS;
}

#define __host__
#define __device__
#define __global__
#define __forceinline__ inline
#define __shared__ static
#define __align__(x) __attribute__((aligned(x)))
#define __launch_bounds__(...)
"""


def _launches(src: str) -> str:
    """k<<<cfg>>>(args)  ->  host_launch(grid, block, smem, [&] { k(args); })"""
    out, i = [], 0
    while True:
        j = src.find("<<<", i)
        if j < 0:
            out.append(src[i:])
            return "".join(out)
        # the kernel name (with template arguments) ends at j
        k = j
        depth = 0
        while k > 0:
            c = src[k - 1]
            if c == ">":
                depth += 1
            elif c == "<":
                depth -= 1
            elif depth == 0 and not (c.isalnum() or c in "_:"):
                break
            k -= 1
        name = src[k:j]
        e = src.index(">>>", j)
        cfg = [x.strip() for x in _split_top(src[j + 3:e])]
        a0 = src.index("(", e)
        depth, a1 = 0, a0
        while True:
            depth += {"(": 1, ")": -1}.get(src[a1], 0)
            if depth == 0:
                break
            a1 += 1
        args = src[a0 + 1:a1]
        grid, block = cfg[0], cfg[1]
        smem = cfg[2] if len(cfg) > 2 else "0"
        out.append(src[i:k])
        out.append(f"host_launch(dim3({grid}), dim3({block}), (size_t)({smem}), [&] {{ {name}({args}); }})")
        i = a1 + 1


def _split_top(s: str):
    parts, depth, cur = [], 0, ""
    for c in s:
        if c in "([{":
            depth += 1
        elif c in ")]}":
            depth -= 1
        if c == "," and depth == 0:
            parts.append(cur)
            cur = ""
        else:
            cur += c
    parts.append(cur)
    return parts


def source(name: str) -> str:
    """A CUDA source of the library made host-compilable: local includes and the
    runtime header dropped, launches and dynamic shared memory rewritten."""
    src = open(os.path.join(hc.CSRC, name)).read()
    src = re.sub(r'^\s*#include\s+["<](cuda_runtime\.h|cufft\.h|[a-z_0-9]+\.cuh|flints\.h)[">]\s*$', "", src, flags=re.M)
    src = src.replace("#pragma once", "")
    src = re.sub(r"extern __shared__\s+(?:__align__\(\d+\)\s+)?([\w ]+?)\s+(\w+)\[\];",
                 r"\1 *\2 = reinterpret_cast<\1 *>(g_dyn_smem);", src)
    return _launches(src)


def build(tmpdir, name: str, files, driver: str, sanitize: str | None = None) -> str:
    """Compile the given sources (in order) with the runtime stand-ins and ``driver``.
    ``sanitize`` ("address" or "thread", see host_compile.SANITIZE): with the
    sanitizer, device allocations and dynamic shared memory of exactly the requested
    size and filled with 0xff bytes."""
    text = (("#define FLINTS_HOST_SANITIZE 1\n" if sanitize else "") + RUNTIME + '#include "' + hc.ROOT
            + '/include/flints.h"\n' + "".join(source(f) + "\n" for f in files) + driver)
    return hc.build(tmpdir, name, text, warp="none", sanitize=sanitize)

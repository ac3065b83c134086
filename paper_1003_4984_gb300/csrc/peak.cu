// Arithmetic-throughput probe: the FP32 and FP64 fused multiply-add rates of
// the GPU this library runs on, measured with the same clocks and power state
// as the lens kernels timed beside it.  The lens kernels are bound by these
// pipes (the mixed path by FP32, the FP64 path by FP64), so their roofline
// fractions are taken against these measured rates.
#include <cstdio>

#include "common.cuh"

namespace flints {
namespace {

constexpr int CHAINS = 8;  // independent multiply-add chains per thread (hides the pipe latency)
__device__ double g_sink;  // written only if a chain reaches an impossible value: keeps the chains live

template <class T>
__global__ void __launch_bounds__(256) fma_chain_kernel(int iters, T b, T c) {
    T a[CHAINS];
#pragma unroll
    for (int i = 0; i < CHAINS; ++i) a[i] = (T)(threadIdx.x + i) * (T)1e-3;
    for (int it = 0; it < iters; ++it) {
#pragma unroll
        for (int u = 0; u < 16; ++u) {
#pragma unroll
            for (int i = 0; i < CHAINS; ++i) a[i] = fma(a[i], b, c);
        }
    }
    T s = 0;
#pragma unroll
    for (int i = 0; i < CHAINS; ++i) s += a[i];
    if (s == (T)-1.2345) g_sink = (double)s;  // never true: the chains stay positive
}

template <class T>
cudaError_t run(int iters, double *tflops, cudaStream_t st) {
    int sms = device_sm_count();
    int per_sm = 0;
    cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, fma_chain_kernel<T>, 256, 0);
    if (e != cudaSuccess) return e;
    if (per_sm < 1) per_sm = 1;
    const int blocks = sms * per_sm;
    cudaEvent_t e0, e1;
    if ((e = cudaEventCreate(&e0)) != cudaSuccess) return e;
    if ((e = cudaEventCreate(&e1)) != cudaSuccess) {
        cudaEventDestroy(e0);
        return e;
    }
    // b < 1 and c small: the chains converge to c / (1 - b) and stay finite and normal
    const T b = (T)0.999, c = (T)1e-4;
    fma_chain_kernel<T><<<blocks, 256, 0, st>>>(iters / 4 > 0 ? iters / 4 : 1, b, c);  // warm-up
    cudaEventRecord(e0, st);
    fma_chain_kernel<T><<<blocks, 256, 0, st>>>(iters, b, c);
    cudaEventRecord(e1, st);
    e = cudaGetLastError();
    if (e == cudaSuccess) e = cudaEventSynchronize(e1);
    float ms = 0.0f;
    if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (e != cudaSuccess) return e;
    const double flops = 2.0 * CHAINS * 16.0 * (double)iters * 256.0 * (double)blocks;
    *tflops = flops / ((double)ms * 1e-3) / 1e12;
    return cudaSuccess;
}

thread_local char g_msg[256] = "no error";

}  // namespace
}  // namespace flints

extern "C" int flints_measure_fma_peak(int precision, int iters, double *tflops, void *stream) {
    using namespace flints;
    if (!tflops) {
        snprintf(g_msg, sizeof g_msg, "flints_measure_fma_peak: tflops is NULL");
        return FLINTS_EINVAL;
    }
    if (iters < 1 || iters > (1 << 24)) {
        snprintf(g_msg, sizeof g_msg, "flints_measure_fma_peak: iters %d outside [1, 2^24]", iters);
        return FLINTS_EINVAL;
    }
    if (precision != FLINTS_FP64 && precision != FLINTS_MIXED) {
        snprintf(g_msg, sizeof g_msg, "flints_measure_fma_peak: precision must be FLINTS_FP64 or FLINTS_MIXED");
        return FLINTS_EINVAL;
    }
    cudaStream_t st = (cudaStream_t)stream;
    const cudaError_t e = precision == FLINTS_FP64 ? run<double>(iters, tflops, st) : run<float>(iters, tflops, st);
    if (e != cudaSuccess) {
        snprintf(g_msg, sizeof g_msg, "flints_measure_fma_peak: %s", cudaGetErrorString(e));
        return FLINTS_ECUDA;
    }
    return FLINTS_OK;
}

extern "C" const char *flints_measure_last_error(void) { return flints::g_msg; }

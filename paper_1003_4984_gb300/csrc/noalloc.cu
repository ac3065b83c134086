// Lensing entry point that allocates no device memory (flints_lens_noalloc).
//
// Some callers cannot call cudaMalloc: serving runtimes that reserve all
// device memory for their own pool up front (a library allocation would fail
// or fragment that pool), and embedding hosts whose allocator policy forbids
// the library from allocating behind their back.  For them this file keeps the
// working memory of one lensing call -- spectrum, xi table nodes,
// interpolation coefficients and event counters -- in a file-scope __device__
// array of fixed size, and runs the same tabulation and lens kernels as the
// plan-based entry points.  Each call copies the spectrum from host memory and
// synchronises its stream once (to read xi(0) back).
//
// Host code must not use the array's name as a device address: in host code
// it is only a stand-in.  The device address is obtained once per device with
// cudaGetSymbolAddress, with that device current, on the first call made on
// that device; that first call should come before any stream capture begins.
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <mutex>

#include "common.cuh"

namespace flints {
namespace {

constexpr int NA_MAX_LMAX = 8192;
constexpr int NA_MAX_INTERVALS = 8192;
constexpr int NA_MAX_DEVICES = 64;

// scratch layout (bytes, each piece 256-byte aligned)
constexpr size_t al(size_t x) { return (x + 255) / 256 * 256; }
constexpr size_t OFF_CL = 0;
constexpr size_t OFF_CLBB = OFF_CL + al(sizeof(double) * (NA_MAX_LMAX + 1));
constexpr size_t OFF_F = OFF_CLBB + al(sizeof(double) * (NA_MAX_LMAX + 1));
constexpr size_t OFF_G = OFF_F + al(sizeof(double) * (NA_MAX_INTERVALS + 1));
constexpr size_t OFF_FM = OFF_G + al(sizeof(double) * (NA_MAX_INTERVALS + 1));
constexpr size_t OFF_GM = OFF_FM + al(sizeof(double) * (NA_MAX_INTERVALS + 1));
constexpr size_t OFF_C64 = OFF_GM + al(sizeof(double) * (NA_MAX_INTERVALS + 1));
constexpr size_t OFF_C32 = OFF_C64 + al(sizeof(Coef64) * NA_MAX_INTERVALS);
constexpr size_t OFF_CNT = OFF_C32 + al(sizeof(float4) * 2 * NA_MAX_INTERVALS);
constexpr size_t OFF_QUEUE = OFF_CNT + al(sizeof(unsigned long long) * CNT_N);
constexpr size_t SCRATCH_BYTES = OFF_QUEUE + al(sizeof(unsigned long long));

// The scratch array: every GPU that loads this library holds it until exit.
static __device__ __align__(256) unsigned char g_noalloc_scratch[SCRATCH_BYTES];

std::mutex g_mu;
unsigned char *g_addr[NA_MAX_DEVICES] = {nullptr};

thread_local char g_msg[512] = "no error";

int na_fail(int code, const char *fmt, ...) {
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(g_msg, sizeof g_msg, fmt, ap);
    va_end(ap);
    return code;
}

}  // namespace
}  // namespace flints

using namespace flints;

extern "C" const char *flints_noalloc_last_error(void) { return g_msg; }

extern "C" int flints_lens_noalloc(int64_t nside, int lmax, const double *cl, const double *cl_bb, int spin, int K,
                                   int precision, int64_t first, int64_t count, const double *map,
                                   const double *defl, double *out, double *var, uint8_t *status, void *stream) {
    if (nside < 1 || nside > 16384) return na_fail(FLINTS_EINVAL, "flints_lens_noalloc: nside outside [1, 16384]");
    if (lmax < 0 || lmax > NA_MAX_LMAX)
        return na_fail(FLINTS_EINVAL, "flints_lens_noalloc: lmax %d exceeds the fixed maximum %d", lmax, NA_MAX_LMAX);
    if (!cl) return na_fail(FLINTS_EINVAL, "flints_lens_noalloc: cl is NULL");
    if (spin != 0 && spin != 2) return na_fail(FLINTS_EINVAL, "flints_lens_noalloc: spin must be 0 or 2");
    if (!(K == 16 || K == 24 || K == 32 || K == 48))
        return na_fail(FLINTS_EINVAL, "flints_lens_noalloc: K must be 16, 24, 32 or 48");
    if (precision != FLINTS_FP64 && precision != FLINTS_MIXED)
        return na_fail(FLINTS_EINVAL, "flints_lens_noalloc: bad precision");
    const int64_t npix = 12 * nside * nside;
    if (first < 0 || count < 0 || first > npix || count > npix - first)
        return na_fail(FLINTS_EINVAL, "flints_lens_noalloc: target range outside the map");
    if (count == 0) return FLINTS_OK;
    if (!map || !defl || !out) return na_fail(FLINTS_EINVAL, "flints_lens_noalloc: NULL data pointer");
    // alignment of the plan-based entry points: deflections 16 bytes, two-component
    // maps and outputs 16 bytes, one-component maps, outputs and variances 8 bytes
    const uintptr_t vec_align = spin == 0 ? 7u : 15u;
    if (((uintptr_t)defl & 15u) || ((uintptr_t)map & vec_align) || ((uintptr_t)out & vec_align) ||
        ((uintptr_t)var & 7u))
        return na_fail(FLINTS_EINVAL,
                       "flints_lens_noalloc: misaligned buffer (defl 16 bytes; map, out %d bytes; var 8 bytes)",
                       spin == 0 ? 8 : 16);
    for (int l = 0; l <= lmax; ++l)
        if (!std::isfinite(cl[l]) || (spin == 2 && cl_bb && !std::isfinite(cl_bb[l])))
            return na_fail(FLINTS_EINVAL, "flints_lens_noalloc: non-finite spectrum value at l = %d", l);

    // the table grid and search disc: the same rule as flints_plan
    const TableGrid tg = table_grid(nside, K, lmax, cl, spin == 2 ? cl_bb : nullptr);
    const int n = tg.n;
    const double t_max = tg.t_max;
    if (n > NA_MAX_INTERVALS)
        return na_fail(FLINTS_EINVAL,
                       "flints_lens_noalloc: the xi table needs %d intervals, above the fixed maximum %d", n,
                       NA_MAX_INTERVALS);
    const int R_rings = tg.R_rings;
    if (2 * R_rings + 2 > 32) return na_fail(FLINTS_EINVAL, "flints_lens_noalloc: search disc spans too many rings");

    // device address of the scratch array, set up once per device
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return na_fail(FLINTS_ECUDA, "cudaGetDevice: %s", cudaGetErrorString(e));
    if (dev < 0 || dev >= NA_MAX_DEVICES) return na_fail(FLINTS_EINVAL, "flints_lens_noalloc: device index too large");
    unsigned char *base;
    {
        std::lock_guard<std::mutex> lk(g_mu);
        if (!g_addr[dev]) {
            void *p = nullptr;
            e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
            if (e != cudaSuccess || !p)
                return na_fail(FLINTS_ECUDA, "cudaGetSymbolAddress: %s", cudaGetErrorString(e));
            g_addr[dev] = static_cast<unsigned char *>(p);
        }
        base = g_addr[dev];
    }
    double *d_cl = reinterpret_cast<double *>(base + OFF_CL);
    double *d_clbb = (spin == 2 && cl_bb) ? reinterpret_cast<double *>(base + OFF_CLBB) : nullptr;
    double *d_f = reinterpret_cast<double *>(base + OFF_F);
    double *d_g = reinterpret_cast<double *>(base + OFF_G);
    double *d_fm = reinterpret_cast<double *>(base + OFF_FM);
    double *d_gm = reinterpret_cast<double *>(base + OFF_GM);
    Coef64 *d_c64 = reinterpret_cast<Coef64 *>(base + OFF_C64);
    float4 *d_c32 = reinterpret_cast<float4 *>(base + OFF_C32);
    unsigned long long *d_cnt = reinterpret_cast<unsigned long long *>(base + OFF_CNT);
    unsigned long long *d_queue = reinterpret_cast<unsigned long long *>(base + OFF_QUEUE);
    cudaStream_t st = (cudaStream_t)stream;
    const size_t ncl = (size_t)lmax + 1, nn = (size_t)n + 1;

#define NA_CK(call, what)                                                                 \
    do {                                                                                  \
        cudaError_t e_ = (call);                                                          \
        if (e_ != cudaSuccess) return na_fail(FLINTS_ECUDA, "%s: %s", what, cudaGetErrorString(e_)); \
    } while (0)
    NA_CK(cudaMemcpyAsync(d_cl, cl, ncl * sizeof(double), cudaMemcpyHostToDevice, st), "copy cl");
    if (d_clbb) NA_CK(cudaMemcpyAsync(d_clbb, cl_bb, ncl * sizeof(double), cudaMemcpyHostToDevice, st), "copy cl_bb");
    // the array keeps the previous call's contents: clear what must start at zero
    NA_CK(cudaMemsetAsync(d_fm, 0, nn * sizeof(double), st), "clear xi- nodes");
    NA_CK(cudaMemsetAsync(d_gm, 0, nn * sizeof(double), st), "clear xi- slopes");
    NA_CK(cudaMemsetAsync(d_cnt, 0, CNT_N * sizeof(unsigned long long), st), "clear counters");
    NA_CK(cudaMemsetAsync(d_queue, 0, sizeof(unsigned long long), st), "clear tile queue");
    NA_CK(launch_xi_table(spin, lmax, d_cl, d_clbb, t_max, n, d_f, d_g, d_fm, d_gm, st), "xi table kernel");
    double xi0 = 0.0;
    NA_CK(cudaMemcpyAsync(&xi0, d_f, sizeof(double), cudaMemcpyDeviceToHost, st), "read xi(0)");
    NA_CK(cudaStreamSynchronize(st), "xi table");
    if (!(xi0 > 0.0) || !std::isfinite(xi0))
        return na_fail(FLINTS_EINVAL, "flints_lens_noalloc: xi(0) = %g is not positive", xi0);
    NA_CK(finish_table(d_f, d_g, n, tg.h, xi0, d_c64, d_c32, st), "table coefficients");

    LensArgs a{};
    a.nside = nside;
    a.first = first;
    a.count = count;
    a.map = map;
    a.defl = defl;
    a.out = out;
    a.var = var;
    a.status = status;
    a.stencil = nullptr;
    a.tab.c64 = d_c64;
    a.tab.c32 = d_c32;
    a.tab.t_max = t_max;
    a.tab.inv_h = tg.inv_h;
    a.tab.inv_h_hi = (float)a.tab.inv_h;
    a.tab.inv_h_lo = (float)(a.tab.inv_h - (double)a.tab.inv_h_hi);
    a.tab.n = n;
    a.xi0 = xi0;
    a.r2 = tg.r2;
    a.counters = d_cnt;
    a.queue = d_queue;
    NA_CK(launch_lens(spin, K, precision, a, R_rings, LaunchCfg{0, 0, 0}, st), "lens kernel launch");
#undef NA_CK
    return FLINTS_OK;
}

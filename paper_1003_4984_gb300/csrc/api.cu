// C ABI of the lensing remap (include/flints.h): plans, launches, statistics.
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <algorithm>
#include <vector>

#include "common.cuh"
#include "batch_types.cuh"

namespace flints {
// class index within a precision: 4 * (spin == 2) + index of K in {16, 24, 32, 48}
cudaError_t batch_prepare_p0(int c, int wpb, int *max_blocks_per_sm);
cudaError_t batch_prepare_p1(int c, int wpb, int *max_blocks_per_sm);
cudaError_t batch_launch_p0(int c, const BatchHeader *hdr, const BatchJob *jobs, unsigned long long *next_tile,
                            int wpb, int blocks, cudaStream_t st);
cudaError_t batch_launch_p1(int c, const BatchHeader *hdr, const BatchJob *jobs, unsigned long long *next_tile,
                            int wpb, int blocks, cudaStream_t st);
int batch_fit_wpb_p0(int c);
int batch_fit_wpb_p1(int c);
cudaError_t launch_lens_spin0(int K, int precision, const LensArgs &a, int R_rings, const LaunchCfg &cfg,
                              cudaStream_t st);
cudaError_t launch_lens_spin2(int K, int precision, const LensArgs &a, int R_rings, const LaunchCfg &cfg,
                              cudaStream_t st);
cudaError_t launch_lens_spin2a(int K, int precision, const LensArgs &a, int R_rings, const LaunchCfg &cfg,
                               cudaStream_t st);
cudaError_t launch_lens_spin1(int K, int precision, const LensArgs &a, int R_rings, const LaunchCfg &cfg,
                              cudaStream_t st);

int device_sm_count() {
    int dev = 0, n = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return 1;
    if (cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || n < 1) return 1;
    return n;
}

size_t device_smem_optin() {
    int dev = 0, n = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return 48 * 1024;
    if (cudaDeviceGetAttribute(&n, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev) != cudaSuccess || n < 1)
        return 48 * 1024;
    return (size_t)n;
}

cudaError_t launch_lens(int spin, int K, int precision, const LensArgs &a, int R_rings, const LaunchCfg &cfg,
                        cudaStream_t st) {
    if (spin == 0) return launch_lens_spin0(K, precision, a, R_rings, cfg, st);
    if (spin == 1) return launch_lens_spin1(K, precision, a, R_rings, cfg, st);
    if (spin == 2) return launch_lens_spin2(K, precision, a, R_rings, cfg, st);
    if (spin == SPIN2_AUG) return launch_lens_spin2a(K, precision, a, R_rings, cfg, st);
    return cudaErrorInvalidValue;
}
}  // namespace flints

using namespace flints;

struct flints_plan_s {
    int device;
    int64_t nside;
    int lmax, spin, K, precision;
    unsigned flags;
    double t_max, h, inv_h, xi0, r, r2;
    int n, R_rings;
    double *d_cl, *d_clbb, *d_f, *d_g, *d_fm, *d_gm;
    Coef64 *d_c64, *d_cm64;  // xi+ (spin 0: xi) and, spin 2, xi- interpolation coefficients
    float4 *d_c32, *d_cm32;
    unsigned long long *d_counters;
    unsigned long long *d_queue;  // QUEUE_SLOTS blocks of BATCH_CLASSES tile-queue counters, one block per call
    unsigned queue_next;
    // spin 0 / 2 plans (not augmented): QUEUE_SLOTS one-job tables of the batched class
    // kernel, and its prepared launch shape
    unsigned char *d_jt;
    int jt_wpb, jt_bps;
    int64_t points;
    int64_t device_bytes;  // sum of the plan's device allocations
    LaunchCfg cfg;
};

static thread_local char g_err[512] = "no error";

static int fail(int code, const char *fmt, ...) {
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(g_err, sizeof g_err, fmt, ap);
    va_end(ap);
    return code;
}

static int cuda_fail(cudaError_t e, const char *what) {
    return fail(e == cudaErrorMemoryAllocation ? FLINTS_ENOMEM : FLINTS_ECUDA, "%s: %s", what, cudaGetErrorString(e));
}

#define CK(call, what)                                   \
    do {                                                 \
        cudaError_t e_ = (call);                         \
        if (e_ != cudaSuccess) return cuda_fail(e_, what); \
    } while (0)

static bool supported_K(int K) { return K == 16 || K == 24 || K == 32 || K == 48; }

// one-job table of the batched class kernel (header, then the job), 256-byte slots
static constexpr size_t JT_BYTES = (sizeof(BatchHeader) + sizeof(BatchJob) + 255) / 256 * 256;

struct OneJob {
    BatchHeader h;
    BatchJob j;
};

// Writes a one-job table into device memory from the kernel's parameters: no
// copy-engine transfer, so the call's table never queues behind the caller's own
// host-device copies, and no host staging buffer has to outlive the call.
__global__ void store_one_job(OneJob t, unsigned *dst) {
    static_assert(sizeof(OneJob) % 4 == 0, "word copy");
    const unsigned *src = reinterpret_cast<const unsigned *>(&t);
    for (int i = threadIdx.x; i < (int)(sizeof(OneJob) / 4); i += blockDim.x) dst[i] = src[i];
}

namespace flints {
TableGrid table_grid(int64_t nside, int K, int lmax, const double *cl, const double *cl_bb) {
    TableGrid g{};
    g.r = 1.25 * std::sqrt(K / 3.0) / (double)nside;
    g.r2 = g.r * g.r;
    g.t_max = 4.0 * g.r * g.r;
    double x0 = 0.0, b4num = 0.0;
    for (int l = 0; l <= lmax; ++l) {
        const double ld = (double)l;
        const double c = std::fabs(cl[l]) + (cl_bb ? std::fabs(cl_bb[l]) : 0.0);
        const double a = (2.0 * ld + 1.0) / (4.0 * PI) * c;
        x0 += a;
        if (l >= 4) b4num += a * ((ld - 3) * (ld - 2) * (ld - 1) * ld * (ld + 1) * (ld + 2) * (ld + 3) * (ld + 4) / 384.0);
    }
    const double b4 = x0 > 0 ? b4num / 16.0 / x0 : 0.0;
    g.n = 64;
    if (b4 > 0) {
        const double h = std::pow(384.0 * 1e-11 / b4, 0.25);
        const double want = std::ceil(std::log2(g.t_max / h));
        g.n = want > 16 ? 65536 : (want < 6 ? 64 : (1 << (int)want));
    }
    g.h = g.t_max / g.n;
    g.inv_h = g.n / g.t_max;
    g.R_rings = (int)std::ceil(1.5 * g.r * (double)nside) + 1;
    return g;
}
}  // namespace flints

static void free_plan_memory(flints_plan_s *p) {
    cudaFree(p->d_cl);
    cudaFree(p->d_clbb);
    cudaFree(p->d_f);
    cudaFree(p->d_g);
    cudaFree(p->d_fm);
    cudaFree(p->d_gm);
    cudaFree(p->d_c64);
    cudaFree(p->d_c32);
    cudaFree(p->d_cm64);
    cudaFree(p->d_cm32);
    cudaFree(p->d_counters);
    cudaFree(p->d_queue);
    cudaFree(p->d_jt);
}

extern "C" {

const char *flints_last_error(void) { return g_err; }

int flints_plan(flints_plan_t *out, int64_t nside, int lmax, const double *cl, const double *cl_bb, int spin, int K,
                int precision, unsigned flags, void *stream) {
    if (!out) return fail(FLINTS_EINVAL, "flints_plan: out is NULL");
    *out = nullptr;
    if (nside < 1 || nside > 16384) return fail(FLINTS_EINVAL, "flints_plan: nside %lld outside [1, 16384]", (long long)nside);
    if (lmax < 0 || lmax > 16384) return fail(FLINTS_EINVAL, "flints_plan: lmax %d outside [0, 16384]", lmax);
    if (!cl) return fail(FLINTS_EINVAL, "flints_plan: cl is NULL");
    if (spin != 0 && spin != 1 && spin != 2) return fail(FLINTS_EINVAL, "flints_plan: spin must be 0, 1 or 2");
    if (!supported_K(K)) return fail(FLINTS_EINVAL, "flints_plan: K must be 16, 24, 32 or 48 (got %d)", K);
    if (12 * nside * nside < K) return fail(FLINTS_EINVAL, "flints_plan: K exceeds the pixel count");
    if (precision != FLINTS_FP64 && precision != FLINTS_MIXED)
        return fail(FLINTS_EINVAL, "flints_plan: precision must be FLINTS_FP64 or FLINTS_MIXED");
    if (flags & ~(unsigned)(FLINTS_SPIN2_AUGMENTED | FLINTS_ROTATE_TO_TARGET | FLINTS_NO_VARIANCE |
                            FLINTS_FORCE_FALLBACK))
        return fail(FLINTS_EINVAL, "flints_plan: unknown flag bits 0x%x", flags);
    if ((flags & FLINTS_SPIN2_AUGMENTED) && spin != 2)
        return fail(FLINTS_EINVAL, "flints_plan: FLINTS_SPIN2_AUGMENTED applies to spin-2 plans");
    if ((flags & FLINTS_ROTATE_TO_TARGET) && spin == 0)
        return fail(FLINTS_EINVAL, "flints_plan: FLINTS_ROTATE_TO_TARGET applies to spin-1 and spin-2 plans");
    for (int l = 0; l <= lmax; ++l) {
        if (!std::isfinite(cl[l]) || (spin != 0 && cl_bb && !std::isfinite(cl_bb[l])))
            return fail(FLINTS_EINVAL, "flints_plan: non-finite spectrum value at l = %d", l);
    }
    cudaStream_t st = (cudaStream_t)stream;
    flints_plan_s *p = new flints_plan_s();
    std::memset(p, 0, sizeof *p);
    cudaGetDevice(&p->device);
    p->nside = nside;
    p->lmax = lmax;
    p->spin = spin;
    p->K = K;
    p->precision = precision;
    p->flags = flags;

    // Table domain and size, and the search disc (the grid rule of table_grid).
    {
        const TableGrid tg = table_grid(nside, K, lmax, cl, spin != 0 ? cl_bb : nullptr);
        p->r = tg.r;
        p->r2 = tg.r2;
        p->t_max = tg.t_max;
        p->n = tg.n;
        p->h = tg.h;
        p->inv_h = tg.inv_h;
        p->R_rings = tg.R_rings;
    }
    if (2 * p->R_rings + 2 > 32) {
        delete p;
        return fail(FLINTS_EINVAL, "flints_plan: search disc spans too many rings");
    }

    const size_t ncl = (size_t)(lmax + 1);
    const size_t nn = (size_t)p->n + 1;
    cudaError_t e;
#define ALLOC(ptr, bytes)                                      \
    do {                                                       \
        e = cudaMalloc((void **)&(ptr), (bytes));              \
        if (e != cudaSuccess) {                                \
            free_plan_memory(p);                               \
            delete p;                                          \
            return cuda_fail(e, "flints_plan: cudaMalloc");    \
        }                                                      \
        p->device_bytes += (int64_t)(bytes);                   \
    } while (0)
    ALLOC(p->d_cl, ncl * sizeof(double));
    if (spin != 0 && cl_bb) {
        ALLOC(p->d_clbb, ncl * sizeof(double));
    }
    ALLOC(p->d_f, nn * sizeof(double));
    ALLOC(p->d_g, nn * sizeof(double));
    ALLOC(p->d_fm, nn * sizeof(double));
    ALLOC(p->d_gm, nn * sizeof(double));
    ALLOC(p->d_c64, (size_t)p->n * sizeof(Coef64));
    ALLOC(p->d_c32, (size_t)p->n * 2 * sizeof(float4));
    if (spin != 0) {
        ALLOC(p->d_cm64, (size_t)p->n * sizeof(Coef64));
        ALLOC(p->d_cm32, (size_t)p->n * 2 * sizeof(float4));
    }
    ALLOC(p->d_counters, CNT_N * sizeof(unsigned long long));
    ALLOC(p->d_queue, (size_t)QUEUE_SLOTS * BATCH_CLASSES * sizeof(unsigned long long));
    if (spin != 1 && !(flags & FLINTS_SPIN2_AUGMENTED)) {
        ALLOC(p->d_jt, (size_t)QUEUE_SLOTS * JT_BYTES);
    }
#undef ALLOC
    auto bail = [&](cudaError_t err, const char *what) {
        free_plan_memory(p);
        delete p;
        return cuda_fail(err, what);
    };
    if ((e = cudaMemcpyAsync(p->d_cl, cl, ncl * sizeof(double), cudaMemcpyHostToDevice, st)) != cudaSuccess)
        return bail(e, "flints_plan: copy cl");
    if (p->d_clbb &&
        (e = cudaMemcpyAsync(p->d_clbb, cl_bb, ncl * sizeof(double), cudaMemcpyHostToDevice, st)) != cudaSuccess)
        return bail(e, "flints_plan: copy cl_bb");
    if ((e = cudaMemsetAsync(p->d_counters, 0, CNT_N * sizeof(unsigned long long), st)) != cudaSuccess)
        return bail(e, "flints_plan: memset");
    if ((e = cudaMemsetAsync(p->d_fm, 0, nn * sizeof(double), st)) != cudaSuccess) return bail(e, "flints_plan: memset");
    if ((e = cudaMemsetAsync(p->d_gm, 0, nn * sizeof(double), st)) != cudaSuccess) return bail(e, "flints_plan: memset");
    if ((e = launch_xi_table(spin, lmax, p->d_cl, p->d_clbb, p->t_max, p->n, p->d_f, p->d_g, p->d_fm, p->d_gm, st)) !=
        cudaSuccess)
        return bail(e, "flints_plan: xi table kernel");
    double xi0 = 0.0;
    if ((e = cudaMemcpyAsync(&xi0, p->d_f, sizeof(double), cudaMemcpyDeviceToHost, st)) != cudaSuccess)
        return bail(e, "flints_plan: read xi(0)");
    if ((e = cudaStreamSynchronize(st)) != cudaSuccess) return bail(e, "flints_plan: xi table");
    if (!(xi0 > 0.0) || !std::isfinite(xi0)) {
        free_plan_memory(p);
        delete p;
        return fail(FLINTS_EINVAL, "flints_plan: xi(0) = %g is not positive", xi0);
    }
    p->xi0 = xi0;
    if ((e = finish_table(p->d_f, p->d_g, p->n, p->h, xi0, p->d_c64, p->d_c32, st)) != cudaSuccess)
        return bail(e, "flints_plan: table coefficients");
    if (spin != 0 && (e = finish_table(p->d_fm, p->d_gm, p->n, p->h, xi0, p->d_cm64, p->d_cm32, st)) != cudaSuccess)
        return bail(e, "flints_plan: xi- table");
    if ((e = cudaStreamSynchronize(st)) != cudaSuccess) return bail(e, "flints_plan: table coefficients");
    *out = p;
    return FLINTS_OK;
}

void flints_free(flints_plan_t p) {
    if (!p) return;
    int cur = 0;
    cudaGetDevice(&cur);
    if (cur != p->device) cudaSetDevice(p->device);
    free_plan_memory(p);
    if (cur != p->device) cudaSetDevice(cur);
    delete p;
}

static int check_device(flints_plan_t p) {
    int cur = -1;
    cudaGetDevice(&cur);
    if (cur != p->device) return fail(FLINTS_EINVAL, "plan was created on device %d, current device is %d", p->device, cur);
    return FLINTS_OK;
}

// nside_tgt = 0: lensing targets (pixels of the plan's grid displaced by defl);
// nside_tgt > 0: the pixel centres of an Nside = nside_tgt grid (supersampling).
static int run(flints_plan_t p, int64_t nside_tgt, int64_t first, int64_t count, const double *map,
               const double *defl, double *out, double *var, uint8_t *status, int64_t *stencil, void *stream) {
    if (!p) return fail(FLINTS_EINVAL, "plan is NULL");
    if (int rc = check_device(p)) return rc;
    const int64_t nt = nside_tgt > 0 ? nside_tgt : p->nside;
    const int64_t npix = 12 * nt * nt;
    if (first < 0 || count < 0 || first > npix || count > npix - first)
        return fail(FLINTS_EINVAL, "target range [%lld, %lld) outside [0, %lld)", (long long)first,
                    (long long)(first + count), (long long)npix);
    if (count == 0) return FLINTS_OK;
    if (!defl && nside_tgt == 0) return fail(FLINTS_EINVAL, "defl is NULL");
    if (!stencil && (!map || !out)) return fail(FLINTS_EINVAL, "map and out must not be NULL");
    // defl and two-component maps/outputs are read and written as 16-byte pairs
    const uintptr_t need = p->spin == 0 ? 7u : 15u;
    if (((uintptr_t)defl & 15u) || (((uintptr_t)map | (uintptr_t)out) & need) ||
        (((uintptr_t)var | (uintptr_t)stencil) & 7u))
        return fail(FLINTS_EINVAL, "defl (and spin 1/2 map and out) must be 16-byte aligned, spin 0 map, out, var and "
                                   "idx 8-byte aligned");
    LensArgs a{};
    a.nside = p->nside;
    a.first = first;
    a.count = count;
    a.map = map;
    a.defl = defl;
    a.out = out;
    a.var = (p->flags & FLINTS_NO_VARIANCE) ? nullptr : var;
    a.force_fallback = (p->flags & FLINTS_FORCE_FALLBACK) ? 1 : 0;
    a.rotate = (p->flags & FLINTS_ROTATE_TO_TARGET) ? 1 : 0;
    a.nside_tgt = nside_tgt;
    a.status = status;
    a.stencil = stencil;
    a.tab.c64 = p->d_c64;
    a.tab.c32 = p->d_c32;
    a.tab.t_max = p->t_max;
    a.tab.inv_h = p->inv_h;
    a.tab.inv_h_hi = (float)p->inv_h;
    a.tab.inv_h_lo = (float)(p->inv_h - (double)a.tab.inv_h_hi);
    a.tab.n = p->n;
    a.tabm = a.tab;
    a.tabm.c64 = p->d_cm64;
    a.tabm.c32 = p->d_cm32;
    a.xi0 = p->xi0;
    a.r2 = p->r2;
    a.counters = p->d_counters;
    // this call's slot: its tile-queue counters (and one-job table), zeroed on the stream
    const unsigned slot = p->queue_next++ % QUEUE_SLOTS;
    unsigned long long *qblock = p->d_queue + (size_t)slot * BATCH_CLASSES;
    cudaStream_t st = (cudaStream_t)stream;
    cudaError_t e;
    if (p->d_jt) {
        // spin 0 / 2: the persistent class kernel of the batched launch, given a one-job
        // table (the same per-tile code; on GB300 this kernel runs the c3 workload 3-4 %
        // faster than the single-range kernel)
        const int cls = 8 * (p->precision == FLINTS_MIXED ? 1 : 0) + 4 * (p->spin == 2 ? 1 : 0) + batch_k_index(p->K);
        const int tp = p->cfg.tile_points > 0 && p->cfg.tile_points < MAX_TILE_POINTS ? p->cfg.tile_points
                                                                                       : MAX_TILE_POINTS;
        const int fit = (cls >> 3) ? batch_fit_wpb_p1(cls & 7) : batch_fit_wpb_p0(cls & 7);
        // default: 8-warp blocks (2 per SM at spin 2, K = 32; on 2^24 targets of the
        // Nside 4096 workload 3.8 % faster than four 4-warp blocks for the same 16 warps per SM)
        int wpb = p->cfg.warps_per_block > 0 ? p->cfg.warps_per_block : 8;
        if (wpb > fit) wpb = fit;
        if (p->jt_wpb != wpb) {
            int mx = 0;
            e = (cls >> 3) ? batch_prepare_p1(cls & 7, wpb, &mx) : batch_prepare_p0(cls & 7, wpb, &mx);
            if (e != cudaSuccess) return cuda_fail(e, "lens kernel set-up");
            if (mx < 1) return fail(FLINTS_EINVAL, "lens kernel: %d warps per block do not fit on an SM", wpb);
            p->jt_wpb = wpb;
            p->jt_bps = mx;
        }
        const int64_t ntiles = (count + tp - 1) / tp;
        OneJob t{};
        t.h.njobs[cls] = 1;
        t.h.total_tiles[cls] = ntiles;
        t.h.tile_pts = tp;
        t.j.a = a;
        t.j.R_rings = p->R_rings;
        t.j.K = p->K;
        t.j.spin = p->spin;
        t.j.precision = p->precision;
        t.j.tile_begin = 0;
        t.j.ntiles = ntiles;
        unsigned char *ds = p->d_jt + (size_t)slot * JT_BYTES;
        store_one_job<<<1, 64, 0, st>>>(t, reinterpret_cast<unsigned *>(ds));
        if ((e = cudaGetLastError()) != cudaSuccess) return cuda_fail(e, "lens job table");
        if ((e = cudaMemsetAsync(qblock + cls, 0, sizeof(unsigned long long), st)) != cudaSuccess)
            return cuda_fail(e, "tile queue reset");
        int bps = p->jt_bps;
        if (p->cfg.blocks_per_sm > 0 && p->cfg.blocks_per_sm < bps) bps = p->cfg.blocks_per_sm;
        int64_t blocks = (int64_t)device_sm_count() * bps;
        const int64_t need = (ntiles + wpb - 1) / wpb;
        if (blocks > need) blocks = need;
        const BatchHeader *hd = reinterpret_cast<const BatchHeader *>(ds);
        const BatchJob *jd = reinterpret_cast<const BatchJob *>(ds + offsetof(OneJob, j));
        e = (cls >> 3) ? batch_launch_p1(cls & 7, hd, jd, qblock, wpb, (int)blocks, st)
                       : batch_launch_p0(cls & 7, hd, jd, qblock, wpb, (int)blocks, st);
        if (e != cudaSuccess) return cuda_fail(e, "lens kernel launch");
        p->points += count;
        return FLINTS_OK;
    }
    // spin 1 and the augmented estimator: the single-range kernel with the slot's queue
    a.queue = qblock;
    if ((e = cudaMemsetAsync(a.queue, 0, sizeof(unsigned long long), st)) != cudaSuccess)
        return cuda_fail(e, "tile queue reset");
    const int mode = (p->flags & FLINTS_SPIN2_AUGMENTED) ? SPIN2_AUG : p->spin;
    e = launch_lens(mode, p->K, p->precision, a, p->R_rings, p->cfg, st);
    if (e != cudaSuccess) return cuda_fail(e, "lens kernel launch");
    p->points += count;
    return FLINTS_OK;
}

int flints_lens_spin0(flints_plan_t p, const double *map, const double *defl, double *out, double *var, void *stream) {
    if (!p) return fail(FLINTS_EINVAL, "plan is NULL");
    if (p->spin != 0) return fail(FLINTS_EINVAL, "flints_lens_spin0 called with a spin-2 plan");
    return run(p, 0, 0, 12 * p->nside * p->nside, map, defl, out, var, nullptr, nullptr, stream);
}

int flints_lens_spin2(flints_plan_t p, const double *qu, const double *defl, double *qu_out, double *var,
                      void *stream) {
    if (!p) return fail(FLINTS_EINVAL, "plan is NULL");
    if (p->spin != 2) return fail(FLINTS_EINVAL, "flints_lens_spin2 called with a plan of spin %d", p->spin);
    return run(p, 0, 0, 12 * p->nside * p->nside, qu, defl, qu_out, var, nullptr, nullptr, stream);
}

int flints_lens_range(flints_plan_t p, int64_t first, int64_t count, const double *map, const double *defl,
                      double *out, double *var, uint8_t *status, void *stream) {
    return run(p, 0, first, count, map, defl, out, var, status, nullptr, stream);
}

int flints_supersample(flints_plan_t p, int64_t nside_out, int64_t first, int64_t count, const double *map,
                       double *out, double *var, uint8_t *status, void *stream) {
    if (!p) return fail(FLINTS_EINVAL, "plan is NULL");
    if (nside_out < 1 || nside_out > 65536)
        return fail(FLINTS_EINVAL, "flints_supersample: nside_out %lld outside [1, 65536]", (long long)nside_out);
    return run(p, nside_out, first, count, map, nullptr, out, var, status, nullptr, stream);
}

int flints_stencil(flints_plan_t p, int64_t first, int64_t count, const double *defl, int64_t *idx, uint8_t *status,
                   void *stream) {
    if (!idx) return fail(FLINTS_EINVAL, "idx is NULL");
    return run(p, 0, first, count, nullptr, defl, nullptr, nullptr, status, idx, stream);
}

// ------------------------------------------------------------------ batches
}  // extern "C"

struct flints_batch_s {
    int device, max_jobs, num_sms;
    size_t table_bytes;       // header + job array
    unsigned char *d_buf;     // device: header, jobs, one work-queue counter per class
    unsigned char *h_buf;     // pinned host staging of header and jobs
    int wpb[BATCH_CLASSES], max_bps[BATCH_CLASSES];  // prepared launch shape per class
    int fit_wpb[BATCH_CLASSES];                      // warps per block that fit in shared memory
};

static BatchHeader *hdr_of(unsigned char *p) { return reinterpret_cast<BatchHeader *>(p); }
static BatchJob *jobs_of(unsigned char *p) { return reinterpret_cast<BatchJob *>(p + sizeof(BatchHeader)); }

static int batch_prepare(flints_batch_s *b, int cls, int wpb) {
    int mx = 0;
    cudaError_t e = (cls >> 3) ? batch_prepare_p1(cls & 7, wpb, &mx) : batch_prepare_p0(cls & 7, wpb, &mx);
    if (e != cudaSuccess) return cuda_fail(e, "batch kernel set-up");
    if (mx < 1) return fail(FLINTS_EINVAL, "batch kernel: %d warps per block do not fit on an SM", wpb);
    b->wpb[cls] = wpb;
    b->max_bps[cls] = mx;
    return FLINTS_OK;
}

extern "C" {

int flints_batch_create(flints_batch_t *out, int max_jobs) {
    if (!out || max_jobs < 1 || max_jobs > (1 << 20)) return fail(FLINTS_EINVAL, "flints_batch_create: bad arguments");
    *out = nullptr;
    flints_batch_s *b = new flints_batch_s();
    std::memset(b, 0, sizeof *b);
    cudaGetDevice(&b->device);
    b->max_jobs = max_jobs;
    b->num_sms = device_sm_count();
    b->table_bytes = sizeof(BatchHeader) + sizeof(BatchJob) * (size_t)max_jobs;
    cudaError_t e = cudaMalloc((void **)&b->d_buf, b->table_bytes + BATCH_CLASSES * sizeof(unsigned long long));
    if (e == cudaSuccess) e = cudaHostAlloc((void **)&b->h_buf, b->table_bytes, cudaHostAllocDefault);
    if (e != cudaSuccess) {
        cudaFree(b->d_buf);
        delete b;
        return cuda_fail(e, "flints_batch_create: allocation");
    }
    std::memset(b->h_buf, 0, b->table_bytes);
    for (int cls = 0; cls < BATCH_CLASSES; ++cls) {
        b->fit_wpb[cls] = (cls >> 3) ? batch_fit_wpb_p1(cls & 7) : batch_fit_wpb_p0(cls & 7);
        if (int rc = batch_prepare(b, cls, b->fit_wpb[cls] < 4 ? b->fit_wpb[cls] : 4)) {
            cudaFree(b->d_buf);
            cudaFreeHost(b->h_buf);
            delete b;
            return rc;
        }
    }
    *out = b;
    return FLINTS_OK;
}

void flints_batch_free(flints_batch_t b) {
    if (!b) return;
    cudaFree(b->d_buf);
    cudaFreeHost(b->h_buf);
    delete b;
}

int flints_batch_stage(flints_batch_t b, const flints_job *jobs, int n, int tile_points) {
    if (!b) return fail(FLINTS_EINVAL, "batch is NULL");
    if (n < 0 || n > b->max_jobs || (n > 0 && !jobs))
        return fail(FLINTS_EINVAL, "flints_batch_stage: %d jobs for a batch of capacity %d", n, b->max_jobs);
    if (tile_points < 0 || tile_points > MAX_TILE_POINTS)
        return fail(FLINTS_EINVAL, "flints_batch_stage: tile_points 0..%d", MAX_TILE_POINTS);
    const int tp = tile_points > 0 ? tile_points : MAX_TILE_POINTS;
    std::vector<BatchJob> v;
    v.reserve(n);
    std::vector<double> cost;
    for (int i = 0; i < n; ++i) {
        const flints_job &j = jobs[i];
        flints_plan_s *p = j.plan;
        if (!p) return fail(FLINTS_EINVAL, "job %d: plan is NULL", i);
        if (p->device != b->device) return fail(FLINTS_EINVAL, "job %d: plan and batch on different devices", i);
        if ((p->flags & FLINTS_SPIN2_AUGMENTED) || p->spin == 1)
            return fail(FLINTS_EINVAL, "job %d: spin-1 and augmented spin-2 plans run through the single-plan entry points",
                        i);
        const int64_t npix = 12 * p->nside * p->nside;
        if (j.first < 0 || j.count < 0 || j.first > npix || j.count > npix - j.first)
            return fail(FLINTS_EINVAL, "job %d: target range outside the map", i);
        if (j.count == 0) continue;
        if (!j.map || !j.defl || !j.out) return fail(FLINTS_EINVAL, "job %d: NULL data pointer", i);
        if (((uintptr_t)j.defl & 15u) || (((uintptr_t)j.map | (uintptr_t)j.out) & (p->spin == 0 ? 7u : 15u)) ||
            ((uintptr_t)j.var & 7u))
            return fail(FLINTS_EINVAL, "job %d: misaligned map, defl, out or var", i);
        BatchJob bj{};
        LensArgs &a = bj.a;
        a.nside = p->nside;
        a.first = j.first;
        a.count = j.count;
        a.map = j.map;
        a.defl = j.defl;
        a.out = j.out;
        a.var = (p->flags & FLINTS_NO_VARIANCE) ? nullptr : j.var;
        a.force_fallback = (p->flags & FLINTS_FORCE_FALLBACK) ? 1 : 0;
        a.rotate = (p->flags & FLINTS_ROTATE_TO_TARGET) ? 1 : 0;
        a.status = j.status;
        a.stencil = nullptr;
        a.tab.c64 = p->d_c64;
        a.tab.c32 = p->d_c32;
        a.tab.t_max = p->t_max;
        a.tab.inv_h = p->inv_h;
        a.tab.inv_h_hi = (float)p->inv_h;
        a.tab.inv_h_lo = (float)(p->inv_h - (double)a.tab.inv_h_hi);
        a.tab.n = p->n;
        a.xi0 = p->xi0;
        a.r2 = p->r2;
        a.counters = p->d_counters;
        bj.R_rings = p->R_rings;
        bj.K = p->K;
        bj.spin = p->spin;
        bj.precision = p->precision;
        bj.ntiles = (j.count + tp - 1) / tp;
        v.push_back(bj);
    }
    // every job is valid: count its points (a refused stage counts none)
    for (int i = 0; i < n; ++i) jobs[i].plan->points += jobs[i].count;
    // classes (precision, spin, K), each in decreasing estimated cost
    // (longest jobs start first)
    auto cls_of = [](const BatchJob &x) { return 8 * x.precision + (x.spin == 2 ? 4 : 0) + batch_k_index(x.K); };
    auto est = [](const BatchJob &x) {
        return (double)x.a.count * x.K * x.K * x.K * (x.spin == 2 ? 4.0 : 1.0);
    };
    std::stable_sort(v.begin(), v.end(), [&](const BatchJob &x, const BatchJob &y) {
        if (cls_of(x) != cls_of(y)) return cls_of(x) < cls_of(y);
        return est(x) > est(y);
    });
    BatchHeader h{};
    h.tile_pts = tp;
    int k = 0;
    for (int cls = 0; cls < BATCH_CLASSES; ++cls) {
        h.job_offset[cls] = k;
        int64_t tiles = 0;
        while (k < (int)v.size() && cls_of(v[k]) == cls) {
            v[k].tile_begin = tiles;
            tiles += v[k].ntiles;
            ++k;
            ++h.njobs[cls];
        }
        h.total_tiles[cls] = tiles;
    }
    *hdr_of(b->h_buf) = h;
    if (!v.empty()) std::memcpy(jobs_of(b->h_buf), v.data(), v.size() * sizeof(BatchJob));
    return FLINTS_OK;
}

int flints_batch_launch(flints_batch_t b, const flints_launch_cfg *cfg, void *stream) {
    if (!b) return fail(FLINTS_EINVAL, "batch is NULL");
    int cur = -1;
    cudaGetDevice(&cur);
    if (cur != b->device) return fail(FLINTS_EINVAL, "batch was created on device %d, current device is %d", b->device, cur);
    const int want = (cfg && cfg->warps_per_block > 0) ? cfg->warps_per_block : 4;
    if (want > 8) return fail(FLINTS_EINVAL, "flints_batch_launch: warps_per_block 1..8");
    cudaStream_t st = (cudaStream_t)stream;
    const BatchHeader *h = hdr_of(b->h_buf);
    int njobs = 0;
    for (int cls = 0; cls < BATCH_CLASSES; ++cls) njobs += h->njobs[cls];
    const size_t bytes = sizeof(BatchHeader) + sizeof(BatchJob) * (size_t)njobs;
    unsigned long long *ctr = reinterpret_cast<unsigned long long *>(b->d_buf + b->table_bytes);
    CK(cudaMemcpyAsync(b->d_buf, b->h_buf, bytes, cudaMemcpyHostToDevice, st), "batch: upload jobs");
    CK(cudaMemsetAsync(ctr, 0, BATCH_CLASSES * sizeof(unsigned long long), st), "batch: reset work queues");
    // every class kernel is launched (an empty class exits at once), so a captured
    // graph runs whatever table is staged later
    for (int cls = 0; cls < BATCH_CLASSES; ++cls) {
        const int wpb = want < b->fit_wpb[cls] ? want : b->fit_wpb[cls];  // a hint: keep within shared memory
        if (b->wpb[cls] != wpb)
            if (int rc = batch_prepare(b, cls, wpb)) return rc;
        int bps = b->max_bps[cls];
        if (cfg && cfg->blocks_per_sm > 0 && cfg->blocks_per_sm < bps) bps = cfg->blocks_per_sm;
        const int blocks = b->num_sms * bps;
        cudaError_t e = (cls >> 3)
                            ? batch_launch_p1(cls & 7, hdr_of(b->d_buf), jobs_of(b->d_buf), ctr, wpb, blocks, st)
                            : batch_launch_p0(cls & 7, hdr_of(b->d_buf), jobs_of(b->d_buf), ctr, wpb, blocks, st);
        if (e != cudaSuccess) return cuda_fail(e, "batch kernel launch");
    }
    return FLINTS_OK;
}

int flints_batch_run(flints_batch_t b, const flints_job *jobs, int n, const flints_launch_cfg *cfg, void *stream) {
    const int tp = cfg ? cfg->tile_points : 0;
    if (int rc = flints_batch_stage(b, jobs, n, tp)) return rc;
    return flints_batch_launch(b, cfg, stream);
}

int flints_lens_batch(const flints_job *jobs, int n, void *stream) {
    if (n < 0 || (n > 0 && !jobs)) return fail(FLINTS_EINVAL, "flints_lens_batch: bad job list");
    if (n == 0) return FLINTS_OK;
    flints_batch_t b = nullptr;
    if (int rc = flints_batch_create(&b, n)) return rc;
    int rc = flints_batch_run(b, jobs, n, nullptr, stream);
    cudaError_t e = cudaStreamSynchronize((cudaStream_t)stream);
    flints_batch_free(b);
    if (rc) return rc;
    if (e != cudaSuccess) return cuda_fail(e, "flints_lens_batch");
    return FLINTS_OK;
}

int flints_get_stats(flints_plan_t p, flints_stats *s, void *stream) {
    if (!p || !s) return fail(FLINTS_EINVAL, "flints_get_stats: NULL argument");
    unsigned long long c[CNT_N] = {0};
    CK(cudaMemcpyAsync(c, p->d_counters, sizeof c, cudaMemcpyDeviceToHost, (cudaStream_t)stream), "read counters");
    CK(cudaStreamSynchronize((cudaStream_t)stream), "read counters");
    s->points = p->points;
    s->nugget = (int64_t)c[CNT_NUGGET];
    s->fallback = (int64_t)c[CNT_FALLBACK];
    s->window = (int64_t)c[CNT_WINDOW];
    s->failed = (int64_t)c[CNT_FAILED];
    return FLINTS_OK;
}

int flints_reset_stats(flints_plan_t p, void *stream) {
    if (!p) return fail(FLINTS_EINVAL, "plan is NULL");
    CK(cudaMemsetAsync(p->d_counters, 0, CNT_N * sizeof(unsigned long long), (cudaStream_t)stream), "reset counters");
    p->points = 0;
    return FLINTS_OK;
}

int flints_plan_set_launch(flints_plan_t p, const flints_launch_cfg *cfg) {
    if (!p) return fail(FLINTS_EINVAL, "plan is NULL");
    if (!cfg) {
        p->cfg = LaunchCfg{0, 0, 0};
        return FLINTS_OK;
    }
    if (cfg->warps_per_block < 0 || cfg->warps_per_block > 8 || cfg->blocks_per_sm < 0 || cfg->blocks_per_sm > 32 ||
        cfg->tile_points < 0 || cfg->tile_points > MAX_TILE_POINTS)
        return fail(FLINTS_EINVAL, "flints_plan_set_launch: warps_per_block 0..8, blocks_per_sm 0..32, tile_points 0..%d",
                    MAX_TILE_POINTS);
    p->cfg = LaunchCfg{cfg->warps_per_block, cfg->blocks_per_sm, cfg->tile_points};
    return FLINTS_OK;
}

int flints_get_info(flints_plan_t p, flints_plan_info *info) {
    if (!p || !info) return fail(FLINTS_EINVAL, "flints_get_info: NULL argument");
    info->nside = p->nside;
    info->lmax = p->lmax;
    info->spin = p->spin;
    info->K = p->K;
    info->precision = p->precision;
    info->t_max = p->t_max;
    info->n_intervals = p->n;
    info->xi0 = p->xi0;
    info->search_radius = p->r;
    info->device_bytes = p->device_bytes;
    return FLINTS_OK;
}

int flints_get_table(flints_plan_t p, int which, double *f, double *g, void *stream) {
    if (!p || !f || !g) return fail(FLINTS_EINVAL, "flints_get_table: NULL argument");
    if (which != 0 && !(which == 1 && p->spin != 0)) return fail(FLINTS_EINVAL, "flints_get_table: bad table index");
    const size_t bytes = ((size_t)p->n + 1) * sizeof(double);
    cudaStream_t st = (cudaStream_t)stream;
    CK(cudaMemcpyAsync(f, which ? p->d_fm : p->d_f, bytes, cudaMemcpyDeviceToHost, st), "read table");
    CK(cudaMemcpyAsync(g, which ? p->d_gm : p->d_g, bytes, cudaMemcpyDeviceToHost, st), "read table");
    CK(cudaStreamSynchronize(st), "read table");
    return FLINTS_OK;
}

}  // extern "C"

// Shared device-side definitions of the lensing remap library (sm_103a).
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include "flints.h"

namespace flints {

constexpr unsigned FULL = 0xffffffffu;
constexpr double PI = 3.141592653589793238462643383279502884;
constexpr double NUGGET_EPS = 1.49e-8;  // sqrt of the double-precision epsilon (Sec. 2.4)
constexpr int MAX_NUGGET_STEPS = 8;      // nugget doubled at most this many times

// ---------------------------------------------------------------------------
// Double-float numbers: value = hi + lo with |lo| <= ulp(hi)/2 after
// normalisation, about 48 significant bits on the FP32 pipe.  The error-free
// transforms are Knuth's TwoSum and the FMA form of Dekker's TwoProduct; the
// __f*_rn intrinsics keep the compiler from contracting or reassociating them.
// ---------------------------------------------------------------------------
struct df {
    float hi, lo;
};

__device__ __forceinline__ df df_from(double x) {
    float h = __double2float_rn(x);
    float l = __double2float_rn(x - (double)h);
    return {h, l};
}
__device__ __forceinline__ double df_to(df a) { return (double)a.hi + (double)a.lo; }

__device__ __forceinline__ df two_sum(float a, float b) {
    float s = __fadd_rn(a, b);
    float bb = __fsub_rn(s, a);
    float e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
    return {s, e};
}
__device__ __forceinline__ df quick_two_sum(float a, float b) {  // needs |a| >= |b|
    float s = __fadd_rn(a, b);
    float e = __fsub_rn(b, __fsub_rn(s, a));
    return {s, e};
}
__device__ __forceinline__ df df_add(df a, df b) {
    df s = two_sum(a.hi, b.hi);
    df t = two_sum(a.lo, b.lo);
    float e = __fadd_rn(s.lo, t.hi);
    s = quick_two_sum(s.hi, e);
    e = __fadd_rn(s.lo, t.lo);
    return quick_two_sum(s.hi, e);
}
// Sum with an error of about 2^-44 relative to the larger operand (not to the
// result): used where the operands are O(1) partial sums or all terms are
// positive, so that no cancellation can magnify it.
__device__ __forceinline__ df df_add_fast(df a, df b) {
    const df s = two_sum(a.hi, b.hi);
    return quick_two_sum(s.hi, __fadd_rn(s.lo, __fadd_rn(a.lo, b.lo)));
}
__device__ __forceinline__ df df_neg(df a) { return {-a.hi, -a.lo}; }
// double-float plus a single float
__device__ __forceinline__ df df_addf(df a, float c) {
    const df s = two_sum(a.hi, c);
    return quick_two_sum(s.hi, __fadd_rn(s.lo, a.lo));
}
__device__ __forceinline__ df df_sub(df a, df b) { return df_add(a, df_neg(b)); }
__device__ __forceinline__ df df_mul(df a, df b) {
    float p = __fmul_rn(a.hi, b.hi);
    float e = __fmaf_rn(a.hi, b.hi, -p);
    e = __fmaf_rn(a.hi, b.lo, e);
    e = __fmaf_rn(a.lo, b.hi, e);
    return quick_two_sum(p, e);
}
__device__ __forceinline__ df df_mulf(df a, float b) {
    float p = __fmul_rn(a.hi, b);
    float e = __fmaf_rn(a.hi, b, -p);
    e = __fmaf_rn(a.lo, b, e);
    return quick_two_sum(p, e);
}
__device__ __forceinline__ df df_sqrt(df a) {
    if (!(a.hi > 0.0f)) return {0.0f, 0.0f};
    float s = __fsqrt_rn(a.hi);
    float p = __fmul_rn(s, s);
    float pe = __fmaf_rn(s, s, -p);
    float r = __fadd_rn(__fsub_rn(__fsub_rn(a.hi, p), pe), a.lo);
    float c = __fdiv_rn(r, __fmul_rn(2.0f, s));
    return quick_two_sum(s, c);
}
__device__ __forceinline__ df df_rcp(df a) {
    float y = __frcp_rn(a.hi);
    // e = 1 - a*y in double-float, then y + y*e
    df ay = df_mulf(a, y);
    df e = df_sub({1.0f, 0.0f}, ay);
    float corr = __fmul_rn(y, e.hi);
    return quick_two_sum(y, corr);
}

// Pivot of a Cholesky column in double-float: l = sqrt(d) and il = 1/l.  Newton-
// Raphson on 1/sqrt from the single-precision rsqrtf(d.hi) = r0 (2 ulp): with
// e = 1 - d r0^2 (|e| < 2^-21, formed from the exact square r0^2 and a double-
// float product), 1/sqrt(d) = r0 (1 - e)^(-1/2) = r0 (1 + e/2 + 3e^2/8 + O(e^3)),
// so il carries a relative error of about 2^-47 typically and 2^-44 at most (the
// roundings of e and of the correction); l = d il.  Requires d.hi > 0 normal.
__device__ __forceinline__ void df_pivot(df d, df &l, df &il) {
    const float r0 = rsqrtf(d.hi);
    const float p = __fmul_rn(r0, r0);
    const float pe = __fmaf_rn(r0, r0, -p);
    const df m = df_mul(d, df{p, pe});                            // 1 - e
    const float e = __fsub_rn(__fsub_rn(1.0f, m.hi), m.lo);        // 1 - m.hi is exact
    const float corr = __fmul_rn(r0, __fmul_rn(e, __fmaf_rn(0.375f, e, 0.5f)));
    il = quick_two_sum(r0, corr);
    l = df_mul(d, il);
}

// Dot-product accumulator: acc -= x*y with the product's rounding error kept;
// the low word is left unnormalised until the end (its error is relative to
// the operands, which are O(1) in the kernels).
struct dfacc {
    float hi, lo;
};
__device__ __forceinline__ void dfacc_sub_prod(dfacc &a, df x, df y) {
    float p = __fmul_rn(x.hi, y.hi);
    float e = __fmaf_rn(x.hi, y.hi, -p);
    e = __fmaf_rn(x.hi, y.lo, e);
    e = __fmaf_rn(x.lo, y.hi, e);
    df s = two_sum(a.hi, -p);
    a.hi = s.hi;
    a.lo = __fsub_rn(a.lo, __fsub_rn(e, s.lo));
}
__device__ __forceinline__ void dfacc_add_prod(dfacc &a, df x, df y) {
    float p = __fmul_rn(x.hi, y.hi);
    float e = __fmaf_rn(x.hi, y.hi, -p);
    e = __fmaf_rn(x.hi, y.lo, e);
    e = __fmaf_rn(x.lo, y.hi, e);
    df s = two_sum(a.hi, p);
    a.hi = s.hi;
    a.lo = __fadd_rn(a.lo, __fadd_rn(e, s.lo));
}
__device__ __forceinline__ df dfacc_val(dfacc a) { return two_sum(a.hi, a.lo); }

// Anchored double-float accumulator for sums of products whose partial sums are
// known to stay within |s| <= B.  The high word h holds C + (high part of the
// sum), C = 6 * 2^e with 2^e >= B, so every value h takes lies in [4, 8] * 2^e:
// adding a product to h rounds it onto that binade's fixed grid (2^(e-21)), the
// amount actually added, h_new - h_old, is exact (Sterbenz), and the rounding
// remainder x*y - (h_new - h_old) is at most half a grid step.  The remainders
// and the cross terms of the double-float operands collect in the low word l,
// whose size stays near the grid step.  A multiply-accumulate is 6 FP32
// instructions (a general double-float one is 12) with an absolute error of
// at most about 2^-46 2^e per step (typically 2^-49 2^e; 2^e <= 2B when the
// anchor is the smallest one above B).  The value is (h - C) + l, the first
// term exact.
struct anc {
    float h, l;
};
__device__ __forceinline__ anc anc_init(df a, float C) {
    anc r;
    r.h = __fadd_rn(C, a.hi);
    r.l = __fadd_rn(a.lo, __fsub_rn(a.hi, __fsub_rn(r.h, C)));  // a.hi minus what h took: exact
    return r;
}
// a -= x*y
__device__ __forceinline__ void anc_sub_prod(anc &a, df x, df y) {
    const float h0 = a.h;
    a.h = __fmaf_rn(-x.hi, y.hi, h0);
    float t = __fmaf_rn(-x.hi, y.hi, __fsub_rn(h0, a.h));  // remainder of the high product
    t = __fmaf_rn(-x.hi, y.lo, t);
    t = __fmaf_rn(-x.lo, y.hi, t);
    a.l = __fadd_rn(a.l, t);
}
// a += x*y
__device__ __forceinline__ void anc_add_prod(anc &a, df x, df y) {
    const float h0 = a.h;
    a.h = __fmaf_rn(x.hi, y.hi, h0);
    float t = __fmaf_rn(x.hi, y.hi, __fsub_rn(h0, a.h));
    t = __fmaf_rn(x.hi, y.lo, t);
    t = __fmaf_rn(x.lo, y.hi, t);
    a.l = __fadd_rn(a.l, t);
}
// a += h*h + 2*h*l + l*l, the square of the unnormalised pair (h, l)
__device__ __forceinline__ void anc_add_sq(anc &a, float h, float l) {
    const float h0 = a.h;
    a.h = __fmaf_rn(h, h, h0);
    float t = __fmaf_rn(h, h, __fsub_rn(h0, a.h));
    t = __fmaf_rn(l, __fmaf_rn(2.0f, h, l), t);
    a.l = __fadd_rn(a.l, t);
}
// Double-float split of x whose high word lies on the grid of [M, 2M) (M = 1.5 * 2^E,
// grid 2^(E-23)), for |x| <= 2^(E-1): differences of two such high words are exact
// in FP32, and the low word keeps x to about 2^(E-48).
__device__ __forceinline__ df df_on_grid(double x, float M) {
    const float h = __fsub_rn(__fadd_rn(__double2float_rn(x), M), M);
    return {h, __double2float_rn(x - (double)h)};
}
// Anchor for partial sums bounded by b >= 0: 6 * 2^e with 2^e > b (b finite).
__device__ __forceinline__ float anc_anchor(float b) {
    const unsigned ex = (__float_as_uint(b) >> 23) & 0xffu;  // b < 2^(ex - 126)
    return __uint_as_float((ex + 1u) << 23) * 6.0f;
}

// ---------------------------------------------------------------------------
// Precision policy: the same kernel source is instantiated for FP64 and for
// double-float.
// ---------------------------------------------------------------------------
template <class R>
struct Ops;

template <>
struct Ops<double> {
    using T = double;
    struct Acc {
        double v;
    };
    static __device__ __forceinline__ T from(double x) { return x; }
    static __device__ __forceinline__ double to(T x) { return x; }
    static __device__ __forceinline__ T zero() { return 0.0; }
    static __device__ __forceinline__ T add(T a, T b) { return a + b; }
    static __device__ __forceinline__ T add_fast(T a, T b) { return a + b; }
    static __device__ __forceinline__ T sub(T a, T b) { return a - b; }
    static __device__ __forceinline__ T mul(T a, T b) { return a * b; }
    static __device__ __forceinline__ T neg(T a) { return -a; }
    static __device__ __forceinline__ T sqrt_(T a) { return sqrt(a); }
    static __device__ __forceinline__ T rcp(T a) { return 1.0 / a; }
    // pivot l = sqrt(d) and 1/l from one reciprocal square root (rsqrt: 1 ulp)
    static __device__ __forceinline__ void pivot(T d, T &l, T &il) {
        il = rsqrt(d);
        l = d * il;
    }
    static __device__ __forceinline__ bool positive(T a) { return a > 0.0; }
    static __device__ __forceinline__ Acc acc(T x) { return {x}; }
    static __device__ __forceinline__ void sub_prod(Acc &a, T x, T y) { a.v = fma(-x, y, a.v); }
    static __device__ __forceinline__ void add_prod(Acc &a, T x, T y) { a.v = fma(x, y, a.v); }
    static __device__ __forceinline__ T val(Acc a) { return a.v; }
    static __device__ __forceinline__ T raw(Acc a) { return a.v; }
    static __device__ __forceinline__ T shfl(T v, int src) { return __shfl_sync(FULL, v, src); }
    static __device__ __forceinline__ T shfl_xor(T v, int m) { return __shfl_xor_sync(FULL, v, m); }
};

template <>
struct Ops<df> {
    using T = df;
    using Acc = dfacc;
    static __device__ __forceinline__ T from(double x) { return df_from(x); }
    static __device__ __forceinline__ double to(T x) { return df_to(x); }
    static __device__ __forceinline__ T zero() { return {0.0f, 0.0f}; }
    static __device__ __forceinline__ T add(T a, T b) { return df_add(a, b); }
    static __device__ __forceinline__ T add_fast(T a, T b) { return df_add_fast(a, b); }
    static __device__ __forceinline__ T sub(T a, T b) { return df_sub(a, b); }
    static __device__ __forceinline__ T mul(T a, T b) { return df_mul(a, b); }
    static __device__ __forceinline__ T neg(T a) { return df_neg(a); }
    static __device__ __forceinline__ T sqrt_(T a) { return df_sqrt(a); }
    static __device__ __forceinline__ T rcp(T a) { return df_rcp(a); }
    static __device__ __forceinline__ void pivot(T d, T &l, T &il) { df_pivot(d, l, il); }
    static __device__ __forceinline__ bool positive(T a) { return a.hi > 0.0f; }
    static __device__ __forceinline__ Acc acc(T x) { return {x.hi, x.lo}; }
    static __device__ __forceinline__ void sub_prod(Acc &a, T x, T y) { dfacc_sub_prod(a, x, y); }
    static __device__ __forceinline__ void add_prod(Acc &a, T x, T y) { dfacc_add_prod(a, x, y); }
    static __device__ __forceinline__ T val(Acc a) { return dfacc_val(a); }
    // the accumulator's two words as stored, unnormalised (acc() reads them back)
    static __device__ __forceinline__ T raw(Acc a) { return {a.hi, a.lo}; }
    static __device__ __forceinline__ T shfl(T v, int src) {
        return {__shfl_sync(FULL, v.hi, src), __shfl_sync(FULL, v.lo, src)};
    }
    static __device__ __forceinline__ T shfl_xor(T v, int m) {
        return {__shfl_xor_sync(FULL, v.hi, m), __shfl_xor_sync(FULL, v.lo, m)};
    }
};

// ---------------------------------------------------------------------------
// HEALPix RING geometry (integer-exact numerators, one rounding each).
// ---------------------------------------------------------------------------
struct Ring {
    double z, s;
    int64_t first;
    int n_in, nq;
    double f;  // phase offset: phi_j = (j + f) pi / (2 nq)
};

// inv3N = 1/(3 Nside), inv3N2 = 1/(3 Nside^2): multiplications replace the
// divisions of the ring formulas (positions then differ from the correctly
// rounded ones by at most a couple of ulps).
__device__ __forceinline__ Ring ring_of(int64_t N, int64_t i, double inv3N, double inv3N2) {
    Ring r;
    const double Nd = (double)N;
    if (i < N) {
        const double id = (double)i;
        r.z = 1.0 - id * id * inv3N2;
        r.s = id * sqrt(6.0 * Nd * Nd - id * id) * inv3N2;
        r.first = 2 * i * (i - 1);
        r.nq = (int)i;
        r.f = 0.5;
    } else if (i <= 3 * N) {
        const double id = (double)i;
        r.z = (4.0 * Nd - 2.0 * id) * inv3N;
        r.s = sqrt((2.0 * id - Nd) * (7.0 * Nd - 2.0 * id)) * inv3N;
        r.first = 2 * N * (N - 1) + 4 * N * (i - N);
        r.nq = (int)N;
        r.f = ((i + N) & 1) ? 0.0 : 0.5;
    } else {
        const int64_t ip = 4 * N - i;
        const double id = (double)ip;
        r.z = -(1.0 - id * id * inv3N2);
        r.s = id * sqrt(6.0 * Nd * Nd - id * id) * inv3N2;
        r.first = 12 * N * N - 2 * ip * (ip + 1);
        r.nq = (int)ip;
        r.f = 0.5;
    }
    r.n_in = 4 * r.nq;
    return r;
}
__device__ __forceinline__ Ring ring_of(int64_t N, int64_t i) {
    return ring_of(N, i, 1.0 / (3.0 * (double)N), 1.0 / (3.0 * (double)N * (double)N));
}

__device__ __forceinline__ int64_t cap_ring_of(int64_t p) {  // largest i with 2i(i-1) <= p
    int64_t i = (int64_t)(0.5 * (1.0 + sqrt(1.0 + 2.0 * (double)p)));
    while (i > 1 && 2 * i * (i - 1) > p) --i;
    while (2 * (i + 1) * i <= p) ++i;
    return i;
}

__device__ __forceinline__ void pix_ring(int64_t N, int64_t p, int64_t &ring, int64_t &j) {
    const int64_t ncap = 2 * N * (N - 1), npix = 12 * N * N;
    if (p < ncap) {
        ring = cap_ring_of(p);
        j = p - 2 * ring * (ring - 1);
    } else if (p < npix - ncap) {
        const int64_t q = p - ncap;
        ring = q / (4 * N) + N;
        j = q - (ring - N) * 4 * N;
    } else {
        const int64_t i = cap_ring_of(npix - 1 - p);
        ring = 4 * N - i;
        j = p - (npix - 2 * i * (i + 1));
    }
}

// last ring whose z is >= z (0 if none)
__device__ __forceinline__ int64_t ring_above(int64_t N, double z) {
    const double za = fabs(z);
    int64_t i;
    if (za <= 2.0 / 3.0) {
        i = (int64_t)floor((double)N * (2.0 - 1.5 * z));
    } else {
        const int64_t in = (int64_t)floor((double)N * sqrt(fmax(3.0 * (1.0 - za), 0.0)));
        i = (z > 0) ? in : 4 * N - 1 - in;
    }
    i = i < 0 ? 0 : (i > 4 * N - 1 ? 4 * N - 1 : i);
    for (int it = 0; it < 3; ++it) {
        if (i >= 1 && ring_of(N, i).z < z) --i;
        if (i + 1 <= 4 * N - 1 && ring_of(N, i + 1).z >= z) ++i;
    }
    return i;
}

// ---------------------------------------------------------------------------
// Launch description.
// ---------------------------------------------------------------------------
// Per-interval cubic coefficients in FP64: p(s) = f + s (m + s (c2 + s c3)).
struct alignas(32) Coef64 {
    double f, m, c2, c3;
};

struct TableDev {
    const Coef64 *c64;  // per interval: f_k, h g_k, c2, c3 (Horner in s)
    const float4 *c32;   // per interval, double-float: (f.hi, f.lo, m.hi, m.lo), (c2.hi, c2.lo, c3.hi, c3.lo)
    double t_max, inv_h;
    float inv_h_hi, inv_h_lo;  // inv_h as a double-float pair
    int n;
};

struct LensArgs {
    int64_t nside;
    int64_t first, count;
    const double *map;
    const double *defl;
    double *out, *var;
    uint8_t *status;
    int64_t *stencil;  // non-NULL: write the stencil and skip the solve
    TableDev tab;
    double xi0;
    double r2;  // squared search radius (chord^2)
    unsigned long long *counters;  // points, nugget, fallback, window, failed
    int force_fallback;            // discard double-float solves (testing aid)
    int64_t nside_tgt;             // > 0: targets are the pixel centres of this grid (no deflection)
    int rotate;                    // spin 2: return P in the frame at n instead of n'
    TableDev tabm;                 // spin 2: xi-/xi+(0) on the same grid (augmented estimator)
    // tile queue of a single-range launch: zero before the launch, warps take tiles by
    // atomicAdd (NULL: a static grid stride over the tiles)
    unsigned long long *queue;
};

// Tile-queue counters a plan keeps: each single-range launch takes the next one, so up
// to this many launches of one plan may be in flight at once.
constexpr int QUEUE_SLOTS = 64;

// Internal kernel mode of the augmented (widely linear) spin-2 estimator.
constexpr int SPIN2_AUG = 3;

// Launch shape chosen by the caller or the autotuner (0 = library default).
// Targets per warp tile (the displacement phase runs one target per lane).
constexpr int MAX_TILE_POINTS = 16;

struct LaunchCfg {
    int warps_per_block, blocks_per_sm, tile_points;
};

enum { CNT_POINTS = 0, CNT_NUGGET = 1, CNT_FALLBACK = 2, CNT_WINDOW = 3, CNT_FAILED = 4, CNT_N = 5 };

// Correlation-table grid and stencil search disc of a K-nearest plan (host).
// The disc has chord radius r = 1.25 sqrt(K/3)/Nside (a cap holding K pixels
// has radius sqrt(K/3)/Nside), so chords between stencil members are <= 2r and
// the table covers t = chord^2 in [0, t_max = 4 r^2]; the interval count is the
// smallest power of two >= 64 (<= 65536) whose cubic Hermite error bound
// h^4/384 max|f''''| stays below 1e-11 of xi(0), with max|f''''| bounded by
// sum_l |a_l| P_l''''(1) / (16 xi(0)), a_l = (2l+1)/(4 pi) |C_l| (+ |C_l^BB|
// when cl_bb is given); R_rings is the number of rings searched on each side.
struct TableGrid {
    double r, r2, t_max, h, inv_h;
    int n, R_rings;
};
TableGrid table_grid(int64_t nside, int K, int lmax, const double *cl, const double *cl_bb);

// Host-side launchers (lens_spin0.cu, lens_spin2.cu, xi_table.cu).
cudaError_t launch_lens(int spin, int K, int precision, const LensArgs &a, int R_rings, const LaunchCfg &cfg,
                        cudaStream_t st);
cudaError_t launch_xi_table(int spin, int lmax, const double *cl_dev, const double *clbb_dev, double t_max,
                            int n, double *f_out, double *g_out, double *fm_out, double *gm_out,
                            cudaStream_t st);
cudaError_t finish_table(double *f, double *g, int n, double h, double xi0, Coef64 *c64, float4 *c32,
                         cudaStream_t st);
int device_sm_count();
size_t device_smem_optin();

}  // namespace flints

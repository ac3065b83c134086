// Harmonic synthesis of a band-limited HEALPix map on the GPU: the unlensed
// input of the remap (Sec. 3.2 draws it from C_l and synthesises it; Table 2
// counts that transform in the total time).  Spin s = 0, 1, 2:
//
//   spin 0:  T(theta, phi) = sum_{l,m} a_lm sY_lm,
//   spin s:  P = -sum_{l,m} (E + iB)_lm sY_lm  (P = Q + iU for s = 2; for s = 1
//            with E_lm = sqrt(l(l+1)) phi_lm it is the gradient d_theta + i d_phi),
//
// with sY_lm(theta, phi) = (-1)^s N_l e^{i m phi} d^l_{m,-s}(theta),
// N_l = sqrt((2l+1)/(4 pi)) (Appendix A), and real E, B fields
// (a_{l,-m} = (-1)^m a_lm^*).  Per ring the sum over l gives coefficients
//
//   spin 0:  F_m = sum_l a_lm N_l d^l_{m,0}                       (m >= 0),
//   spin s:  P_m  = -(-1)^s sum_l (E + iB)_lm N_l d^l_{m,-s},
//            P_-m = -sum_l (E^* + iB^*)_lm N_l d^l_{m,s}            (m >= 1),
//
// and the ring values are the Fourier sums sum_m F_m e^{i m phi_j}, done by
// folding m modulo the ring length n and an inverse DFT of length n.  The
// 2 Nside + 1 equatorial rings (n = 4 Nside) share one batched cuFFT plan.
// The polar rings (n = 4i, i < Nside) use Bluestein's algorithm: with
// w_t = exp(i pi t^2 / n), x_j = sum_k H_k e^{2 pi i jk/n} = w_j (a * b)_j for
// a_k = H_k w_k and b_t = conj(w_t), a linear convolution done with FFTs of
// a power-of-two length M >= 2n - 1; the transforms of b are tabulated per
// ring size at plan time, and the rings of equal M share one batched plan, so
// a plan holds at most 14 cuFFT plans whatever Nside.
//
// The l-sums use the Wigner-d three-term recurrence in l at fixed (m, m'):
//   d^{l+1} = (A_l x - B_l) d^l - C_l d^{l-1},  A_l = (2l+1) l (l+1) / D_l,
//   B_l = (2l+1) m m' / D_l,  C_l = (l+1) sqrt((l^2-m^2)(l^2-m'^2)) / D_l,
//   D_l = l sqrt(((l+1)^2-m^2)((l+1)^2-m'^2)),  x = cos(theta),
// started at l0 = max(m, |m'|) from the closed form
//   d^l_{l,b} = (-1)^{l-b} sqrt((2l)! / ((l+b)!(l-b)!)) c^{l+b} s^{l-b},
//   d^l_{-l,b} = sqrt((2l)! / ((l+b)!(l-b)!)) c^{l-b} s^{l+b}   (c, s = cos, sin theta/2)
// with d^l_{m,m'} = d^l_{-m',-m} when |m'| > m.  The start is formed in
// base-2 logarithms and carried as v 2^E (E an integer, raised in steps of 256
// while |v| > 2^256), so columns whose start underflows (large m near the
// poles) still reach their oscillatory range.  One thread runs the columns of
// one (ring, m) pair for the northern ring and, through
//   d^l_{m,m'}(pi - theta) = (-1)^{l+m} d^l_{m,-m'}(theta),
// for its southern mirror as well.
#include <cuda_runtime.h>
#include <cufft.h>

#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <vector>

#include "common.cuh"
#include "flints.h"

namespace {

using flints::df;

constexpr int CHUNK = 256;  // l values staged per pass in shared memory
constexpr double PI_D = 3.14159265358979323846;

struct SynthRing {
    double x;          // cos(theta)
    double lc, ls;     // log2 cos(theta/2), log2 sin(theta/2)
    double phi0;       // azimuth of the first pixel / pi
    long long first;   // RING index of the first pixel
    long long off;     // equatorial ring: offset of its FFT input; polar ring: offset of its Bluestein slot
    long long fboff;   // polar ring: offset of the transformed chirp for its size
    int n;             // pixels in the ring
    int M;             // polar ring: Bluestein length (0: equatorial ring)
};

// w_t = exp(i pi t^2 / n), with t^2 reduced modulo 2n (exact in integers)
__device__ __forceinline__ double2 chirp(long long t, int n) {
    const long long q = (t * t) % (2LL * n);
    double sp, cp;
    sincospi((double)q / (double)n, &sp, &cp);
    return make_double2(cp, sp);
}

thread_local char g_msg[512] = "no error";

int sfail(int code, const char *fmt, ...) {
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(g_msg, sizeof g_msg, fmt, ap);
    va_end(ap);
    return code;
}

// log2 |d^l0_{m,m'}| (as lg) and sign of the starting value of a column
__device__ __forceinline__ double start_log2(int m, int mp, double lc, double ls, bool &neg) {
    const double inv_ln2 = 1.4426950408889634;
    int l, b, pc, ps;
    if (m >= abs(mp)) {  // first index +l = m, second b = m'
        l = m;
        b = mp;
        pc = l + b;
        ps = l - b;
        neg = ((l - b) & 1) != 0;
    } else if (mp < 0) {  // d_{m,m'} = d_{-m',-m}, first index -m' = +l
        l = -mp;
        b = -m;
        pc = l + b;
        ps = l - b;
        neg = ((l - b) & 1) != 0;
    } else {  // first index -m' = -l
        l = mp;
        b = -m;
        pc = l - b;
        ps = l + b;
        neg = false;
    }
    const double lf = 0.5 * (lgamma(2.0 * l + 1.0) - lgamma((double)(l + b) + 1.0) - lgamma((double)(l - b) + 1.0));
    return lf * inv_ln2 + pc * lc + ps * ls;
}

// One recurrence column carried as v 2^E.
struct Col {
    double v, prev, mult;
    int e;
    __device__ __forceinline__ void init(double lg, bool neg) {
        const double fl = floor(lg);
        e = (int)fl;
        v = exp2(lg - fl);
        if (neg) v = -v;
        prev = 0.0;
        mult = e < -1074 ? 0.0 : ldexp(1.0, e);
    }
    __device__ __forceinline__ void step(double a, double b, double c, double x) {
        const double nv = fma(fma(a, x, -b), v, -c * prev);
        prev = v;
        v = nv;
        if (fabs(v) > 1.157920892373162e77) {  // 2^256
            v *= 8.636168555094445e-78;
            prev *= 8.636168555094445e-78;
            e += 256;
            mult = e < -1074 ? 0.0 : ldexp(1.0, e);
        }
    }
    __device__ __forceinline__ double value() const { return v * mult; }
};

// F layout: spin 0: [ring][m], m = 0..lmax;  spin s: [ring][lmax + m], m = -lmax..lmax.
// Rings are 1..4N-1, stored at index ring-1.  Threads: x = northern ring (1..2N), y = m.
template <int S>
__global__ void __launch_bounds__(128) legendre_kernel(int lmax, int nside, const SynthRing *__restrict__ rings,
                                                       const double2 *__restrict__ alm, const double2 *__restrict__ blm,
                                                       double2 *__restrict__ F) {
    __shared__ double sA[CHUNK], sB[CHUNK], sC[CHUNK];
    __shared__ double2 sWp[CHUNK], sWm[CHUNK];
    const int m = blockIdx.y;
    const int ring = blockIdx.x * blockDim.x + threadIdx.x + 1;  // northern ring incl. the equator
    const int nnorth = 2 * nside;
    const bool active = ring <= nnorth;
    const int NM = S == 0 ? lmax + 1 : 2 * lmax + 1;
    const int l0 = m > S ? m : S;
    const double inv4pi = 1.0 / (4.0 * PI_D);
    SynthRing rg{};
    if (active) rg = rings[ring - 1];
    // columns: A = d_{m,-s}, B = d_{m,+s} (spin 0: A only)
    Col ca{}, cb{};
    if (active && l0 <= lmax) {
        bool neg;
        double lg = start_log2(m, -S, rg.lc, rg.ls, neg);
        ca.init(lg, neg);
        if (S > 0) {
            lg = start_log2(m, S, rg.lc, rg.ls, neg);
            cb.init(lg, neg);
        }
    }
    // accumulators by parity of l + m (e: even, o: odd); the parity is uniform
    // across the block (same l and m), so the branches below do not diverge
    double2 pAe{}, pAo{}, pBe{}, pBo{}, mAe{}, mAo{}, mBe{}, mBo{};
    for (int c0 = l0; c0 <= lmax; c0 += CHUNK) {
        const int c1 = min(c0 + CHUNK, lmax + 1);
        __syncthreads();
        for (int l = c0 + threadIdx.x; l < c1; l += blockDim.x) {
            const int k = l - c0;
            const double ld = (double)l, lp = ld + 1.0;
            const double md = (double)m, sd = (double)S;
            const double den = ld * sqrt((lp * lp - md * md) * (lp * lp - sd * sd));
            if (l == 0 || !(den > 0.0)) {  // l = m = s = 0: d^1 = x d^0
                sA[k] = 1.0;
                sB[k] = 0.0;
                sC[k] = 0.0;
            } else {
                sA[k] = (2.0 * ld + 1.0) * ld * lp / den;
                sB[k] = (2.0 * ld + 1.0) * md * sd / den;  // for m' = +s; m' = -s takes -sB
                sC[k] = lp * sqrt((ld * ld - md * md) * (ld * ld - sd * sd)) / den;
            }
            const double nl = sqrt((2.0 * ld + 1.0) * inv4pi);
            const double2 a = alm[(size_t)l * (lmax + 1) + m];
            if (S == 0) {
                sWp[k] = make_double2(a.x * nl, a.y * nl);
            } else {
                const double2 b = blm ? blm[(size_t)l * (lmax + 1) + m] : make_double2(0.0, 0.0);
                // (E + iB) N and (E^* + iB^*) N
                sWp[k] = make_double2((a.x - b.y) * nl, (a.y + b.x) * nl);
                sWm[k] = make_double2((a.x + b.y) * nl, (b.x - a.y) * nl);
            }
        }
        __syncthreads();
        if (active) {
            for (int l = c0; l < c1; ++l) {
                const int k = l - c0;
                const bool odd = ((l + m) & 1) != 0;
                const double da = ca.value();
                const double2 wp = sWp[k];
                double2 &pa = odd ? pAo : pAe;
                pa.x = fma(wp.x, da, pa.x);
                pa.y = fma(wp.y, da, pa.y);
                if (S > 0) {
                    const double db = cb.value();
                    const double2 wm = sWm[k];
                    double2 &pb = odd ? pBo : pBe;
                    double2 &ma = odd ? mAo : mAe;
                    double2 &mb = odd ? mBo : mBe;
                    pb.x = fma(wp.x, db, pb.x);
                    pb.y = fma(wp.y, db, pb.y);
                    ma.x = fma(wm.x, da, ma.x);
                    ma.y = fma(wm.y, da, ma.y);
                    mb.x = fma(wm.x, db, mb.x);
                    mb.y = fma(wm.y, db, mb.y);
                }
                if (l < lmax) {
                    ca.step(sA[k], -sB[k], sC[k], rg.x);
                    if (S > 0) cb.step(sA[k], sB[k], sC[k], rg.x);
                }
            }
        }
    }
    if (!active) return;
    const int south = 4 * nside - ring;  // mirror ring (== ring at the equator)
    double2 *Fn = F + (size_t)(ring - 1) * NM;
    double2 *Fs = F + (size_t)(south - 1) * NM;
    if (S == 0) {
        Fn[m] = make_double2(pAe.x + pAo.x, pAe.y + pAo.y);
        if (south != ring) Fs[m] = make_double2(pAe.x - pAo.x, pAe.y - pAo.y);
        return;
    }
    // P_m = -(-1)^s sum wp d_{m,-s}; south: d_{m,-s}(pi - t) = (-1)^{l+m} d_{m,s}(t)
    const double sg = (S & 1) ? 1.0 : -1.0;  // -(-1)^s
    Fn[lmax + m] = make_double2(sg * (pAe.x + pAo.x), sg * (pAe.y + pAo.y));
    if (south != ring) Fs[lmax + m] = make_double2(sg * (pBe.x - pBo.x), sg * (pBe.y - pBo.y));
    if (m > 0) {  // P_-m = -sum wm d_{m,s}; south: d_{m,s}(pi - t) = (-1)^{l+m} d_{m,-s}(t)
        Fn[lmax - m] = make_double2(-(mBe.x + mBo.x), -(mBe.y + mBo.y));
        if (south != ring) Fs[lmax - m] = make_double2(-(mAe.x - mAo.x), -(mAe.y - mAo.y));
    }
}

// Fold the coefficients of one ring modulo its length n, with the phase of the
// first pixel: H_k = sum_{m = k mod n} F_m e^{i m phi0}.  Spin 0 (real field,
// F_-m = F_m^*): k = 0..n/2 for a complex-to-real FFT; spin s: k = 0..n-1.
// Double-float form of the same recurrence on the FP32 pipe (the mixed
// precision of the synthesis): the column carried as v 2^E with v a double-
// float pair, rescaled by 2^-64 while |v| > 2^64 (FP32 exponent range);
// coefficients, weights and sums in double-float, the sums (F) written as
// FP64.  Relative accuracy about 1e-13 after 4096 steps.
struct ColDF {
    df v, prev;
    float mult;
    int e;
    __device__ __forceinline__ void init(double lg, bool neg) {
        const double fl = floor(lg);
        e = (int)fl;
        double vd = exp2(lg - fl);
        if (neg) vd = -vd;
        v = flints::df_from(vd);
        prev = df{0.0f, 0.0f};
        mult = e < -126 ? 0.0f : ldexpf(1.0f, e);
    }
    __device__ __forceinline__ void step(df a, df b, df c, df x) {
        const df t = flints::df_sub(flints::df_mul(a, x), b);
        const df nv = flints::df_sub(flints::df_mul(t, v), flints::df_mul(c, prev));
        prev = v;
        v = nv;
        if (fabsf(v.hi) > 1.8446744e19f) {  // 2^64
            const float k = 5.421011e-20f;  // 2^-64
            v = df{v.hi * k, v.lo * k};
            prev = df{prev.hi * k, prev.lo * k};
            e += 64;
            mult = e < -126 ? 0.0f : ldexpf(1.0f, e);
        }
    }
    __device__ __forceinline__ df value() const { return df{v.hi * mult, v.lo * mult}; }
};

template <int S>
__global__ void __launch_bounds__(128) legendre_df_kernel(int lmax, int nside, const SynthRing *__restrict__ rings,
                                                          const double2 *__restrict__ alm,
                                                          const double2 *__restrict__ blm, double2 *__restrict__ F) {
    __shared__ float2 sA[CHUNK], sB[CHUNK], sC[CHUNK];
    __shared__ float4 sWp[CHUNK], sWm[CHUNK];  // (re.hi, re.lo, im.hi, im.lo)
    const int m = blockIdx.y;
    const int ring = blockIdx.x * blockDim.x + threadIdx.x + 1;
    const int nnorth = 2 * nside;
    const bool active = ring <= nnorth;
    const int NM = S == 0 ? lmax + 1 : 2 * lmax + 1;
    const int l0 = m > S ? m : S;
    const double inv4pi = 1.0 / (4.0 * PI_D);
    SynthRing rg{};
    if (active) rg = rings[ring - 1];
    const df x = flints::df_from(rg.x);
    ColDF ca{}, cb{};
    if (active && l0 <= lmax) {
        bool neg;
        double lg = start_log2(m, -S, rg.lc, rg.ls, neg);
        ca.init(lg, neg);
        if (S > 0) {
            lg = start_log2(m, S, rg.lc, rg.ls, neg);
            cb.init(lg, neg);
        }
    }
    using Acc = flints::dfacc;
    struct CAcc {  // complex double-float sum
        Acc re, im;
    };
    CAcc pAe{}, pAo{}, pBe{}, pBo{}, mAe{}, mAo{}, mBe{}, mBo{};
    auto mac = [](CAcc &a, df wr, df wi, df d) {
        flints::dfacc_add_prod(a.re, wr, d);
        flints::dfacc_add_prod(a.im, wi, d);
    };
    auto f2 = [](double v) {
        const df d = flints::df_from(v);
        return make_float2(d.hi, d.lo);
    };
    for (int c0 = l0; c0 <= lmax; c0 += CHUNK) {
        const int c1 = min(c0 + CHUNK, lmax + 1);
        __syncthreads();
        for (int l = c0 + threadIdx.x; l < c1; l += blockDim.x) {
            const int k = l - c0;
            const double ld = (double)l, lp = ld + 1.0;
            const double md = (double)m, sd = (double)S;
            const double den = ld * sqrt((lp * lp - md * md) * (lp * lp - sd * sd));
            if (l == 0 || !(den > 0.0)) {
                sA[k] = f2(1.0);
                sB[k] = f2(0.0);
                sC[k] = f2(0.0);
            } else {
                sA[k] = f2((2.0 * ld + 1.0) * ld * lp / den);
                sB[k] = f2((2.0 * ld + 1.0) * md * sd / den);
                sC[k] = f2(lp * sqrt((ld * ld - md * md) * (ld * ld - sd * sd)) / den);
            }
            const double nl = sqrt((2.0 * ld + 1.0) * inv4pi);
            const double2 a = alm[(size_t)l * (lmax + 1) + m];
            double2 wp, wm = make_double2(0.0, 0.0);
            if (S == 0) {
                wp = make_double2(a.x * nl, a.y * nl);
            } else {
                const double2 b = blm ? blm[(size_t)l * (lmax + 1) + m] : make_double2(0.0, 0.0);
                wp = make_double2((a.x - b.y) * nl, (a.y + b.x) * nl);
                wm = make_double2((a.x + b.y) * nl, (b.x - a.y) * nl);
            }
            const float2 pr = f2(wp.x), pi = f2(wp.y), mr = f2(wm.x), mi = f2(wm.y);
            sWp[k] = make_float4(pr.x, pr.y, pi.x, pi.y);
            sWm[k] = make_float4(mr.x, mr.y, mi.x, mi.y);
        }
        __syncthreads();
        if (active) {
            for (int l = c0; l < c1; ++l) {
                const int k = l - c0;
                const bool odd = ((l + m) & 1) != 0;
                const df da = ca.value();
                const float4 wpf = sWp[k];
                const df wpr{wpf.x, wpf.y}, wpi{wpf.z, wpf.w};
                // the parity is uniform across the block: no divergence, no indexed registers
                if (odd) {
                    mac(pAo, wpr, wpi, da);
                } else {
                    mac(pAe, wpr, wpi, da);
                }
                if (S > 0) {
                    const df db = cb.value();
                    const float4 wmf = sWm[k];
                    const df wmr{wmf.x, wmf.y}, wmi{wmf.z, wmf.w};
                    if (odd) {
                        mac(pBo, wpr, wpi, db);
                        mac(mAo, wmr, wmi, da);
                        mac(mBo, wmr, wmi, db);
                    } else {
                        mac(pBe, wpr, wpi, db);
                        mac(mAe, wmr, wmi, da);
                        mac(mBe, wmr, wmi, db);
                    }
                }
                if (l < lmax) {
                    const float2 A = sA[k], B = sB[k], C = sC[k];
                    const df Ad{A.x, A.y}, Bd{B.x, B.y}, Cd{C.x, C.y};
                    ca.step(Ad, flints::df_neg(Bd), Cd, x);
                    if (S > 0) cb.step(Ad, Bd, Cd, x);
                }
            }
        }
    }
    if (!active) return;
    auto val = [](const Acc &acc) { return flints::df_to(flints::dfacc_val(acc)); };
    auto sum = [&](const CAcc &e_, const CAcc &o_, double sg_o, double sg) {
        return make_double2(sg * (val(e_.re) + sg_o * val(o_.re)), sg * (val(e_.im) + sg_o * val(o_.im)));
    };
    const int south = 4 * nside - ring;
    double2 *Fn = F + (size_t)(ring - 1) * NM;
    double2 *Fs = F + (size_t)(south - 1) * NM;
    if (S == 0) {
        Fn[m] = sum(pAe, pAo, 1.0, 1.0);
        if (south != ring) Fs[m] = sum(pAe, pAo, -1.0, 1.0);
        return;
    }
    const double sg = (S & 1) ? 1.0 : -1.0;  // -(-1)^s
    Fn[lmax + m] = sum(pAe, pAo, 1.0, sg);
    if (south != ring) Fs[lmax + m] = sum(pBe, pBo, -1.0, sg);
    if (m > 0) {
        Fn[lmax - m] = sum(mBe, mBo, 1.0, -1.0);
        if (south != ring) Fs[lmax - m] = sum(mAe, mAo, -1.0, -1.0);
    }
}

// Polar rings (rg.M > 0) write a_k = H_k w_k, k < n, zero-padded to M, into
// their Bluestein slot in A; equatorial rings write H into H.
template <int S>
__global__ void fold_kernel(int lmax, const SynthRing *__restrict__ rings, const double2 *__restrict__ F,
                            double2 *__restrict__ H, double2 *__restrict__ A) {
    const int r = blockIdx.x;  // ring index - 1
    const SynthRing rg = rings[r];
    const int n = rg.n;
    const int NM = S == 0 ? lmax + 1 : 2 * lmax + 1;
    const double2 *Fr = F + (size_t)r * NM;
    const bool polar = rg.M > 0;
    double2 *Hr = polar ? A + rg.off : H + rg.off;
    if (polar)
        for (int k = n + threadIdx.x; k < rg.M; k += blockDim.x) Hr[k] = make_double2(0.0, 0.0);
    const int nk = (S == 0 && !polar) ? n / 2 + 1 : n;
    for (int k = threadIdx.x; k < nk; k += blockDim.x) {
        double hr = 0.0, hi = 0.0;
        if (S == 0) {
            for (int m = k; m <= lmax; m += n) {  // m >= 0, m = k mod n
                double sp, cp;
                sincospi((double)m * rg.phi0, &sp, &cp);
                const double2 f = Fr[m];
                hr += f.x * cp - f.y * sp;
                hi += f.x * sp + f.y * cp;
            }
            for (int m = (k == 0 ? n : n - k); m <= lmax; m += n) {  // m >= 1, -m = k mod n: conj
                double sp, cp;
                sincospi((double)m * rg.phi0, &sp, &cp);
                const double2 f = Fr[m];
                hr += f.x * cp - f.y * sp;
                hi -= f.x * sp + f.y * cp;
            }
        } else {
            // m = k + j n within [-lmax, lmax]
            int m = k - ((k + lmax) / n) * n;
            for (; m <= lmax; m += n) {
                double sp, cp;
                sincospi((double)m * rg.phi0, &sp, &cp);
                const double2 f = Fr[lmax + m];
                hr += f.x * cp - f.y * sp;
                hi += f.x * sp + f.y * cp;
            }
        }
        if (polar) {
            const double2 w = chirp(k, n);
            Hr[k] = make_double2(hr * w.x - hi * w.y, hr * w.y + hi * w.x);
        } else {
            Hr[k] = make_double2(hr, hi);
        }
    }
}

// Bluestein middle step: the transformed slot times the transformed chirp, / M.
__global__ void chirp_mul_kernel(const SynthRing *__restrict__ rings, const int *__restrict__ polar,
                                 const double2 *__restrict__ FB, double2 *__restrict__ A) {
    const SynthRing rg = rings[polar[blockIdx.x]];
    const double inv = 1.0 / (double)rg.M;
    double2 *a = A + rg.off;
    const double2 *b = FB + rg.fboff;
    for (int k = threadIdx.x; k < rg.M; k += blockDim.x) {
        const double2 x = a[k], y = b[k];
        a[k] = make_double2((x.x * y.x - x.y * y.y) * inv, (x.x * y.y + x.y * y.x) * inv);
    }
}

// Bluestein last step: x_j = w_j c_j, written to the ring's pixels.
template <int S>
__global__ void chirp_out_kernel(const SynthRing *__restrict__ rings, const int *__restrict__ polar,
                                 const double2 *__restrict__ A, double *__restrict__ map) {
    const SynthRing rg = rings[polar[blockIdx.x]];
    const double2 *a = A + rg.off;
    for (int j = threadIdx.x; j < rg.n; j += blockDim.x) {
        const double2 w = chirp(j, rg.n), c = a[j];
        const double xr = w.x * c.x - w.y * c.y, xi = w.x * c.y + w.y * c.x;
        if (S == 0) {
            map[rg.first + j] = xr;
        } else {
            reinterpret_cast<double2 *>(map)[rg.first + j] = make_double2(xr, xi);
        }
    }
}

// Chirp b_t = conj(w_t) for |t| < n in a length-M cyclic buffer (one block per ring size).
__global__ void chirp_fill_kernel(const int *__restrict__ sizes_n, const int *__restrict__ sizes_M,
                                  const long long *__restrict__ sizes_off, double2 *__restrict__ FB) {
    const int n = sizes_n[blockIdx.x], M = sizes_M[blockIdx.x];
    double2 *b = FB + sizes_off[blockIdx.x];
    for (int t = threadIdx.x; t < M; t += blockDim.x) {
        double2 v = make_double2(0.0, 0.0);
        if (t < n) {
            const double2 w = chirp(t, n);
            v = make_double2(w.x, -w.y);
        } else if (t > M - n) {
            const double2 w = chirp(M - t, n);
            v = make_double2(w.x, -w.y);
        }
        b[t] = v;
    }
}

}  // namespace

struct flints_synth_s {
    int device;
    int64_t nside;
    int lmax, spin, precision;
    SynthRing *d_rings;
    int *d_polar;      // indices of the polar rings
    double2 *d_F, *d_H, *d_A, *d_FB;
    void *d_work;
    std::vector<SynthRing> rings;
    int npolar;
    cufftHandle belt;                 // equatorial rings, batched
    std::vector<cufftHandle> groups;  // polar rings: one C2C plan per Bluestein length M
    std::vector<long long> group_off; // first slot of each group in A
    bool belt_made;
};

static void synth_release(flints_synth_s *s) {
    if (s->belt_made) cufftDestroy(s->belt);
    for (cufftHandle h : s->groups) cufftDestroy(h);
    cudaFree(s->d_rings);
    cudaFree(s->d_polar);
    cudaFree(s->d_F);
    cudaFree(s->d_H);
    cudaFree(s->d_A);
    cudaFree(s->d_FB);
    cudaFree(s->d_work);
}

static int synth_bail(flints_synth_s *s, int code, const char *what, cudaError_t e = cudaSuccess) {
    synth_release(s);
    delete s;
    if (e != cudaSuccess) return sfail(code, "flints_synth_plan: %s: %s", what, cudaGetErrorString(e));
    return sfail(code, "flints_synth_plan: %s", what);
}

extern "C" {

const char *flints_synth_last_error(void) { return g_msg; }

int flints_synth_plan(flints_synth_t *out, int64_t nside, int lmax, int spin, int precision, void *stream) {
    if (!out) return sfail(FLINTS_EINVAL, "flints_synth_plan: out is NULL");
    *out = nullptr;
    if (nside < 1 || nside > 8192) return sfail(FLINTS_EINVAL, "flints_synth_plan: nside outside [1, 8192]");
    if (spin != 0 && spin != 1 && spin != 2) return sfail(FLINTS_EINVAL, "flints_synth_plan: spin must be 0, 1 or 2");
    if (lmax < spin || lmax > 16384) return sfail(FLINTS_EINVAL, "flints_synth_plan: lmax outside [spin, 16384]");
    if (precision != FLINTS_FP64 && precision != FLINTS_MIXED)
        return sfail(FLINTS_EINVAL, "flints_synth_plan: precision must be FLINTS_FP64 or FLINTS_MIXED");
    const int64_t N = nside;
    const int nr = (int)(4 * N - 1);
    flints_synth_s *s = new flints_synth_s();
    cudaGetDevice(&s->device);
    s->nside = nside;
    s->lmax = lmax;
    s->spin = spin;
    s->precision = precision;
    s->d_rings = nullptr;
    s->d_polar = nullptr;
    s->d_F = s->d_H = s->d_A = s->d_FB = nullptr;
    s->d_work = nullptr;
    s->belt_made = false;
    // ring geometry (host, FP64)
    s->rings.resize(nr);
    for (int i = 1; i <= nr; ++i) {
        SynthRing rg{};
        double z, f;
        int nq;
        long long first;
        if (i < N) {
            nq = i;
            z = 1.0 - (double)i * i / (3.0 * N * N);
            first = 2LL * i * (i - 1);
            f = 0.5;
        } else if (i <= 3 * N) {
            nq = (int)N;
            z = (4.0 * N - 2.0 * i) / (3.0 * N);
            first = 2LL * N * (N - 1) + 4LL * N * (i - N);
            f = ((i + N) & 1) ? 0.0 : 0.5;
        } else {
            const int ip = (int)(4 * N - i);
            nq = ip;
            z = -(1.0 - (double)ip * ip / (3.0 * N * N));
            first = 12LL * N * N - 2LL * ip * (ip + 1);
            f = 0.5;
        }
        const double th = acos(z);
        rg.x = z;
        rg.lc = log2(cos(0.5 * th));
        rg.ls = log2(sin(0.5 * th));
        rg.phi0 = f / (2.0 * nq);
        rg.first = first;
        rg.n = 4 * nq;
        s->rings[i - 1] = rg;
    }
    // equatorial FFT inputs, contiguous in ring order
    const long long nkb = spin == 0 ? 2 * N + 1 : 4 * N;  // per equatorial ring
    for (int i = (int)N; i <= 3 * N; ++i) s->rings[i - 1].off = (long long)(i - N) * nkb;
    const long long hsize = (2 * N + 1) * nkb;
    // polar rings: Bluestein length M = next power of two >= 2n - 1, slots grouped by M
    std::vector<int> polar, sz_n, sz_M;
    std::vector<long long> sz_off;
    std::vector<int> group_M;
    std::vector<int> group_batch;
    long long aoff = 0, fboff = 0;
    for (int i = 1; i < N; ++i) {
        const int n = 4 * i;
        int M = 1;
        while (M < 2 * n - 1) M <<= 1;
        if (group_M.empty() || group_M.back() != M) {
            group_M.push_back(M);
            group_batch.push_back(0);
            s->group_off.push_back(aoff);
        }
        sz_n.push_back(n);
        sz_M.push_back(M);
        sz_off.push_back(fboff);
        for (int r : {i, (int)(4 * N - i)}) {
            SynthRing &rg = s->rings[r - 1];
            rg.M = M;
            rg.off = aoff;
            rg.fboff = fboff;
            aoff += M;
            polar.push_back(r - 1);
            group_batch.back() += 1;
        }
        fboff += M;
    }
    s->npolar = (int)polar.size();
    const size_t NM = spin == 0 ? (size_t)lmax + 1 : 2 * (size_t)lmax + 1;
    cudaError_t e;
    if ((e = cudaMalloc(&s->d_rings, sizeof(SynthRing) * nr)) != cudaSuccess ||
        (e = cudaMalloc(&s->d_F, sizeof(double2) * NM * nr)) != cudaSuccess ||
        (e = cudaMalloc(&s->d_H, sizeof(double2) * (size_t)hsize)) != cudaSuccess)
        return synth_bail(s, e == cudaErrorMemoryAllocation ? FLINTS_ENOMEM : FLINTS_ECUDA, "allocation", e);
    if (s->npolar > 0 &&
        ((e = cudaMalloc(&s->d_polar, sizeof(int) * polar.size())) != cudaSuccess ||
         (e = cudaMalloc(&s->d_A, sizeof(double2) * (size_t)aoff)) != cudaSuccess ||
         (e = cudaMalloc(&s->d_FB, sizeof(double2) * (size_t)fboff)) != cudaSuccess))
        return synth_bail(s, e == cudaErrorMemoryAllocation ? FLINTS_ENOMEM : FLINTS_ECUDA, "allocation", e);
    cudaStream_t st = (cudaStream_t)stream;
    if ((e = cudaMemcpyAsync(s->d_rings, s->rings.data(), sizeof(SynthRing) * nr, cudaMemcpyHostToDevice, st)) !=
        cudaSuccess)
        return synth_bail(s, FLINTS_ECUDA, "copy", e);
    if (s->npolar > 0 && (e = cudaMemcpyAsync(s->d_polar, polar.data(), sizeof(int) * polar.size(),
                                              cudaMemcpyHostToDevice, st)) != cudaSuccess)
        return synth_bail(s, FLINTS_ECUDA, "copy", e);
    // cuFFT plans sharing one work area
    size_t work_max = 0;
    auto make = [&](cufftHandle &h, int n, long long idist, long long odist, cufftType type, int batch) -> bool {
        if (cufftCreate(&h) != CUFFT_SUCCESS) return false;
        cufftSetAutoAllocation(h, 0);
        int nn[1] = {n}, inembed[1] = {(int)idist}, onembed[1] = {(int)odist};
        size_t ws = 0;
        if (cufftMakePlanMany(h, 1, nn, inembed, 1, (int)idist, onembed, 1, (int)odist, type, batch, &ws) !=
            CUFFT_SUCCESS) {
            cufftDestroy(h);
            return false;
        }
        if (ws > work_max) work_max = ws;
        return true;
    };
    if (!make(s->belt, (int)(4 * N), nkb, 4 * N, spin == 0 ? CUFFT_Z2D : CUFFT_Z2Z, (int)(2 * N + 1)))
        return synth_bail(s, FLINTS_ECUDA, "cuFFT plan creation failed");
    s->belt_made = true;
    for (size_t g = 0; g < group_M.size(); ++g) {
        cufftHandle h;
        if (!make(h, group_M[g], group_M[g], group_M[g], CUFFT_Z2Z, group_batch[g]))
            return synth_bail(s, FLINTS_ECUDA, "cuFFT plan creation failed");
        s->groups.push_back(h);
    }
    if (work_max && (e = cudaMalloc(&s->d_work, work_max)) != cudaSuccess)
        return synth_bail(s, FLINTS_ENOMEM, "FFT work area", e);
    cufftSetWorkArea(s->belt, s->d_work);
    for (cufftHandle h : s->groups) cufftSetWorkArea(h, s->d_work);
    // transformed chirps, one per polar ring size
    if (s->npolar > 0) {
        int *d_n = nullptr, *d_M = nullptr;
        long long *d_off = nullptr;
        const size_t ns = sz_n.size();
        if ((e = cudaMalloc(&d_n, sizeof(int) * ns)) != cudaSuccess ||
            (e = cudaMalloc(&d_M, sizeof(int) * ns)) != cudaSuccess ||
            (e = cudaMalloc(&d_off, sizeof(long long) * ns)) != cudaSuccess) {
            cudaFree(d_n);
            cudaFree(d_M);
            return synth_bail(s, FLINTS_ENOMEM, "chirp tables", e);
        }
        cudaMemcpyAsync(d_n, sz_n.data(), sizeof(int) * ns, cudaMemcpyHostToDevice, st);
        cudaMemcpyAsync(d_M, sz_M.data(), sizeof(int) * ns, cudaMemcpyHostToDevice, st);
        cudaMemcpyAsync(d_off, sz_off.data(), sizeof(long long) * ns, cudaMemcpyHostToDevice, st);
        chirp_fill_kernel<<<(unsigned)ns, 256, 0, st>>>(d_n, d_M, d_off, s->d_FB);
        e = cudaGetLastError();
        // forward transforms of the chirps, group by group (one per ring size in a group)
        for (size_t g = 0; e == cudaSuccess && g < group_M.size(); ++g) {
            size_t k0 = 0;
            while (k0 < ns && sz_M[k0] != group_M[g]) ++k0;
            size_t k1 = k0;
            while (k1 < ns && sz_M[k1] == group_M[g]) ++k1;
            cufftHandle h;
            if (!make(h, group_M[g], group_M[g], group_M[g], CUFFT_Z2Z, (int)(k1 - k0))) {
                e = cudaErrorUnknown;
                break;
            }
            void *tmp = nullptr;
            size_t ws = 0;
            cufftGetSize(h, &ws);
            if (ws && cudaMalloc(&tmp, ws) != cudaSuccess) {
                cufftDestroy(h);
                e = cudaErrorMemoryAllocation;
                break;
            }
            cufftSetWorkArea(h, tmp);
            cufftSetStream(h, st);
            cufftDoubleComplex *p = reinterpret_cast<cufftDoubleComplex *>(s->d_FB + sz_off[k0]);
            if (cufftExecZ2Z(h, p, p, CUFFT_FORWARD) != CUFFT_SUCCESS) e = cudaErrorUnknown;
            cudaStreamSynchronize(st);
            cufftDestroy(h);
            cudaFree(tmp);
        }
        cudaStreamSynchronize(st);
        cudaFree(d_n);
        cudaFree(d_M);
        cudaFree(d_off);
        if (e != cudaSuccess) return synth_bail(s, FLINTS_ECUDA, "chirp transforms", e);
    }
    if ((e = cudaStreamSynchronize(st)) != cudaSuccess) return synth_bail(s, FLINTS_ECUDA, "set-up", e);
    *out = s;
    return FLINTS_OK;
}

int flints_synthesize(flints_synth_t s, const double *alm, const double *blm, double *map, void *stream) {
    if (!s) return sfail(FLINTS_EINVAL, "flints_synthesize: plan is NULL");
    if (!alm || !map) return sfail(FLINTS_EINVAL, "flints_synthesize: alm and map must not be NULL");
    if (((uintptr_t)alm | (uintptr_t)map | (uintptr_t)blm) & 15u)
        return sfail(FLINTS_EINVAL, "flints_synthesize: alm, blm and map must be 16-byte aligned");
    int cur = -1;
    cudaGetDevice(&cur);
    if (cur != s->device) return sfail(FLINTS_EINVAL, "flints_synthesize: plan made on another device");
    cudaStream_t st = (cudaStream_t)stream;
    const int N = (int)s->nside, lmax = s->lmax;
    const dim3 grid((2 * N + 127) / 128, lmax + 1);
    const double2 *a = reinterpret_cast<const double2 *>(alm);
    const double2 *b = s->spin == 0 ? nullptr : reinterpret_cast<const double2 *>(blm);
    const int nr = 4 * N - 1;
    const bool mixed = s->precision == FLINTS_MIXED;
    switch (s->spin) {
        case 0:
            if (mixed)
                legendre_df_kernel<0><<<grid, 128, 0, st>>>(lmax, N, s->d_rings, a, b, s->d_F);
            else
                legendre_kernel<0><<<grid, 128, 0, st>>>(lmax, N, s->d_rings, a, b, s->d_F);
            fold_kernel<0><<<nr, 256, 0, st>>>(lmax, s->d_rings, s->d_F, s->d_H, s->d_A);
            break;
        case 1:
            if (mixed)
                legendre_df_kernel<1><<<grid, 128, 0, st>>>(lmax, N, s->d_rings, a, b, s->d_F);
            else
                legendre_kernel<1><<<grid, 128, 0, st>>>(lmax, N, s->d_rings, a, b, s->d_F);
            fold_kernel<1><<<nr, 256, 0, st>>>(lmax, s->d_rings, s->d_F, s->d_H, s->d_A);
            break;
        default:
            if (mixed)
                legendre_df_kernel<2><<<grid, 128, 0, st>>>(lmax, N, s->d_rings, a, b, s->d_F);
            else
                legendre_kernel<2><<<grid, 128, 0, st>>>(lmax, N, s->d_rings, a, b, s->d_F);
            fold_kernel<2><<<nr, 256, 0, st>>>(lmax, s->d_rings, s->d_F, s->d_H, s->d_A);
            break;
    }
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return sfail(FLINTS_ECUDA, "flints_synthesize: kernel launch: %s", cudaGetErrorString(e));
    // equatorial rings: one batched inverse transform straight into the map
    if (cufftSetStream(s->belt, st) != CUFFT_SUCCESS) return sfail(FLINTS_ECUDA, "flints_synthesize: cufftSetStream");
    {
        const SynthRing &r0 = s->rings[N - 1];
        cufftDoubleComplex *in = reinterpret_cast<cufftDoubleComplex *>(s->d_H);
        cufftResult fr = s->spin == 0
                             ? cufftExecZ2D(s->belt, in, reinterpret_cast<cufftDoubleReal *>(map + r0.first))
                             : cufftExecZ2Z(s->belt, in, reinterpret_cast<cufftDoubleComplex *>(map) + r0.first,
                                            CUFFT_INVERSE);
        if (fr != CUFFT_SUCCESS) return sfail(FLINTS_ECUDA, "flints_synthesize: cuFFT execution failed (%d)", (int)fr);
    }
    if (s->npolar == 0) return FLINTS_OK;
    // polar rings: Bluestein convolution
    for (size_t g = 0; g < s->groups.size(); ++g) {
        cufftSetStream(s->groups[g], st);
        cufftDoubleComplex *p = reinterpret_cast<cufftDoubleComplex *>(s->d_A + s->group_off[g]);
        if (cufftExecZ2Z(s->groups[g], p, p, CUFFT_FORWARD) != CUFFT_SUCCESS)
            return sfail(FLINTS_ECUDA, "flints_synthesize: cuFFT execution failed");
    }
    chirp_mul_kernel<<<s->npolar, 256, 0, st>>>(s->d_rings, s->d_polar, s->d_FB, s->d_A);
    for (size_t g = 0; g < s->groups.size(); ++g) {
        cufftDoubleComplex *p = reinterpret_cast<cufftDoubleComplex *>(s->d_A + s->group_off[g]);
        if (cufftExecZ2Z(s->groups[g], p, p, CUFFT_INVERSE) != CUFFT_SUCCESS)
            return sfail(FLINTS_ECUDA, "flints_synthesize: cuFFT execution failed");
    }
    if (s->spin == 0)
        chirp_out_kernel<0><<<s->npolar, 256, 0, st>>>(s->d_rings, s->d_polar, s->d_A, map);
    else
        chirp_out_kernel<1><<<s->npolar, 256, 0, st>>>(s->d_rings, s->d_polar, s->d_A, map);
    e = cudaGetLastError();
    if (e != cudaSuccess) return sfail(FLINTS_ECUDA, "flints_synthesize: kernel launch: %s", cudaGetErrorString(e));
    return FLINTS_OK;
}

void flints_synth_free(flints_synth_t s) {
    if (!s) return;
    int cur = 0;
    cudaGetDevice(&cur);
    if (cur != s->device) cudaSetDevice(s->device);
    synth_release(s);
    if (cur != s->device) cudaSetDevice(cur);
    delete s;
}

}  // extern "C"

// xi tabulation (Sec. 2.5 step 2; Appendix B, last paragraph): values and
// t-derivatives of the correlation function on the grid t_k = k h, in FP64,
// one thread per node, summed over l by three-term recurrences.
//
// Spin 0 (Eq. correlation_func): xi = sum_l (2l+1)/(4 pi) C_l P_l(x),
// x = cos b = 1 - u, u = t/2.  With D_l = P_l - P_{l-1} the Legendre
// recurrence (l+1) P_{l+1} = (2l+1) x P_l - l P_{l-1} becomes
//     D_{l+1} = (l D_l - (2l+1) u P_l) / (l+1),   P_{l+1} = P_l + D_{l+1},
// which forms P_l near x = 1 without cancellation.  P'_{l+1} = P'_{l-1} + (2l+1) P_l.
//
// Spin s = 1, 2 (Eq. spins_correl): xi+ = sum_l (2l+1)/(4 pi) (C^E + C^B) d^l_{ss},
// xi- = sum_l (2l+1)/(4 pi) (C^E - C^B) d^l_{s,-s}, from the Wigner-d
// recurrence in l at fixed (m, m') = (s, +-s):
//     d_{l+1} = a_l (b_l x - m m') d_l - e_l d_{l-1},
//     a_l = (2l+1) / (l((l+1)^2-s^2)),  b_l = l(l+1),  e_l = (l+1)(l^2-s^2) / (l((l+1)^2-s^2)),
// started at l = s from d^s_{ss} = ((1+x)/2)^s and d^s_{s,-s} = ((1-x)/2)^s
// (e_s = 0, so no l = s-1 term is needed).  Because d^l_{ss}(1) = 1 for all l,
// a_l (b_l - s^2) - e_l = 1 and the increments obey
//     D_{l+1} = e_l D_l - a_l b_l u d_l,
// the same cancellation-free form as for spin 0.  x-derivatives follow by
// differentiating the recurrence; d/dt = -1/2 d/dx.
#include "common.cuh"

namespace flints {

__global__ void xi_table_kernel(int spin, int lmax, const double *__restrict__ cl,
                                const double *__restrict__ clbb, double h, int n, double *f, double *g,
                                double *fm, double *gm) {
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k > n) return;
    const double t = (double)k * h;
    const double u = 0.5 * t;
    const double inv4pi = 1.0 / (4.0 * PI);
    if (spin == 0) {
        double acc = cl[0] * inv4pi, dacc = 0.0;
        if (lmax >= 1) {
            double P = 1.0 - u, D = -u, dPm = 0.0, dP = 1.0;
            const double a1 = 3.0 * inv4pi * cl[1];
            acc += a1 * P;
            dacc += a1 * dP;
            for (int l = 1; l < lmax; ++l) {
                const double ld = (double)l;
                const double Dn = (ld * D - (2.0 * ld + 1.0) * u * P) / (ld + 1.0);
                const double Pn = P + Dn;
                const double dPn = dPm + (2.0 * ld + 1.0) * P;
                const double a = (2.0 * ld + 3.0) * inv4pi * cl[l + 1];
                acc += a * Pn;
                dacc += a * dPn;
                P = Pn;
                D = Dn;
                dPm = dP;
                dP = dPn;
            }
        }
        f[k] = acc;
        g[k] = -0.5 * dacc;
        return;
    }
    // spin s = 1 or 2
    const int sp_ = spin == 1 ? 1 : 2;
    const double s2 = (double)(sp_ * sp_);
    double sp = 0.0, dsp = 0.0, sm = 0.0, dsm = 0.0;
    if (lmax >= sp_) {
        const double x = 1.0 - u;
        // ((1+x)/2)^s, ((1-x)/2)^s = (u/2)^s and their x-derivatives
        const double hp = 1.0 - 0.5 * u, hm = 0.5 * u;
        double d = sp_ == 1 ? hp : hp * hp, D = 0.0, dd = sp_ == 1 ? 0.5 : hp, ddm = 0.0;
        double e2 = sp_ == 1 ? hm : hm * hm, de2 = sp_ == 1 ? -0.5 : -hm, e2m = 0.0, de2m = 0.0;
        for (int l = sp_; l <= lmax; ++l) {
            const double ld = (double)l;
            const double bb = clbb ? clbb[l] : 0.0;
            const double wp = (2.0 * ld + 1.0) * inv4pi * (cl[l] + bb);
            const double wm = (2.0 * ld + 1.0) * inv4pi * (cl[l] - bb);
            sp += wp * d;
            dsp += wp * dd;
            sm += wm * e2;
            dsm += wm * de2;
            if (l == lmax) break;
            const double lp = ld + 1.0;
            const double den = ld * (lp * lp - s2);
            const double al = (2.0 * ld + 1.0) / den;
            const double bl = ld * lp;
            const double el = lp * (ld * ld - s2) / den;
            // d^l_{ss}
            const double Dn = el * D - al * bl * u * d;
            const double dn = d + Dn;
            const double ddn = al * (bl * x - s2) * dd + al * bl * d - el * ddm;
            // d^l_{s,-s}
            const double e2n = al * (bl * x + s2) * e2 - el * e2m;
            const double de2n = al * (bl * x + s2) * de2 + al * bl * e2 - el * de2m;
            D = Dn;
            ddm = dd;
            d = dn;
            dd = ddn;
            e2m = e2;
            de2m = de2;
            e2 = e2n;
            de2 = de2n;
        }
    }
    f[k] = sp;
    g[k] = -0.5 * dsp;
    fm[k] = sm;
    gm[k] = -0.5 * dsm;
}

// Normalise by xi(0) = f[0] and form per-interval cubic coefficients in the
// local variable s = t/h - k:  p(s) = f_k + m0 s + c2 s^2 + c3 s^3 with
// m0 = h g_k, m1 = h g_{k+1}, D = f_{k+1} - f_k, c2 = 3D - 2 m0 - m1,
// c3 = m0 + m1 - 2D (the cubic Hermite interpolant of values and slopes).
__global__ void table_coeffs_kernel(double *f, double *g, int n, double h, double xi0, Coef64 *c64,
                                    float4 *c32) {
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= n) return;
    const double inv = 1.0 / xi0;
    const double f0 = f[k] * inv, f1 = f[k + 1] * inv;
    const double m0 = h * g[k] * inv, m1 = h * g[k + 1] * inv;
    const double dlt = f1 - f0;
    const double c2 = 3.0 * dlt - 2.0 * m0 - m1;
    const double c3 = m0 + m1 - 2.0 * dlt;
    c64[k] = Coef64{f0, m0, c2, c3};
    const df a = df_from(f0), b = df_from(m0), c = df_from(c2), d = df_from(c3);
    c32[2 * k] = make_float4(a.hi, a.lo, b.hi, b.lo);
    c32[2 * k + 1] = make_float4(c.hi, c.lo, d.hi, d.lo);
}

__global__ void normalise_kernel(double *f, double *g, int n, double xi0) {
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k > n) return;
    f[k] /= xi0;
    g[k] /= xi0;
}

cudaError_t launch_xi_table(int spin, int lmax, const double *cl_dev, const double *clbb_dev, double t_max,
                            int n, double *f_out, double *g_out, double *fm_out, double *gm_out,
                            cudaStream_t st) {
    const double h = t_max / n;
    const int threads = 128, blocks = (n + 1 + threads - 1) / threads;
    xi_table_kernel<<<blocks, threads, 0, st>>>(spin, lmax, cl_dev, clbb_dev, h, n, f_out, g_out, fm_out,
                                                gm_out);
    return cudaGetLastError();
}

// Normalise the raw node sums of one table (xi or xi-) by xi0, and (for the
// table used by the lens kernels) write the interval coefficients.
cudaError_t finish_table(double *f, double *g, int n, double h, double xi0, Coef64 *c64, float4 *c32,
                         cudaStream_t st) {
    const int threads = 128;
    if (c64) {
        table_coeffs_kernel<<<(n + threads - 1) / threads, threads, 0, st>>>(f, g, n, h, xi0, c64, c32);
        cudaError_t e = cudaGetLastError();
        if (e != cudaSuccess) return e;
    }
    normalise_kernel<<<(n + 1 + threads - 1) / threads, threads, 0, st>>>(f, g, n, xi0);
    return cudaGetLastError();
}

}  // namespace flints

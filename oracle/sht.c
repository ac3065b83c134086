/* Spherical-harmonic synthesis at arbitrary colatitudes: CPU oracle (test
 * infrastructure, FP64).  Only the tests, the smoke check and the CPU-baseline
 * leg of the benchmark load this library; the CUDA path never does.
 *
 * The exact benchmark of the paper (Sec. 3.2: sum the spherical harmonics at
 * the displaced positions) and the synthesis of test maps both reduce to the
 * per-colatitude coefficients
 *
 *     F_m(theta) = sum_{l >= max(|m|,|s|)} a_lm N_l d^l_{m,-s}(theta),
 *     N_l = sqrt((2l+1)/(4 pi)),
 *
 * because sY_lm(theta, phi) = (-1)^s N_l e^{i m phi} d^l_{m,-s}(theta)
 * (Appendix A); the caller then sums F_m e^{i m phi} over m.
 *
 * d^l_{m,m'} is computed by the three-term recurrence in l at fixed (m, m'):
 *   l sqrt(((l+1)^2-m^2)((l+1)^2-m'^2)) d^{l+1}
 *     = (2l+1)(l(l+1) x - m m') d^l - (l+1) sqrt((l^2-m^2)(l^2-m'^2)) d^{l-1},
 * x = cos(theta), started at l0 = max(|m|,|m'|) from the closed form
 *   d^l_{l,m'}  = (-1)^{l-m'} sqrt((2l)!/((l+m')!(l-m')!)) c^{l+m'} s^{l-m'},
 *   d^l_{-l,m'} = sqrt((2l)!/((l+m')!(l-m')!)) c^{l-m'} s^{l+m'},
 *   d^l_{m,-l}  = d^l_{l,-m},
 * with c = cos(theta/2), s = sin(theta/2).  The starting value is formed in
 * logarithms and carried as v * 2^S, so that columns whose start underflows
 * (large m) still reach their oscillatory range accurately.
 *
 * The colatitude derivative used for gradients (spin 0 only) follows from
 *   sin(theta) d/dtheta d^l_{m0} = l x d^l_{m0} - sqrt(l^2 - m^2) d^{l-1}_{m0}.
 */
#include <math.h>
#include <stdlib.h>
#include <string.h>

#define LOG2E 1.4426950408889634
#define RESCALE_AT 1.157920892373162e77 /* 2^256 */
#define RESCALE_BY 8.636168555094445e-78 /* 2^-256 */

static double log_start(int l, int mp, double lc, double ls, int first_plus, int *neg)
{
    /* log |d^l_{+-l, m'}| and its sign; first_plus selects the first index +l. */
    double lg = 0.5 * (lgamma(2.0 * l + 1.0) - lgamma((double)l + mp + 1.0) - lgamma((double)l - mp + 1.0));
    if (first_plus) {
        *neg = ((l - mp) % 2 + 2) % 2;
        return lg + (l + mp) * lc + (l - mp) * ls;
    }
    *neg = 0;
    return lg + (l - mp) * lc + (l + mp) * ls;
}

/* Column of d^l_{m, mp}(theta) for l = l0..lmax accumulated against weights.
 * acc_re/acc_im receive sum_l w_l d^l (w complex, given per l);
 * if dacc != NULL (mp == 0 only), dacc receives sum_l w_l d/dtheta(d^l)*N_l-free. */
static void column(int lmax, int m, int mp, double theta,
                   const double *A, const double *B, const double *C,
                   const double *w_re, const double *w_im,
                   double *acc_re, double *acc_im, double *dacc_re, double *dacc_im)
{
    int l0 = abs(m) > abs(mp) ? abs(m) : abs(mp);
    double x = cos(theta), st = sin(theta);
    double lc = log(cos(0.5 * theta)), ls = log(sin(0.5 * theta));
    int neg = 0;
    double lg;
    if (abs(m) >= abs(mp)) {
        lg = log_start(l0, mp, lc, ls, m >= 0, &neg);
    } else {
        /* |mp| = l0 > |m|: d^l_{m,mp} = d^l_{-mp,-m}; first index -mp = +-l0 */
        lg = log_start(l0, -m, lc, ls, -mp >= 0, &neg);
    }
    double r = 0, i_ = 0, dr = 0, di = 0;
    if (!isfinite(lg)) { /* theta at a pole: start is exactly 0 unless the exponent vanishes */
        lg = -INFINITY;
    }
    int S = 0;
    double v;
    if (lg == -INFINITY) {
        v = 0.0;
    } else {
        double e2 = lg * LOG2E;
        S = (int)floor(e2);
        v = exp2(e2 - S);
        if (neg) v = -v;
    }
    double vprev = 0.0;
    double mult = ldexp(1.0, S);
    for (int l = l0; l <= lmax; ++l) {
        if (l > l0) {
            double vn = A[l - 1] * (x * v) - B[l - 1] * v - C[l - 1] * vprev;
            vprev = v;
            v = vn;
            if (fabs(v) > RESCALE_AT) {
                v *= RESCALE_BY;
                vprev *= RESCALE_BY;
                S += 256;
                mult = ldexp(1.0, S);
            }
        }
        double d = v * mult;
        r += w_re[l] * d;
        i_ += w_im[l] * d;
        if (dacc_re) {
            double dprev = (l > l0) ? vprev * mult : 0.0;
            double dd = (l * x * d - sqrt((double)l * l - (double)m * m) * dprev) / st;
            dr += w_re[l] * dd;
            di += w_im[l] * dd;
        }
    }
    *acc_re = r;
    *acc_im = i_;
    if (dacc_re) { *dacc_re = dr; *dacc_im = di; }
}

static void coefs(int lmax, int m, int mp, double *A, double *B, double *C)
{
    /* d^{l+1} = (A_l x - B_l) d^l - C_l d^{l-1} for l >= max(|m|,|mp|,1) */
    for (int l = 0; l < lmax; ++l) {
        double lp = l + 1.0;
        double den = l * sqrt((lp * lp - (double)m * m) * (lp * lp - (double)mp * mp));
        if (l == 0 || den == 0.0) { /* only reached from l0 = 0 (m = mp = 0): d^1 = x d^0 */
            A[l] = (l == 0) ? 1.0 : 0.0;
            B[l] = 0.0;
            C[l] = 0.0;
            continue;
        }
        A[l] = (2.0 * l + 1.0) * l * lp / den;
        B[l] = (2.0 * l + 1.0) * (double)m * mp / den;
        C[l] = lp * sqrt(((double)l * l - (double)m * m) * ((double)l * l - (double)mp * mp)) / den;
    }
}

/* Per-colatitude coefficients.
 *
 * mode 0: spin 0 values.    out[p][0][m] = F_m (m = 0..lmax)
 * mode 1: spin 0 gradient.  out[p][0][m] = F_m, out[p][1][m] = dF_m/dtheta
 * mode 2: spin 2 (P = -sum (aE + i aB) 2Y_lm over all m).
 *         out[p][0][m] = F+_m = sum_l a_{l,m}  N_l d^l_{m,-2},
 *         out[p][1][m] = F-_m = sum_l a_{l,-m} N_l d^l_{-m,-2},
 *         with a_{l,m} = -(E_lm + i B_lm) and E_{l,-m} = (-1)^m conj(E_lm).
 *
 * alm arrays are (lmax+1)^2 doubles indexed [l*(lmax+1)+m], m >= 0.
 * out_re/out_im are npts*2*(lmax+1) doubles indexed [(p*2+k)*(lmax+1)+m].
 */
void oracle_theta_coeffs(int lmax, int mode,
                         const double *e_re, const double *e_im,
                         const double *b_re, const double *b_im,
                         long npts, const double *theta,
                         double *out_re, double *out_im)
{
    int L1 = lmax + 1;
    memset(out_re, 0, sizeof(double) * npts * 2 * L1);
    memset(out_im, 0, sizeof(double) * npts * 2 * L1);
    int mp = (mode == 2) ? -2 : 0;
    int nsides = (mode == 2) ? 2 : 1;
    /* few directions: parallel over m; many: parallel over directions */
    int over_m = npts < 256;
    long nm = (long)nsides * L1;
#pragma omp parallel if (over_m)
    {
        double *A = malloc(sizeof(double) * L1), *B = malloc(sizeof(double) * L1), *C = malloc(sizeof(double) * L1);
        double *wr = malloc(sizeof(double) * L1), *wi = malloc(sizeof(double) * L1);
#pragma omp for schedule(dynamic, 4)
        for (long it = 0; it < nm; ++it) {
            int side = (int)(it / L1), m0 = (int)(it % L1);
            int m = side ? -m0 : m0;
            if (side && m0 == 0) continue;
            coefs(lmax, m, mp, A, B, C);
            for (int l = 0; l <= lmax; ++l) {
                double nl = sqrt((2.0 * l + 1.0) / (4.0 * M_PI));
                double ar = 0, ai = 0;
                if (l >= m0) {
                    ar = e_re[l * L1 + m0];
                    ai = e_im[l * L1 + m0];
                    if (mode == 2) {
                        double br = b_re ? b_re[l * L1 + m0] : 0.0, bi = b_im ? b_im[l * L1 + m0] : 0.0;
                        if (side) { /* E_{l,-m} = (-1)^m conj(E_lm), likewise B */
                            double sg = (m0 % 2) ? -1.0 : 1.0;
                            ar = sg * ar; ai = -sg * ai; br = sg * br; bi = -sg * bi;
                        }
                        /* a = -(E + i B) */
                        double tr = -(ar - bi), ti = -(ai + br);
                        ar = tr; ai = ti;
                    }
                }
                wr[l] = ar * nl;
                wi[l] = ai * nl;
            }
#pragma omp parallel for schedule(static) if (!over_m)
            for (long p = 0; p < npts; ++p) {
                double r, i_, dr = 0, di = 0;
                column(lmax, m, mp, theta[p], A, B, C, wr, wi, &r, &i_,
                       mode == 1 ? &dr : NULL, mode == 1 ? &di : NULL);
                long o0 = (p * 2 + side) * L1 + m0;
                out_re[o0] = r;
                out_im[o0] = i_;
                if (mode == 1) {
                    long o1 = (p * 2 + 1) * L1 + m0;
                    out_re[o1] = dr;
                    out_im[o1] = di;
                }
            }
        }
        free(A); free(B); free(C); free(wr); free(wi);
    }
}

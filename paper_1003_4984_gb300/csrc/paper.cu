// The paper's own estimator route (Secs. 2.3-2.5): the pixel-centred stencil of
// 9 * 4^(y-1) pixels with the inverse covariance tabulated once per symmetry
// class of central pixels, so that each target costs two triangular
// matrix-vector products instead of a K x K Cholesky factorisation.
//
// The tabulated matrix is L^-1, the factor of S^-1 = L^-T L^-1 (L the Cholesky
// factor of S + n I): the estimate c^T S^-1 y = (L^-1 c) . (L^-1 y) and its
// variance xi(0) (1 - |L^-1 c|^2) then carry the rounding of a triangular
// solve, not that of an explicit inverse (which loses a factor cond(S) ~ 1e8),
// in half the memory of S^-1.
//
// Plan (once per Nside, y and spectrum):
//   1. xi table on [0, t_max], t_max = min((7 / Nc)^2, 4) (every chord between
//      stencil members and from a target to them is below 7 / Nc);
//   2. stencil_kernel: one thread per coarse pixel c (Nc = Nside / 2^(y-1))
//      writes its members (ordering rule of paper_geom.cuh) and its slot;
//   3. linv_kernel: one block per slot: S = xi(chord^2)/xi(0) over the slot
//      representative's members, nugget rule of Sec. 2.4, right-looking
//      Cholesky in shared memory, L^-1 column by column, stored packed by
//      columns (column j, rows j .. K-1, contiguous: coalesced lane loads).
// Per call (apply_kernel): one warp per tile of 32 targets.  Lane l displaces
// target l and locates its coarse pixel (RING ang2pix at Nc); then per target
// (three at a time in groups of 10 lanes for K = 9, one at a time for K = 36)
// the lanes own stencil members l (and l + 32): c_l = xi(|n' - x_l|^2)/xi(0),
// y_l = map[x_l]; lane i accumulates row i of z_c = L^-1 c and z_y = L^-1 y
// (c_j, y_j broadcast by shuffles); value = z_c . z_y and variance
// xi(0) (1 - z_c . z_c), the kriging estimate and its error (Eqs.
// best_temperature_field, gaussvar).
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>

#include "flints.h"
#include "lens.cuh"
#include "paper_geom.cuh"

namespace flints {
namespace paper {

constexpr int SINV_THREADS = 64;

// offset of column j of a K x K lower-triangular matrix packed by columns
__host__ __device__ constexpr int col_start(int K, int j) { return j * K - j * (j - 1) / 2; }

// L^-1 storage per class.  K = 9: packed by columns.  K = 36: the lane-step
// layout that the K = 36 kernel reads with one coalesced load per step: rows
// 0..31 in LS_STEPS steps of 32 lanes, lanes 2p and 2p + 1 sharing rows p and
// 31 - p (the pair's 33 entries in order: row p, columns 0..p, then row
// 31 - p, columns 0..31-p; lane 2p takes positions 0..16, lane 2p + 1
// positions 17..32, position 33 a zero pad), then LS_TAIL steps for rows
// 32..35 (lane l: row 32 + (l & 3), column (l >> 2) + 8t; zero above the
// diagonal).
constexpr int LS_STEPS = 17, LS_TAIL = 5;
__host__ __device__ constexpr int linv_len(int K) { return K == 36 ? (LS_STEPS + LS_TAIL) * 32 : K * (K + 1) / 2; }
// (row, column) of entry e of a K = 36 lane-step block; false for a zero pad
__host__ __device__ inline bool lanestep_entry(int e, int &row, int &col) {
    if (e < LS_STEPS * 32) {
        const int u = e >> 5, L = e & 31, p = L >> 1;
        const int t = (L & 1) ? LS_STEPS + u : u;
        if (t <= p) {
            row = p;
            col = t;
            return true;
        }
        row = 31 - p;
        col = t - p - 1;
        return col <= row;
    }
    const int f = e - LS_STEPS * 32, t = f >> 5, L = f & 31;
    row = 32 + (L & 3);
    col = (L >> 2) + 8 * t;
    return col <= row;
}
constexpr int LDS = STENCIL_MAX + 1;  // padded shared-memory row stride

// unit vector of RING pixel p at Nside N
__device__ __forceinline__ void pix2vec(int64_t N, int64_t p, double &x, double &y, double &z) {
    int64_t i, j;
    pix_ring(N, p, i, j);
    const Ring rg = ring_of(N, i);
    double sp, cp;
    sincospi(((double)j + rg.f) / (2.0 * (double)rg.nq), &sp, &cp);
    x = rg.s * cp;
    y = rg.s * sp;
    z = rg.z;
}

// unit vectors of all pixels of the map grid, (x, y, z, 0) per pixel: built once
// per plan so that the per-target kernel gathers member positions instead of
// recomputing them (FP64 sin/cos/sqrt are scarce on this part)
__global__ void pixvec_kernel(int64_t N, double2 *pv) {
    const int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= 12 * N * N) return;
    double x, y, z;
    pix2vec(N, p, x, y, z);
    pv[2 * p] = make_double2(x, y);
    pv[2 * p + 1] = make_double2(z, 0.0);
}

__device__ __forceinline__ void member_vec(const double2 *pv, int64_t m, double &x, double &y, double &z) {
    const double2 a = __ldg(pv + 2 * m), b = __ldg(pv + 2 * m + 1);
    x = a.x;
    y = a.y;
    z = b.x;
}

// RING pixel at Nside N containing the unit vector (x, y, z) (the ring scheme's
// point location of Gorski et al. 2005: belt by the two edge-line families,
// caps by the distance to the pole, sin(theta) taken from x, y near the poles)
__device__ __forceinline__ int64_t ang2pix(int64_t N, double x, double y, double z) {
    const double Nd = (double)N;
    double phi = atan2(y, x);
    if (phi < 0.0) phi += 2.0 * PI;
    double tt = phi * (2.0 / PI);  // [0, 4)
    if (tt >= 4.0) tt -= 4.0;
    const double za = fabs(z);
    if (za <= 2.0 / 3.0) {
        const double t1 = Nd * (0.5 + tt), t2 = Nd * z * 0.75;
        const int64_t jp = (int64_t)floor(t1 - t2), jm = (int64_t)floor(t1 + t2);
        int64_t ir = N + 1 + jp - jm;  // 1 .. 2N+1, from z = 2/3
        ir = ir < 1 ? 1 : (ir > 2 * N + 1 ? 2 * N + 1 : ir);  // rounding at |z| = 2/3
        const int64_t kshift = 1 - (ir & 1);
        int64_t ip = (jp + jm - N + kshift + 1) / 2;
        ip = pmod(ip, 4 * N);
        return 2 * N * (N - 1) + (ir - 1) * 4 * N + ip;
    }
    const double tp = tt - floor(tt);
    const double st = sqrt(x * x + y * y);
    const double tmp = Nd * st * sqrt(3.0 / (1.0 + za));  // N sqrt(3 (1 - |z|))
    int64_t jp = (int64_t)(tp * tmp), jm = (int64_t)((1.0 - tp) * tmp);
    jp = jp < 0 ? 0 : (jp > N - 1 ? N - 1 : jp);
    jm = jm < 0 ? 0 : (jm > N - 1 - jp ? N - 1 - jp : jm);
    const int64_t ir = jp + jm + 1;  // ring counted from the nearer pole
    int64_t ip = (int64_t)(tt * (double)ir);
    ip = pmod(ip, 4 * ir);
    return z > 0.0 ? 2 * ir * (ir - 1) + ip : 12 * N * N - 2 * ir * (ir + 1) + ip;
}

// ---------------------------------------------------------------- plan kernels
__global__ void stencil_kernel(int64_t Nc, int k, int K, int32_t *members, int32_t *slot, int *bad) {
    const int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= 12 * Nc * Nc) return;
    int32_t mem[STENCIL_MAX];
    const int n = stencil_members(Nc, k, c, mem);
    int32_t *dst = members + c * K;
    if (n < 0 || n > K) {
        atomicAdd(bad, 1);
        for (int m = 0; m < K; ++m) dst[m] = -1;
    } else {
        for (int m = 0; m < K; ++m) dst[m] = m < n ? mem[m] : -1;
    }
    int64_t i, j;
    ring_and_pos(Nc, c, i, j);
    slot[c] = (int32_t)slot_of(Nc, i, j);
}

struct LinvArgs {
    int64_t Nc, N, nslot;
    int K;
    const int32_t *members;
    TableDev tab;
    double *linv;                  // [nslot][K (K + 1) / 2], L^-1 packed by columns
    int *slot_steps;               // [nslot]: nugget doublings, -1 = no factor found
    unsigned long long *max_t;     // bits of the largest member-pair chord^2
    int *counts;                   // [0]: slots with a raised nugget, [1]: failed slots
};

__global__ void __launch_bounds__(SINV_THREADS) linv_kernel(LinvArgs a) {
    __shared__ double S[STENCIL_MAX * LDS], Li[STENCIL_MAX * LDS];
    __shared__ double px[STENCIL_MAX], py[STENCIL_MAX], pz[STENCIL_MAX];
    __shared__ int n_sh, bad;
    const int tid = threadIdx.x, nt = blockDim.x, K = a.K;
    for (int64_t sl = blockIdx.x; sl < a.nslot; sl += gridDim.x) {
        const int64_t rep = slot_rep(a.Nc, sl);
        const int32_t *mem = a.members + rep * K;
        if (tid == 0) {
            int n = 0;
            while (n < K && mem[n] >= 0) ++n;
            n_sh = n;
        }
        __syncthreads();
        const int n = n_sh;
        for (int m = tid; m < n; m += nt) pix2vec(a.N, mem[m], px[m], py[m], pz[m]);
        __syncthreads();
        double tmax = 0.0;
        double nug = NUGGET_EPS;
        int steps = 0;
        bool ok = false;
        for (; steps <= MAX_NUGGET_STEPS; ++steps) {
            for (int e = tid; e < n * n; e += nt) {
                const int i = e / n, j = e - (e / n) * n;
                if (j > i) continue;
                if (i == j) {
                    S[i * LDS + j] = 1.0 + nug;
                } else {
                    const double dx = px[i] - px[j], dy = py[i] - py[j], dz = pz[i] - pz[j];
                    const double t = dx * dx + dy * dy + dz * dz;
                    tmax = fmax(tmax, t);
                    S[i * LDS + j] = table_eval<double>(a.tab, t);
                }
            }
            if (tid == 0) bad = 0;
            __syncthreads();
            // right-looking Cholesky of the lower triangle, in place
            for (int kk = 0; kk < n; ++kk) {
                if (tid == 0) {
                    const double d = S[kk * LDS + kk];
                    if (d > 0.0) S[kk * LDS + kk] = sqrt(d); else bad = 1;
                }
                __syncthreads();
                if (bad) break;
                const double lkk = S[kk * LDS + kk];
                for (int i = kk + 1 + tid; i < n; i += nt) S[i * LDS + kk] /= lkk;
                __syncthreads();
                const int w = n - kk - 1;
                for (int e = tid; e < w * w; e += nt) {
                    const int i = kk + 1 + e / w, j = kk + 1 + (e - (e / w) * w);
                    if (j <= i) S[i * LDS + j] -= S[i * LDS + kk] * S[j * LDS + kk];
                }
                __syncthreads();
            }
            if (!bad) {
                ok = true;
                break;
            }
            nug *= 2.0;
            __syncthreads();
        }
        // L^-1, one column per thread: L x = e_col by forward substitution
        if (ok) {
            for (int col = tid; col < n; col += nt) {
                for (int i = 0; i < col; ++i) Li[i * LDS + col] = 0.0;
                for (int i = col; i < n; ++i) {
                    double acc = i == col ? 1.0 : 0.0;
                    for (int m = col; m < i; ++m) acc = fma(-S[i * LDS + m], Li[m * LDS + col], acc);
                    Li[i * LDS + col] = acc / S[i * LDS + i];
                }
            }
        }
        __syncthreads();
        // L^-1 in the class's storage layout; zero outside the n x n block
        double *dst = a.linv + sl * (int64_t)linv_len(K);
        if (K == 36) {
            for (int e = tid; e < linv_len(36); e += nt) {
                int i, j;
                const bool v = lanestep_entry(e, i, j);
                dst[e] = (ok && v && i < n && j < n) ? Li[i * LDS + j] : 0.0;
            }
        } else {
            for (int j = 0; j < K; ++j) {
                for (int i = j + tid; i < K; i += nt)
                    dst[col_start(K, j) + i - j] = (ok && i < n && j < n) ? Li[i * LDS + j] : 0.0;
            }
        }
        // the largest pair chord (block reduction through atomics on the bit pattern)
        if (tmax > 0.0) atomicMax(a.max_t, (unsigned long long)__double_as_longlong(tmax));
        if (tid == 0) {
            a.slot_steps[sl] = ok ? steps : -1;
            if (!ok) atomicAdd(a.counts + 1, 1);
            else if (steps > 0) atomicAdd(a.counts, 1);
        }
        __syncthreads();
    }
}

// ------------------------------------------------- spin 1 and 2 fields
// Pixel table of spin-s plans: (cos phi, sin phi), (z, sin theta) per pixel:
// x = s cos phi, y = s sin phi as in pix2vec, plus the local frame.
__device__ __forceinline__ void pix_frame(int64_t N, int64_t p, double &c, double &sn, double &z, double &s) {
    int64_t i, j;
    pix_ring(N, p, i, j);
    const Ring rg = ring_of(N, i);
    sincospi(((double)j + rg.f) / (2.0 * (double)rg.nq), &sn, &c);
    z = rg.z;
    s = rg.s;
}

__global__ void pixframe_kernel(int64_t N, double2 *pv) {
    const int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= 12 * N * N) return;
    double c, sn, z, s;
    pix_frame(N, p, c, sn, z, s);
    pv[2 * p] = make_double2(c, sn);
    pv[2 * p + 1] = make_double2(z, s);
}

// Spin-S class blocks: C_ij = xi+(t_ij)/xi+(0) exp(iS(a_ij - a_ji - pi)) over
// the representative's members (unit diagonal, Eqs. v_spins, spins_correl; the
// pi, from frames referred to the direction of travel, matters for odd S), the
// nugget rule of Sec. 2.4, a Hermitian right-looking Cholesky C + n I = L L^H
// in shared memory, L^-1 column by column; written as complex entries in the
// class's storage layout (as the spin-0 blocks).
template <int S>
__global__ void __launch_bounds__(SINV_THREADS) linv_kernel_c(LinvArgs a, double2 *linvc) {
    __shared__ double Sr[STENCIL_MAX * LDS], Si[STENCIL_MAX * LDS], Lr[STENCIL_MAX * LDS], Lim[STENCIL_MAX * LDS];
    __shared__ double px[STENCIL_MAX], py[STENCIL_MAX], pz[STENCIL_MAX], ps[STENCIL_MAX], pc[STENCIL_MAX],
        psn[STENCIL_MAX];
    __shared__ int n_sh, bad;
    const int tid = threadIdx.x, nt = blockDim.x, K = a.K;
    for (int64_t sl = blockIdx.x; sl < a.nslot; sl += gridDim.x) {
        const int64_t rep = slot_rep(a.Nc, sl);
        const int32_t *mem = a.members + rep * K;
        if (tid == 0) {
            int n = 0;
            while (n < K && mem[n] >= 0) ++n;
            n_sh = n;
        }
        __syncthreads();
        const int n = n_sh;
        for (int m = tid; m < n; m += nt) {
            pix_frame(a.N, mem[m], pc[m], psn[m], pz[m], ps[m]);
            px[m] = ps[m] * pc[m];
            py[m] = ps[m] * psn[m];
        }
        __syncthreads();
        double tmax = 0.0;
        double nug = NUGGET_EPS;
        int steps = 0;
        bool ok = false;
        for (; steps <= MAX_NUGGET_STEPS; ++steps) {
            for (int e = tid; e < n * n; e += nt) {
                const int i = e / n, j = e - (e / n) * n;
                if (j > i) continue;
                if (i == j) {
                    Sr[i * LDS + j] = 1.0 + nug;
                    Si[i * LDS + j] = 0.0;
                } else {
                    const double dx = px[j] - px[i], dy = py[j] - py[i], dz = pz[j] - pz[i];
                    const double t = dx * dx + dy * dy + dz * dz;
                    tmax = fmax(tmax, t);
                    const double f = table_eval<double>(a.tab, t);
                    const Cx<double> ph = pair_phase<double, S>(dx, dy, dz, pz[i], ps[i], pc[i], psn[i], pz[j], ps[j],
                                                                pc[j], psn[j]);
                    Sr[i * LDS + j] = f * ph.re;
                    Si[i * LDS + j] = f * ph.im;
                }
            }
            if (tid == 0) bad = 0;
            __syncthreads();
            for (int kk = 0; kk < n; ++kk) {
                if (tid == 0) {
                    const double d = Sr[kk * LDS + kk];
                    if (d > 0.0) Sr[kk * LDS + kk] = sqrt(d); else bad = 1;
                }
                __syncthreads();
                if (bad) break;
                const double lkk = Sr[kk * LDS + kk];
                for (int i = kk + 1 + tid; i < n; i += nt) {
                    Sr[i * LDS + kk] /= lkk;
                    Si[i * LDS + kk] /= lkk;
                }
                __syncthreads();
                const int w = n - kk - 1;
                for (int e = tid; e < w * w; e += nt) {
                    const int i = kk + 1 + e / w, j = kk + 1 + (e - (e / w) * w);
                    if (j <= i) {  // A_ij -= L_ik conj(L_jk)
                        const double ar = Sr[i * LDS + kk], ai = Si[i * LDS + kk];
                        const double br = Sr[j * LDS + kk], bi = Si[j * LDS + kk];
                        Sr[i * LDS + j] -= ar * br + ai * bi;
                        Si[i * LDS + j] -= ai * br - ar * bi;
                    }
                }
                __syncthreads();
            }
            if (!bad) {
                ok = true;
                break;
            }
            nug *= 2.0;
            __syncthreads();
        }
        if (ok) {  // L^-1 by columns: X_cc = 1/L_cc, X_ic = -(sum_{c<=m<i} L_im X_mc)/L_ii
            for (int col = tid; col < n; col += nt) {
                for (int i = 0; i < col; ++i) {
                    Lr[i * LDS + col] = 0.0;
                    Lim[i * LDS + col] = 0.0;
                }
                for (int i = col; i < n; ++i) {
                    double accr = i == col ? 1.0 : 0.0, acci = 0.0;
                    for (int m = col; m < i; ++m) {
                        const double lr = Sr[i * LDS + m], li = Si[i * LDS + m];
                        const double xr = Lr[m * LDS + col], xi = Lim[m * LDS + col];
                        accr -= lr * xr - li * xi;
                        acci -= lr * xi + li * xr;
                    }
                    const double d = Sr[i * LDS + i];
                    Lr[i * LDS + col] = accr / d;
                    Lim[i * LDS + col] = acci / d;
                }
            }
        }
        __syncthreads();
        double2 *dst = linvc + sl * (int64_t)linv_len(K);
        if (K == 36) {
            for (int e = tid; e < linv_len(36); e += nt) {
                int i, j;
                const bool v = lanestep_entry(e, i, j);
                const bool in = ok && v && i < n && j < n;
                dst[e] = make_double2(in ? Lr[i * LDS + j] : 0.0, in ? Lim[i * LDS + j] : 0.0);
            }
        } else {
            for (int j = 0; j < K; ++j) {
                for (int i = j + tid; i < K; i += nt) {
                    const bool in = ok && i < n && j < n;
                    dst[col_start(K, j) + i - j] = make_double2(in ? Lr[i * LDS + j] : 0.0, in ? Lim[i * LDS + j] : 0.0);
                }
            }
        }
        if (tmax > 0.0) atomicMax(a.max_t, (unsigned long long)__double_as_longlong(tmax));
        if (tid == 0) {
            a.slot_steps[sl] = ok ? steps : -1;
            if (!ok) atomicAdd(a.counts + 1, 1);
            else if (steps > 0) atomicAdd(a.counts, 1);
        }
        __syncthreads();
    }
}

// ---------------------------------------------------------------- apply kernel
struct ApplyArgs {
    int64_t N, Nc, first, count, nside_tgt;
    const double *map, *defl;
    double *out, *var;
    uint8_t *status;
    const int32_t *members, *slot;
    const double *linv;
    const double2 *pv;             // [12 N^2][2]: (x, y), (z, 0) of every map pixel (FP64 plans)
    const float4 *pvf;             // [12 N^2][2]: double-float (x, y), (z, 0) (mixed plans)
    const float2 *linvf;           // double-float L^-1 blocks (mixed plans)
    const int *slot_steps;
    TableDev tab;
    TableDev tabm;                 // augmented plans: xi-/xi+(0) on the same grid
    double xi0;
    unsigned long long *counters;  // points, nugget, -, window, failed
};

constexpr int APPLY_WARPS = 4;
constexpr int GROUP = 10;  // lanes per target when K <= 10 (three targets per warp)

// value, variance and status of target p from v = w . y and qc = w . c
// true when target p is a lensing target whose deflection is not finite (its
// outputs are NaN: target_of placed it at NaN)
__device__ __forceinline__ bool bad_deflection(const ApplyArgs &a, int64_t p) {
    if (a.nside_tgt > 0) return false;
    const double2 dd = __ldg(reinterpret_cast<const double2 *>(a.defl) + p);
    return !(isfinite(dd.x) && isfinite(dd.y));
}

__device__ __forceinline__ void finish_point(const ApplyArgs &a, int64_t p, int32_t sl, double v, double qc,
                                             bool any_win, unsigned long long &n_win, unsigned long long &n_nug,
                                             unsigned long long &n_fail) {
    const int steps = __ldg(a.slot_steps + sl);
    const bool bad = bad_deflection(a, p);
    uint8_t st = bad ? FLINTS_ST_INPUT : 0;
    if (steps > 0) st |= FLINTS_ST_NUGGET;
    if (any_win) st |= FLINTS_ST_WINDOW;
    if (steps < 0 || bad) {
        st |= FLINTS_ST_FAILED;
        v = __longlong_as_double(0x7ff8000000000000ll);
        qc = v;
    }
    a.out[p] = v;
    if (a.var) a.var[p] = a.xi0 * (1.0 - qc);
    if (a.status) a.status[p] = st;
    n_win += any_win;
    n_nug += steps > 0;
    n_fail += steps < 0 || bad;
}

// Target p (displaced pixel first + p, or the pixel centre of the nside_tgt
// grid) and the coarse pixel holding it; p >= count leaves the defaults.
__device__ __forceinline__ void target_of(const ApplyArgs &a, int64_t p, double &x, double &y, double &z,
                                          int64_t &c) {
    if (p >= a.count) return;
    const int64_t pix = a.first + p;
    if (a.nside_tgt > 0) {
        pix2vec(a.nside_tgt, pix, x, y, z);
    } else {
        int64_t i, j;
        pix_ring(a.N, pix, i, j);
        const Ring rg = ring_of(a.N, i);
        double sp, cp;
        sincospi(((double)j + rg.f) / (2.0 * (double)rg.nq), &sp, &cp);
        const double nx = rg.s * cp, ny = rg.s * sp, nz = rg.z;
        const double2 dd = __ldg(reinterpret_cast<const double2 *>(a.defl) + p);
        const double dl2 = dd.x * dd.x + dd.y * dd.y;
        x = nx;
        y = ny;
        z = nz;
        if (!(isfinite(dd.x) && isfinite(dd.y))) x = y = z = __longlong_as_double(0x7ff8000000000000ll);
        if (dl2 > 0.0) {
            // geodesic step of length |d| along d_theta e_theta + d_phi e_phi:
            // n' = cos|d| n + (sin|d|/|d|) (d_theta e_theta + d_phi e_phi).  For
            // |d| < 1/16 both factors are their Taylor series in |d|^2 to the
            // |d|^8 term (the next terms are below 3e-19); larger steps use sincos.
            double kk, cd;
            if (dl2 < 0.00390625) {
                kk = fma(dl2, fma(dl2, fma(dl2, fma(dl2, 1.0 / 362880.0, -1.0 / 5040.0), 1.0 / 120.0), -1.0 / 6.0), 1.0);
                cd = fma(dl2, fma(dl2, fma(dl2, fma(dl2, 1.0 / 40320.0, -1.0 / 720.0), 1.0 / 24.0), -0.5), 1.0);
            } else {
                const double dl = sqrt(dl2);
                double sd;
                sincos(dl, &sd, &cd);
                kk = sd / dl;
            }
            const double tx = dd.x * nz * cp - dd.y * sp;
            const double ty = dd.x * nz * sp + dd.y * cp;
            const double tz = -dd.x * rg.s;
            x = cd * nx + kk * tx;
            y = cd * ny + kk * ty;
            z = cd * nz + kk * tz;
        }
    }
    c = ang2pix(a.Nc, x, y, z);
    // a non-finite target yields NaN outputs; keep its index inside the grid
    c = (c < 0 || c >= 12 * a.Nc * a.Nc) ? 0 : c;
}

template <int K>
__global__ void __launch_bounds__(APPLY_WARPS * 32) apply_kernel(ApplyArgs a) {
    __shared__ double stx[APPLY_WARPS][32], sty[APPLY_WARPS][32], stz[APPLY_WARPS][32];
    __shared__ int64_t scp[APPLY_WARPS][32];
    __shared__ double sc[APPLY_WARPS][K > GROUP ? K : 1], sy[APPLY_WARPS][K > GROUP ? K : 1];
    // per target of the tile: w . y, w . c, class and window flag, finished one
    // target per lane after the tile
    __shared__ double rv[APPLY_WARPS][32], rq[APPLY_WARPS][32];
    __shared__ int32_t rsl[APPLY_WARPS][32];
    __shared__ unsigned char rwin[APPLY_WARPS][32];
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    const int64_t ntiles = (a.count + 31) / 32;
    unsigned long long n_win = 0, n_nug = 0, n_fail = 0;
    for (int64_t tile = (int64_t)blockIdx.x * APPLY_WARPS + wid; tile < ntiles;
         tile += (int64_t)gridDim.x * APPLY_WARPS) {
        // ---- lane l: target l of the tile and its coarse pixel
        {
            double x = 0.0, y = 0.0, z = 1.0;
            int64_t c = 0;
            target_of(a, tile * 32 + lane, x, y, z, c);
            scp[wid][lane] = c;
            stx[wid][lane] = x;
            sty[wid][lane] = y;
            stz[wid][lane] = z;
        }
        __syncwarp();
        const int npt = a.count - tile * 32 < 32 ? (int)(a.count - tile * 32) : 32;
        if constexpr (K <= GROUP) {
            // three targets at a time, one per group of GROUP lanes (lanes 30, 31 idle)
            const int g = lane / GROUP, l = lane - g * GROUP, base = g * GROUP;
            for (int q0 = 0; q0 < npt; q0 += 3) {
                const int q = q0 + g;
                const bool has = g < 3 && q < npt;
                double tx = 0.0, ty = 0.0, tz = 0.0;
                int64_t c = 0;
                if (has) {
                    tx = stx[wid][q];
                    ty = sty[wid][q];
                    tz = stz[wid][q];
                    c = scp[wid][q];
                }
                const int32_t sl = has ? __ldg(a.slot + c) : 0;
                double cv = 0.0, yv = 0.0;
                bool win = false;
                if (has && l < K) {
                    const int32_t m = __ldg(a.members + c * K + l);
                    if (m >= 0) {
                        double mx, my, mz;
                        member_vec(a.pv, m, mx, my, mz);
                        const double dx = tx - mx, dy = ty - my, dz = tz - mz;
                        const double t = dx * dx + dy * dy + dz * dz;
                        win = t > a.tab.t_max;
                        cv = table_eval<double>(a.tab, t);
                        yv = __ldg(a.map + m);
                    }
                }
                // z_c = L^-1 c, z_y = L^-1 y: lane l of the group accumulates row l
                const double *Lr = a.linv + (int64_t)sl * linv_len(K);
                double zc = 0.0, zy = 0.0;
#pragma unroll
                for (int j = 0; j < K; ++j) {
                    const double cj = __shfl_sync(FULL, cv, base + j);
                    const double yj = __shfl_sync(FULL, yv, base + j);
                    if (has && l < K && l >= j) {
                        const double e = __ldg(Lr + col_start(K, j) + l - j);
                        zc = fma(e, cj, zc);
                        zy = fma(e, yj, zy);
                    }
                }
                // group sums over lanes 0 .. GROUP-1: fold 8-9 onto 0-1, then halve 8 -> 1
                double vs = zc * zy, qs = zc * zc;
#pragma unroll
                for (int o = 8; o >= 1; o >>= 1) {
                    const double tv = __shfl_sync(FULL, vs, lane + o), tq = __shfl_sync(FULL, qs, lane + o);
                    if (l < o && l + o < GROUP) {
                        vs += tv;
                        qs += tq;
                    }
                }
                const unsigned wb = __ballot_sync(FULL, win);
                if (has && l == 0) {
                    rv[wid][q] = vs;
                    rq[wid][q] = qs;
                    rsl[wid][q] = sl;
                    rwin[wid][q] = ((wb >> base) & ((1u << GROUP) - 1u)) != 0;
                }
            }
        } else {
            // one target at a time; lanes own members l and l + 32.  Consecutive
            // targets in one coarse pixel reuse the members' positions and data.
            int64_t prev = -1;
            double m0x = 0.0, m0y = 0.0, m0z = 0.0, y0 = 0.0, m1x = 0.0, m1y = 0.0, m1z = 0.0, y1 = 0.0;
            bool v0 = false, v1 = false;
            for (int q = 0; q < npt; ++q) {
                const double tx = stx[wid][q], ty = sty[wid][q], tz = stz[wid][q];
                const int64_t c = scp[wid][q];
                const int32_t sl = __ldg(a.slot + c);
                if (c != prev) {
                    prev = c;
                    const int32_t *mem = a.members + c * K;
                    v0 = false;
                    v1 = false;
                    y0 = 0.0;
                    y1 = 0.0;
                    if (lane < K) {
                        const int32_t m = __ldg(mem + lane);
                        if (m >= 0) {
                            member_vec(a.pv, m, m0x, m0y, m0z);
                            y0 = __ldg(a.map + m);
                            v0 = true;
                        }
                    }
                    if (lane + 32 < K) {
                        const int32_t m = __ldg(mem + lane + 32);
                        if (m >= 0) {
                            member_vec(a.pv, m, m1x, m1y, m1z);
                            y1 = __ldg(a.map + m);
                            v1 = true;
                        }
                    }
                }
                double c0 = 0.0, c1 = 0.0;
                bool win = false;
                if (v0) {
                    const double dx = tx - m0x, dy = ty - m0y, dz = tz - m0z;
                    const double t = dx * dx + dy * dy + dz * dz;
                    win |= t > a.tab.t_max;
                    c0 = table_eval<double>(a.tab, t);
                }
                if (v1) {
                    const double dx = tx - m1x, dy = ty - m1y, dz = tz - m1z;
                    const double t = dx * dx + dy * dy + dz * dz;
                    win |= t > a.tab.t_max;
                    c1 = table_eval<double>(a.tab, t);
                }
                // z_c = L^-1 c, z_y = L^-1 y from the lane-step block; c and y go to
                // the warp's shared slots.  Rows 0..31: lanes 2p, 2p + 1 run through
                // the 33 entries of rows p and 31 - p (lane 2p switches from row p
                // to row 31 - p after column p; the two halves of row 31 - p are
                // joined by a shuffle).  Rows 32..35: lane l takes row 32 + (l & 3)
                // on columns (l >> 2) + 8t, eight partial sums joined by shuffles.
                static_assert(K == 36, "the lane-step layout is laid out for K = 36");
                const double *Lr = a.linv + (int64_t)sl * linv_len(K);
                __syncwarp();
                sc[wid][lane] = c0;
                sy[wid][lane] = y0;
                if (lane < K - 32) {
                    sc[wid][32 + lane] = c1;
                    sy[wid][32 + lane] = y1;
                }
                __syncwarp();
                const int pp = lane >> 1, odd = lane & 1;
                double zca = 0.0, zya = 0.0, zc0 = 0.0, zy0 = 0.0, zc1 = 0.0, zy1 = 0.0;
#pragma unroll
                for (int u = 0; u < LS_STEPS; ++u) {
                    const int t = odd ? LS_STEPS + u : u;
                    if (!odd && u == pp + 1) {
                        zca = zc0;
                        zya = zy0;
                        zc0 = 0.0;
                        zy0 = 0.0;
                    }
                    int j = t <= pp ? t : t - pp - 1;
                    j = j < K ? j : K - 1;  // the zero pad
                    const double e = __ldg(Lr + u * 32 + lane);
                    zc0 = fma(e, sc[wid][j], zc0);
                    zy0 = fma(e, sy[wid][j], zy0);
                }
                const double zcb = zc0 + __shfl_xor_sync(FULL, zc0, 1), zyb = zy0 + __shfl_xor_sync(FULL, zy0, 1);
                {
                    const int g = lane >> 2;
#pragma unroll
                    for (int t = 0; t < LS_TAIL; ++t) {
                        const int j = g + 8 * t < K ? g + 8 * t : K - 1;  // zero entries past the diagonal
                        const double e = __ldg(Lr + (LS_STEPS + t) * 32 + lane);
                        zc1 = fma(e, sc[wid][j], zc1);
                        zy1 = fma(e, sy[wid][j], zy1);
                    }
#pragma unroll
                    for (int o = 4; o < 32; o <<= 1) {
                        zc1 += __shfl_xor_sync(FULL, zc1, o);
                        zy1 += __shfl_xor_sync(FULL, zy1, o);
                    }
                }
                // even lanes count rows p and 31 - p, lanes 0..3 rows 32..35, each once
                double v = odd ? 0.0 : zca * zya + zcb * zyb, qc = odd ? 0.0 : zca * zca + zcb * zcb;
                if (lane < K - 32) {
                    v = fma(zc1, zy1, v);
                    qc = fma(zc1, zc1, qc);
                }
#pragma unroll
                for (int o = 16; o > 0; o >>= 1) {
                    v += __shfl_xor_sync(FULL, v, o);
                    qc += __shfl_xor_sync(FULL, qc, o);
                }
                const bool any_win = __any_sync(FULL, win);
                if (lane == 0) {
                    rv[wid][q] = v;
                    rq[wid][q] = qc;
                    rsl[wid][q] = sl;
                    rwin[wid][q] = any_win;
                }
            }
        }
        __syncwarp();
        if (lane < npt)
            finish_point(a, tile * 32 + lane, rsl[wid][lane], rv[wid][lane], rq[wid][lane], rwin[wid][lane] != 0,
                         n_win, n_nug, n_fail);
        __syncwarp();
    }
    // counts of every lane, summed over the warp
    const unsigned w_win = __reduce_add_sync(FULL, (unsigned)n_win);
    const unsigned w_nug = __reduce_add_sync(FULL, (unsigned)n_nug);
    const unsigned w_fail = __reduce_add_sync(FULL, (unsigned)n_fail);
    if (lane == 0 && a.counters) {
        if (w_win) atomicAdd(a.counters + CNT_WINDOW, (unsigned long long)w_win);
        if (w_nug) atomicAdd(a.counters + CNT_NUGGET, (unsigned long long)w_nug);
        if (w_fail) atomicAdd(a.counters + CNT_FAILED, (unsigned long long)w_fail);
    }
}

// -------------------------------------------- augmented spin 2 (xi+, xi-)
// Class blocks of the widely linear estimator: the real 2K x 2K form of the
// Hermitian covariance G_ab = xi+(t)/xi+(0) exp(2i(a_ab - a_ba)) and the
// pseudo-covariance C_ab = xi-(t)/xi+(0) exp(2i(a_ab + a_ba)) of P = Q + iU,
// rows and columns (Q_0..Q_{K-1}, U_0..U_{K-1}):
//   A[Q_a][Q_b] = Re(G + C),  A[U_a][Q_b] = Im(G + C),  A[U_a][U_b] = Re(G - C)
// (absent members: unit rows), nugget rule of Sec. 2.4, Cholesky and L^-1 in
// dynamic shared memory, L^-1 packed by columns (2K (2K + 1) / 2 entries).
__global__ void __launch_bounds__(SINV_THREADS) linv_kernel_aug(LinvArgs a, TableDev tabm, double *linva) {
    extern __shared__ double dsm[];
    __shared__ double px[STENCIL_MAX], py[STENCIL_MAX], pz[STENCIL_MAX], ps[STENCIL_MAX], pc[STENCIL_MAX],
        psn[STENCIL_MAX];
    __shared__ int n_sh, bad;
    const int tid = threadIdx.x, nt = blockDim.x, K = a.K, N = 2 * a.K, ld = N + 1;
    double *S = dsm, *Li = dsm + N * ld;
    for (int64_t sl = blockIdx.x; sl < a.nslot; sl += gridDim.x) {
        const int64_t rep = slot_rep(a.Nc, sl);
        const int32_t *mem = a.members + rep * K;
        if (tid == 0) {
            int n = 0;
            while (n < K && mem[n] >= 0) ++n;
            n_sh = n;
        }
        __syncthreads();
        const int n = n_sh;
        for (int m = tid; m < n; m += nt) {
            pix_frame(a.N, mem[m], pc[m], psn[m], pz[m], ps[m]);
            px[m] = ps[m] * pc[m];
            py[m] = ps[m] * psn[m];
        }
        __syncthreads();
        double tmax = 0.0;
        double nug = NUGGET_EPS;
        int steps = 0;
        bool ok = false;
        for (; steps <= MAX_NUGGET_STEPS; ++steps) {
            for (int e = tid; e < N * N; e += nt) {
                const int i = e / N, j = e - (e / N) * N;
                if (j > i) continue;
                const int mi = i < K ? i : i - K, mj = j < K ? j : j - K;
                double v;
                if (mi >= n || mj >= n) {
                    v = i == j ? 1.0 : 0.0;
                } else if (mi == mj) {
                    v = i == j ? 1.0 + nug : 0.0;  // xi-(0) = 0: no coupling of Q_a and U_a
                } else {
                    const double dx = px[mj] - px[mi], dy = py[mj] - py[mi], dz = pz[mj] - pz[mi];
                    const double t = dx * dx + dy * dy + dz * dz;
                    tmax = fmax(tmax, t);
                    const double fp = table_eval<double>(a.tab, t), fm = table_eval<double>(tabm, t);
                    Cx<double> php, phm;
                    pair_phases_pm<double>(dx, dy, dz, pz[mi], ps[mi], pc[mi], psn[mi], pz[mj], ps[mj], pc[mj], psn[mj],
                                           php, phm);
                    const double gr = fp * php.re, gi = fp * php.im, cr = fm * phm.re, ci = fm * phm.im;
                    const bool ui = i >= K, uj = j >= K;
                    v = !ui ? gr + cr : (uj ? gr - cr : gi + ci);
                }
                S[i * ld + j] = v;
            }
            if (tid == 0) bad = 0;
            __syncthreads();
            for (int kk = 0; kk < N; ++kk) {
                if (tid == 0) {
                    const double d = S[kk * ld + kk];
                    if (d > 0.0) S[kk * ld + kk] = sqrt(d); else bad = 1;
                }
                __syncthreads();
                if (bad) break;
                const double lkk = S[kk * ld + kk];
                for (int i = kk + 1 + tid; i < N; i += nt) S[i * ld + kk] /= lkk;
                __syncthreads();
                const int w = N - kk - 1;
                for (int e = tid; e < w * w; e += nt) {
                    const int i = kk + 1 + e / w, j = kk + 1 + (e - (e / w) * w);
                    if (j <= i) S[i * ld + j] -= S[i * ld + kk] * S[j * ld + kk];
                }
                __syncthreads();
            }
            if (!bad) {
                ok = true;
                break;
            }
            nug *= 2.0;
            __syncthreads();
        }
        if (ok) {
            for (int col = tid; col < N; col += nt) {
                for (int i = 0; i < col; ++i) Li[i * ld + col] = 0.0;
                for (int i = col; i < N; ++i) {
                    double acc = i == col ? 1.0 : 0.0;
                    for (int m = col; m < i; ++m) acc = fma(-S[i * ld + m], Li[m * ld + col], acc);
                    Li[i * ld + col] = acc / S[i * ld + i];
                }
            }
        }
        __syncthreads();
        double *dst = linva + sl * (int64_t)(N * (N + 1) / 2);
        for (int j = 0; j < N; ++j) {
            for (int i = j + tid; i < N; i += nt) dst[col_start(N, j) + i - j] = ok ? Li[i * ld + j] : 0.0;
        }
        if (tmax > 0.0) atomicMax(a.max_t, (unsigned long long)__double_as_longlong(tmax));
        if (tid == 0) {
            a.slot_steps[sl] = ok ? steps : -1;
            if (!ok) atomicAdd(a.counts + 1, 1);
            else if (steps > 0) atomicAdd(a.counts, 1);
        }
        __syncthreads();
    }
}

// ------------------------------------------------- spin-1/2 apply (FP64)
// value conj(z_c) . z_y (Q, U; or d_theta, d_phi for spin 1) and variance of
// target p
__device__ __forceinline__ void finish_point_s2(const ApplyArgs &a, int64_t p, int32_t sl, double vr, double vi,
                                                double qc, bool any_win, unsigned long long &n_win,
                                                unsigned long long &n_nug, unsigned long long &n_fail) {
    const int steps = __ldg(a.slot_steps + sl);
    const bool bad = bad_deflection(a, p);
    uint8_t st = bad ? FLINTS_ST_INPUT : 0;
    if (steps > 0) st |= FLINTS_ST_NUGGET;
    if (any_win) st |= FLINTS_ST_WINDOW;
    if (steps < 0 || bad) {
        st |= FLINTS_ST_FAILED;
        vr = vi = qc = __longlong_as_double(0x7ff8000000000000ll);
    }
    reinterpret_cast<double2 *>(a.out)[p] = make_double2(vr, vi);
    if (a.var) a.var[p] = a.xi0 * (1.0 - qc);
    if (a.status) a.status[p] = st;
    n_win += any_win;
    n_nug += steps > 0;
    n_fail += steps < 0 || bad;
}

// c_m = xi+(t)/xi+(0) exp(iS(a_tm - a_mt - pi)) of member m for the target
// (t, frame) and its two field components; returns false for an absent member
template <int S>
__device__ __forceinline__ bool member_s2(const ApplyArgs &a, int32_t m, double tx, double ty, double tz, double tzz,
                                         double ts, double tc, double tsn, double &cr, double &ci, double &yr,
                                         double &yi, bool &win) {
    if (m < 0) return false;
    const double2 f0 = __ldg(a.pv + 2 * m), f1 = __ldg(a.pv + 2 * m + 1);  // (cos, sin phi), (z, s)
    const double mx = f1.y * f0.x, my = f1.y * f0.y, mz = f1.x;
    const double dx = mx - tx, dy = my - ty, dz = mz - tz;
    const double t = dx * dx + dy * dy + dz * dz;
    win |= t > a.tab.t_max;
    const double f = table_eval<double>(a.tab, t);
    const Cx<double> ph = pair_phase<double, S>(dx, dy, dz, tzz, ts, tc, tsn, f1.x, f1.y, f0.x, f0.y);
    cr = f * ph.re;
    ci = f * ph.im;
    const double2 q = __ldg(reinterpret_cast<const double2 *>(a.map) + m);
    yr = q.x;
    yi = q.y;
    return true;
}

template <int K, int S>
__global__ void __launch_bounds__(APPLY_WARPS * 32) apply_kernel_s2(ApplyArgs a) {
    __shared__ double stx[APPLY_WARPS][32], sty[APPLY_WARPS][32], stz[APPLY_WARPS][32];
    __shared__ double sts[APPLY_WARPS][32], stc[APPLY_WARPS][32], stn[APPLY_WARPS][32];
    __shared__ int64_t scp[APPLY_WARPS][32];
    constexpr int KS = K > GROUP ? K : 1;
    __shared__ double sxr[APPLY_WARPS][KS], sxi[APPLY_WARPS][KS], syr[APPLY_WARPS][KS], syi[APPLY_WARPS][KS];
    __shared__ double rvr[APPLY_WARPS][32], rvi[APPLY_WARPS][32], rq[APPLY_WARPS][32];
    __shared__ int32_t rsl[APPLY_WARPS][32];
    __shared__ unsigned char rwin[APPLY_WARPS][32];
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    const int64_t ntiles = (a.count + 31) / 32;
    const int64_t mirror_from = 6 * a.Nc * a.Nc + 2 * a.Nc;  // first pixel of coarse ring 2 Nc + 1
    unsigned long long n_win = 0, n_nug = 0, n_fail = 0;
    for (int64_t tile = (int64_t)blockIdx.x * APPLY_WARPS + wid; tile < ntiles;
         tile += (int64_t)gridDim.x * APPLY_WARPS) {
        {
            double x = 0.0, y = 0.0, z = 1.0;
            int64_t c = 0;
            target_of(a, tile * 32 + lane, x, y, z, c);
            const double sn = sqrt(x * x + y * y);
            scp[wid][lane] = c;
            stx[wid][lane] = x;
            sty[wid][lane] = y;
            stz[wid][lane] = z;
            sts[wid][lane] = sn;
            stc[wid][lane] = sn > 1e-12 ? x / sn : 1.0;
            stn[wid][lane] = sn > 1e-12 ? y / sn : 0.0;
        }
        __syncwarp();
        const int npt = a.count - tile * 32 < 32 ? (int)(a.count - tile * 32) : 32;
        if constexpr (K <= GROUP) {
            const int g = lane / GROUP, l = lane - g * GROUP, base = g * GROUP;
            for (int q0 = 0; q0 < npt; q0 += 3) {
                const int q = q0 + g;
                const bool has = g < 3 && q < npt;
                const int qq = has ? q : 0;
                const int64_t c = scp[wid][qq];
                const int32_t sl = has ? __ldg(a.slot + c) : 0;
                const double msign = c >= mirror_from ? -1.0 : 1.0;  // conj(L^-1) for mirrored classes
                double cr = 0.0, ci = 0.0, yr = 0.0, yi = 0.0;
                bool win = false;
                if (has && l < K)
                    member_s2<S>(a, __ldg(a.members + c * K + l), stx[wid][qq], sty[wid][qq], stz[wid][qq],
                              stz[wid][qq], sts[wid][qq], stc[wid][qq], stn[wid][qq], cr, ci, yr, yi, win);
                // z_c = L^-1 conj(c), z_y = L^-1 y: lane l of the group accumulates row l
                const double2 *Lr = reinterpret_cast<const double2 *>(a.linv) + (int64_t)sl * linv_len(K);
                double zcr = 0.0, zci = 0.0, zyr = 0.0, zyi = 0.0;
#pragma unroll
                for (int j = 0; j < K; ++j) {
                    const double xr = __shfl_sync(FULL, cr, base + j), xi = -__shfl_sync(FULL, ci, base + j);
                    const double ur = __shfl_sync(FULL, yr, base + j), ui = __shfl_sync(FULL, yi, base + j);
                    if (has && l < K && l >= j) {
                        const double2 e = __ldg(Lr + col_start(K, j) + l - j);
                        const double ei = msign * e.y;
                        zcr = fma(e.x, xr, fma(-ei, xi, zcr));
                        zci = fma(e.x, xi, fma(ei, xr, zci));
                        zyr = fma(e.x, ur, fma(-ei, ui, zyr));
                        zyi = fma(e.x, ui, fma(ei, ur, zyi));
                    }
                }
                double vr = zcr * zyr + zci * zyi, vi = zcr * zyi - zci * zyr, qs = zcr * zcr + zci * zci;
#pragma unroll
                for (int o = 8; o >= 1; o >>= 1) {
                    const double tr = __shfl_sync(FULL, vr, lane + o), ti = __shfl_sync(FULL, vi, lane + o);
                    const double tq = __shfl_sync(FULL, qs, lane + o);
                    if (l < o && l + o < GROUP) {
                        vr += tr;
                        vi += ti;
                        qs += tq;
                    }
                }
                const unsigned wb = __ballot_sync(FULL, win);
                if (has && l == 0) {
                    rvr[wid][q] = vr;
                    rvi[wid][q] = vi;
                    rq[wid][q] = qs;
                    rsl[wid][q] = sl;
                    rwin[wid][q] = ((wb >> base) & ((1u << GROUP) - 1u)) != 0;
                }
            }
        } else {
            static_assert(K == 36, "the lane-step layout is laid out for K = 36");
            for (int q = 0; q < npt; ++q) {
                const int64_t c = scp[wid][q];
                const int32_t sl = __ldg(a.slot + c);
                const double msign = c >= mirror_from ? -1.0 : 1.0;
                const double tx = stx[wid][q], ty = sty[wid][q], tz = stz[wid][q];
                const double ts = sts[wid][q], tc = stc[wid][q], tn = stn[wid][q];
                const int32_t *mem = a.members + c * K;
                double c0r = 0.0, c0i = 0.0, y0r = 0.0, y0i = 0.0, c1r = 0.0, c1i = 0.0, y1r = 0.0, y1i = 0.0;
                bool win = false;
                member_s2<S>(a, __ldg(mem + lane), tx, ty, tz, tz, ts, tc, tn, c0r, c0i, y0r, y0i, win);
                if (lane + 32 < K)
                    member_s2<S>(a, __ldg(mem + lane + 32), tx, ty, tz, tz, ts, tc, tn, c1r, c1i, y1r, y1i, win);
                const double2 *Lr = reinterpret_cast<const double2 *>(a.linv) + (int64_t)sl * linv_len(K);
                __syncwarp();
                sxr[wid][lane] = c0r;
                sxi[wid][lane] = -c0i;
                syr[wid][lane] = y0r;
                syi[wid][lane] = y0i;
                if (lane < K - 32) {
                    sxr[wid][32 + lane] = c1r;
                    sxi[wid][32 + lane] = -c1i;
                    syr[wid][32 + lane] = y1r;
                    syi[wid][32 + lane] = y1i;
                }
                __syncwarp();
                // the lane-step block as in the spin-0 kernel, complex
                const int pp = lane >> 1, odd = lane & 1;
                double acr = 0.0, aci = 0.0, ayr = 0.0, ayi = 0.0;  // row p (even lanes)
                double zcr = 0.0, zci = 0.0, zyr = 0.0, zyi = 0.0;
#pragma unroll
                for (int u = 0; u < LS_STEPS; ++u) {
                    const int t = odd ? LS_STEPS + u : u;
                    if (!odd && u == pp + 1) {
                        acr = zcr;
                        aci = zci;
                        ayr = zyr;
                        ayi = zyi;
                        zcr = zci = zyr = zyi = 0.0;
                    }
                    int j = t <= pp ? t : t - pp - 1;
                    j = j < K ? j : K - 1;  // the zero pad
                    const double2 e = __ldg(Lr + u * 32 + lane);
                    const double ei = msign * e.y;
                    const double xr = sxr[wid][j], xi = sxi[wid][j], ur = syr[wid][j], ui = syi[wid][j];
                    zcr = fma(e.x, xr, fma(-ei, xi, zcr));
                    zci = fma(e.x, xi, fma(ei, xr, zci));
                    zyr = fma(e.x, ur, fma(-ei, ui, zyr));
                    zyi = fma(e.x, ui, fma(ei, ur, zyi));
                }
                const double bcr = zcr + __shfl_xor_sync(FULL, zcr, 1), bci = zci + __shfl_xor_sync(FULL, zci, 1);
                const double byr = zyr + __shfl_xor_sync(FULL, zyr, 1), byi = zyi + __shfl_xor_sync(FULL, zyi, 1);
                double tcr = 0.0, tci = 0.0, tyr = 0.0, tyi = 0.0;  // rows 32..35
                {
                    const int g = lane >> 2;
#pragma unroll
                    for (int t = 0; t < LS_TAIL; ++t) {
                        const int j = g + 8 * t < K ? g + 8 * t : K - 1;  // zero entries past the diagonal
                        const double2 e = __ldg(Lr + (LS_STEPS + t) * 32 + lane);
                        const double ei = msign * e.y;
                        const double xr = sxr[wid][j], xi = sxi[wid][j], ur = syr[wid][j], ui = syi[wid][j];
                        tcr = fma(e.x, xr, fma(-ei, xi, tcr));
                        tci = fma(e.x, xi, fma(ei, xr, tci));
                        tyr = fma(e.x, ur, fma(-ei, ui, tyr));
                        tyi = fma(e.x, ui, fma(ei, ur, tyi));
                    }
#pragma unroll
                    for (int o = 4; o < 32; o <<= 1) {
                        tcr += __shfl_xor_sync(FULL, tcr, o);
                        tci += __shfl_xor_sync(FULL, tci, o);
                        tyr += __shfl_xor_sync(FULL, tyr, o);
                        tyi += __shfl_xor_sync(FULL, tyi, o);
                    }
                }
                // even lanes count rows p and 31 - p, lanes 0..3 rows 32..35, each once
                double vr = 0.0, vi = 0.0, qc = 0.0;
                if (!odd) {
                    vr = acr * ayr + aci * ayi + bcr * byr + bci * byi;
                    vi = acr * ayi - aci * ayr + bcr * byi - bci * byr;
                    qc = acr * acr + aci * aci + bcr * bcr + bci * bci;
                }
                if (lane < K - 32) {
                    vr += tcr * tyr + tci * tyi;
                    vi += tcr * tyi - tci * tyr;
                    qc += tcr * tcr + tci * tci;
                }
#pragma unroll
                for (int o = 16; o > 0; o >>= 1) {
                    vr += __shfl_xor_sync(FULL, vr, o);
                    vi += __shfl_xor_sync(FULL, vi, o);
                    qc += __shfl_xor_sync(FULL, qc, o);
                }
                const bool any_win = __any_sync(FULL, win);
                if (lane == 0) {
                    rvr[wid][q] = vr;
                    rvi[wid][q] = vi;
                    rq[wid][q] = qc;
                    rsl[wid][q] = sl;
                    rwin[wid][q] = any_win;
                }
            }
        }
        __syncwarp();
        if (lane < npt)
            finish_point_s2(a, tile * 32 + lane, rsl[wid][lane], rvr[wid][lane], rvi[wid][lane], rq[wid][lane],
                            rwin[wid][lane] != 0, n_win, n_nug, n_fail);
        __syncwarp();
    }
    const unsigned w_win = __reduce_add_sync(FULL, (unsigned)n_win);
    const unsigned w_nug = __reduce_add_sync(FULL, (unsigned)n_nug);
    const unsigned w_fail = __reduce_add_sync(FULL, (unsigned)n_fail);
    if (lane == 0 && a.counters) {
        if (w_win) atomicAdd(a.counters + CNT_WINDOW, (unsigned long long)w_win);
        if (w_nug) atomicAdd(a.counters + CNT_NUGGET, (unsigned long long)w_nug);
        if (w_fail) atomicAdd(a.counters + CNT_FAILED, (unsigned long long)w_fail);
    }
}

// Widely linear estimate per target: b_Q, b_U (the columns of (<P_i P_0^*>,
// <P_i P_0>) in the real form) and x = (Q_i, U_i); Z_Q = L^-1 b_Q, Z_U = L^-1
// b_U, z_x = L^-1 x; (Q, U) = (Z_Q . z_x, Z_U . z_x), variance xi+(0) (1 -
// (|Z_Q|^2 + |Z_U|^2)/2).  A class mirrored by z -> -z uses D L^-1 D, D =
// diag(I, -I): its Q-U entries change sign.  One target per warp; lane l owns
// rows l + 32t of the 2K.
template <int K>
__global__ void __launch_bounds__(APPLY_WARPS * 32) apply_kernel_aug(ApplyArgs a) {
    constexpr int N = 2 * K, T = (N + 31) / 32;
    __shared__ double stx[APPLY_WARPS][32], sty[APPLY_WARPS][32], stz[APPLY_WARPS][32];
    __shared__ double sts[APPLY_WARPS][32], stc[APPLY_WARPS][32], stn[APPLY_WARPS][32];
    __shared__ int64_t scp[APPLY_WARPS][32];
    __shared__ double sbq[APPLY_WARPS][N], sbu[APPLY_WARPS][N], sx[APPLY_WARPS][N];
    __shared__ double rvr[APPLY_WARPS][32], rvi[APPLY_WARPS][32], rq[APPLY_WARPS][32];
    __shared__ int32_t rsl[APPLY_WARPS][32];
    __shared__ unsigned char rwin[APPLY_WARPS][32];
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    const int64_t ntiles = (a.count + 31) / 32;
    const int64_t mirror_from = 6 * a.Nc * a.Nc + 2 * a.Nc;  // first pixel of coarse ring 2 Nc + 1
    unsigned long long n_win = 0, n_nug = 0, n_fail = 0;
    for (int64_t tile = (int64_t)blockIdx.x * APPLY_WARPS + wid; tile < ntiles;
         tile += (int64_t)gridDim.x * APPLY_WARPS) {
        {
            double x = 0.0, y = 0.0, z = 1.0;
            int64_t c = 0;
            target_of(a, tile * 32 + lane, x, y, z, c);
            const double sn = sqrt(x * x + y * y);
            scp[wid][lane] = c;
            stx[wid][lane] = x;
            sty[wid][lane] = y;
            stz[wid][lane] = z;
            sts[wid][lane] = sn;
            stc[wid][lane] = sn > 1e-12 ? x / sn : 1.0;
            stn[wid][lane] = sn > 1e-12 ? y / sn : 0.0;
        }
        __syncwarp();
        const int npt = a.count - tile * 32 < 32 ? (int)(a.count - tile * 32) : 32;
        for (int q = 0; q < npt; ++q) {
            const int64_t c = scp[wid][q];
            const int32_t sl = __ldg(a.slot + c);
            const bool mir = c >= mirror_from;
            const double tx = stx[wid][q], ty = sty[wid][q], tz = stz[wid][q];
            const double ts = sts[wid][q], tc = stc[wid][q], tn = stn[wid][q];
            bool win = false;
            __syncwarp();
#pragma unroll
            for (int h = 0; h < (K + 31) / 32; ++h) {
                const int m = lane + 32 * h;
                if (m < K) {
                    const int32_t pm = __ldg(a.members + c * K + m);
                    double bq0 = 0.0, bq1 = 0.0, bu0 = 0.0, bu1 = 0.0, xq = 0.0, xu = 0.0;
                    if (pm >= 0) {
                        const double2 f0 = __ldg(a.pv + 2 * pm), f1 = __ldg(a.pv + 2 * pm + 1);
                        const double mx = f1.y * f0.x, my = f1.y * f0.y, mz = f1.x;
                        const double dx = mx - tx, dy = my - ty, dz = mz - tz;
                        const double t = dx * dx + dy * dy + dz * dz;
                        win |= t > a.tab.t_max;
                        const double fp = table_eval<double>(a.tab, t), fm = table_eval<double>(a.tabm, t);
                        Cx<double> php, phm;  // of (target -> member); G_i0 takes the conjugate Hermitian phase
                        pair_phases_pm<double>(dx, dy, dz, tz, ts, tc, tn, f1.x, f1.y, f0.x, f0.y, php, phm);
                        const double gr = fp * php.re, gi = -fp * php.im, cr = fm * phm.re, ci = fm * phm.im;
                        bq0 = gr + cr;
                        bq1 = gi + ci;
                        bu0 = ci - gi;
                        bu1 = gr - cr;
                        const double2 qu = __ldg(reinterpret_cast<const double2 *>(a.map) + pm);
                        xq = qu.x;
                        xu = qu.y;
                    }
                    sbq[wid][m] = bq0;
                    sbq[wid][K + m] = bq1;
                    sbu[wid][m] = bu0;
                    sbu[wid][K + m] = bu1;
                    sx[wid][m] = xq;
                    sx[wid][K + m] = xu;
                }
            }
            __syncwarp();
            const double *Lr = a.linv + (int64_t)sl * (N * (N + 1) / 2);
            double zq[T], zu[T], zx[T];
#pragma unroll
            for (int t = 0; t < T; ++t) zq[t] = zu[t] = zx[t] = 0.0;
#pragma unroll 2
            for (int j = 0; j < N; ++j) {
                const double bqj = sbq[wid][j], buj = sbu[wid][j], xj = sx[wid][j];
                const int cs = col_start(N, j) - j;
#pragma unroll
                for (int t = 0; t < T; ++t) {
                    const int r = lane + 32 * t;
                    if (r < N && r >= j) {
                        double e = __ldg(Lr + cs + r);
                        if (mir && ((r < K) != (j < K))) e = -e;
                        zq[t] = fma(e, bqj, zq[t]);
                        zu[t] = fma(e, buj, zu[t]);
                        zx[t] = fma(e, xj, zx[t]);
                    }
                }
            }
            double vq = 0.0, vu = 0.0, nn = 0.0;
#pragma unroll
            for (int t = 0; t < T; ++t) {
                vq = fma(zq[t], zx[t], vq);
                vu = fma(zu[t], zx[t], vu);
                nn = fma(zq[t], zq[t], fma(zu[t], zu[t], nn));
            }
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) {
                vq += __shfl_xor_sync(FULL, vq, o);
                vu += __shfl_xor_sync(FULL, vu, o);
                nn += __shfl_xor_sync(FULL, nn, o);
            }
            const bool any_win = __any_sync(FULL, win);
            if (lane == 0) {
                rvr[wid][q] = vq;
                rvi[wid][q] = vu;
                rq[wid][q] = 0.5 * nn;
                rsl[wid][q] = sl;
                rwin[wid][q] = any_win;
            }
        }
        __syncwarp();
        if (lane < npt)
            finish_point_s2(a, tile * 32 + lane, rsl[wid][lane], rvr[wid][lane], rvi[wid][lane], rq[wid][lane],
                            rwin[wid][lane] != 0, n_win, n_nug, n_fail);
        __syncwarp();
    }
    const unsigned w_win = __reduce_add_sync(FULL, (unsigned)n_win);
    const unsigned w_nug = __reduce_add_sync(FULL, (unsigned)n_nug);
    const unsigned w_fail = __reduce_add_sync(FULL, (unsigned)n_fail);
    if (lane == 0 && a.counters) {
        if (w_win) atomicAdd(a.counters + CNT_WINDOW, (unsigned long long)w_win);
        if (w_nug) atomicAdd(a.counters + CNT_NUGGET, (unsigned long long)w_nug);
        if (w_fail) atomicAdd(a.counters + CNT_FAILED, (unsigned long long)w_fail);
    }
}

// ------------------------------------------------------- mixed precision
// The same route with the per-target arithmetic in double-float (pairs of FP32,
// about 2^-44 relative per operation) on the FP32 pipe: member positions from a
// double-float pixel table, chords and the correlation lookup in double-float,
// z_c = L^-1 c and z_y = L^-1 y accumulated from double-float L^-1 blocks; the
// target position and its coarse pixel stay FP64.  Chords between nearby unit
// vectors lose the positions' absolute error (2^-48) relative to the chord:
// about 1e-10 of chord^2 at Nside 4096.
__global__ void pixvec_df_kernel(int64_t N, float4 *pvf) {
    const int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= 12 * N * N) return;
    double x, y, z;
    pix2vec(N, p, x, y, z);
    const df dx = df_from(x), dy = df_from(y), dz = df_from(z);
    pvf[2 * p] = make_float4(dx.hi, dx.lo, dy.hi, dy.lo);
    pvf[2 * p + 1] = make_float4(dz.hi, dz.lo, 0.0f, 0.0f);
}

__global__ void to_df_kernel(const double *src, float2 *dst, int64_t n) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const df v = df_from(src[i]);
    dst[i] = make_float2(v.hi, v.lo);
}

__device__ __forceinline__ void member_vec_df(const float4 *pvf, int64_t m, df &x, df &y, df &z) {
    const float4 u = __ldg(pvf + 2 * m), v = __ldg(pvf + 2 * m + 1);
    x = {u.x, u.y};
    y = {u.z, u.w};
    z = {v.x, v.y};
}

// |t - m|^2 of double-float unit vectors: the differences' high words cancel
// exactly or leave a two_sum error, and the squares are positive
__device__ __forceinline__ df chord2_df(df tx, df ty, df tz, df mx, df my, df mz) {
    const df dx = df_add_fast(tx, df_neg(mx)), dy = df_add_fast(ty, df_neg(my)), dz = df_add_fast(tz, df_neg(mz));
    return df_add_fast(df_add_fast(df_mul(dx, dx), df_mul(dy, dy)), df_mul(dz, dz));
}

__device__ __forceinline__ df shfl_df(df v, int src) {
    return {__shfl_sync(FULL, v.hi, src), __shfl_sync(FULL, v.lo, src)};
}
__device__ __forceinline__ df shfl_xor_df(df v, int o) {
    return {__shfl_xor_sync(FULL, v.hi, o), __shfl_xor_sync(FULL, v.lo, o)};
}
__device__ __forceinline__ df ld_df(const float2 *p) {
    const float2 v = __ldg(p);
    return {v.x, v.y};
}

// A double as a double-float pair without FP64 instructions: hi = x with its
// mantissa truncated to 24 bits (bit operations), lo = the next 29 bits rounded
// to 24 (integer to float, exact power-of-two scaling), |x - (hi + lo)| <=
// 2^-47 |x|.  Values below the float normal range become 0, beyond it +-inf;
// NaN stays NaN.
__device__ __forceinline__ df split_double(double x) {
    const unsigned long long b = (unsigned long long)__double_as_longlong(x);
    const unsigned sign = (unsigned)(b >> 32) & 0x80000000u;
    const int e = (int)((b >> 52) & 0x7ff);
    const unsigned long long mant = b & 0xfffffffffffffull;
    if (e == 0x7ff) return {__uint_as_float(sign | 0x7f800000u | (mant ? 0x400000u : 0u)), 0.0f};
    const int fe = e - 1023 + 127;
    if (fe <= 0) return {__uint_as_float(sign), 0.0f};
    if (fe >= 255) return {__uint_as_float(sign | 0x7f800000u), 0.0f};
    const float hi = __uint_as_float(sign | ((unsigned)fe << 23) | (unsigned)(mant >> 29));
    // the low bits' unit 2^(e - 1075), applied in two exact steps when it lies
    // below the float normal range (fe > 0 keeps le > -52)
    const int le = e - 1075 + 127;
    float lo = __uint2float_rn((unsigned)(mant & 0x1fffffffu)) * __uint_as_float((unsigned)(le > 0 ? le : le + 64) << 23);
    if (le <= 0) lo *= 5.42101086242752217e-20f;  // 2^-64
    return {hi, __uint_as_float(__float_as_uint(lo) | sign)};
}

template <int K>
__global__ void __launch_bounds__(APPLY_WARPS * 32) apply_kernel_df(ApplyArgs a) {
    __shared__ df stx[APPLY_WARPS][32], sty[APPLY_WARPS][32], stz[APPLY_WARPS][32];
    __shared__ int64_t scp[APPLY_WARPS][32];
    __shared__ df sc[APPLY_WARPS][K > GROUP ? K : 1], sy[APPLY_WARPS][K > GROUP ? K : 1];
    // per target of the tile: w . y, w . c, class and window flag, finished one
    // target per lane after the tile (the double conversions then cost one
    // instruction per 32 targets)
    __shared__ df rv[APPLY_WARPS][32], rq[APPLY_WARPS][32];
    __shared__ int32_t rsl[APPLY_WARPS][32];
    __shared__ unsigned char rwin[APPLY_WARPS][32];
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    const int64_t ntiles = (a.count + 31) / 32;
    const float tmaxf = (float)a.tab.t_max;
    unsigned long long n_win = 0, n_nug = 0, n_fail = 0;
    for (int64_t tile = (int64_t)blockIdx.x * APPLY_WARPS + wid; tile < ntiles;
         tile += (int64_t)gridDim.x * APPLY_WARPS) {
        {
            double x = 0.0, y = 0.0, z = 1.0;
            int64_t c = 0;
            target_of(a, tile * 32 + lane, x, y, z, c);
            scp[wid][lane] = c;
            stx[wid][lane] = split_double(x);
            sty[wid][lane] = split_double(y);
            stz[wid][lane] = split_double(z);
        }
        __syncwarp();
        const int npt = a.count - tile * 32 < 32 ? (int)(a.count - tile * 32) : 32;
        if constexpr (K <= GROUP) {
            const int g = lane / GROUP, l = lane - g * GROUP, base = g * GROUP;
            for (int q0 = 0; q0 < npt; q0 += 3) {
                const int q = q0 + g;
                const bool has = g < 3 && q < npt;
                int64_t c = 0;
                df tx{0.0f, 0.0f}, ty{0.0f, 0.0f}, tz{1.0f, 0.0f};
                if (has) {
                    tx = stx[wid][q];
                    ty = sty[wid][q];
                    tz = stz[wid][q];
                    c = scp[wid][q];
                }
                const int32_t sl = has ? __ldg(a.slot + c) : 0;
                df cv{0.0f, 0.0f}, yv{0.0f, 0.0f};
                bool win = false;
                if (has && l < K) {
                    const int32_t m = __ldg(a.members + c * K + l);
                    if (m >= 0) {
                        df mx, my, mz;
                        member_vec_df(a.pvf, m, mx, my, mz);
                        const df t = chord2_df(tx, ty, tz, mx, my, mz);
                        win = t.hi > tmaxf;
                        cv = table_eval<df>(a.tab, t);
                        yv = split_double(__ldg(a.map + m));
                    }
                }
                const float2 *Lr = a.linvf + (int64_t)sl * linv_len(K);
                dfacc zc{0.0f, 0.0f}, zy{0.0f, 0.0f};
#pragma unroll
                for (int j = 0; j < K; ++j) {
                    const df cj = shfl_df(cv, base + j), yj = shfl_df(yv, base + j);
                    if (has && l < K && l >= j) {
                        const df e = ld_df(Lr + col_start(K, j) + l - j);
                        dfacc_add_prod(zc, e, cj);
                        dfacc_add_prod(zy, e, yj);
                    }
                }
                const df zcv = dfacc_val(zc), zyv = dfacc_val(zy);
                df vs = df_mul(zcv, zyv), qs = df_mul(zcv, zcv);
#pragma unroll
                for (int o = 8; o >= 1; o >>= 1) {
                    const df tv = shfl_df(vs, lane + o), tq = shfl_df(qs, lane + o);
                    if (l < o && l + o < GROUP) {
                        vs = df_add_fast(vs, tv);
                        qs = df_add_fast(qs, tq);
                    }
                }
                const unsigned wb = __ballot_sync(FULL, win);
                if (has && l == 0) {
                    rv[wid][q] = vs;
                    rq[wid][q] = qs;
                    rsl[wid][q] = sl;
                    rwin[wid][q] = ((wb >> base) & ((1u << GROUP) - 1u)) != 0;
                }
            }
        } else {
            static_assert(K == 36, "the split of rows 32 .. K-1 is laid out for K = 36");
            int64_t prev = -1;
            df m0x{0.0f, 0.0f}, m0y{0.0f, 0.0f}, m0z{0.0f, 0.0f}, y0{0.0f, 0.0f};
            df m1x{0.0f, 0.0f}, m1y{0.0f, 0.0f}, m1z{0.0f, 0.0f}, y1{0.0f, 0.0f};
            bool v0 = false, v1 = false;
            for (int q = 0; q < npt; ++q) {
                const df tx = stx[wid][q], ty = sty[wid][q], tz = stz[wid][q];
                const int64_t c = scp[wid][q];
                const int32_t sl = __ldg(a.slot + c);
                if (c != prev) {
                    prev = c;
                    const int32_t *mem = a.members + c * K;
                    v0 = false;
                    v1 = false;
                    y0 = {0.0f, 0.0f};
                    y1 = {0.0f, 0.0f};
                    const int32_t mA = __ldg(mem + lane);
                    if (mA >= 0) {
                        member_vec_df(a.pvf, mA, m0x, m0y, m0z);
                        y0 = split_double(__ldg(a.map + mA));
                        v0 = true;
                    }
                    if (lane + 32 < K) {
                        const int32_t mB = __ldg(mem + lane + 32);
                        if (mB >= 0) {
                            member_vec_df(a.pvf, mB, m1x, m1y, m1z);
                            y1 = split_double(__ldg(a.map + mB));
                            v1 = true;
                        }
                    }
                }
                df c0{0.0f, 0.0f}, c1{0.0f, 0.0f};
                bool win = false;
                if (v0) {
                    const df t = chord2_df(tx, ty, tz, m0x, m0y, m0z);
                    win |= t.hi > tmaxf;
                    c0 = table_eval<df>(a.tab, t);
                }
                if (v1) {
                    const df t = chord2_df(tx, ty, tz, m1x, m1y, m1z);
                    win |= t.hi > tmaxf;
                    c1 = table_eval<df>(a.tab, t);
                }
                const float2 *Lr = a.linvf + (int64_t)sl * linv_len(K);
                __syncwarp();
                sc[wid][lane] = c0;
                sy[wid][lane] = y0;
                if (lane < K - 32) {
                    sc[wid][32 + lane] = c1;
                    sy[wid][32 + lane] = y1;
                }
                __syncwarp();
                // the lane-step block, as in the FP64 kernel
                const int pp = lane >> 1, odd = lane & 1;
                dfacc zca{0.0f, 0.0f}, zya{0.0f, 0.0f}, zc0{0.0f, 0.0f}, zy0{0.0f, 0.0f};
                dfacc zc1{0.0f, 0.0f}, zy1{0.0f, 0.0f};
#pragma unroll
                for (int u = 0; u < LS_STEPS; ++u) {
                    const int t = odd ? LS_STEPS + u : u;
                    if (!odd && u == pp + 1) {
                        zca = zc0;
                        zya = zy0;
                        zc0 = {0.0f, 0.0f};
                        zy0 = {0.0f, 0.0f};
                    }
                    int j = t <= pp ? t : t - pp - 1;
                    j = j < K ? j : K - 1;  // the zero pad
                    const df e = ld_df(Lr + u * 32 + lane);
                    dfacc_add_prod(zc0, e, sc[wid][j]);
                    dfacc_add_prod(zy0, e, sy[wid][j]);
                }
                const df zc0v = dfacc_val(zc0), zy0v = dfacc_val(zy0);
                const df zcb = df_add_fast(zc0v, shfl_xor_df(zc0v, 1)), zyb = df_add_fast(zy0v, shfl_xor_df(zy0v, 1));
                df zc1v, zy1v;
                {
                    const int g = lane >> 2;
#pragma unroll
                    for (int t = 0; t < LS_TAIL; ++t) {
                        const int j = g + 8 * t < K ? g + 8 * t : K - 1;  // zero entries past the diagonal
                        const df e = ld_df(Lr + (LS_STEPS + t) * 32 + lane);
                        dfacc_add_prod(zc1, e, sc[wid][j]);
                        dfacc_add_prod(zy1, e, sy[wid][j]);
                    }
                    zc1v = dfacc_val(zc1);
                    zy1v = dfacc_val(zy1);
#pragma unroll
                    for (int o = 4; o < 32; o <<= 1) {
                        zc1v = df_add_fast(zc1v, shfl_xor_df(zc1v, o));
                        zy1v = df_add_fast(zy1v, shfl_xor_df(zy1v, o));
                    }
                }
                const df zcav = dfacc_val(zca), zyav = dfacc_val(zya);
                df v{0.0f, 0.0f}, qc{0.0f, 0.0f};
                if (!odd) {  // even lanes count rows p and 31 - p, lanes 0..3 rows 32..35, each once
                    v = df_add_fast(df_mul(zcav, zyav), df_mul(zcb, zyb));
                    qc = df_add_fast(df_mul(zcav, zcav), df_mul(zcb, zcb));
                }
                if (lane < K - 32) {
                    v = df_add_fast(v, df_mul(zc1v, zy1v));
                    qc = df_add_fast(qc, df_mul(zc1v, zc1v));
                }
#pragma unroll
                for (int o = 16; o > 0; o >>= 1) {
                    v = df_add_fast(v, shfl_xor_df(v, o));
                    qc = df_add_fast(qc, shfl_xor_df(qc, o));
                }
                const bool any_win = __any_sync(FULL, win);
                if (lane == 0) {
                    rv[wid][q] = v;
                    rq[wid][q] = qc;
                    rsl[wid][q] = sl;
                    rwin[wid][q] = any_win;
                }
            }
        }
        __syncwarp();
        if (lane < npt)
            finish_point(a, tile * 32 + lane, rsl[wid][lane], df_to(rv[wid][lane]), df_to(rq[wid][lane]),
                         rwin[wid][lane] != 0, n_win, n_nug, n_fail);
        __syncwarp();
    }
    // counts of every lane, summed over the warp
    const unsigned w_win = __reduce_add_sync(FULL, (unsigned)n_win);
    const unsigned w_nug = __reduce_add_sync(FULL, (unsigned)n_nug);
    const unsigned w_fail = __reduce_add_sync(FULL, (unsigned)n_fail);
    if (lane == 0 && a.counters) {
        if (w_win) atomicAdd(a.counters + CNT_WINDOW, (unsigned long long)w_win);
        if (w_nug) atomicAdd(a.counters + CNT_NUGGET, (unsigned long long)w_nug);
        if (w_fail) atomicAdd(a.counters + CNT_FAILED, (unsigned long long)w_fail);
    }
}

// ------------------------------------------- spin 1 and 2, double-float
// Mixed spin-s plans: a double-float frame table ((cos phi, sin phi), (z, s) as
// float pairs, 32 B per pixel) and complex double-float L^-1 blocks (float4 per
// entry: re.hi, re.lo, im.hi, im.lo); chords, correlation lookups, transport
// phases and the complex triangular products in double-float.
__global__ void pixframe_df_kernel(int64_t N, float4 *pvf) {
    const int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= 12 * N * N) return;
    double c, sn, z, s;
    pix_frame(N, p, c, sn, z, s);
    const df a = split_double(c), b = split_double(sn), d = split_double(z), e = split_double(s);
    pvf[2 * p] = make_float4(a.hi, a.lo, b.hi, b.lo);
    pvf[2 * p + 1] = make_float4(d.hi, d.lo, e.hi, e.lo);
}

__global__ void to_df_c_kernel(const double2 *src, float4 *dst, int64_t n) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const double2 v = src[i];
    const df r = split_double(v.x), m = split_double(v.y);
    dst[i] = make_float4(r.hi, r.lo, m.hi, m.lo);
}

// c = xi+(t)/xi+(0) exp(iS(a_tm - a_mt - pi)) and the field of member m in double-float
template <int S>
__device__ __forceinline__ bool member_s2_df(const ApplyArgs &a, int32_t m, df tx, df ty, df tz, df ts, df tc,
                                            df tsn, float tmaxf, Cx<df> &cv, Cx<df> &yv, bool &win) {
    if (m < 0) return false;
    const float4 f0 = __ldg(a.pvf + 2 * m), f1 = __ldg(a.pvf + 2 * m + 1);
    const df mc{f0.x, f0.y}, msn{f0.z, f0.w}, mz{f1.x, f1.y}, ms{f1.z, f1.w};
    const df mx = df_mul(ms, mc), my = df_mul(ms, msn);
    const df dx = df_add_fast(mx, df_neg(tx)), dy = df_add_fast(my, df_neg(ty)), dz = df_add_fast(mz, df_neg(tz));
    const df t = df_add_fast(df_add_fast(df_mul(dx, dx), df_mul(dy, dy)), df_mul(dz, dz));
    win |= t.hi > tmaxf;
    const df f = table_eval<df>(a.tab, t);
    const Cx<df> ph = pair_phase<df, S>(dx, dy, dz, tz, ts, tc, tsn, mz, ms, mc, msn);
    cv.re = df_mul(f, ph.re);
    cv.im = df_mul(f, ph.im);
    const double2 q = __ldg(reinterpret_cast<const double2 *>(a.map) + m);
    yv.re = split_double(q.x);
    yv.im = split_double(q.y);
    return true;
}

// z += e x for complex double-float e (imaginary part times msign) and x
__device__ __forceinline__ void cmac_df(dfacc &zr, dfacc &zi, const df er, const df ei, const df xr, const df xi) {
    dfacc_add_prod(zr, er, xr);
    dfacc_sub_prod(zr, ei, xi);
    dfacc_add_prod(zi, er, xi);
    dfacc_add_prod(zi, ei, xr);
}

__device__ __forceinline__ df shfl_df2(df v, int src) {
    return {__shfl_sync(FULL, v.hi, src), __shfl_sync(FULL, v.lo, src)};
}

template <int K, int S>
__global__ void __launch_bounds__(APPLY_WARPS * 32) apply_kernel_s2_df(ApplyArgs a) {
    __shared__ df stx[APPLY_WARPS][32], sty[APPLY_WARPS][32], stz[APPLY_WARPS][32];
    __shared__ df sts[APPLY_WARPS][32], stc[APPLY_WARPS][32], stn[APPLY_WARPS][32];
    __shared__ int64_t scp[APPLY_WARPS][32];
    constexpr int KS = K > GROUP ? K : 1;
    __shared__ df sxr[APPLY_WARPS][KS], sxi[APPLY_WARPS][KS], syr[APPLY_WARPS][KS], syi[APPLY_WARPS][KS];
    __shared__ df rvr[APPLY_WARPS][32], rvi[APPLY_WARPS][32], rq[APPLY_WARPS][32];
    __shared__ int32_t rsl[APPLY_WARPS][32];
    __shared__ unsigned char rwin[APPLY_WARPS][32];
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    const int64_t ntiles = (a.count + 31) / 32;
    const int64_t mirror_from = 6 * a.Nc * a.Nc + 2 * a.Nc;  // first pixel of coarse ring 2 Nc + 1
    const float tmaxf = (float)a.tab.t_max;
    const df zero{0.0f, 0.0f};
    unsigned long long n_win = 0, n_nug = 0, n_fail = 0;
    for (int64_t tile = (int64_t)blockIdx.x * APPLY_WARPS + wid; tile < ntiles;
         tile += (int64_t)gridDim.x * APPLY_WARPS) {
        {
            double x = 0.0, y = 0.0, z = 1.0;
            int64_t c = 0;
            target_of(a, tile * 32 + lane, x, y, z, c);
            const double sn = sqrt(x * x + y * y);
            scp[wid][lane] = c;
            stx[wid][lane] = split_double(x);
            sty[wid][lane] = split_double(y);
            stz[wid][lane] = split_double(z);
            sts[wid][lane] = split_double(sn);
            stc[wid][lane] = split_double(sn > 1e-12 ? x / sn : 1.0);
            stn[wid][lane] = split_double(sn > 1e-12 ? y / sn : 0.0);
        }
        __syncwarp();
        const int npt = a.count - tile * 32 < 32 ? (int)(a.count - tile * 32) : 32;
        if constexpr (K <= GROUP) {
            const int g = lane / GROUP, l = lane - g * GROUP, base = g * GROUP;
            for (int q0 = 0; q0 < npt; q0 += 3) {
                const int q = q0 + g;
                const bool has = g < 3 && q < npt;
                const int qq = has ? q : 0;
                const int64_t c = scp[wid][qq];
                const int32_t sl = has ? __ldg(a.slot + c) : 0;
                const bool mir = c >= mirror_from;
                Cx<df> cv{zero, zero}, yv{zero, zero};
                bool win = false;
                if (has && l < K)
                    member_s2_df<S>(a, __ldg(a.members + c * K + l), stx[wid][qq], sty[wid][qq], stz[wid][qq],
                                 sts[wid][qq], stc[wid][qq], stn[wid][qq], tmaxf, cv, yv, win);
                const float4 *Lr = reinterpret_cast<const float4 *>(a.linvf) + (int64_t)sl * linv_len(K);
                dfacc zcr{0.0f, 0.0f}, zci{0.0f, 0.0f}, zyr{0.0f, 0.0f}, zyi{0.0f, 0.0f};
#pragma unroll
                for (int j = 0; j < K; ++j) {
                    const df xr = shfl_df2(cv.re, base + j), xi = df_neg(shfl_df2(cv.im, base + j));
                    const df ur = shfl_df2(yv.re, base + j), ui = shfl_df2(yv.im, base + j);
                    if (has && l < K && l >= j) {
                        const float4 e4 = __ldg(Lr + col_start(K, j) + l - j);
                        const df er{e4.x, e4.y}, ei = mir ? df{-e4.z, -e4.w} : df{e4.z, e4.w};
                        cmac_df(zcr, zci, er, ei, xr, xi);
                        cmac_df(zyr, zyi, er, ei, ur, ui);
                    }
                }
                const df ar = dfacc_val(zcr), ai = dfacc_val(zci), br = dfacc_val(zyr), bi = dfacc_val(zyi);
                df vr = df_add_fast(df_mul(ar, br), df_mul(ai, bi));
                df vi = df_add_fast(df_mul(ar, bi), df_neg(df_mul(ai, br)));
                df qs = df_add_fast(df_mul(ar, ar), df_mul(ai, ai));
#pragma unroll
                for (int o = 8; o >= 1; o >>= 1) {
                    const df tr = shfl_df2(vr, lane + o), ti = shfl_df2(vi, lane + o), tq = shfl_df2(qs, lane + o);
                    if (l < o && l + o < GROUP) {
                        vr = df_add_fast(vr, tr);
                        vi = df_add_fast(vi, ti);
                        qs = df_add_fast(qs, tq);
                    }
                }
                const unsigned wb = __ballot_sync(FULL, win);
                if (has && l == 0) {
                    rvr[wid][q] = vr;
                    rvi[wid][q] = vi;
                    rq[wid][q] = qs;
                    rsl[wid][q] = sl;
                    rwin[wid][q] = ((wb >> base) & ((1u << GROUP) - 1u)) != 0;
                }
            }
        } else {
            static_assert(K == 36, "the lane-step layout is laid out for K = 36");
            for (int q = 0; q < npt; ++q) {
                const int64_t c = scp[wid][q];
                const int32_t sl = __ldg(a.slot + c);
                const bool mir = c >= mirror_from;
                const df tx = stx[wid][q], ty = sty[wid][q], tz = stz[wid][q];
                const df ts = sts[wid][q], tc = stc[wid][q], tn = stn[wid][q];
                const int32_t *mem = a.members + c * K;
                Cx<df> c0{zero, zero}, y0{zero, zero}, c1{zero, zero}, y1{zero, zero};
                bool win = false;
                member_s2_df<S>(a, __ldg(mem + lane), tx, ty, tz, ts, tc, tn, tmaxf, c0, y0, win);
                if (lane + 32 < K) member_s2_df<S>(a, __ldg(mem + lane + 32), tx, ty, tz, ts, tc, tn, tmaxf, c1, y1, win);
                const float4 *Lr = reinterpret_cast<const float4 *>(a.linvf) + (int64_t)sl * linv_len(K);
                __syncwarp();
                sxr[wid][lane] = c0.re;
                sxi[wid][lane] = df_neg(c0.im);
                syr[wid][lane] = y0.re;
                syi[wid][lane] = y0.im;
                if (lane < K - 32) {
                    sxr[wid][32 + lane] = c1.re;
                    sxi[wid][32 + lane] = df_neg(c1.im);
                    syr[wid][32 + lane] = y1.re;
                    syi[wid][32 + lane] = y1.im;
                }
                __syncwarp();
                const int pp = lane >> 1, odd = lane & 1;
                dfacc acr{0.0f, 0.0f}, aci{0.0f, 0.0f}, ayr{0.0f, 0.0f}, ayi{0.0f, 0.0f};
                dfacc zcr{0.0f, 0.0f}, zci{0.0f, 0.0f}, zyr{0.0f, 0.0f}, zyi{0.0f, 0.0f};
#pragma unroll
                for (int u = 0; u < LS_STEPS; ++u) {
                    const int t = odd ? LS_STEPS + u : u;
                    if (!odd && u == pp + 1) {
                        acr = zcr;
                        aci = zci;
                        ayr = zyr;
                        ayi = zyi;
                        zcr = zci = zyr = zyi = dfacc{0.0f, 0.0f};
                    }
                    int j = t <= pp ? t : t - pp - 1;
                    j = j < K ? j : K - 1;  // the zero pad
                    const float4 e4 = __ldg(Lr + u * 32 + lane);
                    const df er{e4.x, e4.y}, ei = mir ? df{-e4.z, -e4.w} : df{e4.z, e4.w};
                    cmac_df(zcr, zci, er, ei, sxr[wid][j], sxi[wid][j]);
                    cmac_df(zyr, zyi, er, ei, syr[wid][j], syi[wid][j]);
                }
                const df b0r = dfacc_val(zcr), b0i = dfacc_val(zci), b1r = dfacc_val(zyr), b1i = dfacc_val(zyi);
                const df bcr = df_add_fast(b0r, shfl_xor_df(b0r, 1)), bci = df_add_fast(b0i, shfl_xor_df(b0i, 1));
                const df byr = df_add_fast(b1r, shfl_xor_df(b1r, 1)), byi = df_add_fast(b1i, shfl_xor_df(b1i, 1));
                dfacc tcr{0.0f, 0.0f}, tci{0.0f, 0.0f}, tyr{0.0f, 0.0f}, tyi{0.0f, 0.0f};
                {
                    const int g = lane >> 2;
#pragma unroll
                    for (int t = 0; t < LS_TAIL; ++t) {
                        const int j = g + 8 * t < K ? g + 8 * t : K - 1;  // zero entries past the diagonal
                        const float4 e4 = __ldg(Lr + (LS_STEPS + t) * 32 + lane);
                        const df er{e4.x, e4.y}, ei = mir ? df{-e4.z, -e4.w} : df{e4.z, e4.w};
                        cmac_df(tcr, tci, er, ei, sxr[wid][j], sxi[wid][j]);
                        cmac_df(tyr, tyi, er, ei, syr[wid][j], syi[wid][j]);
                    }
                }
                df t1r = dfacc_val(tcr), t1i = dfacc_val(tci), t2r = dfacc_val(tyr), t2i = dfacc_val(tyi);
#pragma unroll
                for (int o = 4; o < 32; o <<= 1) {
                    t1r = df_add_fast(t1r, shfl_xor_df(t1r, o));
                    t1i = df_add_fast(t1i, shfl_xor_df(t1i, o));
                    t2r = df_add_fast(t2r, shfl_xor_df(t2r, o));
                    t2i = df_add_fast(t2i, shfl_xor_df(t2i, o));
                }
                const df aar = dfacc_val(acr), aai = dfacc_val(aci), abr = dfacc_val(ayr), abi = dfacc_val(ayi);
                df vr = zero, vi = zero, qc = zero;
                if (!odd) {  // even lanes count rows p and 31 - p, lanes 0..3 rows 32..35, each once
                    vr = df_add_fast(df_add_fast(df_mul(aar, abr), df_mul(aai, abi)),
                                     df_add_fast(df_mul(bcr, byr), df_mul(bci, byi)));
                    vi = df_add_fast(df_add_fast(df_mul(aar, abi), df_neg(df_mul(aai, abr))),
                                     df_add_fast(df_mul(bcr, byi), df_neg(df_mul(bci, byr))));
                    qc = df_add_fast(df_add_fast(df_mul(aar, aar), df_mul(aai, aai)),
                                     df_add_fast(df_mul(bcr, bcr), df_mul(bci, bci)));
                }
                if (lane < K - 32) {
                    vr = df_add_fast(vr, df_add_fast(df_mul(t1r, t2r), df_mul(t1i, t2i)));
                    vi = df_add_fast(vi, df_add_fast(df_mul(t1r, t2i), df_neg(df_mul(t1i, t2r))));
                    qc = df_add_fast(qc, df_add_fast(df_mul(t1r, t1r), df_mul(t1i, t1i)));
                }
#pragma unroll
                for (int o = 16; o > 0; o >>= 1) {
                    vr = df_add_fast(vr, shfl_xor_df(vr, o));
                    vi = df_add_fast(vi, shfl_xor_df(vi, o));
                    qc = df_add_fast(qc, shfl_xor_df(qc, o));
                }
                const bool any_win = __any_sync(FULL, win);
                if (lane == 0) {
                    rvr[wid][q] = vr;
                    rvi[wid][q] = vi;
                    rq[wid][q] = qc;
                    rsl[wid][q] = sl;
                    rwin[wid][q] = any_win;
                }
            }
        }
        __syncwarp();
        if (lane < npt)
            finish_point_s2(a, tile * 32 + lane, rsl[wid][lane], df_to(rvr[wid][lane]), df_to(rvi[wid][lane]),
                            df_to(rq[wid][lane]), rwin[wid][lane] != 0, n_win, n_nug, n_fail);
        __syncwarp();
    }
    const unsigned w_win = __reduce_add_sync(FULL, (unsigned)n_win);
    const unsigned w_nug = __reduce_add_sync(FULL, (unsigned)n_nug);
    const unsigned w_fail = __reduce_add_sync(FULL, (unsigned)n_fail);
    if (lane == 0 && a.counters) {
        if (w_win) atomicAdd(a.counters + CNT_WINDOW, (unsigned long long)w_win);
        if (w_nug) atomicAdd(a.counters + CNT_NUGGET, (unsigned long long)w_nug);
        if (w_fail) atomicAdd(a.counters + CNT_FAILED, (unsigned long long)w_fail);
    }
}

}  // namespace paper
}  // namespace flints

using namespace flints;
using namespace flints::paper;

struct flints_paper_s {
    int device;
    int64_t nside, nside_c, nslot;
    int y, K, lmax, n;
    double t_max, h, inv_h, xi0, max_pair_t;
    int64_t nugget_slots, failed_slots;
    double *d_cl, *d_f, *d_g, *d_fm, *d_gm;
    Coef64 *d_c64;
    float4 *d_c32;
    int32_t *d_members, *d_slot;
    int *d_steps, *d_scratch;
    double *d_linv;
    double2 *d_pv;
    float4 *d_pvf;
    float2 *d_linvf;
    int precision, spin;
    unsigned flags;
    double *d_clbb;
    Coef64 *d_cm64;
    float4 *d_cm32;
    unsigned long long *d_counters, *d_maxt;
    int64_t points;
    int64_t device_bytes;  // sum of the plan's device allocations
};

static thread_local char g_perr[512] = "no error";

static int pfail(int code, const char *fmt, ...) {
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(g_perr, sizeof g_perr, fmt, ap);
    va_end(ap);
    return code;
}

static int pcuda(cudaError_t e, const char *what) {
    return pfail(e == cudaErrorMemoryAllocation ? FLINTS_ENOMEM : FLINTS_ECUDA, "%s: %s", what, cudaGetErrorString(e));
}

static void paper_release(flints_paper_s *p) {
    cudaFree(p->d_cl);
    cudaFree(p->d_f);
    cudaFree(p->d_g);
    cudaFree(p->d_fm);
    cudaFree(p->d_gm);
    cudaFree(p->d_c64);
    cudaFree(p->d_c32);
    cudaFree(p->d_members);
    cudaFree(p->d_slot);
    cudaFree(p->d_steps);
    cudaFree(p->d_scratch);
    cudaFree(p->d_linv);
    cudaFree(p->d_pv);
    cudaFree(p->d_clbb);
    cudaFree(p->d_cm64);
    cudaFree(p->d_cm32);
    cudaFree(p->d_pvf);
    cudaFree(p->d_linvf);
    cudaFree(p->d_counters);
    cudaFree(p->d_maxt);
}

// interval count of the xi table on [0, t_max]: the cubic Hermite error bound
// h^4/384 max|f4| below 1e-11 (f4 bounded through the fourth derivatives of
// P_l at 1, weights |C_l| (+ |C_l^BB| for spin 2)), a power of two in [64, 65536]
static int table_intervals(const double *cl, const double *cl_bb, int lmax, double t_max) {
    double x0 = 0.0, b4num = 0.0;
    for (int l = 0; l <= lmax; ++l) {
        const double ld = (double)l;
        const double a = (2.0 * ld + 1.0) / (4.0 * PI) * (std::fabs(cl[l]) + (cl_bb ? std::fabs(cl_bb[l]) : 0.0));
        x0 += a;
        if (l >= 4) b4num += a * ((ld - 3) * (ld - 2) * (ld - 1) * ld * (ld + 1) * (ld + 2) * (ld + 3) * (ld + 4) / 384.0);
    }
    const double b4 = x0 > 0 ? b4num / 16.0 / x0 : 0.0;
    if (!(b4 > 0)) return 64;
    const double h = std::pow(384.0 * 1e-11 / b4, 0.25);
    const double want = std::ceil(std::log2(t_max / h));
    return want > 16 ? 65536 : (want < 6 ? 64 : (1 << (int)want));
}

extern "C" {

const char *flints_paper_last_error(void) { return g_perr; }

int flints_paper_plan(flints_paper_t *out, int64_t nside, int lmax, const double *cl, const double *cl_bb, int y,
                      int spin, int precision, unsigned flags, void *stream) {
    if (!out) return pfail(FLINTS_EINVAL, "flints_paper_plan: out is NULL");
    *out = nullptr;
    if (y != 1 && y != 2) return pfail(FLINTS_EINVAL, "flints_paper_plan: level y must be 1 or 2 (got %d)", y);
    const int k = 1 << (y - 1);
    if (nside < 1 || nside > 8192 || nside % k != 0)
        return pfail(FLINTS_EINVAL, "flints_paper_plan: nside %lld must be in [1, 8192] and divisible by %d",
                     (long long)nside, k);
    if (lmax < 0 || lmax > 16384) return pfail(FLINTS_EINVAL, "flints_paper_plan: lmax %d outside [0, 16384]", lmax);
    if (!cl) return pfail(FLINTS_EINVAL, "flints_paper_plan: cl is NULL");
    if (precision != FLINTS_FP64 && precision != FLINTS_MIXED)
        return pfail(FLINTS_EINVAL, "flints_paper_plan: precision must be FLINTS_FP64 or FLINTS_MIXED");
    if (spin < 0 || spin > 2) return pfail(FLINTS_EINVAL, "flints_paper_plan: spin must be 0, 1 or 2 (got %d)", spin);
    if (flags & ~(unsigned)FLINTS_SPIN2_AUGMENTED)
        return pfail(FLINTS_EINVAL, "flints_paper_plan: unknown flag bits 0x%x", flags);
    const bool aug = (flags & FLINTS_SPIN2_AUGMENTED) != 0;
    if (aug && (spin != 2 || precision != FLINTS_FP64))
        return pfail(FLINTS_EINVAL, "flints_paper_plan: FLINTS_SPIN2_AUGMENTED needs a spin-2 FP64 plan");
    if (spin == 0) cl_bb = nullptr;
    for (int l = 0; l <= lmax; ++l)
        if (!std::isfinite(cl[l]) || (cl_bb && !std::isfinite(cl_bb[l])))
            return pfail(FLINTS_EINVAL, "flints_paper_plan: non-finite spectrum value at l = %d", l);
    cudaStream_t st = (cudaStream_t)stream;
    flints_paper_s *p = new flints_paper_s();
    std::memset(p, 0, sizeof *p);
    cudaGetDevice(&p->device);
    p->nside = nside;
    p->nside_c = nside / k;
    p->y = y;
    p->K = 9 * k * k;
    p->lmax = lmax;
    p->precision = precision;
    p->spin = spin;
    p->flags = flags;
    p->nslot = slot_count(p->nside_c);
    const double Dc = 7.0 / (double)p->nside_c;
    p->t_max = Dc * Dc < 4.0 ? Dc * Dc : 4.0;  // 4: the chord^2 of antipodal points
    p->n = table_intervals(cl, cl_bb, lmax, p->t_max);
    p->h = p->t_max / p->n;
    p->inv_h = p->n / p->t_max;
    const int64_t npc = 12 * p->nside_c * p->nside_c;
    const size_t nn = (size_t)p->n + 1;
    cudaError_t e;
    auto bail = [&](cudaError_t err, const char *what) {
        paper_release(p);
        delete p;
        return pcuda(err, what);
    };
#define PALLOC(ptr, bytes)                                                                                   \
    do {                                                                                                     \
        if ((e = cudaMalloc((void **)&(ptr), (bytes))) != cudaSuccess) return bail(e, "flints_paper_plan: cudaMalloc"); \
        p->device_bytes += (int64_t)(bytes);                                                                 \
    } while (0)
    PALLOC(p->d_cl, (size_t)(lmax + 1) * sizeof(double));
    PALLOC(p->d_f, nn * sizeof(double));
    PALLOC(p->d_g, nn * sizeof(double));
    PALLOC(p->d_fm, nn * sizeof(double));
    PALLOC(p->d_gm, nn * sizeof(double));
    PALLOC(p->d_c64, (size_t)p->n * sizeof(Coef64));
    PALLOC(p->d_c32, (size_t)p->n * 2 * sizeof(float4));
    PALLOC(p->d_members, (size_t)npc * p->K * sizeof(int32_t));
    PALLOC(p->d_slot, (size_t)npc * sizeof(int32_t));
    PALLOC(p->d_steps, (size_t)p->nslot * sizeof(int));
    PALLOC(p->d_scratch, 4 * sizeof(int));
    const int64_t lv = aug ? (int64_t)(2 * p->K) * (2 * p->K + 1) / 2 : (int64_t)linv_len(p->K) * (spin != 0 ? 2 : 1);
    PALLOC(p->d_linv, (size_t)p->nslot * lv * sizeof(double));
    if (aug) {
        PALLOC(p->d_cm64, (size_t)p->n * sizeof(Coef64));
        PALLOC(p->d_cm32, (size_t)p->n * 2 * sizeof(float4));
    }
    if (cl_bb) PALLOC(p->d_clbb, (size_t)(lmax + 1) * sizeof(double));
    if (precision == FLINTS_MIXED) {
        PALLOC(p->d_pvf, (size_t)12 * nside * nside * 2 * sizeof(float4));
        PALLOC(p->d_linvf, (size_t)p->nslot * linv_len(p->K) * (spin != 0 ? 2 : 1) * sizeof(float2));
    } else {
        PALLOC(p->d_pv, (size_t)12 * nside * nside * 2 * sizeof(double2));
    }
    PALLOC(p->d_counters, CNT_N * sizeof(unsigned long long));
    PALLOC(p->d_maxt, sizeof(unsigned long long));
#undef PALLOC
    if ((e = cudaMemcpyAsync(p->d_cl, cl, (size_t)(lmax + 1) * sizeof(double), cudaMemcpyHostToDevice, st)) !=
        cudaSuccess)
        return bail(e, "flints_paper_plan: copy cl");
    if (cl_bb &&
        (e = cudaMemcpyAsync(p->d_clbb, cl_bb, (size_t)(lmax + 1) * sizeof(double), cudaMemcpyHostToDevice, st)) !=
            cudaSuccess)
        return bail(e, "flints_paper_plan: copy cl_bb");
    if ((e = cudaMemsetAsync(p->d_fm, 0, nn * sizeof(double), st)) != cudaSuccess) return bail(e, "memset");
    if ((e = cudaMemsetAsync(p->d_gm, 0, nn * sizeof(double), st)) != cudaSuccess) return bail(e, "memset");
    if ((e = cudaMemsetAsync(p->d_scratch, 0, 4 * sizeof(int), st)) != cudaSuccess) return bail(e, "memset");
    if ((e = cudaMemsetAsync(p->d_counters, 0, CNT_N * sizeof(unsigned long long), st)) != cudaSuccess)
        return bail(e, "memset");
    if ((e = cudaMemsetAsync(p->d_maxt, 0, sizeof(unsigned long long), st)) != cudaSuccess) return bail(e, "memset");
    if ((e = launch_xi_table(spin, lmax, p->d_cl, p->d_clbb, p->t_max, p->n, p->d_f, p->d_g, p->d_fm, p->d_gm, st)) !=
        cudaSuccess)
        return bail(e, "flints_paper_plan: xi table kernel");
    double xi0 = 0.0;
    if ((e = cudaMemcpyAsync(&xi0, p->d_f, sizeof(double), cudaMemcpyDeviceToHost, st)) != cudaSuccess)
        return bail(e, "flints_paper_plan: read xi(0)");
    if ((e = cudaStreamSynchronize(st)) != cudaSuccess) return bail(e, "flints_paper_plan: xi table");
    if (!(xi0 > 0.0) || !std::isfinite(xi0)) {
        paper_release(p);
        delete p;
        return pfail(FLINTS_EINVAL, "flints_paper_plan: xi(0) = %g is not positive", xi0);
    }
    p->xi0 = xi0;
    if ((e = finish_table(p->d_f, p->d_g, p->n, p->h, xi0, p->d_c64, p->d_c32, st)) != cudaSuccess)
        return bail(e, "flints_paper_plan: table coefficients");
    if (aug && (e = finish_table(p->d_fm, p->d_gm, p->n, p->h, xi0, p->d_cm64, p->d_cm32, st)) != cudaSuccess)
        return bail(e, "flints_paper_plan: xi- table coefficients");
    if (precision == FLINTS_MIXED && spin != 0)
        pixframe_df_kernel<<<(unsigned)((12 * nside * nside + 255) / 256), 256, 0, st>>>(nside, p->d_pvf);
    else if (precision == FLINTS_MIXED)
        pixvec_df_kernel<<<(unsigned)((12 * nside * nside + 255) / 256), 256, 0, st>>>(nside, p->d_pvf);
    else if (spin != 0)
        pixframe_kernel<<<(unsigned)((12 * nside * nside + 255) / 256), 256, 0, st>>>(nside, p->d_pv);
    else
        pixvec_kernel<<<(unsigned)((12 * nside * nside + 255) / 256), 256, 0, st>>>(nside, p->d_pv);
    if ((e = cudaGetLastError()) != cudaSuccess) return bail(e, "flints_paper_plan: pixel vector kernel");
    stencil_kernel<<<(unsigned)((npc + 127) / 128), 128, 0, st>>>(p->nside_c, k, p->K, p->d_members, p->d_slot,
                                                                 p->d_scratch + 2);
    if ((e = cudaGetLastError()) != cudaSuccess) return bail(e, "flints_paper_plan: stencil kernel");
    LinvArgs sa{};
    sa.Nc = p->nside_c;
    sa.N = nside;
    sa.nslot = p->nslot;
    sa.K = p->K;
    sa.members = p->d_members;
    sa.tab.c64 = p->d_c64;
    sa.tab.c32 = p->d_c32;
    sa.tab.t_max = p->t_max;
    sa.tab.inv_h = p->inv_h;
    sa.tab.inv_h_hi = (float)p->inv_h;
    sa.tab.inv_h_lo = (float)(p->inv_h - (double)sa.tab.inv_h_hi);
    sa.tab.n = p->n;
    sa.linv = p->d_linv;
    sa.slot_steps = p->d_steps;
    sa.max_t = p->d_maxt;
    sa.counts = p->d_scratch;
    const int64_t grid = p->nslot < 152 * 16 ? p->nslot : 152 * 16;
    if (aug) {
        TableDev tm = sa.tab;
        tm.c64 = p->d_cm64;
        tm.c32 = p->d_cm32;
        const size_t dsm = (size_t)2 * (2 * p->K) * (2 * p->K + 1) * sizeof(double);
        if ((e = cudaFuncSetAttribute(linv_kernel_aug, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)dsm)) !=
            cudaSuccess)
            return bail(e, "flints_paper_plan: shared memory of the augmented factor");
        linv_kernel_aug<<<(unsigned)grid, SINV_THREADS, dsm, st>>>(sa, tm, p->d_linv);
    } else if (spin == 2)
        linv_kernel_c<2><<<(unsigned)grid, SINV_THREADS, 0, st>>>(sa, reinterpret_cast<double2 *>(p->d_linv));
    else if (spin == 1)
        linv_kernel_c<1><<<(unsigned)grid, SINV_THREADS, 0, st>>>(sa, reinterpret_cast<double2 *>(p->d_linv));
    else
        linv_kernel<<<(unsigned)grid, SINV_THREADS, 0, st>>>(sa);
    if ((e = cudaGetLastError()) != cudaSuccess) return bail(e, "flints_paper_plan: L^-1 kernel");
    if (precision == FLINTS_MIXED) {
        const int64_t nl = p->nslot * (int64_t)linv_len(p->K);
        if (spin != 0)
            to_df_c_kernel<<<(unsigned)((nl + 255) / 256), 256, 0, st>>>(reinterpret_cast<const double2 *>(p->d_linv),
                                                                        reinterpret_cast<float4 *>(p->d_linvf), nl);
        else
            to_df_kernel<<<(unsigned)((nl + 255) / 256), 256, 0, st>>>(p->d_linv, p->d_linvf, nl);
        if ((e = cudaGetLastError()) != cudaSuccess) return bail(e, "flints_paper_plan: double-float L^-1");
    }
    int scratch[4] = {0, 0, 0, 0};
    unsigned long long maxt = 0;
    if ((e = cudaMemcpyAsync(scratch, p->d_scratch, sizeof scratch, cudaMemcpyDeviceToHost, st)) != cudaSuccess)
        return bail(e, "flints_paper_plan: read counts");
    if ((e = cudaMemcpyAsync(&maxt, p->d_maxt, sizeof maxt, cudaMemcpyDeviceToHost, st)) != cudaSuccess)
        return bail(e, "flints_paper_plan: read chord bound");
    if ((e = cudaStreamSynchronize(st)) != cudaSuccess) return bail(e, "flints_paper_plan: tabulation");
    double mt;
    std::memcpy(&mt, &maxt, sizeof mt);
    p->max_pair_t = mt;
    p->nugget_slots = scratch[0];
    p->failed_slots = scratch[1];
    if (scratch[2] != 0) {
        paper_release(p);
        delete p;
        return pfail(FLINTS_EINVAL, "flints_paper_plan: %d coarse pixels with an inconsistent neighbour set", scratch[2]);
    }
    if (mt > p->t_max) {
        paper_release(p);
        delete p;
        return pfail(FLINTS_EINVAL, "flints_paper_plan: stencil chord^2 %g exceeds the table domain %g", mt, p->t_max);
    }
    if (precision == FLINTS_MIXED) {  // only the double-float blocks are kept
        cudaFree(p->d_linv);
        p->d_linv = nullptr;
        p->device_bytes -= (int64_t)((size_t)p->nslot * lv * sizeof(double));
    }
    *out = p;
    return FLINTS_OK;
}

void flints_paper_free(flints_paper_t p) {
    if (!p) return;
    int cur = 0;
    cudaGetDevice(&cur);
    if (cur != p->device) cudaSetDevice(p->device);
    paper_release(p);
    if (cur != p->device) cudaSetDevice(cur);
    delete p;
}

static int paper_run(flints_paper_t p, int64_t nside_tgt, int64_t first, int64_t count, const double *map,
                     const double *defl, double *out, double *var, uint8_t *status, void *stream) {
    if (!p) return pfail(FLINTS_EINVAL, "plan is NULL");
    int cur = -1;
    cudaGetDevice(&cur);
    if (cur != p->device) return pfail(FLINTS_EINVAL, "plan was created on device %d, current device is %d", p->device, cur);
    if (nside_tgt < 0 || nside_tgt > 16384) return pfail(FLINTS_EINVAL, "nside_out %lld outside [1, 16384]", (long long)nside_tgt);
    const int64_t nt = nside_tgt > 0 ? nside_tgt : p->nside;
    const int64_t npix = 12 * nt * nt;
    if (first < 0 || count < 0 || first > npix || count > npix - first)
        return pfail(FLINTS_EINVAL, "target range [%lld, %lld) outside [0, %lld)", (long long)first,
                     (long long)(first + count), (long long)npix);
    if (count == 0) return FLINTS_OK;
    if (!map || !out) return pfail(FLINTS_EINVAL, "map and out must not be NULL");
    if (nside_tgt == 0 && !defl) return pfail(FLINTS_EINVAL, "defl is NULL");
    const uintptr_t need = p->spin != 0 ? 15u : 7u;
    if (((uintptr_t)defl & 15u) || (((uintptr_t)map | (uintptr_t)out) & need) || ((uintptr_t)var & 7u))
        return pfail(FLINTS_EINVAL, "defl (and spin-2 map and out) must be 16-byte aligned, map, out and var 8-byte "
                                    "aligned");
    ApplyArgs a{};
    a.N = p->nside;
    a.Nc = p->nside_c;
    a.first = first;
    a.count = count;
    a.nside_tgt = nside_tgt;
    a.map = map;
    a.defl = defl;
    a.out = out;
    a.var = var;
    a.status = status;
    a.members = p->d_members;
    a.slot = p->d_slot;
    a.linv = p->d_linv;
    a.pv = p->d_pv;
    a.pvf = p->d_pvf;
    a.linvf = p->d_linvf;
    a.slot_steps = p->d_steps;
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
    a.counters = p->d_counters;
    const int64_t tiles = (count + 31) / 32;
    const int64_t want = (tiles + APPLY_WARPS - 1) / APPLY_WARPS;
    const int64_t cap = (int64_t)device_sm_count() * 16;
    const unsigned grid = (unsigned)(want < cap ? want : cap);
    cudaStream_t st = (cudaStream_t)stream;
    const bool mixed = p->precision == FLINTS_MIXED;
    if (p->flags & FLINTS_SPIN2_AUGMENTED) {
        if (p->K == 9)
            apply_kernel_aug<9><<<grid, APPLY_WARPS * 32, 0, st>>>(a);
        else
            apply_kernel_aug<36><<<grid, APPLY_WARPS * 32, 0, st>>>(a);
    } else if (p->spin != 0) {
        const bool k9 = p->K == 9, s2 = p->spin == 2;
        if (mixed) {
            if (k9) {
                if (s2) apply_kernel_s2_df<9, 2><<<grid, APPLY_WARPS * 32, 0, st>>>(a);
                else apply_kernel_s2_df<9, 1><<<grid, APPLY_WARPS * 32, 0, st>>>(a);
            } else {
                if (s2) apply_kernel_s2_df<36, 2><<<grid, APPLY_WARPS * 32, 0, st>>>(a);
                else apply_kernel_s2_df<36, 1><<<grid, APPLY_WARPS * 32, 0, st>>>(a);
            }
        } else {
            if (k9) {
                if (s2) apply_kernel_s2<9, 2><<<grid, APPLY_WARPS * 32, 0, st>>>(a);
                else apply_kernel_s2<9, 1><<<grid, APPLY_WARPS * 32, 0, st>>>(a);
            } else {
                if (s2) apply_kernel_s2<36, 2><<<grid, APPLY_WARPS * 32, 0, st>>>(a);
                else apply_kernel_s2<36, 1><<<grid, APPLY_WARPS * 32, 0, st>>>(a);
            }
        }
    } else if (p->K == 9) {
        if (mixed)
            apply_kernel_df<9><<<grid, APPLY_WARPS * 32, 0, st>>>(a);
        else
            apply_kernel<9><<<grid, APPLY_WARPS * 32, 0, st>>>(a);
    } else {
        if (mixed)
            apply_kernel_df<36><<<grid, APPLY_WARPS * 32, 0, st>>>(a);
        else
            apply_kernel<36><<<grid, APPLY_WARPS * 32, 0, st>>>(a);
    }
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return pcuda(e, "paper apply kernel launch");
    p->points += count;
    return FLINTS_OK;
}

int flints_paper_lens(flints_paper_t p, int64_t first, int64_t count, const double *map, const double *defl,
                      double *out, double *var, uint8_t *status, void *stream) {
    return paper_run(p, 0, first, count, map, defl, out, var, status, stream);
}

int flints_paper_supersample(flints_paper_t p, int64_t nside_out, int64_t first, int64_t count, const double *map,
                             double *out, double *var, uint8_t *status, void *stream) {
    if (nside_out < 1) return pfail(FLINTS_EINVAL, "nside_out must be positive");
    return paper_run(p, nside_out, first, count, map, nullptr, out, var, status, stream);
}

int flints_paper_get_info(flints_paper_t p, flints_paper_info *info, void *stream) {
    if (!p || !info) return pfail(FLINTS_EINVAL, "plan and info must not be NULL");
    unsigned long long c[CNT_N];
    cudaError_t e = cudaMemcpyAsync(c, p->d_counters, sizeof c, cudaMemcpyDeviceToHost, (cudaStream_t)stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize((cudaStream_t)stream);
    if (e != cudaSuccess) return pcuda(e, "flints_paper_get_info");
    info->nside = p->nside;
    info->nside_coarse = p->nside_c;
    info->y = p->y;
    info->K = p->K;
    info->slots = p->nslot;
    info->t_max = p->t_max;
    info->n_intervals = p->n;
    info->xi0 = p->xi0;
    info->table_bytes = (int64_t)p->nslot * linv_len(p->K) * 8 +
                        12 * p->nside_c * p->nside_c * (int64_t)(p->K + 1) * 4 + 12 * p->nside * p->nside * 32;
    info->precision = p->precision;
    info->spin = p->spin;
    info->flags = p->flags;
    if (p->flags & FLINTS_SPIN2_AUGMENTED)
        info->table_bytes += (int64_t)p->nslot * ((2 * p->K) * (2 * p->K + 1) / 2 - linv_len(p->K)) * 8;
    else if (p->spin != 0)
        info->table_bytes += (int64_t)p->nslot * linv_len(p->K) * 8;
    info->max_pair_t = p->max_pair_t;
    info->nugget_slots = p->nugget_slots;
    info->failed_slots = p->failed_slots;
    info->points = p->points;
    info->window = (int64_t)c[CNT_WINDOW];
    info->device_bytes = p->device_bytes;
    return FLINTS_OK;
}

int flints_paper_tables(flints_paper_t p, int32_t *members, int32_t *slot, double *linv, void *stream) {
    if (!p) return pfail(FLINTS_EINVAL, "plan is NULL");
    if (linv && !p->d_linv)  // refused before any copy is queued
        return pfail(FLINTS_EINVAL, "flints_paper_tables: mixed plans keep only double-float L^-1 blocks");
    cudaStream_t st = (cudaStream_t)stream;
    const int64_t npc = 12 * p->nside_c * p->nside_c;
    cudaError_t e = cudaSuccess;
    if (members)
        e = cudaMemcpyAsync(members, p->d_members, (size_t)npc * p->K * sizeof(int32_t), cudaMemcpyDeviceToDevice, st);
    if (e == cudaSuccess && slot)
        e = cudaMemcpyAsync(slot, p->d_slot, (size_t)npc * sizeof(int32_t), cudaMemcpyDeviceToDevice, st);
    if (e == cudaSuccess && linv)
        e = cudaMemcpyAsync(linv, p->d_linv,
                            (size_t)p->nslot *
                                ((p->flags & FLINTS_SPIN2_AUGMENTED) ? (2 * p->K) * (2 * p->K + 1) / 2
                                                                      : linv_len(p->K) * (p->spin != 0 ? 2 : 1)) *
                                sizeof(double),
                            cudaMemcpyDeviceToDevice, st);
    if (e != cudaSuccess) return pcuda(e, "flints_paper_tables");
    return FLINTS_OK;
}

}  // extern "C"

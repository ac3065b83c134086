// Fused lensing-remap kernel: one warp per target point (Secs. 2.1-2.5, 3.1).
//
// Per tile of up to 16 (MAX_TILE_POINTS) consecutive RING targets a warp first
// displaces all of them (one per lane, FP64), then, point by point:
//   1. stencil search: the rings whose circle comes within the search radius r
//      of n' (one ring per lane), the pixel range of each ring that can lie
//      inside the disc, candidates enumerated in increasing RING index;
//   2. exact K-nearest selection: FP32 keys of all candidates pre-select, FP64
//      squared chords of the selected (or near-tied) ones decide, warp bitonic
//      sorts on (chord^2, RING index); the K-th chord must lie inside the disc;
//   3. covariance assembly S_ij = xi(t_ij)/xi(0) (+ nugget on the diagonal)
//      and c_i = xi(t_i)/xi(0), spin 2 with the parallel-transport phase
//      exp(2i(a_ij - a_ji)); lower triangle spread over the lanes;
//   4. Cholesky of the matrix bordered by the right-hand-side rows c and y,
//      so that the factor's bordered rows are the forward solves z_c, z_y:
//      right-looking in FP64 for N <= 32 (all lanes share the rank-one
//      updates), split left-looking otherwise and in double-float (anchored
//      accumulators); the nugget is doubled while a pivot is not positive
//      (Sec. 2.4);
//   5. value = z_c^H z_y, variance = xi(0) (1 - |z_c|^2) (Eqs.
//      best_temperature_field, gaussvar, major_eq, gaussvar_pol).
// Precision R = double (FP64 path) or df (double-float on the FP32 pipe, the
// mixed path: FP64 geometry and selection, double-float assembly, factor and
// solves, FP64 fallback for points whose double-float factor fails).
#pragma once
#include <cstddef>
#include <type_traits>

#include "common.cuh"

namespace flints {

template <class T>
struct Cx {
    T re, im;
};

template <int K>
struct Shape {
    static constexpr int NSLOT = K > 32 ? 256 : 128;  // candidate slots
    static constexpr int SPL = NSLOT / 32;            // slots per lane
    static constexpr int RPL = (K + 31) / 32;         // matrix rows per lane
    static constexpr int LD = K + 1;                  // padded row stride
    static constexpr int NTRI = K * (K + 1) / 2;
};

struct PointA {
    double x, y, z, s, cph, sph, phi;
    double rot_re, rot_im;  // spin 2: parallel-transport phase from the frame at n' to the frame at n
    int64_t ic;
    int flags;
    float zf, sf, phif;  // FP32 copies for the candidate-range arithmetic
};

struct RingRec {
    double z, s, f;
    double inv2nq;  // 1 / (2 nq): pixel j of the ring sits at phi = pi (j + f) inv2nq
    int64_t first;
    int n_in, j0, cnt, end, jref;
    // FP32 pre-selection key of pixel j of this ring:
    //   a32 + b32 sin^2(pi (j - jref + frac) / n_in)
    float a32, b32, frac, inv_n;
};

template <int K, int SPIN, class R>
struct WarpSmem {
    using Elem = typename std::conditional<SPIN == 1 || SPIN == 2, Cx<typename Ops<R>::T>, typename Ops<R>::T>::type;
    static constexpr int NSLOT = Shape<K>::NSLOT;
    // packed lower triangle of S + n I (row i starts at i(i+1)/2), then the two
    // bordered right-hand-side rows (c and y), K entries each; the augmented
    // spin-2 system is real, 2K x 2K, with three bordered rows (Q and U
    // cross-covariances of the target, and the data)
    static constexpr int MAT = SPIN == SPIN2_AUG ? (2 * K) * (2 * K + 1) / 2 + 3 * (2 * K) : K * (K + 1) / 2 + 2 * K;
    using T = typename Ops<R>::T;
    PointA pts[MAX_TILE_POINTS];
    // neighbour offsets X_i - n', and neighbour z, sin(theta), cos(phi), sin(phi),
    // in the solve's precision (FP64 or double-float; both 8 bytes, so the two
    // views of a warp's slice share every offset)
    T gx[K], gy[K], gz[K], gnz[K], gns[K], gnc[K], gnsn[K];
    // spin 2: per-neighbour target phase Phi0_i = phase(n' -> X_i), tangent-plane
    // coordinates (u, v) of X_i - n' at n', and squared chords to n'
    typename Ops<R>::T p0r[K], p0i[K], pu[K], pv[K];
    float ktf[K];  // squared chords to n' (FP32, for the spherical-excess correction)
    union U {
        struct Cand {
            RingRec rings[32];
            double cx[NSLOT], cy[NSLOT], cz[NSLOT], cc[NSLOT], cs[NSLOT];
            uint32_t cpix[NSLOT];
        } cand;
        Elem mat[MAT];
    } u;
};

template <int K>
__device__ __forceinline__ int tri(int i, int k) {
    return i < K ? i * (i + 1) / 2 + k : K * (K + 1) / 2 + (i - K) * K + k;
}

// ------------------------------------------------------------------ helpers
__device__ __forceinline__ bool key_less(unsigned long long ka, unsigned ia, unsigned long long kb, unsigned ib) {
    return ka < kb || (ka == kb && ia < ib);
}

// Ascending bitonic sort of 32*SPL (key, id) pairs; element e = s*32 + lane.
template <int SPL>
__device__ __forceinline__ void bitonic_sort(unsigned long long (&key)[SPL], unsigned (&id)[SPL], int lane) {
    constexpr int N = 32 * SPL;
#pragma unroll
    for (int k = 2; k <= N; k <<= 1) {
#pragma unroll
        for (int j = k >> 1; j > 0; j >>= 1) {
#pragma unroll
            for (int s = 0; s < SPL; ++s) {
                const int e = s * 32 + lane;
                const bool up = (e & k) == 0;
                if (j >= 32) {
                    const int ps = s ^ (j >> 5);
                    if (ps > s) {
                        const bool sw = up ? key_less(key[ps], id[ps], key[s], id[s])
                                           : key_less(key[s], id[s], key[ps], id[ps]);
                        if (sw) {
                            const unsigned long long tk = key[s];
                            key[s] = key[ps];
                            key[ps] = tk;
                            const unsigned ti = id[s];
                            id[s] = id[ps];
                            id[ps] = ti;
                        }
                    }
                } else {
                    const unsigned long long pk = __shfl_xor_sync(FULL, key[s], j);
                    const unsigned pi = __shfl_xor_sync(FULL, id[s], j);
                    const bool lower = (lane & j) == 0;
                    const bool keep_min = (lower == up);
                    const bool partner_less = key_less(pk, pi, key[s], id[s]);
                    if (keep_min ? partner_less : (!partner_less && (pk != key[s] || pi != id[s]))) {
                        key[s] = pk;
                        id[s] = pi;
                    }
                }
            }
        }
    }
}

// Ascending bitonic sort of 32*SPL packed 64-bit keys; element e = s*32 + lane.
template <int SPL>
__device__ __forceinline__ void bitonic_sort_packed(unsigned long long (&key)[SPL], int lane) {
    constexpr int N = 32 * SPL;
#pragma unroll
    for (int k = 2; k <= N; k <<= 1) {
#pragma unroll
        for (int j = k >> 1; j > 0; j >>= 1) {
#pragma unroll
            for (int s = 0; s < SPL; ++s) {
                const int e = s * 32 + lane;
                const bool up = (e & k) == 0;
                if (j >= 32) {
                    const int ps = s ^ (j >> 5);
                    if (ps > s) {
                        const unsigned long long lo = key[s] < key[ps] ? key[s] : key[ps];
                        const unsigned long long hi = key[s] < key[ps] ? key[ps] : key[s];
                        key[s] = up ? lo : hi;
                        key[ps] = up ? hi : lo;
                    }
                } else {
                    const unsigned long long pk = __shfl_xor_sync(FULL, key[s], j);
                    const bool keep_min = (((lane & j) == 0) == up);
                    key[s] = keep_min ? (pk < key[s] ? pk : key[s]) : (pk > key[s] ? pk : key[s]);
                }
            }
        }
    }
}

template <class R>
__device__ __forceinline__ typename Ops<R>::T table_eval(const TableDev &tab, typename Ops<R>::T t);

template <>
__device__ __forceinline__ double table_eval<double>(const TableDev &tab, double t) {
    const double x = t * tab.inv_h;
    int k = (int)x;
    k = k > tab.n - 1 ? tab.n - 1 : (k < 0 ? 0 : k);
    const double s = x - (double)k;
    const double2 c01 = __ldg(reinterpret_cast<const double2 *>(tab.c64 + k));
    const double2 c23 = __ldg(reinterpret_cast<const double2 *>(tab.c64 + k) + 1);
    return fma(s, fma(s, fma(s, c23.y, c23.x), c01.y), c01.x);
}

template <>
__device__ __forceinline__ df table_eval<df>(const TableDev &tab, df t) {
    const df x = df_mul(t, df{tab.inv_h_hi, tab.inv_h_lo});
    float kf = floorf(x.hi);
    df s = two_sum(__fsub_rn(x.hi, kf), x.lo);
    if (s.hi < 0.0f) {
        kf -= 1.0f;
        s = df_add(s, {1.0f, 0.0f});
    }
    int k = (int)kf;
    if (k > tab.n - 1) {
        s = df_add(s, {(float)(k - (tab.n - 1)), 0.0f});
        k = tab.n - 1;
    } else if (k < 0) {
        s = df_add(s, {(float)k, 0.0f});
        k = 0;
    }
    const float4 c0 = __ldg(&tab.c32[2 * k]);
    const float4 c1 = __ldg(&tab.c32[2 * k + 1]);
    // p = f + s (m0 + s (c2 + s c3)).  The curvature terms c2, c3 of a table that
    // meets the grid rule are below ~1e-4 of xi(0), so s (c2 + s c3) is formed in
    // FP32 (absolute error ~1e-12, far inside the tolerance of this path); m0 plus
    // that term, and the outer step, in double-float.
    const float q = __fmul_rn(s.hi, __fmaf_rn(s.hi, c1.z, c1.x));
    const df r = df_addf(df{c0.z, c0.w}, q);
    // f and s (m0 + ...) are both at most xi(0) = 1 in size: the sum's error is
    // about 2^-44 absolute
    return df_add_fast(df_mul(r, s), df{c0.x, c0.y});
}

template <class R, int S>
__device__ __forceinline__ Cx<typename Ops<R>::T> pair_phase_uv(
    typename Ops<R>::T dx, typename Ops<R>::T dy, typename Ops<R>::T dz, typename Ops<R>::T zi,
    typename Ops<R>::T si, typename Ops<R>::T ci, typename Ops<R>::T sni, typename Ops<R>::T zj,
    typename Ops<R>::T sj, typename Ops<R>::T cj, typename Ops<R>::T snj, typename Ops<R>::T &u_out,
    typename Ops<R>::T &v_out);

// exp(is(a_ij - a_ji - pi)) for the pair (i -> j) with d = X_j - X_i, spin s = S,
// from the projections of d on the local bases at both ends: with e_theta =
// (z cos phi, z sin phi, -s) and e_phi = (-sin phi, cos phi, 0),
//   A = d.e_theta = z (dx cos phi + dy sin phi) - s dz,  B = d.e_phi = dy cos phi - dx sin phi.
// At j, d points along the direction of travel (angle a_ji + pi), so with
// q = (A1 + i B1)(A2 - i B2) the phase is (q / |q|)^s.
template <class R, int S>
__device__ __forceinline__ Cx<typename Ops<R>::T> pair_phase(typename Ops<R>::T dx, typename Ops<R>::T dy,
                                                             typename Ops<R>::T dz, typename Ops<R>::T zi,
                                                             typename Ops<R>::T si, typename Ops<R>::T ci,
                                                             typename Ops<R>::T sni, typename Ops<R>::T zj,
                                                             typename Ops<R>::T sj, typename Ops<R>::T cj,
                                                             typename Ops<R>::T snj) {
    typename Ops<R>::T u_dummy, v_dummy;
    return pair_phase_uv<R, S>(dx, dy, dz, zi, si, ci, sni, zj, sj, cj, snj, u_dummy, v_dummy);
}

// As pair_phase, also returning the projections (A1, B1) of d on e_theta, e_phi at i.
template <class R, int S>
__device__ __forceinline__ Cx<typename Ops<R>::T> pair_phase_uv(
    typename Ops<R>::T dx, typename Ops<R>::T dy, typename Ops<R>::T dz, typename Ops<R>::T zi,
    typename Ops<R>::T si, typename Ops<R>::T ci, typename Ops<R>::T sni, typename Ops<R>::T zj,
    typename Ops<R>::T sj, typename Ops<R>::T cj, typename Ops<R>::T snj, typename Ops<R>::T &u_out,
    typename Ops<R>::T &v_out) {
    using O = Ops<R>;
    using T = typename O::T;
    const T h1 = O::add(O::mul(dx, ci), O::mul(dy, sni));
    const T A1 = O::sub(O::mul(zi, h1), O::mul(si, dz));
    const T B1 = O::sub(O::mul(dy, ci), O::mul(dx, sni));
    u_out = A1;
    v_out = B1;
    const T h2 = O::add(O::mul(dx, cj), O::mul(dy, snj));
    const T A2 = O::sub(O::mul(zj, h2), O::mul(sj, dz));
    const T B2 = O::sub(O::mul(dy, cj), O::mul(dx, snj));
    const T qr = O::add(O::mul(A1, A2), O::mul(B1, B2));
    const T qi = O::sub(O::mul(B1, A2), O::mul(A1, B2));
    if constexpr (S == 1) {
        const T den1 = O::add(O::mul(qr, qr), O::mul(qi, qi));
        if (!O::positive(den1)) return {O::from(1.0), O::zero()};  // coincident points: no rotation
        T l, il;
        O::pivot(den1, l, il);  // il = 1/|q|
        return {O::mul(qr, il), O::mul(qi, il)};
    }
    // s = 2: q^2 / |q|^2
    const T qr2 = O::mul(qr, qr), qi2 = O::mul(qi, qi);
    const T nre = O::sub(qr2, qi2);
    const T qri = O::mul(qr, qi);
    const T nim = O::add(qri, qri);
    const T den = O::add(qr2, qi2);
    if (!O::positive(den)) return {O::from(1.0), O::zero()};  // coincident points: no rotation
    const T inv = O::rcp(den);
    return {O::mul(nre, inv), O::mul(nim, inv)};
}

// --------------------------------------------------- assemble, factor, solve
// Neighbour geometry in precision R (FP64 arrays, or their double-float copies).
template <class R, class SM>
struct Geom;
template <class SM>
struct Geom<double, SM> {
    static __device__ __forceinline__ double x(const SM &s, int i) { return s.gx[i]; }
    static __device__ __forceinline__ double y(const SM &s, int i) { return s.gy[i]; }
    static __device__ __forceinline__ double z(const SM &s, int i) { return s.gz[i]; }
    static __device__ __forceinline__ double nz(const SM &s, int i) { return s.gnz[i]; }
    static __device__ __forceinline__ double ns(const SM &s, int i) { return s.gns[i]; }
    static __device__ __forceinline__ double nc(const SM &s, int i) { return s.gnc[i]; }
    static __device__ __forceinline__ double nsn(const SM &s, int i) { return s.gnsn[i]; }
};
template <class SM>
struct Geom<df, SM> {
    static __device__ __forceinline__ df x(const SM &s, int i) { return s.gx[i]; }
    static __device__ __forceinline__ df y(const SM &s, int i) { return s.gy[i]; }
    static __device__ __forceinline__ df z(const SM &s, int i) { return s.gz[i]; }
    static __device__ __forceinline__ df nz(const SM &s, int i) { return s.gnz[i]; }
    static __device__ __forceinline__ df ns(const SM &s, int i) { return s.gns[i]; }
    static __device__ __forceinline__ df nc(const SM &s, int i) { return s.gnc[i]; }
    static __device__ __forceinline__ df nsn(const SM &s, int i) { return s.gnsn[i]; }
};

template <class R>
__device__ __forceinline__ Cx<typename Ops<R>::T> cx_conj(Cx<typename Ops<R>::T> a) {
    return {a.re, Ops<R>::neg(a.im)};
}

// Pair phase through the target (spin 2): with Phi0_i = phase(n' -> X_i),
//   phase(X_i -> X_j) = conj(Phi0_i) Phi0_j exp(-2iE_ij),
// E_ij the spherical excess of the triangle (n', X_i, X_j), tan(E/2) = x =
// (u_i v_j - v_i u_j) / (4 - (t_i + t_j + t_ij)/2) (Van Oosterom-Strackee, with
// (u, v) the tangent-plane coordinates at n' and t the squared chords), and
// exp(-2iE) = (1 - ix)^4 / (1 + x^2)^2, i.e. 1 + delta with
//   delta = (-8x^2 - 4ix(1 - x^2)) / (1 + x^2)^2
// (spin 1: exp(-iE) = (1 - ix)^2 / (1 + x^2), delta = (-2x^2 - 2ix) / (1 + x^2)).
// E is of order |X_i - n'||X_j - n'|, so delta is a small correction computed
// in FP32 (the double-float path; the FP64 path uses the direct vector form,
// cheaper in FP64 than the divisions below).
struct Holo32 {
    float dr, di;
};
template <int S>
__device__ __forceinline__ Holo32 holonomy32(float ui, float vi, float uj, float vj, float ti, float tj, float tij) {
    // x and w feed a correction of order x that is needed to FP32 accuracy only:
    // the fast divisions (2 ulp) suffice
    const float x = __fdividef(ui * vj - vi * uj, 4.0f - 0.5f * (ti + tj + tij));
    const float x2 = x * x;
    const float w = __fdividef(1.0f, 1.0f + x2);
    if constexpr (S == 1) return {-2.0f * x2 * w, -2.0f * x * w};  // exp(-iE) = (1 - ix)^2 / (1 + x^2)
    const float q = w * w;
    return {-8.0f * x2 * q, -4.0f * x * (1.0f - x2) * q};
}

// conj(a) b (1 + delta), delta from holonomy32.  a and b are unit complex
// numbers, so the two real dot products are anchored sums of products bounded
// by 1 (anchor 6); the FP32 correction b delta joins their low words.
__device__ __forceinline__ Cx<df> transported_phase(Cx<df> a, Cx<df> b, const Holo32 &h) {
    anc ar{6.0f, 0.0f}, ai{6.0f, 0.0f};
    anc_add_prod(ar, a.re, b.re);
    anc_add_prod(ar, a.im, b.im);
    anc_add_prod(ai, a.re, b.im);
    anc_sub_prod(ai, a.im, b.re);
    const float hr = __fsub_rn(ar.h, 6.0f), hi = __fsub_rn(ai.h, 6.0f);  // exact
    const float br = __fadd_rn(hr, ar.l), bi = __fadd_rn(hi, ai.l);        // FP32 values for the correction
    const float cr = br * h.dr - bi * h.di, ci = br * h.di + bi * h.dr;
    return {two_sum(hr, __fadd_rn(ar.l, cr)), two_sum(hi, __fadd_rn(ai.l, ci))};
}

// Both spin-2 phases of the pair (i -> j), d = X_j - X_i: exp(2i(a_ij - a_ji)) of
// the Hermitian covariance <P_i P_j^*> (as pair_phase) and exp(2i(a_ij + a_ji)) of
// the pseudo-covariance <P_i P_j>.  With w_i = A1 + iB1 and w_j = A2 + iB2 the
// projections of d on the local bases at both ends, they are
// (w_i conj(w_j))^2 / |w_i w_j|^2 and (w_i w_j)^2 / |w_i w_j|^2.
template <class R>
__device__ __forceinline__ void pair_phases_pm(typename Ops<R>::T dx, typename Ops<R>::T dy, typename Ops<R>::T dz,
                                               typename Ops<R>::T zi, typename Ops<R>::T si, typename Ops<R>::T ci,
                                               typename Ops<R>::T sni, typename Ops<R>::T zj, typename Ops<R>::T sj,
                                               typename Ops<R>::T cj, typename Ops<R>::T snj,
                                               Cx<typename Ops<R>::T> &php, Cx<typename Ops<R>::T> &phm) {
    using O = Ops<R>;
    using T = typename O::T;
    const T A1 = O::sub(O::mul(zi, O::add(O::mul(dx, ci), O::mul(dy, sni))), O::mul(si, dz));
    const T B1 = O::sub(O::mul(dy, ci), O::mul(dx, sni));
    const T A2 = O::sub(O::mul(zj, O::add(O::mul(dx, cj), O::mul(dy, snj))), O::mul(sj, dz));
    const T B2 = O::sub(O::mul(dy, cj), O::mul(dx, snj));
    const T aa = O::mul(A1, A2), bb = O::mul(B1, B2), ab = O::mul(A1, B2), ba = O::mul(B1, A2);
    const T qpr = O::add(aa, bb), qpi = O::sub(ba, ab);  // w_i conj(w_j)
    const T qmr = O::sub(aa, bb), qmi = O::add(ab, ba);  // w_i w_j
    const T den = O::add(O::mul(qpr, qpr), O::mul(qpi, qpi));
    if (!O::positive(den)) {  // coincident points
        php = {O::from(1.0), O::zero()};
        phm = {O::zero(), O::zero()};
        return;
    }
    const T inv = O::rcp(den);
    const T pri = O::mul(qpr, qpi), mri = O::mul(qmr, qmi);
    php = {O::mul(O::sub(O::mul(qpr, qpr), O::mul(qpi, qpi)), inv), O::mul(O::add(pri, pri), inv)};
    phm = {O::mul(O::sub(O::mul(qmr, qmr), O::mul(qmi, qmi)), inv), O::mul(O::add(mri, mri), inv)};
}

// Split left-looking Cholesky of an N x N packed lower triangle (row i starts
// at i(i+1)/2) bordered by NB right-hand-side rows stored after it (row N + b
// holds the conjugate of the b-th right-hand side); on return the bordered rows
// hold conj(L^-1 conj(rhs)).  At column j the NROW - j active rows are spread
// over 32/s lane groups of s lanes, s the largest power of two with
// (NROW - j) s <= 32, and each group splits the dot product over k < j and
// reduces it with shuffles.  Elem is real (Ops<R>::T) or complex (Cx<T>).
// Returns false when a pivot is not positive.
template <int N, int NB, class R, class Elem>
__device__ __forceinline__ bool bordered_cholesky(Elem *mat, int lane) {
    using O = Ops<R>;
    using T = typename O::T;
    constexpr bool CPLX = !std::is_same<Elem, T>::value;
    constexpr int NROW = N + NB;
    constexpr int NT = (NROW + 31) / 32;  // row slots per lane at s = 1
    for (int j = 0; j < N; ++j) {
        const int nrows = NROW - j;
        int s = 1;
        while ((s << 1) * nrows <= 32) s <<= 1;
        const int g = 32 / s;
        const int part = lane & (s - 1), grp = lane / s;
        const Elem *Lj = mat + tri<N>(j, 0);
        Elem srow[NT];
#pragma unroll
        for (int t = 0; t < NT; ++t) {
            if (t > 0 && j + t * g >= NROW) break;  // warp-uniform: no row left for this slot
            const int r = j + grp + t * g;
            const bool act = r < NROW;
            const int rr = act ? r : j;
            const Elem *Lr = mat + tri<N>(rr, 0);
            if constexpr (!CPLX) {
                typename O::Acc acc = O::acc((part == 0 && act) ? Lr[j] : O::zero());
                typename O::Acc acc2 = O::acc(O::zero());
                if (act) {
                    int k = part;
                    for (; k + s < j; k += 2 * s) {  // two independent chains
                        O::sub_prod(acc, Lr[k], Lj[k]);
                        O::sub_prod(acc2, Lr[k + s], Lj[k + s]);
                    }
                    if (k < j) O::sub_prod(acc, Lr[k], Lj[k]);
                }
                T v = O::add_fast(O::val(acc), O::val(acc2));
                for (int o = 1; o < s; o <<= 1) v = O::add_fast(v, O::shfl_xor(v, o));
                srow[t] = v;
            } else {
                const Elem a0 = Lr[j];
                typename O::Acc ar = O::acc((part == 0 && act) ? a0.re : O::zero());
                typename O::Acc ai = O::acc((part == 0 && act) ? a0.im : O::zero());
                typename O::Acc br = O::acc(O::zero()), bi = O::acc(O::zero());
                if (act)
                    for (int k = part; k < j; k += s) {  // real and imaginary parts in two chains each
                        const Elem a = Lr[k], b = Lj[k];
                        O::sub_prod(ar, a.re, b.re);
                        O::sub_prod(br, a.im, b.im);
                        O::sub_prod(ai, a.im, b.re);
                        O::add_prod(bi, a.re, b.im);
                    }
                T vr = O::add_fast(O::val(ar), O::val(br)), vi = O::add_fast(O::val(ai), O::val(bi));
                for (int o = 1; o < s; o <<= 1) {
                    vr = O::add_fast(vr, O::shfl_xor(vr, o));
                    vi = O::add_fast(vi, O::shfl_xor(vi, o));
                }
                srow[t].re = vr;
                srow[t].im = vi;
            }
        }
        // pivot: row j is held by lane 0 (group 0, part 0, t = 0)
        T d;
        if constexpr (!CPLX) {
            d = O::shfl(srow[0], 0);
        } else {
            d = O::shfl(srow[0].re, 0);
        }
        if (!O::positive(d)) return false;
        T ljj, il;
        O::pivot(d, ljj, il);
        __syncwarp();
        if (part == 0) {
#pragma unroll
            for (int t = 0; t < NT; ++t) {
                const int r = j + grp + t * g;
                if (t > 0 && j + t * g >= NROW) break;
                if (r < NROW) {
                    Elem v;
                    if constexpr (!CPLX) {
                        v = (r == j) ? ljj : O::mul(srow[t], il);
                    } else {
                        if (r == j) {
                            v.re = ljj;
                            v.im = O::zero();
                        } else {
                            v.re = O::mul(srow[t].re, il);
                            v.im = O::mul(srow[t].im, il);
                        }
                    }
                    mat[tri<N>(r, j)] = v;
                }
            }
        }
        __syncwarp();
    }
    return true;
}

// Right-looking form of the same factorisation.  Step j takes the pivot of
// column j, scales the column, and applies the rank-one update
// A_rc -= L_rj conj(L_cj) to every trailing entry (j < c <= r, bordered rows
// included), the entries spread round-robin over the 32 lanes.  Trailing
// entries are kept as unnormalised accumulators between steps (for double-
// float the running TwoSum word and the collected error word) and normalised
// when they become part of a column.  Compared with the split left-looking
// form, every lane stays busy until the last few columns and no shuffle
// reductions are needed.
template <int N, int NB, class R, class Elem>
__device__ __forceinline__ bool bordered_cholesky_rl(Elem *mat, int lane) {
    using O = Ops<R>;
    using T = typename O::T;
    constexpr bool CPLX = !std::is_same<Elem, T>::value;
    constexpr int NROW = N + NB;
    for (int j = 0; j < N; ++j) {
        // pivot
        T d;
        if constexpr (CPLX) {
            d = O::val(O::acc(mat[tri<N>(j, j)].re));
        } else {
            d = O::val(O::acc(mat[tri<N>(j, j)]));
        }
        __syncwarp();  // every lane has read the pivot before lane 0 overwrites it below
        if (!O::positive(d)) return false;
        T ljj, il;
        O::pivot(d, ljj, il);
        // column j
        for (int r = j + 1 + lane; r < NROW; r += 32) {
            Elem a = mat[tri<N>(r, j)];
            if constexpr (CPLX) {
                a.re = O::mul(O::val(O::acc(a.re)), il);
                a.im = O::mul(O::val(O::acc(a.im)), il);
            } else {
                a = O::mul(O::val(O::acc(a)), il);
            }
            mat[tri<N>(r, j)] = a;
        }
        if (lane == 0) {
            if constexpr (CPLX) {
                mat[tri<N>(j, j)] = Elem{ljj, O::zero()};
            } else {
                mat[tri<N>(j, j)] = ljj;
            }
        }
        __syncwarp();
        // rank-one update of the trailing entries: the triangle of rows and
        // columns j+1..N-1 (m(m+1)/2 entries, walked as q = ri(ri+1)/2 + ci),
        // then the NB bordered rows (m entries each)
        const int m = N - 1 - j;
        const int ntri = m * (m + 1) / 2, ntot = ntri + NB * m;
        int ri = 0, ci = lane;
        while (ci > ri) {
            ci -= ri + 1;
            ++ri;
        }
        int br = -1, bc = 0;
        for (int q = lane; q < ntot; q += 32) {
            int r, c;
            if (q < ntri) {
                r = j + 1 + ri;
                c = j + 1 + ci;
                ci += 32;
                while (ci > ri) {
                    ci -= ri + 1;
                    ++ri;
                }
            } else {
                if (br < 0) {
                    const int qq = q - ntri;
                    br = qq / m;
                    bc = qq - br * m;
                }
                r = N + br;
                c = j + 1 + bc;
                bc += 32;
                while (bc >= m) {
                    bc -= m;
                    ++br;
                }
            }
            Elem a = mat[tri<N>(r, c)];
            const Elem x = mat[tri<N>(r, j)], y = mat[tri<N>(c, j)];
            if constexpr (CPLX) {  // a -= x conj(y)
                typename O::Acc ar = O::acc(a.re), ai = O::acc(a.im);
                O::sub_prod(ar, x.re, y.re);
                O::sub_prod(ai, x.im, y.re);
                O::sub_prod(ar, x.im, y.im);
                O::add_prod(ai, x.re, y.im);
                a.re = O::raw(ar);
                a.im = O::raw(ai);
            } else {
                typename O::Acc ac = O::acc(a);
                O::sub_prod(ac, x, y);
                a = O::raw(ac);
            }
            mat[tri<N>(r, c)] = a;
        }
        __syncwarp();
    }
    return true;
}

// Double-float form of the split left-looking factorisation with anchored
// accumulators (struct anc).  The partial sums of column j are bounded by the
// Cauchy-Schwarz inequality: every matrix row r has |L_r| <= sqrt(A_rr) =
// sqrt(1 + n) and so has the pivot row, the covariance rows (c; b_Q, b_U of the
// augmented system) have |L^-1 c|^2 <= 1 (resp. <= 2) because the variance they
// leave is non-negative, and their entries are at most 1: every sum over k < j
// of L_rk conj(L_jk), plus A_rj, stays below 2.5, anchor C = 6.  The last
// bordered row holds the data, whose solve L^-1 y has no a-priori bound; its
// anchor is taken per column from |y_j| + |(L^-1 y)_{<j}| (the running norm of
// the entries already computed, carried in every lane), so its grid follows the
// size of its own sums.  Compared with bordered_cholesky<N, NB, df> only the
// accumulation differs (6 instead of 12 FP32 instructions per real
// multiply-accumulate); the error per step is about 2^-46 of the bound instead
// of 2^-48 of the products.
template <int N, int NB, class Elem>
__device__ __forceinline__ bool bordered_cholesky_anchored(Elem *mat, int lane) {
    using O = Ops<df>;
    constexpr bool CPLX = !std::is_same<Elem, df>::value;
    constexpr int NROW = N + NB;
    constexpr int NT = (NROW + 31) / 32;
    constexpr float C_BOUNDED = 6.0f;
    float ynorm2 = 0.0f;  // |(L^-1 y)_{<j}|^2 of the data row (row NROW - 1), FP32, identical in every lane
    for (int j = 0; j < N; ++j) {
        // s = 2^ls lanes per row group: the largest power of two with (NROW - j) s <= 32,
        // i.e. ls = 5 - ceil(log2(NROW - j)) (at least 0); g = 32 / s groups
        const int nrows = NROW - j;
        const int cl2 = nrows > 1 ? 32 - __clz(nrows - 1) : 0;
        const int ls = cl2 < 5 ? 5 - cl2 : 0;
        const int s = 1 << ls, g = 32 >> ls;
        const int part = lane & (s - 1), grp = lane >> ls;
        const Elem *Lj = mat + tri<N>(j, 0);
        // anchor of the data row at this column (its initial entry plus the running
        // norm; the square root from rsqrtf, within a few ulps, is covered by 1.01)
        float cy;
        {
            const Elem y0 = mat[tri<N>(NROW - 1, j)];
            float ay;
            if constexpr (CPLX) {
                ay = fmaxf(fabsf(y0.re.hi), fabsf(y0.im.hi));
            } else {
                ay = fabsf(y0.hi);
            }
            const float yn = fmaxf(ynorm2, 1e-30f);
            cy = anc_anchor(fmaf(1.01f, ay + yn * rsqrtf(yn), 1e-30f));
        }
        Elem srow[NT];
#pragma unroll
        for (int t = 0; t < NT; ++t) {
            if (t > 0 && j + t * g >= NROW) break;  // warp-uniform: no row left for this slot
            const int r = j + grp + t * g;
            const bool act = r < NROW;
            const int rr = act ? r : j;
            const float C = (rr == NROW - 1) ? cy : C_BOUNDED;
            const Elem *Lr = mat + tri<N>(rr, 0);
            if constexpr (!CPLX) {
                anc acc = anc_init((part == 0 && act) ? Lr[j] : O::zero(), C);
                anc acc2 = anc_init(O::zero(), C);
                if (act) {
                    int k = part;
                    for (; k + s < j; k += 2 * s) {  // two independent chains
                        anc_sub_prod(acc, Lr[k], Lj[k]);
                        anc_sub_prod(acc2, Lr[k + s], Lj[k + s]);
                    }
                    if (k < j) anc_sub_prod(acc, Lr[k], Lj[k]);
                }
                float H = __fadd_rn(__fsub_rn(acc.h, C), __fsub_rn(acc2.h, C));  // exact: grid values in range
                float Lw = __fadd_rn(acc.l, acc2.l);
                for (int o = 1; o < s; o <<= 1) {
                    H = __fadd_rn(H, __shfl_xor_sync(FULL, H, o));
                    Lw = __fadd_rn(Lw, __shfl_xor_sync(FULL, Lw, o));
                }
                srow[t] = two_sum(H, Lw);
            } else {
                const Elem a0 = Lr[j];
                anc ar = anc_init((part == 0 && act) ? a0.re : O::zero(), C);
                anc ai = anc_init((part == 0 && act) ? a0.im : O::zero(), C);
                anc br = anc_init(O::zero(), C), bi = anc_init(O::zero(), C);
                if (act)
                    for (int k = part; k < j; k += s) {  // real and imaginary parts in two chains each
                        const Elem a = Lr[k], b = Lj[k];
                        anc_sub_prod(ar, a.re, b.re);
                        anc_sub_prod(br, a.im, b.im);
                        anc_sub_prod(ai, a.im, b.re);
                        anc_add_prod(bi, a.re, b.im);
                    }
                float Hr = __fadd_rn(__fsub_rn(ar.h, C), __fsub_rn(br.h, C));
                float Hi = __fadd_rn(__fsub_rn(ai.h, C), __fsub_rn(bi.h, C));
                float Lr_ = __fadd_rn(ar.l, br.l), Li_ = __fadd_rn(ai.l, bi.l);
                for (int o = 1; o < s; o <<= 1) {
                    Hr = __fadd_rn(Hr, __shfl_xor_sync(FULL, Hr, o));
                    Hi = __fadd_rn(Hi, __shfl_xor_sync(FULL, Hi, o));
                    Lr_ = __fadd_rn(Lr_, __shfl_xor_sync(FULL, Lr_, o));
                    Li_ = __fadd_rn(Li_, __shfl_xor_sync(FULL, Li_, o));
                }
                srow[t].re = two_sum(Hr, Lr_);
                srow[t].im = two_sum(Hi, Li_);
            }
        }
        // pivot: row j is held by lane 0 (group 0, part 0, t = 0)
        df d;
        if constexpr (!CPLX) {
            d = O::shfl(srow[0], 0);
        } else {
            d = O::shfl(srow[0].re, 0);
        }
        if (!O::positive(d)) return false;
        df ljj, il;
        O::pivot(d, ljj, il);
        // the data row's new entry (held by the parts of its group) joins the running norm
        {
            const int ty = (NROW - 1 - j) >> (5 - ls), gy = (NROW - 1 - j) - ty * g;
            float vr = 0.0f, vi = 0.0f;
#pragma unroll
            for (int t = 0; t < NT; ++t) {
                if (t == ty) {
                    if constexpr (!CPLX) {
                        vr = srow[t].hi;
                    } else {
                        vr = srow[t].re.hi;
                        vi = srow[t].im.hi;
                    }
                }
            }
            vr = __shfl_sync(FULL, vr, gy * s) * il.hi;
            if constexpr (CPLX) vi = __shfl_sync(FULL, vi, gy * s) * il.hi;
            ynorm2 = fmaf(vr, vr, fmaf(vi, vi, ynorm2));
        }
        __syncwarp();
        if (part == 0) {
#pragma unroll
            for (int t = 0; t < NT; ++t) {
                const int r = j + grp + t * g;
                if (t > 0 && j + t * g >= NROW) break;
                if (r < NROW) {
                    Elem v;
                    if constexpr (!CPLX) {
                        v = (r == j) ? ljj : O::mul(srow[t], il);
                    } else {
                        if (r == j) {
                            v.re = ljj;
                            v.im = O::zero();
                        } else {
                            v.re = O::mul(srow[t].re, il);
                            v.im = O::mul(srow[t].im, il);
                        }
                    }
                    mat[tri<N>(r, j)] = v;
                }
            }
        }
        __syncwarp();
    }
    return true;
}

// Choice between the forms, measured on GB300 (c3-like targets): in FP64 the
// pipe executes inactive lanes too, so the right-looking form's fuller lanes
// win for N <= 32 (spin 2, K = 32: +15 %); for larger N the left-looking form's
// register accumulators win (right-looking was 28 % slower in FP64 at N = 48).
// Double-float factors use the left-looking form with anchored accumulators
// (the right-looking form's memory-resident accumulators were 21 % slower).
template <int N, int NB, class R, class Elem>
__device__ __forceinline__ bool factor_bordered(Elem *mat, int lane) {
    if constexpr (std::is_same<R, double>::value && N <= 32)
        return bordered_cholesky_rl<N, NB, R>(mat, lane);
    else if constexpr (std::is_same<R, df>::value)
        return bordered_cholesky_anchored<N, NB>(mat, lane);
    else
        return bordered_cholesky<N, NB, R>(mat, lane);
}

// Returns false when a pivot of S + nugget I is not positive.

//
// Factorisation: left-looking Cholesky of the matrix bordered by the two
// right-hand-side rows (row K holds c (spin 2: c0 = <P(n') P_i^*>), row K+1
// holds conj(y)); the factor's bordered rows are then conj(L^-1 conj(c)) and
// conj(L^-1 y), so the forward solves need no separate pass.  At column j the
// K+2-j active rows are spread over 32/s lane groups of s lanes, s the largest
// power of two with (K+2-j) s <= 32, and each group splits the dot product
// over k < j and reduces it with shuffles.
template <int K, int SPIN, class R, class SM>
__device__ bool solve_point(SM &sm, const PointA &P, int lane, double nugget, const TableDev &tab,
                            const double (&keyd)[Shape<K>::RPL], const double (&yre)[Shape<K>::RPL],
                            const double (&yim)[Shape<K>::RPL], double &val_re, double &val_im,
                            double &var_rel) {
    using O = Ops<R>;
    using T = typename O::T;
    using G = Geom<R, SM>;
    constexpr int RPL = Shape<K>::RPL, NTRI = Shape<K>::NTRI;
    using Elem = typename SM::Elem;
    Elem *mat = sm.u.mat;

    // ---- spin 2: per-neighbour target phases and tangent coordinates
    if constexpr (SPIN == 1 || SPIN == 2) {
#pragma unroll
        for (int r = 0; r < RPL; ++r) {
            const int i = lane + 32 * r;
            if (i < K) {
                T u, v;
                const Cx<T> ph = pair_phase_uv<R, SPIN>(G::x(sm, i), G::y(sm, i), G::z(sm, i), O::from(P.z), O::from(P.s),
                                                  O::from(P.cph), O::from(P.sph), G::nz(sm, i), G::ns(sm, i),
                                                  G::nc(sm, i), G::nsn(sm, i), u, v);
                sm.p0r[i] = ph.re;
                sm.p0i[i] = ph.im;
                sm.pu[i] = u;
                sm.pv[i] = v;
            }
        }
        __syncwarp();
    }

    // ---- assembly of the lower triangle
    {
        // anchor of the squared chords in the double-float path: every chord between
        // stencil members is at most the table's t_max
        [[maybe_unused]] const float ct = anc_anchor((float)tab.t_max * 1.0001f);
        int i = 0, j = lane;  // q = lane -> (i, j) with q = i(i+1)/2 + j
        while (j > i) {
            j -= i + 1;
            ++i;
        }
        for (int q = lane; q < NTRI; q += 32) {
            Elem e;
            if (i == j) {
                if constexpr (SPIN == 0) {
                    e = O::from(1.0 + nugget);
                } else {
                    e.re = O::from(1.0 + nugget);
                    e.im = O::zero();
                }
            } else {
                T t;
                [[maybe_unused]] T dx, dy, dz;
                if constexpr (std::is_same<R, double>::value) {
                    dx = O::sub(G::x(sm, j), G::x(sm, i));
                    dy = O::sub(G::y(sm, j), G::y(sm, i));
                    dz = O::sub(G::z(sm, j), G::z(sm, i));
                    t = O::add_fast(O::add_fast(O::mul(dx, dx), O::mul(dy, dy)), O::mul(dz, dz));
                } else {
                    // the offsets' high words share one grid (df_on_grid), so their
                    // differences are exact; the squared chord is an anchored sum
                    // (every partial sum <= t_max)
                    anc ta{ct, 0.0f};
                    anc_add_sq(ta, __fsub_rn(sm.gx[j].hi, sm.gx[i].hi), __fsub_rn(sm.gx[j].lo, sm.gx[i].lo));
                    anc_add_sq(ta, __fsub_rn(sm.gy[j].hi, sm.gy[i].hi), __fsub_rn(sm.gy[j].lo, sm.gy[i].lo));
                    anc_add_sq(ta, __fsub_rn(sm.gz[j].hi, sm.gz[i].hi), __fsub_rn(sm.gz[j].lo, sm.gz[i].lo));
                    t = two_sum(__fsub_rn(ta.h, ct), ta.l);
                }
                const T fv = table_eval<R>(tab, t);
                if constexpr (SPIN == 0) {
                    e = fv;
                } else {
                    Cx<T> ph;
                    if constexpr (std::is_same<R, double>::value) {
                        // FP64: the direct vector form is cheaper than the transported form's divisions
                        ph = pair_phase<R, SPIN>(dx, dy, dz, G::nz(sm, i), G::ns(sm, i), G::nc(sm, i), G::nsn(sm, i),
                                           G::nz(sm, j), G::ns(sm, j), G::nc(sm, j), G::nsn(sm, j));
                    } else {
                        const Holo32 hol = holonomy32<SPIN>(sm.pu[i].hi, sm.pv[i].hi, sm.pu[j].hi, sm.pv[j].hi, sm.ktf[i],
                                                      sm.ktf[j], t.hi);
                        ph = transported_phase(Cx<df>{sm.p0r[i], sm.p0i[i]}, Cx<df>{sm.p0r[j], sm.p0i[j]}, hol);
                    }
                    e.re = O::mul(fv, ph.re);
                    e.im = O::mul(fv, ph.im);
                }
            }
            mat[q] = e;
            j += 32;
            while (j > i) {
                j -= i + 1;
                ++i;
            }
        }
    }
    // ---- bordered rows: row K = c (spin 2: c0), row K+1 = conj(y)
#pragma unroll
    for (int r = 0; r < RPL; ++r) {
        const int i = lane + 32 * r;
        if (i < K) {
            const T fv = table_eval<R>(tab, O::from(keyd[r]));
            if constexpr (SPIN == 0) {
                mat[tri<K>(K, i)] = fv;
                mat[tri<K>(K + 1, i)] = O::from(yre[r]);
            } else {
                // target -> neighbour phase from the prologue
                const Cx<T> ph{sm.p0r[i], sm.p0i[i]};
                Elem c0, yc;
                c0.re = O::mul(fv, ph.re);
                c0.im = O::mul(fv, ph.im);
                yc.re = O::from(yre[r]);
                yc.im = O::from(-yim[r]);
                mat[tri<K>(K, i)] = c0;
                mat[tri<K>(K + 1, i)] = yc;
            }
        }
    }
    __syncwarp();

    if (!factor_bordered<K, 2, R>(mat, lane)) return false;
    // ---- value = z_c^H z_y = sum_k row_K[k] conj(row_K+1[k]);  variance = 1 - |z_c|^2
    double vr = 0.0, vi = 0.0, nc = 0.0;
    if constexpr (std::is_same<R, df>::value) {
        // double-float products and lane reduction on the FP32 pipe, one conversion at the end
        dfacc ar{0.0f, 0.0f}, ai{0.0f, 0.0f}, an{0.0f, 0.0f};
#pragma unroll
        for (int r = 0; r < RPL; ++r) {
            const int k = lane + 32 * r;
            if (k < K) {
                const Elem c = mat[tri<K>(K, k)], y = mat[tri<K>(K + 1, k)];
                if constexpr (SPIN == 0) {
                    dfacc_add_prod(ar, c, y);
                    dfacc_add_prod(an, c, c);
                } else {  // (cr + i ci)(yr - i yi)
                    dfacc_add_prod(ar, c.re, y.re);
                    dfacc_add_prod(ar, c.im, y.im);
                    dfacc_add_prod(ai, c.im, y.re);
                    dfacc_sub_prod(ai, c.re, y.im);
                    dfacc_add_prod(an, c.re, c.re);
                    dfacc_add_prod(an, c.im, c.im);
                }
            }
        }
        df dr = dfacc_val(ar), di = dfacc_val(ai), dn = dfacc_val(an);
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            dr = df_add(dr, O::shfl_xor(dr, o));  // the value's terms may cancel: full sum
            if constexpr (SPIN != 0) di = df_add(di, O::shfl_xor(di, o));
            dn = df_add_fast(dn, O::shfl_xor(dn, o));  // non-negative terms
        }
        vr = df_to(dr);
        vi = df_to(di);
        nc = df_to(dn);
    } else {
#pragma unroll
        for (int r = 0; r < RPL; ++r) {
            const int k = lane + 32 * r;
            if (k < K) {
                const Elem c = mat[tri<K>(K, k)], y = mat[tri<K>(K + 1, k)];
                if constexpr (SPIN == 0) {
                    vr = fma(c, y, vr);
                    nc = fma(c, c, nc);
                } else {
                    // (cr + i ci)(yr - i yi)
                    vr = fma(c.re, y.re, fma(c.im, y.im, vr));
                    vi = fma(c.im, y.re, fma(-c.re, y.im, vi));
                    nc = fma(c.re, c.re, fma(c.im, c.im, nc));
                }
            }
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            vr += __shfl_xor_sync(FULL, vr, o);
            vi += __shfl_xor_sync(FULL, vi, o);
            nc += __shfl_xor_sync(FULL, nc, o);
        }
    }
    val_re = vr;
    val_im = vi;
    var_rel = 1.0 - nc;
    return true;
}

// Augmented (widely linear) spin-2 estimate.  With G = <P P^H> / xi+(0) (xi+
// and the pair phases) and C = <P P^T> / xi+(0) (xi- and the pseudo-phases),
// the real vector x = (Q_1..Q_K, U_1..U_K) has covariance xi+(0)/2 A with
//   A = [[Re(G + C), Im(C - G)], [Im(G + C), Re(G - C)]]
// (diagonal 1; the nugget n is added to it as to G), and the target's (Q, U)
// the cross-covariances xi+(0)/2 (b_Q, b_U) built the same way from G_i0, C_i0.
// Then Q = b_Q^T A^-1 x, U = b_U^T A^-1 x, and E|P - P^|^2 = xi+(0)(1 -
// (|L^-1 b_Q|^2 + |L^-1 b_U|^2)/2).  The factor of A bordered by the rows b_Q,
// b_U and x gives all three solves.
template <int K, class R, class SM>
__device__ bool solve_point_aug(SM &sm, const PointA &P, int lane, double nugget, const TableDev &tab,
                                const TableDev &tabm, const double (&keyd)[Shape<K>::RPL],
                                const double (&yre)[Shape<K>::RPL], const double (&yim)[Shape<K>::RPL],
                                double &val_re, double &val_im, double &var_rel) {
    using O = Ops<R>;
    using T = typename O::T;
    using G = Geom<R, SM>;
    constexpr int RPL = Shape<K>::RPL, NTRI = Shape<K>::NTRI, N = 2 * K;
    T *mat = sm.u.mat;
    // ---- assembly: each pair (i >= j) of neighbours gives four entries of A
    {
        int i = 0, j = lane;
        while (j > i) {
            j -= i + 1;
            ++i;
        }
        for (int q = lane; q < NTRI; q += 32) {
            if (i == j) {
                mat[tri<N>(i, i)] = O::from(1.0 + nugget);
                mat[tri<N>(K + i, K + i)] = O::from(1.0 + nugget);
                mat[tri<N>(K + i, i)] = O::zero();
            } else {
                const T dx = O::sub(G::x(sm, j), G::x(sm, i));
                const T dy = O::sub(G::y(sm, j), G::y(sm, i));
                const T dz = O::sub(G::z(sm, j), G::z(sm, i));
                const T t = O::add_fast(O::add_fast(O::mul(dx, dx), O::mul(dy, dy)), O::mul(dz, dz));
                const T fp = table_eval<R>(tab, t), fm = table_eval<R>(tabm, t);
                Cx<T> php, phm;
                pair_phases_pm<R>(dx, dy, dz, G::nz(sm, i), G::ns(sm, i), G::nc(sm, i), G::nsn(sm, i), G::nz(sm, j),
                                  G::ns(sm, j), G::nc(sm, j), G::nsn(sm, j), php, phm);
                const T gr = O::mul(fp, php.re), gi = O::mul(fp, php.im);
                const T cr = O::mul(fm, phm.re), ci = O::mul(fm, phm.im);
                mat[tri<N>(i, j)] = O::add(gr, cr);
                mat[tri<N>(K + i, K + j)] = O::sub(gr, cr);
                mat[tri<N>(K + i, j)] = O::add(gi, ci);
                mat[tri<N>(K + j, i)] = O::sub(ci, gi);
            }
            j += 32;
            while (j > i) {
                j -= i + 1;
                ++i;
            }
        }
    }
    // ---- bordered rows: N = b_Q, N + 1 = b_U, N + 2 = x
#pragma unroll
    for (int r = 0; r < RPL; ++r) {
        const int i = lane + 32 * r;
        if (i < K) {
            const T t0 = O::from(keyd[r]);
            const T fp = table_eval<R>(tab, t0), fm = table_eval<R>(tabm, t0);
            Cx<T> php, phm;  // of (n' -> X_i); G_i0 takes the conjugate Hermitian phase
            pair_phases_pm<R>(G::x(sm, i), G::y(sm, i), G::z(sm, i), O::from(P.z), O::from(P.s), O::from(P.cph),
                              O::from(P.sph), G::nz(sm, i), G::ns(sm, i), G::nc(sm, i), G::nsn(sm, i), php, phm);
            const T gr = O::mul(fp, php.re), gi = O::neg(O::mul(fp, php.im));
            const T cr = O::mul(fm, phm.re), ci = O::mul(fm, phm.im);
            mat[tri<N>(N, i)] = O::add(gr, cr);
            mat[tri<N>(N, K + i)] = O::add(gi, ci);
            mat[tri<N>(N + 1, i)] = O::sub(ci, gi);
            mat[tri<N>(N + 1, K + i)] = O::sub(gr, cr);
            mat[tri<N>(N + 2, i)] = O::from(yre[r]);
            mat[tri<N>(N + 2, K + i)] = O::from(yim[r]);
        }
    }
    __syncwarp();
    if (!factor_bordered<N, 3, R>(mat, lane)) return false;
    double vq = 0.0, vu = 0.0, nn = 0.0;
    for (int k = lane; k < N; k += 32) {
        const double zq = O::to(mat[tri<N>(N, k)]), zu = O::to(mat[tri<N>(N + 1, k)]);
        const double zx = O::to(mat[tri<N>(N + 2, k)]);
        vq = fma(zq, zx, vq);
        vu = fma(zu, zx, vu);
        nn = fma(zq, zq, fma(zu, zu, nn));
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        vq += __shfl_xor_sync(FULL, vq, o);
        vu += __shfl_xor_sync(FULL, vu, o);
        nn += __shfl_xor_sync(FULL, nn, o);
    }
    val_re = vq;
    val_im = vu;
    var_rel = 1.0 - 0.5 * nn;
    return true;
}

template <int K, int SPIN, class R, class SM>
__device__ __forceinline__ bool solve_any(SM &sm, const PointA &P, int lane, double nugget, const LensArgs &a,
                                          const double (&keyd)[Shape<K>::RPL], const double (&yre)[Shape<K>::RPL],
                                          const double (&yim)[Shape<K>::RPL], double &vre, double &vim,
                                          double &vrel) {
    if constexpr (SPIN == SPIN2_AUG)
        return solve_point_aug<K, R>(sm, P, lane, nugget, a.tab, a.tabm, keyd, yre, yim, vre, vim, vrel);
    else
        return solve_point<K, SPIN, R>(sm, P, lane, nugget, a.tab, keyd, yre, yim, vre, vim, vrel);
}

// ------------------------------------------------------------------ kernel
struct Counters {
    unsigned long long nug = 0, fb = 0, win = 0, fail = 0;
};

__device__ __forceinline__ void flush_counters(Counters &cnt, unsigned long long *dst, int lane) {
    if (lane == 0 && dst) {
        if (cnt.nug) atomicAdd(dst + CNT_NUGGET, cnt.nug);
        if (cnt.fb) atomicAdd(dst + CNT_FALLBACK, cnt.fb);
        if (cnt.win) atomicAdd(dst + CNT_WINDOW, cnt.win);
        if (cnt.fail) atomicAdd(dst + CNT_FAILED, cnt.fail);
    }
    cnt = Counters{};
}

template <int K, int SPIN, int MIXED>
constexpr size_t warp_smem_bytes() {
    using SMd = WarpSmem<K, SPIN, double>;
    using SMf = WarpSmem<K, SPIN, df>;
    static_assert(offsetof(SMd, gx) == offsetof(SMf, gx) && offsetof(SMd, ktf) == offsetof(SMf, ktf) &&
                      offsetof(SMd, u) == offsetof(SMf, u),
                  "the FP64 and double-float views of a warp slice must share their layout");
    constexpr size_t WS = sizeof(SMd) > sizeof(SMf) ? sizeof(SMd) : sizeof(SMf);
    return (WS + 15) / 16 * 16;
}

// One tile of `tile_pts` (<= MAX_TILE_POINTS) consecutive targets of a launch, processed by
// one warp whose shared-memory slice starts at `wbase`.
template <int K, int SPIN, int MIXED>
__device__ __forceinline__ void process_tile(const LensArgs &a, int R_rings, int64_t tile, int tile_pts,
                                          unsigned char *wbase, int lane, Counters &ctr) {
    using SMd = WarpSmem<K, SPIN, double>;
    using SMf = WarpSmem<K, SPIN, df>;
    constexpr int SPL = Shape<K>::SPL, RPL = Shape<K>::RPL, NSLOT = Shape<K>::NSLOT;
    SMd &sm = *reinterpret_cast<SMd *>(wbase);
    const int64_t N = a.nside;
    const double inv3N = 1.0 / (3.0 * (double)N), inv3N2 = inv3N / (double)N;
    // ------------------------------------------------ phase A: displace
    {
        const int64_t p = tile * tile_pts + lane;
        PointA P{};
        if (lane < tile_pts && p < a.count) {
            const int64_t pix = a.first + p;
            int64_t ring, jj;
            // supersampling: the target is a pixel centre of the finer grid, undisplaced
            const bool grid = a.nside_tgt > 0;
            pix_ring(grid ? a.nside_tgt : N, pix, ring, jj);
            const Ring rg = grid ? ring_of(a.nside_tgt, ring) : ring_of(N, ring, inv3N, inv3N2);
            double sp, cp;
            sincospi(((double)jj + rg.f) / (2.0 * (double)rg.nq), &sp, &cp);
            const double nx = rg.s * cp, ny = rg.s * sp, nz = rg.z;
            const double2 dd = grid ? make_double2(0.0, 0.0) : __ldg(reinterpret_cast<const double2 *>(a.defl) + p);
            const double dl = sqrt(dd.x * dd.x + dd.y * dd.y);
            double x = nx, y = ny, z = nz;
            if (dl > 0.0) {
                double sd, cd;
                sincos(dl, &sd, &cd);
                const double k = sd / dl;
                // e_theta = (z cos phi, z sin phi, -s), e_phi = (-sin phi, cos phi, 0)
                const double tx = dd.x * nz * cp - dd.y * sp;
                const double ty = dd.x * nz * sp + dd.y * cp;
                const double tz = -dd.x * rg.s;
                x = cd * nx + k * tx;
                y = cd * ny + k * ty;
                z = cd * nz + k * tz;
            }
            const double s = sqrt(x * x + y * y);
            P.x = x;
            P.y = y;
            P.z = z;
            P.s = s;
            if (s > 1e-12) {
                P.cph = x / s;
                P.sph = y / s;
            } else {
                P.cph = 1.0;
                P.sph = 0.0;
                P.flags |= FLINTS_ST_POLE;
            }
            P.phi = atan2(y, x);
            P.rot_re = 1.0;
            P.rot_im = 0.0;
            if (SPIN != 0 && a.rotate && dl > 0.0) {
                // P(n) = P(n') exp(is(a_nn' - a_n'n - pi)) with a_uv the angle at u, from
                // e_theta towards e_phi, of the geodesic towards v: the field parallel-
                // transported back along the deflection.  At n the direction is
                // (d_theta, d_phi) itself; at n' it is (n . e_theta(n'), n . e_phi(n')).
                const double w1r = dd.x, w1i = dd.y;
                const double cq = P.cph, sq = P.sph;
                const double w2r = nx * z * cq + ny * z * sq - nz * s, w2i = ny * cq - nx * sq;
                const double n1 = w1r * w1r + w1i * w1i, n2 = w2r * w2r + w2i * w2i;
                if (n1 > 0.0 && n2 > 0.0) {
                    if (SPIN == 1) {
                        const double inv = -rsqrt(n1 * n2);  // exp(-i pi) for odd spin
                        P.rot_re = (w1r * w2r + w1i * w2i) * inv;  // w1 conj(w2) / |w1 w2|
                        P.rot_im = (w1i * w2r - w1r * w2i) * inv;
                    } else {
                        const double a1r = w1r * w1r - w1i * w1i, a1i = 2.0 * w1r * w1i;
                        const double a2r = w2r * w2r - w2i * w2i, a2i = 2.0 * w2r * w2i;
                        const double inv = 1.0 / (n1 * n2);
                        P.rot_re = (a1r * a2r + a1i * a2i) * inv;  // a1 conj(a2)
                        P.rot_im = (a1i * a2r - a1r * a2i) * inv;
                    }
                }
            }
            if (!grid && !(isfinite(dd.x) && isfinite(dd.y))) {
                // a non-finite deflection is not taken as none: the point is not solved
                const double nan = __longlong_as_double(0x7ff8000000000000ll);
                P.x = P.y = P.z = P.s = P.phi = nan;
                P.flags = FLINTS_ST_INPUT;
                z = nan;
            }
            P.zf = (float)P.z;
            P.sf = (float)P.s;
            P.phif = (float)P.phi;
            P.ic = ring_above(N, z);
        }
        if (lane < MAX_TILE_POINTS) sm.pts[lane] = P;
    }
    __syncwarp();

    // ------------------------------------------------ phase B: per point
    for (int q = 0; q < tile_pts; ++q) {
        const int64_t p = tile * tile_pts + q;
        if (p >= a.count) break;
        const PointA P = sm.pts[q];
        int flags = P.flags;
        // rings of the search disc, one per lane
        int cnt = 0;
        {
            RingRec rec{};
            const int64_t i = P.ic - R_rings + lane;
            if (lane < 2 * R_rings + 2 && i >= 1 && i <= 4 * N - 1) {
                // exact ring latitude in FP64 (needed for the selected neighbours' positions);
                // the candidate range and the FP32 key terms in FP32, with
                // ds = s' - s_r = -dz (z' + z_r)/(s' + s_r), accurate to FP32 from FP64 dz
                const Ring rg = ring_of(N, i, inv3N, inv3N2);
                const double dz = P.z - rg.z;
                const float dzf = (float)dz;
                const float zrf = (float)rg.z, srf = (float)rg.s;
                const float dsf = -dzf * ((P.zf + zrf) / (P.sf + srf));
                const float lbf = fmaf(dzf, dzf, dsf * dsf);
                const float r2f = (float)a.r2;
                if (lbf <= r2f * 1.00001f) {
                    const float den = 4.0f * P.sf * srf;
                    const float qv = den > 0.0f ? (r2f * 1.00001f - lbf) / den : 2.0f;
                    int j0 = 0, c = rg.n_in;
                    const float stepf = (float)rg.n_in * 0.15915494309189535f;  // pixels per radian
                    if (qv < 1.0f) {
                        const float half = 2.0f * asinf(sqrtf(fmaxf(qv, 0.0f)));
                        const float lo = (P.phif - half) * stepf - (float)rg.f;
                        const float hi = (P.phif + half) * stepf - (float)rg.f;
                        // FP32 rounding moves lo and hi by < 0.02 pixel for Nside <= 16384
                        const int jl = (int)floorf(lo - 0.03125f), jh = (int)ceilf(hi + 0.03125f);
                        const int cc = jh - jl + 1;
                        if (cc < rg.n_in) {
                            c = cc;
                            // jl >= -n_in - 2 (phi' from atan2 is in [-pi, pi], half < pi) and
                            // jl <= n_in / 2: two conditional wraps give jl mod n_in
                            int m = jl;
                            if (m < 0) m += rg.n_in;
                            if (m < 0) m += rg.n_in;
                            j0 = m;
                        }
                    }
                    // FP32 key terms: chord^2 = dz^2 + ds^2 + 4 s' s sin^2(dphi/2) with
                    // dphi/2 = pi (j + f - u') / n_in, u' = phi' n_in / (2 pi) in FP64
                    const double u = P.phi * ((double)rg.n_in * (0.5 / PI));
                    const double jr = floor(u - rg.f + 0.5);
                    rec.frac = (float)((jr + rg.f) - u);
                    // |u| <= n_in / 2, so jr lies in [-n_in / 2 - 1, n_in / 2 + 1]: one wrap each way
                    int jri = (int)jr;
                    if (jri < 0) jri += rg.n_in;
                    if (jri >= rg.n_in) jri -= rg.n_in;
                    rec.jref = jri;
                    rec.a32 = lbf;
                    rec.b32 = den;
                    rec.inv_n = 1.0f / (float)rg.n_in;
                    rec.z = rg.z;
                    rec.s = rg.s;
                    rec.f = rg.f;
                    rec.first = rg.first;
                    rec.n_in = rg.n_in;
                    rec.inv2nq = 1.0 / (2.0 * (double)rg.nq);  // beside ring_of's square root, not in the placement chain
                    rec.j0 = j0;
                    rec.cnt = c;
                    cnt = c;
                }
            }
            // inclusive scan of counts
            int incl = cnt;
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const int v = __shfl_up_sync(FULL, incl, o);
                if (lane >= o) incl += v;
            }
            rec.end = incl;
            sm.u.cand.rings[lane] = rec;
            cnt = __shfl_sync(FULL, incl, 31);  // total candidates
        }
        const int C = cnt;
        __syncwarp();
        bool fail = false;
        if (flags & FLINTS_ST_INPUT) {
            fail = true;
            flags |= FLINTS_ST_FAILED;
        } else if (C > NSLOT || C < K) {
            fail = true;
            flags |= FLINTS_ST_WINDOW | FLINTS_ST_FAILED;
        }
        // selected neighbours: FP64 key bits and candidate id per owned row
        unsigned long long key[RPL];
        unsigned id[RPL];
        if (!fail) {
            // 1. FP32 keys of all candidates, packed with the candidate id (ids follow
            //    the RING index, so equal keys order by pixel), one sort
            unsigned long long pk[SPL];
#pragma unroll
            for (int s = 0; s < SPL; ++s) {
                const int c = s * 32 + lane;
                pk[s] = ~0ull;
                if (c < C) {
                    int lo = 0, hi = 31;  // ring holding candidate c: first r with end > c
                    while (lo < hi) {
                        const int mid = (lo + hi) >> 1;
                        if (sm.u.cand.rings[mid].end > c) hi = mid;
                        else lo = mid + 1;
                    }
                    const RingRec &rr = sm.u.cand.rings[lo];
                    const int k = c - (rr.end - rr.cnt);
                    const int w = rr.j0 + rr.cnt - rr.n_in;  // wrapped count
                    const int jj = (w > 0) ? (k < w ? k : rr.j0 + (k - w)) : rr.j0 + k;
                    int dj = jj - rr.jref;
                    if (dj > rr.n_in / 2) dj -= rr.n_in;
                    if (dj < -(rr.n_in / 2)) dj += rr.n_in;
                    const float sn = sinpif(((float)dj + rr.frac) * rr.inv_n);
                    const float k32 = fmaf(rr.b32, sn * sn, rr.a32);
                    sm.u.cand.cpix[c] = ((uint32_t)lo << 24) | (uint32_t)jj;
                    pk[s] = ((unsigned long long)__float_as_uint(fmaxf(k32, 0.0f)) << 32) | (unsigned)c;
                }
            }
            bitonic_sort_packed<SPL>(pk, lane);
            // 2. exact set unless the K-th and (K+1)-th FP32 keys are within 2^-16
            const unsigned long long ka = __shfl_sync(FULL, pk[(K - 1) >> 5], (K - 1) & 31);
            const unsigned long long kb = __shfl_sync(FULL, pk[K >> 5], K & 31);
            const float fa = __uint_as_float((unsigned)(ka >> 32)), fb = __uint_as_float((unsigned)(kb >> 32));
            const bool exact = (C == K) || (fb - fa > fb * 1.52587890625e-05f);
            __syncwarp();
            // 3. FP64 positions and keys: of the K selected (fast) or of all candidates
            auto place = [&](int c) -> unsigned long long {
                const uint32_t pkd = sm.u.cand.cpix[c];
                const RingRec &rr = sm.u.cand.rings[pkd >> 24];
                const int jj = (int)(pkd & 0xffffffu);
                double sp, cp;
                sincospi(((double)jj + rr.f) * rr.inv2nq, &sp, &cp);
                const double cx = rr.s * cp, cy = rr.s * sp, cz = rr.z;
                const double ex = P.x - cx, ey = P.y - cy, ez = P.z - cz;
                sm.u.cand.cx[c] = cx;
                sm.u.cand.cy[c] = cy;
                sm.u.cand.cz[c] = cz;
                sm.u.cand.cc[c] = cp;
                sm.u.cand.cs[c] = sp;
                return (unsigned long long)__double_as_longlong(ex * ex + ey * ey + ez * ez);
            };
            if (exact) {
#pragma unroll
                for (int r = 0; r < RPL; ++r) {
                    key[r] = 0x7ff0000000000000ull;
                    id[r] = 0xffffffffu;
                    if (lane + 32 * r < K) {
                        const unsigned c = (unsigned)(pk[r] & 0xffffffffu);
                        key[r] = place((int)c);
                        id[r] = c;
                    }
                }
                __syncwarp();
                bitonic_sort<RPL>(key, id, lane);
            } else {
                // Near-tie at the K-th place.  A candidate whose FP32 key exceeds the
                // K-th one by more than the margin is farther than the true K-th
                // neighbour (FP32 keys are within 2^-17 relative), so FP64 keys are
                // needed only for the FP32-ranked candidates below that threshold.
                const unsigned thr = __float_as_uint(fa * (1.0f + 1.52587890625e-05f));
                int hi = 0;
#pragma unroll
                for (int s = 0; s < SPL; ++s) hi += __popc(__ballot_sync(FULL, (unsigned)(pk[s] >> 32) <= thr));
                constexpr int S2 = RPL + 1 <= 2 ? 2 : 4;  // power of two >= RPL + 1, <= SPL
                static_assert(S2 <= SPL, "near-tie slots exceed the candidate slots");
                if (hi <= 32 * S2) {
                    unsigned long long k2[S2];
                    unsigned i2[S2];
#pragma unroll
                    for (int s = 0; s < S2; ++s) {
                        k2[s] = 0x7ff0000000000000ull;
                        i2[s] = 0xffffffffu;
                        if (s * 32 + lane < hi) {
                            const unsigned c = (unsigned)(pk[s] & 0xffffffffu);
                            k2[s] = place((int)c);
                            i2[s] = c;
                        }
                    }
                    __syncwarp();
                    bitonic_sort<S2>(k2, i2, lane);
#pragma unroll
                    for (int r = 0; r < RPL; ++r) {
                        key[r] = k2[r];
                        id[r] = i2[r];
                    }
                } else {
                    // a wide tie (many equidistant candidates): FP64 keys of all
                    unsigned long long k2[SPL];
                    unsigned i2[SPL];
#pragma unroll
                    for (int s = 0; s < SPL; ++s) {
                        const int c = s * 32 + lane;
                        k2[s] = 0x7ff0000000000000ull;
                        i2[s] = 0xffffffffu;
                        if (c < C) {
                            k2[s] = place(c);
                            i2[s] = (unsigned)c;
                        }
                    }
                    __syncwarp();
                    bitonic_sort<SPL>(k2, i2, lane);
#pragma unroll
                    for (int r = 0; r < RPL; ++r) {
                        key[r] = k2[r];
                        id[r] = i2[r];
                    }
                }
            }
            // K-th neighbour inside the disc?
            const unsigned long long kK = __shfl_sync(FULL, key[(K - 1) >> 5], (K - 1) & 31);
            if (__longlong_as_double((long long)kK) > a.r2) {
                fail = true;
                flags |= FLINTS_ST_WINDOW | FLINTS_ST_FAILED;
            }
        }
        __syncwarp();
        double keyd[RPL], yre[RPL], yim[RPL];
        uint32_t pixr[RPL];
        if (!fail) {
#pragma unroll
            for (int r = 0; r < RPL; ++r) {
                const int i = lane + 32 * r;
                keyd[r] = 0.0;
                yre[r] = 0.0;
                yim[r] = 0.0;
                pixr[r] = 0;
                if (i < K) {
                    const unsigned c = id[r];
                    keyd[r] = __longlong_as_double((long long)key[r]);
                    sm.ktf[i] = (float)keyd[r];
                    const double cx = sm.u.cand.cx[c], cy = sm.u.cand.cy[c], cz = sm.u.cand.cz[c];
                    const double ox = cx - P.x, oy = cy - P.y, oz = cz - P.z;
                    const uint32_t pkd = sm.u.cand.cpix[c];
                    const RingRec &rr = sm.u.cand.rings[pkd >> 24];
                    // sin(theta) of the neighbour is its ring's s (cx, cy = s (cos phi, sin phi))
                    const double ns = rr.s, nc = sm.u.cand.cc[c], nsn = sm.u.cand.cs[c];
                    pixr[r] = (uint32_t)(rr.first + (pkd & 0xffffffu));
                    if (MIXED) {
                        SMf &smf = *reinterpret_cast<SMf *>(wbase);
                        // offsets |X_i - n'| <= r (the K-th chord is inside the disc): high
                        // words on the grid of [M, 2M), M = 1.5 * 2^E with 2^E >= 4 r
                        const float Mg = 0.25f * anc_anchor(4.0f * sqrtf((float)a.r2));
                        smf.gx[i] = df_on_grid(ox, Mg);
                        smf.gy[i] = df_on_grid(oy, Mg);
                        smf.gz[i] = df_on_grid(oz, Mg);
                        smf.gnz[i] = df_from(cz);
                        smf.gns[i] = df_from(ns);
                        smf.gnc[i] = df_from(nc);
                        smf.gnsn[i] = df_from(nsn);
                    } else {
                        sm.gx[i] = ox;
                        sm.gy[i] = oy;
                        sm.gz[i] = oz;
                        sm.gnz[i] = cz;
                        sm.gns[i] = ns;
                        sm.gnc[i] = nc;
                        sm.gnsn[i] = nsn;
                    }
                }
            }
        }
        __syncwarp();
        if (a.stencil) {
            if (!fail) {
#pragma unroll
                for (int r = 0; r < RPL; ++r) {
                    const int i = lane + 32 * r;
                    if (i < K) a.stencil[p * K + i] = (int64_t)pixr[r];
                }
            } else {
                for (int i = lane; i < K; i += 32) a.stencil[p * K + i] = -1;
            }
            if (lane == 0) {
                if (a.status) a.status[p] = (uint8_t)flags;
                if (flags & FLINTS_ST_WINDOW) ++ctr.win;
                if (flags & FLINTS_ST_FAILED) ++ctr.fail;
            }
            continue;
        }
        double vre = __longlong_as_double(0x7ff8000000000000ll), vim = vre, vrel = vre;
        if (!fail) {
#pragma unroll
            for (int r = 0; r < RPL; ++r) {
                const int i = lane + 32 * r;
                if (i < K) {
                    if (SPIN == 0) {
                        yre[r] = __ldg(a.map + pixr[r]);
                    } else {
                        const double2 v = __ldg(reinterpret_cast<const double2 *>(a.map) + pixr[r]);
                        yre[r] = v.x;
                        yim[r] = v.y;
                    }
                }
            }
            bool solved = false;
            if (MIXED) {
                SMf &smf = *reinterpret_cast<SMf *>(wbase);
                solved = solve_any<K, SPIN, df>(smf, P, lane, NUGGET_EPS, a, keyd, yre, yim, vre, vim, vrel);
                __syncwarp();
                if (a.force_fallback) solved = false;
                if (!solved) {
                    // FP64 fallback: widen the double-float geometry in place (offsets keep
                    // ~2^-48 of their own size, the O(1) terms ~2^-48 absolute)
                    flags |= FLINTS_ST_FALLBACK;
                    for (int i = lane; i < K; i += 32) {
                        const double g[7] = {df_to(smf.gx[i]), df_to(smf.gy[i]), df_to(smf.gz[i]), df_to(smf.gnz[i]),
                                             df_to(smf.gns[i]), df_to(smf.gnc[i]), df_to(smf.gnsn[i])};
                        sm.gx[i] = g[0];
                        sm.gy[i] = g[1];
                        sm.gz[i] = g[2];
                        sm.gnz[i] = g[3];
                        sm.gns[i] = g[4];
                        sm.gnc[i] = g[5];
                        sm.gnsn[i] = g[6];
                    }
                    __syncwarp();
                }
            }
            double nug = NUGGET_EPS;
            for (int step = 0; !solved && step <= MAX_NUGGET_STEPS; ++step) {
                if (step > 0) {
                    nug *= 2.0;
                    flags |= FLINTS_ST_NUGGET;
                }
                solved = solve_any<K, SPIN, double>(sm, P, lane, nug, a, keyd, yre, yim, vre, vim, vrel);
                __syncwarp();
            }
            if (!solved) {
                flags |= FLINTS_ST_FAILED;
                vre = vim = vrel = __longlong_as_double(0x7ff8000000000000ll);
            }
        }
        if (lane == 0) {
            if (SPIN == 0) {
                a.out[p] = vre;
            } else {
                reinterpret_cast<double2 *>(a.out)[p] =
                    make_double2(vre * P.rot_re - vim * P.rot_im, vre * P.rot_im + vim * P.rot_re);
            }
            if (a.var) a.var[p] = a.xi0 * vrel;
            if (a.status) a.status[p] = (uint8_t)flags;
            if (flags & FLINTS_ST_NUGGET) ++ctr.nug;
            if (flags & FLINTS_ST_FALLBACK) ++ctr.fb;
            if (flags & FLINTS_ST_WINDOW) ++ctr.win;
            if (flags & FLINTS_ST_FAILED) ++ctr.fail;
        }
        __syncwarp();
    }
}

// Single-launch kernel: warps take the tiles of one target range from the launch's
// queue (a static grid stride when no queue is given).
template <int K, int SPIN, int MIXED>
__global__ void __launch_bounds__(256, 2) lens_kernel(LensArgs a, int R_rings, int tile_pts) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, wpb = blockDim.x >> 5;
    unsigned char *wbase = smem_raw + (size_t)warp * warp_smem_bytes<K, SPIN, MIXED>();
    const int64_t ntiles = (a.count + tile_pts - 1) / tile_pts;
    Counters ctr;
    if (a.queue) {
        // dynamic tiles: the cost of a tile varies (candidate counts, near ties), and
        // taking the next free tile keeps every warp busy to the end of the launch
        for (;;) {
            unsigned long long t = 0;
            if (lane == 0) t = atomicAdd(a.queue, 1ull);
            t = __shfl_sync(FULL, t, 0);
            if ((int64_t)t >= ntiles) break;
            process_tile<K, SPIN, MIXED>(a, R_rings, (int64_t)t, tile_pts, wbase, lane, ctr);
        }
    } else {
        for (int64_t tile = (int64_t)blockIdx.x * wpb + warp; tile < ntiles; tile += (int64_t)gridDim.x * wpb)
            process_tile<K, SPIN, MIXED>(a, R_rings, tile, tile_pts, wbase, lane, ctr);
    }
    flush_counters(ctr, a.counters, lane);
}

template <int K, int SPIN, int MIXED>
cudaError_t launch_one(const LensArgs &a, int R_rings, const LaunchCfg &cfg, int num_sms, cudaStream_t st) {
    int wpb = cfg.warps_per_block > 0 ? cfg.warps_per_block : 4;
    const int tile_pts = cfg.tile_points > 0 && cfg.tile_points < MAX_TILE_POINTS ? cfg.tile_points : MAX_TILE_POINTS;
    // the launch shape is a hint: keep the block within the opt-in shared memory
    const int fit = (int)(device_smem_optin() / warp_smem_bytes<K, SPIN, MIXED>());
    if (wpb > fit) wpb = fit > 0 ? fit : 1;
    const size_t smem = (size_t)wpb * warp_smem_bytes<K, SPIN, MIXED>();
    auto kern = lens_kernel<K, SPIN, MIXED>;
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    int per_sm = 0;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, wpb * 32, smem);
    if (e != cudaSuccess) return e;
    if (per_sm < 1) return cudaErrorInvalidConfiguration;
    if (cfg.blocks_per_sm > 0 && cfg.blocks_per_sm < per_sm) per_sm = cfg.blocks_per_sm;
    const int64_t ntiles = (a.count + tile_pts - 1) / tile_pts;
    int64_t blocks = (int64_t)num_sms * per_sm;
    const int64_t need = (ntiles + wpb - 1) / wpb;
    if (blocks > need) blocks = need;
    if (blocks < 1) blocks = 1;
    kern<<<(unsigned)blocks, wpb * 32, smem, st>>>(a, R_rings, tile_pts);
    return cudaGetLastError();
}

}  // namespace flints

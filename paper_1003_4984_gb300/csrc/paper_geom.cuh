// HEALPix base-face geometry in integer arithmetic for the pixel-centred
// stencil of Sec. 2.3 and its S^-1 tabulation (Sec. 2.4).
//
// Faces: the sphere is cut into 12 base faces; face f holds pixels (f, ix, iy),
// 0 <= ix, iy < N.  Face f has ring coordinate jrll(f) (in units of N rings) and
// azimuth coordinate jpll(f) (in units of pi/4):
//     jrll = 2 2 2 2 3 3 3 3 4 4 4 4,   jpll = 1 3 5 7 0 2 4 6 1 3 5 7.
// The face point (X, Y) in [0, 1]^2 lies on ring coordinate rho = jrll - X - Y,
// in the polar caps (rho < 1 or rho > 3) at azimuth (pi/4)(jpll + (X - Y)/rho')
// with rho' = rho or 4 - rho, in the belt at (pi/4)(jpll + X - Y).  Pixel
// vertices are the images of the integer face points (u/N, v/N), so two
// vertices coincide exactly when their integer keys (R, Phi) below agree.
//
// All functions are host-device and use integer arithmetic only.
#pragma once
#include <cmath>
#include <cstdint>

namespace flints {
namespace paper {

__host__ __device__ __forceinline__ int face_jrll(int f) { return f < 4 ? 2 : (f < 8 ? 3 : 4); }
__host__ __device__ __forceinline__ int face_jpll(int f) {
    const int q = f & 3;
    return (f >= 4 && f < 8) ? 2 * q : 2 * q + 1;
}

// pixels per quarter ring (the ring holds 4 nq pixels), rings 1 .. 4N-1
__host__ __device__ __forceinline__ int64_t ring_nq(int64_t N, int64_t i) {
    return i < N ? i : (i > 3 * N ? 4 * N - i : N);
}
// azimuth of pixel j of ring i: phi = (2 j + sh) pi / (4 nq)
__host__ __device__ __forceinline__ int ring_sh(int64_t N, int64_t i) {
    if (i < N || i > 3 * N) return 1;
    return ((i + N) & 1) ? 0 : 1;
}
__host__ __device__ __forceinline__ int64_t ring_start(int64_t N, int64_t i) {
    if (i < N) return 2 * i * (i - 1);
    if (i <= 3 * N) return 2 * N * (N - 1) + 4 * N * (i - N);
    const int64_t ip = 4 * N - i;
    return 12 * N * N - 2 * ip * (ip + 1);
}

// ring i (1-based) and position j (0-based) of RING pixel p
__host__ __device__ __forceinline__ void ring_and_pos(int64_t N, int64_t p, int64_t &i, int64_t &j) {
    const int64_t ncap = 2 * N * (N - 1), npix = 12 * N * N;
    if (p < ncap) {
        int64_t r = (int64_t)(0.5 * (1.0 + sqrt(1.0 + 2.0 * (double)p)));
        while (r > 1 && 2 * r * (r - 1) > p) --r;
        while (2 * (r + 1) * r <= p) ++r;
        i = r;
        j = p - 2 * r * (r - 1);
    } else if (p < npix - ncap) {
        const int64_t q = p - ncap;
        i = q / (4 * N) + N;
        j = q - (i - N) * 4 * N;
    } else {
        const int64_t pp = npix - 1 - p;
        int64_t r = (int64_t)(0.5 * (1.0 + sqrt(1.0 + 2.0 * (double)pp)));
        while (r > 1 && 2 * r * (r - 1) > pp) --r;
        while (2 * (r + 1) * r <= pp) ++r;
        i = 4 * N - r;
        j = p - (npix - 2 * r * (r + 1));
    }
}

struct Xyf {
    int64_t ix, iy;
    int f;
};

__host__ __device__ __forceinline__ int64_t pmod(int64_t a, int64_t m) {
    const int64_t r = a % m;
    return r < 0 ? r + m : r;
}

// Face coordinates of pixel j of ring i.  Caps: the quarter q = j / nq is the
// face; ix + iy and ix - iy follow from the ring and the position.  Belt: with
// P = 2j - i - ks and Q = -2j - i - 2 + ks (ks = 1 on rings with phi_0 = 0),
// 2 ix = (jrll - jpll) N + P and 2 iy = (jrll + jpll) N + Q modulo 8N, both in
// [0, 2N); each fixes an odd residue of (jrll -+ jpll) mod 8, and the pair of
// residues names the face.
__host__ __device__ __forceinline__ Xyf ring2xyf(int64_t N, int64_t i, int64_t j) {
    Xyf r;
    if (i < N) {
        const int64_t q = j / i;
        const int64_t s = 2 * N - 1 - i, d = 2 * (j - q * i) + 1 - i;
        r.ix = (s + d) / 2;
        r.iy = (s - d) / 2;
        r.f = (int)q;
        return r;
    }
    if (i > 3 * N) {
        const int64_t nq = 4 * N - i;
        const int64_t q = j / nq;
        const int64_t s = nq - 1, d = 2 * (j - q * nq) + 1 - nq;
        r.ix = (s + d) / 2;
        r.iy = (s - d) / 2;
        r.f = 8 + (int)q;
        return r;
    }
    const int64_t ks = (i - N) & 1;
    const int64_t pA = pmod(2 * j - i - ks, 8 * N), pB = pmod(-2 * j - i - 2 + ks, 8 * N);
    const int64_t kA = pA / N, kB = pB / N;
    const int64_t A = pA - kA * N + ((kA & 1) ? 0 : N);
    const int64_t B = pB - kB * N + ((kB & 1) ? 0 : N);
    const int a = (int)((kA & 1) ? (8 - kA) & 7 : (9 - kA) & 7);  // jrll - jpll mod 8
    const int b = (int)((kB & 1) ? (8 - kB) & 7 : (9 - kB) & 7);  // jrll + jpll mod 8
    // face + 1 in the nibble ((a >> 1) * 4 + (b >> 1)); 0 marks residue pairs no
    // face has: (a, b) = (1,3) 0, (7,5) 1, (5,7) 2, (3,1) 3, (3,3) 4, (1,5) 5,
    // (7,7) 6, (5,1) 7, (3,5) 8, (1,7) 9, (7,1) 10, (5,3) 11
    constexpr uint64_t FACE_OF = 0x720b30c80954a610ull;
    r.ix = A / 2;
    r.iy = B / 2;
    r.f = (int)((FACE_OF >> (4 * ((a >> 1) * 4 + (b >> 1)))) & 15) - 1;
    return r;
}

// RING index (and ring, position) of pixel (f, ix, iy)
__host__ __device__ __forceinline__ int64_t xyf2ring(int64_t N, int64_t ix, int64_t iy, int f, int64_t &ring,
                                                     int64_t &pos) {
    const int64_t jr = (int64_t)face_jrll(f) * N - ix - iy - 1;
    const int64_t nq = ring_nq(N, jr);
    const int64_t ks = (jr >= N && jr <= 3 * N) ? ((jr - N) & 1) : 0;
    int64_t jp = ((int64_t)face_jpll(f) * nq + ix - iy + 1 + ks) / 2;
    if (jp > 4 * nq) jp -= 4 * nq;
    if (jp < 1) jp += 4 * nq;
    ring = jr;
    pos = jp - 1;
    return ring_start(N, jr) + jp - 1;
}

// Exact key of the vertex at integer face point (u, v) of face f: ring
// coordinate R = jrll N - u - v in [0, 4N] and azimuth Phi in units of
// pi/(4 nq(R)), reduced modulo 8 nq(R); the poles have Phi = 0.
__host__ __device__ __forceinline__ uint64_t vertex_key(int64_t N, int64_t u, int64_t v, int f) {
    const int64_t R = (int64_t)face_jrll(f) * N - u - v;
    if (R <= 0) return 0;
    if (R >= 4 * N) return (uint64_t)(4 * N) << 32;
    const int64_t nq = R < N ? R : (R > 3 * N ? 4 * N - R : N);
    const int64_t phi = pmod((int64_t)face_jpll(f) * nq + u - v, 8 * nq);
    return ((uint64_t)R << 32) | (uint64_t)phi;
}

__host__ __device__ __forceinline__ void pixel_vertex_keys(int64_t N, const Xyf &p, uint64_t (&k)[4]) {
    k[0] = vertex_key(N, p.ix, p.iy, p.f);
    k[1] = vertex_key(N, p.ix + 1, p.iy, p.f);
    k[2] = vertex_key(N, p.ix, p.iy + 1, p.f);
    k[3] = vertex_key(N, p.ix + 1, p.iy + 1, p.f);
}

// Symmetry class ("slot") of coarse pixel j of ring i at Nside Nc.  The grid is
// invariant under the reflection z -> -z (ring i -> 4Nc - i, same j), under
// rotations by pi/2 (j -> j + nq) and, on rings whose stencil lies wholly in
// the equatorial belt, under the rotation by one pixel.  Folded ring
// i' = min(i, 4Nc - i); rings Nc + 3 <= i' <= 2Nc (stencil inside the belt)
// share one slot; the others have one slot per position j mod nq(i').
__host__ __device__ __forceinline__ int64_t slot_base(int64_t Nc, int64_t ip) {
    // sum of nq(r) over folded rings r < ip
    if (ip <= Nc) return (ip - 1) * ip / 2;
    return (Nc - 1) * Nc / 2 + (ip - Nc) * Nc;
}
__host__ __device__ __forceinline__ int64_t slot_last_private(int64_t Nc) {
    return (Nc + 2 < 2 * Nc) ? Nc + 2 : 2 * Nc;
}
__host__ __device__ __forceinline__ int64_t slot_count(int64_t Nc) {
    const int64_t priv = slot_base(Nc, slot_last_private(Nc) + 1);
    return priv + (Nc > 2 ? Nc - 2 : 0);
}
__host__ __device__ __forceinline__ int64_t slot_of(int64_t Nc, int64_t i, int64_t j) {
    const int64_t ip = i < 4 * Nc - i ? i : 4 * Nc - i;
    if (ip > slot_last_private(Nc)) return slot_base(Nc, slot_last_private(Nc) + 1) + (ip - Nc - 3);
    const int64_t q = ip < Nc ? ip : Nc;
    return slot_base(Nc, ip) + j % q;
}
// representative coarse pixel (north hemisphere, first quarter) of a slot
__host__ __device__ __forceinline__ int64_t slot_rep(int64_t Nc, int64_t s) {
    const int64_t last = slot_last_private(Nc);
    const int64_t priv = slot_base(Nc, last + 1);
    if (s >= priv) return ring_start(Nc, Nc + 3 + (s - priv));
    // largest ring ip with slot_base(ip) <= s
    int64_t lo = 1, hi = last;
    while (lo < hi) {
        const int64_t mid = (lo + hi + 1) / 2;
        if (slot_base(Nc, mid) <= s) lo = mid; else hi = mid - 1;
    }
    return ring_start(Nc, lo) + (s - slot_base(Nc, lo));
}


// Largest stencil the tabulated path builds: 9 * 4^(y-1) members for y <= 2.
constexpr int STENCIL_MAX = 36;

// Members of the level-y stencil of coarse pixel c (Nside Nc), as RING indices
// at N = Nc k, k = 2^(y-1): the pixel and the pixels of the Nc grid sharing a
// vertex with it (found among rings i-2 .. i+2 within 3 pixels of its azimuth),
// each replaced by its k^2 sub-pixels (fx, fy) = (k ix + a, k iy + b).
//
// Order (the rule that lets symmetric pixels share one S^-1): members sorted by
// (s r, dphi), r the member's ring, s = +1 for c in the northern half (ring <=
// 2Nc) and -1 in the southern, dphi the member's azimuth minus c's, wrapped to
// (-pi, pi] and compared as exact fractions of a quarter turn.  Rotations of the
// grid keep r and dphi, the reflection z -> -z keeps dphi and maps s r to
// s r - 4N, so every pixel of a slot lists its members in corresponding order.
//
// Returns the member count (9 k^2, or 8 k^2 next to the points where three
// faces meet, 7 k^2 at Nc = 1) or -1 when more than 8 neighbours are found.
__host__ __device__ inline int stencil_members(int64_t Nc, int k, int64_t c, int32_t *out) {
    const int64_t N = Nc * k;
    int64_t ic, jc;
    ring_and_pos(Nc, c, ic, jc);
    const Xyf xc = ring2xyf(Nc, ic, jc);
    uint64_t kc[4];
    pixel_vertex_keys(Nc, xc, kc);
    Xyf co[9];
    int nc = 0;
    co[nc++] = xc;
    const int64_t nqc = ring_nq(Nc, ic);
    const int shc = ring_sh(Nc, ic);
    const int64_t r0 = ic - 2 < 1 ? 1 : ic - 2, r1 = ic + 2 > 4 * Nc - 1 ? 4 * Nc - 1 : ic + 2;
    for (int64_t r = r0; r <= r1; ++r) {
        const int64_t nqr = ring_nq(Nc, r), nin = 4 * nqr;
        // position of c's azimuth in ring r's pixel units
        const double x = (double)((2 * jc + shc) * nqr) / (double)(2 * nqc) - 0.5 * (double)ring_sh(Nc, r);
        int64_t lo = (int64_t)floor(x - 3.0), cnt = (int64_t)ceil(x + 3.0) - lo + 1;
        if (cnt >= nin) {
            lo = 0;
            cnt = nin;
        }
        for (int64_t t = 0; t < cnt; ++t) {
            const int64_t jj = pmod(lo + t, nin);
            if (r == ic && jj == jc) continue;
            const Xyf xr = ring2xyf(Nc, r, jj);
            uint64_t kr[4];
            pixel_vertex_keys(Nc, xr, kr);
            bool share = false;
            for (int u = 0; u < 4; ++u)
                for (int v = 0; v < 4; ++v) share |= (kc[u] == kr[v]);
            if (share) {
                if (nc == 9) return -1;
                co[nc++] = xr;
            }
        }
    }
    if (nc * k * k > STENCIL_MAX) return -1;
    const int64_t s = ic <= 2 * Nc ? 1 : -1;
    const int64_t uc = 2 * jc + shc;  // c's azimuth: uc / (2 nqc) quarter turns
    int64_t key1[STENCIL_MAX], num[STENCIL_MAX], den[STENCIL_MAX];
    int32_t pix[STENCIL_MAX];
    int n = 0;
    for (int m = 0; m < nc; ++m) {
        for (int b = 0; b < k; ++b) {
            for (int a = 0; a < k; ++a) {
                int64_t ring, pos;
                const int64_t p = xyf2ring(N, co[m].ix * k + a, co[m].iy * k + b, co[m].f, ring, pos);
                const int64_t nq = ring_nq(N, ring);
                // dphi = ((2 pos + sh) nqc - uc nq) / (2 nq nqc) quarter turns, wrapped to (-2, 2]
                const int64_t d = 2 * nq * nqc;
                int64_t q = (2 * pos + ring_sh(N, ring)) * nqc - uc * nq;
                if (q > 2 * d) q -= 4 * d;
                if (q <= -2 * d) q += 4 * d;
                // insertion into the sorted prefix
                int at = n;
                while (at > 0) {
                    const bool less = (s * ring < key1[at - 1]) ||
                                      (s * ring == key1[at - 1] && q * den[at - 1] < num[at - 1] * d);
                    if (!less) break;
                    key1[at] = key1[at - 1];
                    num[at] = num[at - 1];
                    den[at] = den[at - 1];
                    pix[at] = pix[at - 1];
                    --at;
                }
                key1[at] = s * ring;
                num[at] = q;
                den[at] = d;
                pix[at] = (int32_t)p;
                ++n;
            }
        }
    }
    for (int m = 0; m < n; ++m) out[m] = pix[m];
    return n;
}

}  // namespace paper
}  // namespace flints

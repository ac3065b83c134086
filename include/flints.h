/* flints.h -- C ABI of the GB300 lensing remap (FLINTS kriging interpolation).
 *
 * The library computes, for every target HEALPix pixel, the value of an
 * isotropic Gaussian field at the displaced direction n' = n + d(n) and the
 * Gaussian variance of that estimate, from the K nearest pixels of an unlensed
 * RING-ordered map (Lavaux & Wandelt, "Fast and optimal CMB lensing using
 * statistical interpolation on the sphere").
 *
 *   Displacement   Sec. 3.1, lensed-direction equation:
 *                  n' = cos|d| n + sin|d| (d_theta e_theta + d_phi e_phi)/|d|.
 *   Covariances    Eq. fundamental_variance / Eq. correlation_func (spin 0),
 *                  Eq. v_spins / Eq. spins_correl (spin s = 1, 2).
 *   Estimate       Eq. best_temperature_field and Eq. gaussvar (spin 0),
 *                  Eq. major_eq and Eq. gaussvar_pol (spin s).
 *   Regularisation Sec. 2.4: Cholesky of S + n I with n = 1.49e-8.
 *   xi tabulation  Sec. 2.5 step 2 and Appendix B: cubic interpolation.
 *
 * Conventions shared by every entry point
 * ---------------------------------------
 * - Map buffers are RING ordered, Npix = 12 Nside^2.  Spin-0 maps are double
 *   [Npix]; spin-2 maps are interleaved (Q, U) double [Npix][2], Q and U given
 *   in the local (e_theta, e_phi) frame of each pixel; spin-1 maps likewise
 *   hold the two components of a tangent vector field (e.g. a deflection
 *   (d_theta, d_phi), the real and imaginary parts of P = d_theta + i d_phi).
 * - Deflections are double [count][2] = (d_theta, d_phi) in radians, the
 *   components of d in the local basis at the target pixel.
 * - Outputs: value double [count] (spin 0) or [count][2] (spin 1, 2: the two
 *   components in the local frame at n'); variance double [count] (may be
 *   NULL; spin s: of P); status uint8 [count]
 *   (may be NULL; FLINTS_ST_* bits, 0 = clean).
 * - All data pointers are DEVICE pointers owned by the caller and must not
 *   overlap.  Deflections and two-component maps and outputs (spin 1, 2) must
 *   be 16-byte aligned, one-component maps, outputs and variances 8-byte
 *   aligned.  Calls are asynchronous on the given CUDA
 *   stream (cudaStream_t passed as void*, NULL = legacy default stream); the
 *   caller synchronises the stream before reading results.
 * - Errors found on the host (bad arguments, CUDA launch failures, allocation
 *   failure) are returned synchronously as flints_status codes and described
 *   by flints_last_error().  Per-point numerical events are never errors:
 *   they set status bits and are counted in flints_stats.
 * - A plan owns its device memory (xi tables, counters) and is bound to the
 *   device that was current when it was created.  Plans are not thread-safe:
 *   use one plan per host thread or serialise calls on it.  Each lens call of
 *   a plan takes the next of the plan's 64 slots (a tile-queue counter the
 *   warps take their tiles from and, for spin 0 and 2, the one-job table of
 *   the persistent kernel the call launches), so at most 64 calls of one plan
 *   may be in flight on the GPU at once, on one stream or several.
 */
#ifndef FLINTS_H
#define FLINTS_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct flints_plan_s *flints_plan_t;

typedef enum {
    FLINTS_OK = 0,
    FLINTS_EINVAL = 1,   /* invalid argument (see flints_last_error) */
    FLINTS_ENOMEM = 2,   /* device allocation failed */
    FLINTS_ECUDA = 3     /* a CUDA runtime call or kernel launch failed */
    /* 4 and 5 are reserved: no entry point waits on the device, so none
     * returns a timeout */
} flints_status;

/* precision */
enum { FLINTS_FP64 = 0, FLINTS_MIXED = 1 };

/* plan flags */
enum {
    /* spin 2: augmented (widely linear) estimator.  The paper's spin-2 kriging
     * (Sec. 2.2) conditions on the Hermitian covariance <P_i P_j^*> (xi+) alone;
     * with this flag (Q, U) at the target are the Gaussian conditional mean given
     * (Q_i, U_i) of the stencil, which also uses the pseudo-covariance
     * <P_i P_j> = xi-(beta) exp(2i(a_ij + a_ji)): a 2K x 2K real system.  Equal to
     * the default when C^BB = C^EE (xi- = 0); strictly more precise otherwise.
     * Not accepted by the batch entry points. */
    FLINTS_SPIN2_AUGMENTED = 1u,
    /* spin s = 1, 2: return P in the frame at the target pixel n instead of the
     * frame at the displaced direction n': P(n') times exp(is(a_nn' - a_n'n - pi)),
     * a_uv the angle at u (from e_theta towards e_phi) of the geodesic towards v,
     * i.e. the field parallel-transported back along the deflection (Sec. 3.1
     * remaps P = Q + iU; the rotation is this library's reading) */
    FLINTS_ROTATE_TO_TARGET = 2u,
    FLINTS_NO_VARIANCE = 4u, /* skip the variance output even if a buffer is given */
    /* testing aid (mixed plans): every double-float solve is discarded and the
     * point is re-solved by the FP64 fallback, so that path can be checked on
     * well-conditioned inputs; results carry FLINTS_ST_FALLBACK */
    FLINTS_FORCE_FALLBACK = 256u
};

/* per-point status bits */
enum {
    FLINTS_ST_NUGGET = 1u,    /* S + 1.49e-8 I had a non-positive pivot; nugget raised (x2 steps) */
    FLINTS_ST_FALLBACK = 2u,  /* mixed path: point re-solved in FP64 */
    FLINTS_ST_WINDOW = 4u,    /* stencil not inside the search disc (K-nearest path) or a member chord
                                 beyond the table (tabulated route): the point is not solved */
    FLINTS_ST_FAILED = 8u,    /* no result (no positive-definite factor, stencil outside the disc or
                                 non-finite deflection): outputs are NaN */
    FLINTS_ST_POLE = 16u,     /* displaced direction within 1e-12 rad of a pole (spin-2 frame undefined) */
    FLINTS_ST_INPUT = 32u     /* the target's deflection is not finite (with FLINTS_ST_FAILED) */
};

typedef struct {
    int64_t points;      /* points launched since the plan was created or stats reset (host
                          * count: a batch counts its jobs when they are staged, once; a
                          * refused call counts none) */
    int64_t nugget;      /* points with FLINTS_ST_NUGGET */
    int64_t fallback;    /* points with FLINTS_ST_FALLBACK */
    int64_t window;      /* points with FLINTS_ST_WINDOW */
    int64_t failed;      /* points with FLINTS_ST_FAILED */
} flints_stats;

typedef struct {
    int64_t nside;
    int lmax, spin, K, precision;
    double t_max;        /* tabulated squared-chord domain [0, t_max] */
    int n_intervals;     /* cubic Hermite intervals of the xi table */
    double xi0;          /* xi(0) (spin 0) or xi+(0) (spin 1, 2) */
    double search_radius;/* chord radius of the stencil disc */
    int64_t device_bytes;/* device memory the plan holds: its spectrum and xi tables,
                          * interpolation coefficients, counters and launch queues */
} flints_plan_info;

/* Create a plan: copy the spectrum to the device and tabulate xi on the GPU
 * (Sec. 2.5 steps 1-2; Appendix B).
 *   out        receives the plan (NULL on failure).
 *   nside      HEALPix resolution, 1 <= nside <= 16384.
 *   lmax       band limit, 0 <= lmax <= 16384.
 *   cl         HOST pointer, [lmax+1]: C_l^TT (spin 0), C_l^EE (spin 2), or the
 *              gradient-mode spectrum of a spin-1 field (a deflection
 *              d = grad phi: C^E_l = l(l+1) C^phiphi_l).
 *   cl_bb      HOST pointer, [lmax+1] C_l^BB (spin 1: curl mode), or NULL for
 *              B = 0.  Ignored for spin 0.
 *   spin       0, 1 or 2.  Spin-1 xi+- use d^l_{1,+-1}; the spin-s phases are
 *              exp(is(a_ij - a_ji - pi)), frames referred to the geodesic's
 *              direction of travel (the pi matters for odd s).  Spin-1 plans
 *              run through flints_lens_range / flints_supersample.
 *   K          stencil size: 16, 24, 32 or 48.
 *   precision  FLINTS_FP64 or FLINTS_MIXED.
 *   flags      FLINTS_* plan flags.
 *   stream     CUDA stream for the tabulation (the call returns after it).
 * Returns FLINTS_EINVAL for out-of-range arguments or a spectrum whose
 * xi(0) is not positive and finite. */
int flints_plan(flints_plan_t *out, int64_t nside, int lmax, const double *cl,
                const double *cl_bb, int spin, int K, int precision,
                unsigned flags, void *stream);

/* Lens a whole spin-0 map: out[p] = T(n_p + d(n_p)) for p = 0..Npix-1.
 *   map   device [Npix];  defl device [Npix][2];
 *   out   device [Npix];  var device [Npix] or NULL. */
int flints_lens_spin0(flints_plan_t plan, const double *map, const double *defl,
                      double *out, double *var, void *stream);

/* Lens a whole spin-2 map: (Q, U) at n_p + d(n_p) in the frame at n'.
 *   qu    device [Npix][2]; defl device [Npix][2];
 *   qu_out device [Npix][2]; var device [Npix] or NULL (variance of P = Q+iU). */
int flints_lens_spin2(flints_plan_t plan, const double *qu, const double *defl,
                      double *qu_out, double *var, void *stream);

/* Lens the contiguous target range [first, first+count) of a map whose spin
 * is the plan's.  map is the whole source map; defl, out, var and status are
 * indexed from 0 for pixel `first`.  count may be 0. */
int flints_lens_range(flints_plan_t plan, int64_t first, int64_t count,
                      const double *map, const double *defl, double *out,
                      double *var, uint8_t *status, void *stream);

/* Supersampling (Sec. 2.6 and Table 1 of the paper: a map at Nside predicted
 * at the pixel centres of a finer grid): interpolate the plan's map at the
 * centres of RING pixels [first, first+count) of an Nside = nside_out grid
 * (1..65536; any value, usually 2 x the plan's Nside), with no deflection.
 * map is the whole source map at the plan's Nside (device, [Npix] or
 * [Npix][2]); out, var and status are indexed from 0 for pixel `first`
 * (spin 2: Q, U in the frame at the target).  Errors and status as for
 * flints_lens_range. */
int flints_supersample(flints_plan_t plan, int64_t nside_out, int64_t first, int64_t count,
                       const double *map, double *out, double *var, uint8_t *status,
                       void *stream);

/* Stencil of the range [first, first+count): the K nearest RING pixels to
 * each displaced direction, sorted by (squared chord, pixel index), written
 * to idx device int64 [count][K], 8-byte aligned (the neighbour search of the
 * lens kernels, exposed for verification).  status as for flints_lens_range. */
int flints_stencil(flints_plan_t plan, int64_t first, int64_t count,
                   const double *defl, int64_t *idx, uint8_t *status,
                   void *stream);

/* Launch shape of a plan's lens launches (the autotuner's knobs).
 *   warps_per_block 1..8 (0: 8 for spin-0 and spin-2 plans, 4 for spin-1 and
 *   augmented ones; lowered to what fits in shared memory),
 *   blocks_per_sm cap (0: as many as fit),
 *   tile_points targets per warp tile 1..16 (0: 16).  cfg NULL restores the
 *   defaults.  Results do not depend on the launch shape. */
typedef struct {
    int warps_per_block, blocks_per_sm, tile_points;
} flints_launch_cfg;
int flints_plan_set_launch(flints_plan_t plan, const flints_launch_cfg *cfg);

/* One job of a batched launch: a target range of one plan. */
typedef struct {
    flints_plan_t plan;
    int64_t first, count;
    const double *map, *defl;
    double *out, *var;
    uint8_t *status;
} flints_job;

/* Run n jobs (plans may differ in Nside, K, spin and precision) as one
 * persistent launch per precision class on `stream`, then synchronise the
 * stream.  Convenience form of the batch objects below: it allocates a
 * temporary batch, so it cannot be captured in a CUDA graph. */
int flints_lens_batch(const flints_job *jobs, int n, void *stream);

/* Batch objects for the persistent batched launch.
 *   flints_batch_create: device job table and work queues for up to
 *     max_jobs jobs, plus pinned host staging (allocates; not capturable).
 *   flints_batch_stage: host-only: validate the jobs, order them by precision
 *     class and decreasing estimated cost, cut them into tiles of tile_points
 *     targets (1..16; 0: 16), write the table into the pinned staging buffer.
 *   flints_batch_launch: upload the staged table, reset the work queues and
 *     launch the two persistent kernels (FP64 and mixed jobs) on `stream`:
 *     stream operations only, so it can be captured in a CUDA graph; a replay
 *     runs whatever table was staged last.  The warps_per_block of cfg must
 *     have been used by an earlier launch before capture (changing it
 *     reconfigures the kernel).  Jobs of one batch must not write overlapping
 *     outputs.
 *   flints_batch_run: stage + launch (tile size from cfg).
 * Errors: FLINTS_EINVAL for bad jobs (message names the job index). */
typedef struct flints_batch_s *flints_batch_t;
int flints_batch_create(flints_batch_t *out, int max_jobs);
int flints_batch_stage(flints_batch_t batch, const flints_job *jobs, int n, int tile_points);
int flints_batch_launch(flints_batch_t batch, const flints_launch_cfg *cfg, void *stream);
int flints_batch_run(flints_batch_t batch, const flints_job *jobs, int n, const flints_launch_cfg *cfg,
                     void *stream);
void flints_batch_free(flints_batch_t batch);

/* Device counters of per-point events (synchronises `stream`). */
int flints_get_stats(flints_plan_t plan, flints_stats *s, void *stream);
int flints_reset_stats(flints_plan_t plan, void *stream);

/* Plan parameters (host data; no device access). */
int flints_get_info(flints_plan_t plan, flints_plan_info *info);

/* Copy the plan's xi table to the host: f and g receive n_intervals+1 values
 * of xi/xi0 and d(xi/xi0)/dt at t_k = k t_max / n_intervals (which = 0:
 * xi or xi+, which = 1: xi-).  Synchronises `stream`. */
int flints_get_table(flints_plan_t plan, int which, double *f, double *g, void *stream);

/* Message describing the last error returned on the calling thread. */
const char *flints_last_error(void);

/* Harmonic synthesis of a band-limited map on the GPU: the unlensed input of
 * the remap (Sec. 3.2 synthesises it from C_l; Table 2 counts the transform in
 * the total).  With sY_lm = (-1)^s N_l e^{i m phi} d^l_{m,-s}(theta) (Appendix A):
 *   spin 0: T = sum_lm a_lm Y_lm;
 *   spin s = 1, 2: P = -sum_lm (E + iB)_lm sY_lm, written as (Re P, Im P):
 *     (Q, U) for s = 2; (d_theta, d_phi) for s = 1 when E_lm = sqrt(l(l+1)) phi_lm.
 * E, B are real fields (a_{l,-m} = (-1)^m conj(a_lm)); only m >= 0 is given.
 *   flints_synth_plan: ring geometry, work arrays (about (4 Nside - 1)(2 lmax + 1)
 *     + 2 Npix complex doubles) and the cuFFT plans for Nside (1..8192), lmax
 *     (spin..16384) and spin (0, 1, 2).  precision FLINTS_FP64: the l-recurrence
 *     in FP64; FLINTS_MIXED: in double-float on the FP32 pipe (relative error
 *     about 1e-13 at lmax 4096).  Allocates; not capturable.
 *   flints_synthesize: alm (and blm for spin 1, 2; NULL = 0) DEVICE complex
 *     double [lmax+1][lmax+1] (index [l][m], m <= l read), 16-byte aligned;
 *     map DEVICE double [Npix] (spin 0) or [Npix][2] (spin 1, 2), RING order.
 *     Asynchronous on `stream`: an l-recurrence kernel, a folding kernel and
 *     one inverse FFT per ring size.
 * Errors: FLINTS_EINVAL (arguments), FLINTS_ENOMEM, FLINTS_ECUDA; the message
 * is returned by flints_synth_last_error. */
typedef struct flints_synth_s *flints_synth_t;
int flints_synth_plan(flints_synth_t *out, int64_t nside, int lmax, int spin, int precision, void *stream);
int flints_synthesize(flints_synth_t plan, const double *alm, const double *blm, double *map, void *stream);
void flints_synth_free(flints_synth_t plan);
const char *flints_synth_last_error(void);

/* Lens the target range [first, first+count) without allocating any device
 * memory.  The paper has no counterpart: this entry point exists for callers
 * that cannot call cudaMalloc -- serving runtimes that hand all device memory
 * to their own pool up front (an allocation by the library would fail or
 * fragment it) and hosts whose allocator policy forbids the library from
 * allocating.  It runs the same xi tabulation and lens kernels as
 * flints_plan + flints_lens_range, with their working memory (spectrum, table,
 * coefficients, counters, under 1 MB) in a fixed file-scope device array that
 * every GPU loading the library holds until the process exits.
 *   Arguments: as flints_plan (cl, cl_bb are HOST pointers) followed by the
 *   target range and the DEVICE buffers of flints_lens_range, with the same
 *   alignment rules (defl 16 bytes; map and out 16 bytes for spin 2, 8 bytes
 *   for spin 0; var 8 bytes).
 *   Limits: lmax <= 8192 and a xi table of at most 8192 intervals; larger
 *   requests return FLINTS_EINVAL with a message naming the limit.
 *   Set-up: the first call on each device looks up the array's device address
 *   (cudaGetSymbolAddress) with that device current; make that first call
 *   before any stream capture begins.
 *   Stream use: the call copies the spectrum from host memory and synchronises
 *   `stream` once, after the tabulation, to read xi(0) back; the lens kernel is
 *   then left running asynchronously on `stream`.
 *   Sharing: all calls use the same array and it keeps the last call's
 *   contents (the call clears what must start at zero).  Calls whose work
 *   overlaps on the GPU (different streams or threads) race on it: serialise
 *   them.
 *   Errors: flints_status codes; message in flints_noalloc_last_error(). */
int flints_lens_noalloc(int64_t nside, int lmax, const double *cl, const double *cl_bb, int spin,
                        int K, int precision, int64_t first, int64_t count, const double *map,
                        const double *defl, double *out, double *var, uint8_t *status,
                        void *stream);
const char *flints_noalloc_last_error(void);

/* Measured fused multiply-add throughput of the current device, for roofline
 * fractions.  The paper has no counterpart: this is a measurement utility.
 * One kernel of independent multiply-add chains (8 per thread, every SM filled
 * to its occupancy limit) runs `iters` rounds of 128 multiply-adds per thread
 * after a shorter warm-up launch, timed with CUDA events on `stream`;
 * *tflops = 2 x multiply-adds / seconds / 1e12.
 *   precision: FLINTS_MIXED measures the FP32 pipe (the double-float path's
 *   arithmetic), FLINTS_FP64 the FP64 pipe.  iters in [1, 2^24].
 *   Synchronises `stream`.  Errors: FLINTS_EINVAL, FLINTS_ECUDA; message in
 *   flints_measure_last_error(). */
int flints_measure_fma_peak(int precision, int iters, double *tflops, void *stream);
const char *flints_measure_last_error(void);

/* Release a plan and its device memory (NULL is allowed). */
void flints_free(flints_plan_t plan);

/* The paper's estimator route with tabulated inverses (Secs. 2.3-2.5): the
 * pixel-centred stencil at level y and the inverse covariance computed once per
 * class of central pixels, then triangular matrix-vector products per target.
 * Spin 0, 1 and 2 (Hermitian or augmented), FP64 or mixed precision.
 *
 * Stencil (Sec. 2.3, neighbours() with the NESTED hierarchy): the target's
 * pixel at Nside_c = Nside / 2^(y-1) and the pixels of that grid sharing a
 * vertex with it (8; 7 at the 24 pixels next to the points where three base
 * faces meet; 6 at Nside_c = 1), each replaced by its 4^(y-1) sub-pixels at
 * Nside: K = 9 * 4^(y-1) members (8 or 7 * 4^(y-1) where fewer neighbours).
 * The paper's "pixelization at Nside/y" is read as Nside / 2^(y-1), the grid
 * whose pixels hold 4^(y-1) pixels each.
 *
 * Classes (Sec. 2.4): the grid is invariant under z -> -z, under rotations by
 * pi/2 and, for central pixels whose stencil lies wholly in the equatorial
 * belt (folded coarse ring Nside_c + 3 .. 2 Nside_c), under the rotation by
 * one pixel; with members listed in an order those symmetries keep, one
 * inverse serves a whole class: about Nside_c^2 / 2 + 4 Nside_c of them.  The
 * tabulated matrix is L^-1, L the Cholesky factor of S + n I
 * (S = xi(chord^2)/xi(0), nugget n = 1.49e-8 doubled, at most 8 times, while a
 * pivot is not positive): value = (L^-1 c) . (L^-1 y) = c^T S^-1 y and
 * variance xi(0) (1 - |L^-1 c|^2), without the cond(S) loss of an explicit
 * S^-1 and in half its memory.
 *
 * flints_paper_plan: y = 1 or 2; nside in [1, 8192] and divisible by
 *   2^(y-1); cl HOST [lmax+1] (spin 0: C_l; spin 2: C_l^EE), cl_bb HOST
 *   [lmax+1] or NULL (spin 1, 2: C_l^BB; ignored for spin 0); spin 0, 1 or 2
 *   (spin s: the member covariances carry the transport phases
 *   exp(is(a_ij - a_ji - pi)) with xi+, classes mirrored by z -> -z use
 *   conj(L^-1)); flags 0 or FLINTS_SPIN2_AUGMENTED (spin 2, FP64: the widely
 *   linear estimator with xi+ and xi-, the class factor that of the real
 *   2K x 2K system of (Q_i, U_i), D L^-1 D with D = diag(I, -I) for mirrored
 *   classes; L^-1 blocks 2K (2K + 1) / 2 doubles packed by columns);
 *   precision FLINTS_FP64, or FLINTS_MIXED: the per-target chords,
 *   correlation lookups and triangular products in double-float on the FP32
 *   pipe (target position and location FP64; the L^-1 blocks computed in FP64
 *   and kept as double-float).
 *   Builds on `stream` the xi table(s) on [0, min((7 / Nside_c)^2, 4)]
 *   (interval count by the rule of flints_plan), a table of the map pixels'
 *   positions (and frames, spin 1, 2), the stencil table and the L^-1 blocks,
 *   then synchronises `stream`.  Device memory: 32 bytes per map pixel,
 *   12 Nside_c^2 (K + 1) int32, slots * len doubles (len below; complex
 *   blocks twice that), reported by flints_paper_get_info as table_bytes,
 *   plus the xi tables (device_bytes is the whole).
 *   Errors: FLINTS_EINVAL (arguments; a stencil chord beyond the table
 *   domain), FLINTS_ENOMEM, FLINTS_ECUDA; message in flints_paper_last_error().
 * flints_paper_lens: lensed values at targets first .. first+count-1 (RING
 *   pixels of the plan's grid displaced along defl, as flints_lens_range).
 *   map DEVICE [12 Nside^2] (spin 1, 2: [12 Nside^2][2] = (d_theta, d_phi) or
 *   (Q, U), 16-byte aligned; else 8-byte aligned), defl DEVICE [count][2]
 *   (16-byte aligned; entry i belongs to pixel first + i), out DEVICE [count]
 *   (spin 1, 2: [count][2] in the frame at the displaced direction, 16-byte
 *   aligned), var DEVICE [count] (may be NULL), status DEVICE [count] (may be
 *   NULL; FLINTS_ST_NUGGET
 *   when the class needed a raised nugget, FLINTS_ST_WINDOW when a chord fell
 *   beyond the table domain, FLINTS_ST_FAILED with NaN outputs when no factor
 *   was found).  Asynchronous on `stream`.
 * flints_paper_supersample: values at the centres of pixels first ..
 *   first+count-1 of the grid nside_out (1..16384; Sec. 2.6); otherwise as
 *   above.
 * flints_paper_get_info: plan sizes and counters (synchronises `stream`).
 * flints_paper_tables: copies the stencil table (members DEVICE [12 Nside_c^2]
 *   [K] int32 RING indices at Nside, -1 past the member count), the class of
 *   each coarse pixel (slot DEVICE [12 Nside_c^2] int32) and the L^-1 blocks
 *   (linv DEVICE [slots][len] doubles, complex (re, im) pairs for spin 1, 2,
 *   zero past the member count; augmented plans: the real 2K x 2K factor packed
 *   by columns; else K = 9: len = 45, packed by columns: column j, rows j .. 8,
 *   from offset
 *   9 j - j (j - 1) / 2; K = 36: len = 704, the lane-step layout: entry
 *   32 u + l (u < 17) holds, for p = l / 2 and t = u (l even) or 17 + u (l
 *   odd), row p column t when t <= p, else row 31 - p column t - p - 1 (zero
 *   when that column exceeds the row); entry 544 + 32 t + l (t < 5) holds row
 *   32 + l % 4, column l / 4 + 8 t (zero above the diagonal)) into caller
 *   buffers; any may be NULL.  Mixed plans keep only double-float blocks:
 *   linv must be NULL for them (FLINTS_EINVAL otherwise).
 * flints_paper_free: releases the plan (NULL is allowed). */
typedef struct flints_paper_s *flints_paper_t;
typedef struct flints_paper_info {
    int64_t nside;          /* map grid */
    int64_t nside_coarse;   /* Nside / 2^(y-1) */
    int y, K;               /* level and stencil size 9 * 4^(y-1) */
    int64_t slots;          /* classes of central pixels (L^-1 blocks) */
    double t_max;           /* xi table domain [0, t_max] in chord^2 */
    int n_intervals;
    double xi0;
    int64_t table_bytes;    /* pixel table + stencil table + class map + L^-1 blocks */
    double max_pair_t;      /* largest chord^2 between members of a stencil */
    int64_t nugget_slots;   /* classes whose factor needed a raised nugget */
    int64_t failed_slots;   /* classes without a positive-definite factor */
    int64_t points;         /* targets processed so far */
    int64_t window;         /* targets with a chord beyond the table domain */
    int precision;          /* FLINTS_FP64 or FLINTS_MIXED */
    int spin;               /* 0, 1 or 2 */
    unsigned flags;         /* FLINTS_SPIN2_AUGMENTED or 0 */
    int64_t device_bytes;   /* all device memory the plan holds: table_bytes plus the
                             * spectrum, xi tables, coefficients and counters */
} flints_paper_info;
int flints_paper_plan(flints_paper_t *out, int64_t nside, int lmax, const double *cl, const double *cl_bb, int y,
                      int spin, int precision, unsigned flags, void *stream);
int flints_paper_lens(flints_paper_t plan, int64_t first, int64_t count, const double *map, const double *defl,
                      double *out, double *var, uint8_t *status, void *stream);
int flints_paper_supersample(flints_paper_t plan, int64_t nside_out, int64_t first, int64_t count,
                             const double *map, double *out, double *var, uint8_t *status, void *stream);
int flints_paper_get_info(flints_paper_t plan, flints_paper_info *info, void *stream);
int flints_paper_tables(flints_paper_t plan, int32_t *members, int32_t *slot, double *linv, void *stream);
void flints_paper_free(flints_paper_t plan);
const char *flints_paper_last_error(void);


#ifdef __cplusplus
}
#endif
#endif /* FLINTS_H */

/*
 * gw.h -- C ABI of the GB300 W-projection gridding / degridding library.
 *
 * The library implements the data-parallel hot path of convolutional
 * gridding with a w-projection gridding convolution function (GCF) as
 * formulated in "High-Performance Gridding For Radio Interferometric Image
 * Synthesis" (Muscat, arXiv:2111.04141):
 *
 *   uvw -> index selection        Section 3.3.5 (pre-processing), Section 2.3.6
 *   binning by grid tile          Section 3.3.5 ("SS" ordering mode)
 *   w-kernel tables               Section 1.7.1 (W-projection), Section 2.3.6
 *   gridding                      Section 2.4.5, Algorithm convgriddingoversampling
 *   degridding (the adjoint)      Section 1.6, Eq. (residualcalc), operator G^T
 *   grid correction               Section 2.4.5, Eq. (hco); Section 3.3.8
 *
 * Conventions shared by every entry point
 * ---------------------------------------
 * - All pointers marked "device" are CUDA device pointers on the device that
 *   was current when the plan was created; "host" pointers are ordinary host
 *   memory.  The caller owns every buffer it passes; the plan owns its
 *   kernel tables and scratch.
 * - Calls are asynchronous on the CUDA stream passed as `cuda_stream`
 *   (a cudaStream_t; NULL means the legacy default stream), except where an
 *   argument asks for a host result (n_dropped), which synchronises that
 *   stream.  Two calls on the same plan must not run concurrently (they
 *   share the plan's scratch); serialise them on one stream.
 * - Errors are returned as gw_status codes; no exception crosses the ABI.
 *   gw_last_error() gives a human-readable message for the calling thread.
 * - Complex numbers are interleaved (re, im) float pairs ("c64") unless the
 *   plan selects a half-precision storage type.
 * - Visibilities are laid out [nrow][nchan][npol]; uvw is [nrow][3] float64
 *   metres; frequencies are [nchan] float64 Hz; the grid and images are
 *   [npol][N][N] c64, row index v (or m), column index u (or l), with the uv
 *   origin on pixel (N/2, N/2).
 */
#ifndef GW_H
#define GW_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define GW_API_VERSION 8

typedef struct gw_plan_s* gw_plan;

typedef enum {
    GW_OK = 0,
    GW_EINVAL = -1,        /* invalid argument (null pointer, bad size, bad descriptor) */
    GW_ENOMEM = -2,        /* a device or host allocation failed */
    GW_ECUDA = -3,         /* a CUDA runtime call failed (see gw_last_error) */
    GW_ETIMEDOUT = -4,     /* a bounded device-side wait gave up */
    GW_EUNSUPPORTED = -5,  /* valid request the library does not implement */
    GW_EDEVICE = -6,       /* called with a different current device than the plan's */
    GW_EBOUNDS = -7        /* a device-side bounds check of the debug build failed */
} gw_status;

/* Storage type of visibilities and of the kernel tables.  The 16-bit kinds
 * are pairs (re in the low 16 bits of a 32-bit word, im in the high 16 bits,
 * little-endian: the memory layout of two consecutive 16-bit values re, im).
 * They change storage only: visibilities and table entries are widened to
 * FP32 on load and every sum is FP32; FP64 is kept for coordinates, index
 * selection and table generation.  Degridded visibilities are rounded to
 * the plan's vis_dtype (to nearest) when stored.  Float16 has a narrow
 * range (|x| <= 65504): visibilities must lie in it, and float16 tables are
 * stored scaled by 2^table_exp2 (gw_plan_info), undone in FP32. */
typedef enum {
    GW_C64 = 0,            /* complex float32 pairs, 8 bytes */
    GW_BF16X2 = 1,         /* complex bfloat16 pairs, 4 bytes */
    GW_F16X2 = 2           /* complex float16 pairs, 4 bytes */
} gw_dtype;

/* Plan descriptor.  Defines the imaging problem; see gw_plan_create. */
typedef struct {
    int32_t grid_n;          /* N: grid side, even, 8 <= N <= 32768 */
    double cell_rad;         /* pixel size in direction cosines; L = N * cell_rad */
    int32_t support_min;     /* odd, >= 1: GCF support of the w = 0 plane (taper support) */
    int32_t support_max;     /* odd, >= support_min: support of the outermost w-plane */
    int32_t oversample;      /* beta: even, 2 <= beta <= 256 */
    int32_t n_wplanes;       /* P >= 1; P == 1 ignores w (2-D gridding) */
    double w_max_lambda;     /* > 0 when P > 1: |w| (wavelengths) of the outermost plane */
    int32_t npol;            /* 1 .. 4 polarisations gridded together (Section 3.3.4) */
    int32_t vis_dtype;       /* gw_dtype of visibilities passed to gw_grid_vis / gw_degrid_vis */
    int32_t table_dtype;     /* gw_dtype the kernel tables are stored in */
    int64_t max_vis_per_call;/* scratch sizing: visibilities processed per internal chunk
                                (0 = 2^23); larger calls are processed in chunks */
} gw_plan_desc;

/* One visibility's index record (output of the index stage, 16 bytes).
 * For a valid record: the record sits at pixel (ku + ou/beta, kv + ov/beta)
 * of the grid; ou, ov in [-beta/2, beta/2); plane in [0, P); flags bit 0 =
 * valid (Bounded Records Assumption, Section 2.3.1), bit 1 = w < 0 (the
 * conjugate kernel is used).  Invalid records are all zeros. */
typedef struct {
    int32_t ku, kv;
    int16_t ou, ov;
    int16_t plane;
    uint16_t flags;
} gw_index_rec;

#define GW_FLAG_VALID 1u
#define GW_FLAG_CONJ 2u

/* Read-only facts about a plan (gw_plan_info). */
typedef struct {
    int32_t grid_n, npol, oversample, n_wplanes;
    int32_t grid_tile_u, grid_tile_v;  /* gridder tile (footprint-mode bins), pixels */
    int32_t degrid_tile;      /* degridder tile side (centre-mode bins), pixels */
    int32_t device;           /* CUDA device ordinal the plan lives on */
    int64_t table_elems;      /* complex elements in all kernel tables */
    int64_t chunk_vis;        /* visibilities per internal chunk */
    double field;             /* L = N * cell_rad */
    double taper_c;           /* PSWF bandwidth c = pi * support_min / 2 */
    double table_scale;       /* global kernel scale (w = 0, o = 0 slice sums to 1) */
    int32_t vis_dtype, table_dtype;  /* gw_dtype of the plan */
    int32_t table_exp2;       /* 16-bit tables store round(K * 2^table_exp2); 0 for
                                 GW_C64 and GW_BF16X2; for GW_F16X2 chosen so the largest
                                 entry (w = 0, o = 0 centre tap) lies in [2^14, 2^15) */
    int32_t plane_groups;     /* plane groups the binned gridder uses under the current
                                 tuning (gw_tuning.plane_groups; 1 = tiles only) */
    int64_t table_bytes;      /* device bytes of the kernel tables (shared with clones) */
    int64_t scratch_bytes;    /* device bytes of this plan's own scratch */
} gw_plan_info;

/* Launch tuning of a plan (gw_plan_set_tuning).  Zero fields mean defaults.
 * No counterpart in the thesis: these are implementation choices that an
 * autotuner may pick per workload; results do not depend on them beyond
 * FP32 summation order. */
typedef struct {
    int32_t item_max;       /* records per gridding / staged-degridding work item:
                               0 = 1024, else 64 .. 2^20 (smaller items spread small
                               jobs over more SMs, larger ones commit less often) */
    int32_t degrid_kernel;  /* 0 = automatic, 1 = shared-memory staged, 2 = global gather */
    int32_t grid_kernel;    /* gw_grid_vis / _compensated: 0 = automatic (direct for chunks of
                               at most 16,384 visibilities and 2^22 tap updates, else
                               binned), 1 = binned register-tile gridder, 2 = direct
                               (one global atomic per tap and polarisation, no bins) */
    int32_t compress_min_gain; /* gw_grid_vis_compressed: 0 = always compress; g in
                               1..1000 = first compress a sample (the first rows, up to
                               2^18 visibilities; the call synchronises the stream) and grid
                               without compression when fewer than g per mille of its valid
                               records merge (n_gridded then counts the valid records) */
    int32_t plane_groups;   /* binned gridding in gw_grid_vis / _host / _compressed: bins
                               keyed by (w-plane group, tile) and served group by group, so
                               one group's kernel tables stay in L2 (Section 3.3.5 "SS"
                               ordering): 0 = automatic (FP32 tables above 128 MB: one
                               group per 64 MB of padded tables; otherwise 1),
                               1 = tiles only, n in 2..16 (at most the w-planes) = n
                               groups of consecutive planes */
} gw_tuning;

/* ------------------------------------------------------------------------
 * Plan lifetime
 * ------------------------------------------------------------------------ */

/* Create a plan on the current CUDA device: validates the descriptor,
 * computes the per-plane w and support (w_p = w_max (p/(P-1))^2; S_p = the
 * odd integer nearest S_min + (S_max - S_min) p/(P-1), ties up), builds the
 * kernel tables on the device in FP64 (prolate spheroidal taper psi_0 with
 * c = pi S_min / 2 times the w-screen exp(+j 2 pi w_p (n - 1)), Fourier
 * transformed by Gauss-Legendre quadrature and sampled at offsets
 * t - o/beta, Section 1.7.1 and Section 2.3.6), stores them as table_dtype,
 * computes the corrector, and allocates scratch.  Work is issued on
 * `cuda_stream`; the call synchronises it before returning.
 * Errors: GW_EINVAL (null arguments or a descriptor outside the ranges
 * above, or a field of view whose corners reach l^2 + m^2 >= 1 when P > 1),
 * GW_ENOMEM, GW_ECUDA.  On error *out is set to NULL. */
gw_status gw_plan_create(const gw_plan_desc* desc, void* cuda_stream, gw_plan* out);

/* A plan with the same descriptor that shares src's kernel tables (no table
 * generation) and owns its own scratch, sized by max_vis_per_call (0 =
 * 2^23).  A plan and its clones may run concurrently on different streams;
 * one plan must not run two calls at once (its scratch is reused).  The
 * tables are freed with the last plan that uses them.  Tuning is copied.
 * Errors: GW_EINVAL, GW_EDEVICE, GW_ENOMEM, GW_ECUDA. */
gw_status gw_plan_clone(gw_plan src, int64_t max_vis_per_call, void* cuda_stream, gw_plan* out);

gw_status gw_plan_set_tuning(gw_plan plan, const gw_tuning* tuning);
gw_status gw_plan_get_tuning(gw_plan plan, gw_tuning* out);

/* Test hooks (no thesis counterpart).  gw_debug_fail_alloc(n), n > 0: the
 * n-th allocation the library makes from now on (device memory, or the host
 * objects of a plan) fails as if the device or host were out of memory, and
 * the hook switches itself off; n = 0 switches it off.  The failing call
 * returns GW_ENOMEM after freeing what it had allocated; nothing reaches the
 * GPU.  Process-wide, not thread-safe with concurrent plan calls; meant for
 * tests of the error paths.  gw_debug_live_plans(): plans (and clones)
 * created and not yet destroyed in this process; gw_debug_live_bytes(): bytes
 * of device memory the library has allocated and not freed. */
gw_status gw_debug_fail_alloc(int64_t n);
int64_t gw_debug_live_plans(void);
int64_t gw_debug_live_bytes(void);

/* Synchronises `cuda_stream` and reads the plan's device status word (no
 * thesis counterpart): GW_ETIMEDOUT if, since the last check, a bounded
 * device-side wait of the gridding kernel gave up (its producer / consumer
 * hand-over waits at most about two seconds; the kernel then returns and
 * that call's grid is incomplete); GW_EBOUNDS if a kernel of the debug build
 * (libgw_debug.so, compiled with GW_DEBUG_BOUNDS) found an index outside
 * its buffer (the access is skipped, so that call's result is wrong but
 * nothing faults); else GW_OK.  The word is cleared when read.  Calls that
 * return n_dropped check it the same way.
 * Errors: GW_EINVAL, GW_EDEVICE, GW_ECUDA, GW_ETIMEDOUT, GW_EBOUNDS. */
gw_status gw_plan_device_status(gw_plan plan, void* cuda_stream);

/* Free all device memory of the plan.  NULL is accepted.  The caller must
 * ensure no work using the plan is still in flight. */
gw_status gw_plan_destroy(gw_plan plan);

gw_status gw_plan_info_get(gw_plan plan, gw_plan_info* out);

/* ------------------------------------------------------------------------
 * Hot path
 * ------------------------------------------------------------------------ */

/* Gridding (Section 2.4.5, Algorithm convgriddingoversampling, Gridding Step,
 * with the w-projection GCF): for every visibility (row r, channel c),
 *     grid[pol][kv + tv][ku + tu] += K(tv, tu) * vis[r][c][pol] * weight[r][c][pol]
 * over the S_p x S_p taps of its plane, K the table slice for its offset
 * (conjugated when w < 0).  The grid is ACCUMULATED (+=), so repeated calls
 * and chunked inputs add linearly; zero it first for a fresh image.
 *   uvw_m    device, [nrow][3] float64, metres
 *   freq_hz  device, [nchan] float64, Hz
 *   vis      device, [nrow][nchan][npol] complex of the plan's vis_dtype;
 *            GW_C64: 16-byte aligned when npol is even (8-byte otherwise);
 *            16-bit kinds: 4-byte aligned
 *   weight   device, [nrow][nchan][npol] float32, or NULL for unit weights
 *   grid     device, [npol][N][N] c64, accumulated
 *   n_dropped host, optional: receives the number of visibilities dropped by
 *            the Bounded Records Assumption (Section 2.3.1) or invalid
 *            coordinates; when non-NULL the call synchronises the stream.
 * nrow * nchan may be 0 (no work).  Errors: GW_EINVAL, GW_EDEVICE, GW_ECUDA. */
gw_status gw_grid_vis(gw_plan plan, const double* uvw_m, const double* freq_hz, int64_t nrow,
                      int32_t nchan, const void* vis, const float* weight, void* grid,
                      int64_t* n_dropped, void* cuda_stream);

/* gw_grid_vis from HOST inputs (no thesis counterpart): uvw_h, freq_h,
 * vis_h and weight_h (optional) are host arrays with the layouts of
 * gw_grid_vis; grid is on the device.  The rows are processed in steps
 * whose host-to-device copies run on the plan's own copy stream while the
 * previous step is gridded on `cuda_stream` (two device staging sets, events
 * between the streams).  Host arrays should be page-locked for the copies
 * to overlap; the caller must keep them unchanged until the stream reaches
 * the end of the call.  The first call allocates the staging (grown on
 * demand).  Errors: as gw_grid_vis, and GW_ENOMEM. */
gw_status gw_grid_vis_host(gw_plan plan, const double* uvw_h, const double* freq_h, int64_t nrow,
                           int32_t nchan, const void* vis_h, const float* weight_h, void* grid,
                           int64_t* n_dropped, void* cuda_stream);

/* Gridding with compensated commits (the Kahan-style variant of
 * gw_grid_vis; same arguments plus grid_err).  Each grid point's partial
 * sum over a work item is committed with an atomic add that returns the
 * previous value; the exact rounding error of that FP32 addition
 * (Knuth's TwoSum) is accumulated into grid_err.  grid + grid_err is then
 * the sum of the commits with the FP32 commit rounding removed to first
 * order; gw_grid_fold forms it.
 *   grid_err device, [npol][N][N] c64, 8-byte aligned, caller-owned;
 *            zero it together with the grid, pass the same buffer to every
 *            call that accumulates into that grid, then call gw_grid_fold.
 * Errors as gw_grid_vis, and GW_EINVAL for a null grid_err. */
gw_status gw_grid_vis_compensated(gw_plan plan, const double* uvw_m, const double* freq_hz,
                                  int64_t nrow, int32_t nchan, const void* vis,
                                  const float* weight, void* grid, void* grid_err,
                                  int64_t* n_dropped, void* cuda_stream);

/* Gridding with full compression (Section 3.3.5, "Full Compression"):
 * visibilities that fall on the same pixel of the beta-oversampled grid,
 * in the same w-plane and with the same sign of w, are summed (weights
 * applied) before gridding, so the gridder sees each distinct record once.
 * The result equals gw_grid_vis up to FP32 summation order.  Arguments as
 * gw_grid_vis, plus n_gridded (host, optional): receives the number of
 * records gridded after compression (summed over internal chunks:
 * compression acts within a chunk of max_vis_per_call visibilities); when
 * non-NULL the call synchronises the stream.  The first call allocates the
 * plan's compression scratch (a hash table of 2^ceil(log2(2 chunk)) keys).
 * Errors: GW_EINVAL, GW_EDEVICE, GW_ENOMEM, GW_ECUDA. */
gw_status gw_grid_vis_compressed(gw_plan plan, const double* uvw_m, const double* freq_hz,
                                 int64_t nrow, int32_t nchan, const void* vis,
                                 const float* weight, void* grid, int64_t* n_gridded,
                                 int64_t* n_dropped, void* cuda_stream);

/* W-stacking (Section 1.7.1, "Correction of the W-term in the (l,m)-plane"):
 * each visibility is gridded with the plan's 2-D kernel (the plan must have
 * n_wplanes == 1) onto the grid of its w-layer, layer
 * l = clamp(floor((w_lambda - w_min) / dw + 1/2), 0, n_layers - 1),
 * dw = (w_max - w_min) / (n_layers - 1), computed in FP64 like the index
 * stage (records beyond the range use the outermost layer).
 *   layers  device, [n_layers][npol][N][N] c64, accumulated (+=)
 * Other arguments as gw_grid_vis.  The image is then formed by an
 * unnormalised inverse FFT of each layer grid, gw_wstack_combine (which
 * applies the centring shift), then gw_grid_correct(+1).  The first call allocates
 * the plan's layered bins.  Errors: GW_EINVAL, GW_EDEVICE, GW_ENOMEM, GW_ECUDA. */
gw_status gw_grid_vis_wstack(gw_plan plan, const double* uvw_m, const double* freq_hz,
                             int64_t nrow, int32_t nchan, const void* vis, const float* weight,
                             int32_t n_layers, double w_min_lambda, double w_max_lambda,
                             void* layers, int64_t* n_dropped, void* cuda_stream);

/* image[pol][i][j] += sum_l layer_images[l][pol][i][j] * exp(+j 2 pi w_l (n_ij - 1)),
 * w_l = w_min + l dw as in gw_grid_vis_wstack, n_ij - 1 = -r^2 / (1 + sqrt(1 - r^2)),
 * r^2 = l_j^2 + m_i^2, l_j = (j - N/2) cell_rad, m_i = (i - N/2) cell_rad: the
 * w-screen correction of each layer's image (Eq. (lmwcorr)) and their sum.
 * n_ij - 1 and each screen's phase are formed in FP64 and reduced modulo 2 pi;
 * the screens (a rotation recursion re-anchored every 8 layers) and the sum
 * are FP32.  layer_images: device [n_layers][npol][N][N]
 * c64, the unnormalised inverse FFTs of the layer grids as gridded (not
 * shifted: the centring, a circular shift by N/2 of each transform, is
 * applied in the read; N even); image: device
 * [npol][N][N] c64, accumulated.  Errors: GW_EINVAL, GW_EDEVICE, GW_ECUDA. */
gw_status gw_wstack_combine(gw_plan plan, const void* layer_images, int32_t n_layers,
                            double w_min_lambda, double w_max_lambda, void* image,
                            void* cuda_stream);

/* Hybrid Gridding with a column pruner (Section 2.4, Algorithm (hybrid)),
 * for 2-D plans (n_wplanes == 1, grid_n % 4 == 0, oversample % 4 == 0).
 * Four steps:
 *   gw_hybrid_grid   Gridding Step: each visibility is convolved along u with
 *                    the plan's oversampled 1-D GCF (support_min taps) and
 *                    put on the nearest of beta*N rows along v:
 *                    fine[kv*beta + ov][ku + t][pol] += c(t - ou/beta) * vis;
 *                    fine: device [beta*N][N][npol] c64 (polarisations
 *                    interleaved, so one tap's updates are contiguous),
 *                    accumulated; 16-byte aligned when npol is even.
 *   gw_hybrid_prune  Pruning Step: each column is sampled down by beta/2 onto
 *                    2N rows through the pruning GCF Z, the zeroth-order PSWF
 *                    with odd support sz on the 2x grid (normalised taps):
 *                    pruned[pol][k][u] = sum_r Z(k - 2r/beta) fine[r][u][pol];
 *                    pruned: device [npol][2N][N] c64, overwritten.
 *   gw_hybrid_shift  pruned *= (-1)^(k + u) before an unnormalised inverse FFT.
 *   gw_hybrid_image  Correction Step: keeps rows N/2 .. 3N/2 - 1 of the
 *                    transform `raw` ([npol][2N][N]), re-centres them and
 *                    applies h_co(l) h_pr(m) (Eq. (hhy)); image: device
 *                    [npol][N][N] c64, overwritten.
 * A visibility is dropped (and counted) when the index stage drops it or
 * its pruning window leaves the 2N rows.  The pruner of a support is built
 * on first use (synchronous).  Errors: GW_EINVAL, GW_EDEVICE, GW_ENOMEM,
 * GW_ECUDA. */
gw_status gw_hybrid_grid(gw_plan plan, const double* uvw_m, const double* freq_hz, int64_t nrow,
                         int32_t nchan, const void* vis, const float* weight, int32_t sz,
                         void* fine, int64_t* n_dropped, void* cuda_stream);
gw_status gw_hybrid_prune(gw_plan plan, int32_t sz, const void* fine, void* pruned,
                          void* cuda_stream);
gw_status gw_hybrid_shift(gw_plan plan, void* pruned, void* cuda_stream);
gw_status gw_hybrid_image(gw_plan plan, int32_t sz, const void* raw, void* image,
                          void* cuda_stream);

/* grid += grid_err, then grid_err = 0 (device, both [npol][N][N] c64):
 * ends a sequence of gw_grid_vis_compensated calls.  Asynchronous on the
 * stream.  Errors: GW_EINVAL, GW_EDEVICE, GW_ECUDA. */
gw_status gw_grid_fold(gw_plan plan, void* grid, void* grid_err, void* cuda_stream);

/* Degridding, the adjoint of gw_grid_vis with unit weights:
 *     vis_out[r][c][pol] = sum_{tv,tu} conj(K(tv, tu)) * grid[pol][kv + tv][ku + tu]
 * vis_out (device, [nrow][nchan][npol] of the plan's vis_dtype) is
 * OVERWRITTEN; dropped visibilities receive 0.  Other arguments as above. */
gw_status gw_degrid_vis(gw_plan plan, const double* uvw_m, const double* freq_hz, int64_t nrow,
                        int32_t nchan, const void* grid, void* vis_out, int64_t* n_dropped,
                        void* cuda_stream);

/* Degridding without any allocation.  The thesis has no counterpart; this
 * exists for callers that cannot call cudaMalloc once they are running (a
 * process whose device memory is all handed to another allocator at
 * start-up, or a loop that must not take the driver's allocation lock).
 * Same contract and result as gw_degrid_vis, but its scratch (index records
 * and centre-tile bins) lives in one file-scope device array of about
 * 2.25 MiB (2,360,320 bytes) that every GPU loading the library holds until
 * exit; nothing is allocated.  The driver allocates that array when it loads
 * the library module that holds it, which gw_plan_create does (together with
 * every kernel this call launches), so a process that creates its plans
 * before handing its device memory to another allocator can call this
 * without any allocation.  Each call looks up the array's device address
 * (cudaGetSymbolAddress, no allocation once loaded).
 * Limits: nrow * nchan <= 65536 and grid_n <= 8192, else GW_EINVAL with the
 * limit in gw_last_error().  All calls share the one array and each call overwrites
 * it: calls whose GPU work overlaps (different streams, or different plans
 * on the same device) race; serialise them. */
gw_status gw_degrid_vis_static(gw_plan plan, const double* uvw_m, const double* freq_hz,
                               int64_t nrow, int32_t nchan, const void* grid, void* vis_out,
                               int64_t* n_dropped, void* cuda_stream);

/* Device-count variants of gw_grid_vis / gw_degrid_vis for CUDA graphs.
 * No thesis counterpart: a serving loop captures one call into a graph and
 * replays it for jobs of different sizes.  The row count is read from
 * device memory (*d_nrow, int64) when the kernels run, clamped to
 * [0, max_nrow]; buffers are sized for max_nrow rows.  The call makes no
 * allocation and no synchronisation (so it can be captured) and must fit
 * one chunk: max_nrow * nchan <= the plan's max_vis_per_call, else
 * GW_EINVAL.  No weights; dropped records are skipped and not reported.
 * gw_degrid_vis_devcount zeroes and writes rows [0, *d_nrow) of vis_out. */
gw_status gw_grid_vis_devcount(gw_plan plan, const double* uvw_m, const double* freq_hz,
                               const int64_t* d_nrow, int64_t max_nrow, int32_t nchan,
                               const void* vis, void* grid, void* cuda_stream);
gw_status gw_degrid_vis_devcount(gw_plan plan, const double* uvw_m, const double* freq_hz,
                                 const int64_t* d_nrow, int64_t max_nrow, int32_t nchan,
                                 const void* grid, void* vis_out, void* cuda_stream);

/* gw_grid_vis_devcount with the grid read back to the host while it is
 * still being computed.  No thesis counterpart (serving: a job's latency
 * includes bringing its grid to the host).  The gridder runs once per band
 * of grid-tile rows (n_bands bands of about equal height, at most the number
 * of tile rows, in [1, 64]); a band's tiles receive updates only from its own
 * work items, so when its launch ends its grid rows are final and are
 * copied to host_grid ([npol][N][N] complex64, page-locked host memory,
 * 8-byte aligned; rows of every polarisation plane) on a copy stream of the
 * plan while the next band grids.  Work issued later on cuda_stream waits
 * for the last copy, so a stream synchronise (or an event) covers the
 * result in host memory.  `grid` (device) accumulates as in
 * gw_grid_vis_devcount (zero it first for a fresh grid) and holds the same
 * values.  No allocation and no synchronisation after the plan's first call
 * (which creates the copy stream and its events): the call can be captured
 * into a CUDA graph.  GW_EINVAL for n_bands out of range, a null or
 * misaligned host_grid, or the gw_grid_vis_devcount conditions. */
gw_status gw_grid_vis_devcount_readback(gw_plan plan, const double* uvw_m,
                                        const double* freq_hz, const int64_t* d_nrow,
                                        int64_t max_nrow, int32_t nchan, const void* vis,
                                        void* grid, void* host_grid, int32_t n_bands,
                                        void* cuda_stream);

/* Grid correction (Correction Step, Section 2.3 / 3.3.8), in place on
 * image (device, [npol][N][N] c64):
 *     image[pol][i][j] *= s(i, j) * h(m_i) * h(l_j),
 *     h(l) = 1 / (chat(l) sinc_beta(l)),  l = (pixel - N/2) / N,
 * chat the Fourier transform of the truncated, oversampled w = 0 table
 * (Eq. (hco) of Section 2.4.5 as realised by the table), sinc_beta the
 * nearest-neighbour factor sin(pi l / beta) / (pi l / beta).
 *   direction = +1: image side, applied to the unnormalised inverse FFT of
 *                   a grid prepared with gw_grid_shift; s = (-1)^(i+j)
 *                   re-centres the image on pixel (N/2, N/2).
 *   direction = -1: model side, applied before a forward FFT whose output is
 *                   then passed through gw_grid_shift; s = (-1)^(i+j).
 *   direction =  0: correction only, s = 1.
 * The multiplier is real and diagonal, so +1 and -1 apply the same operator
 * (it is its own adjoint).  Errors: GW_EINVAL, GW_EDEVICE, GW_ECUDA. */
gw_status gw_grid_correct(gw_plan plan, void* image, int32_t direction, void* cuda_stream);

/* Multiply a [npol][N][N] c64 grid in place by (-1)^(kv+ku): moves the uv
 * origin between pixel (N/2, N/2) and the corner (Section 3.3.6, IFFT Step)
 * for an FFT library.  Errors: GW_EINVAL, GW_EDEVICE, GW_ECUDA. */
gw_status gw_grid_shift(gw_plan plan, void* grid, void* cuda_stream);

/* ------------------------------------------------------------------------
 * Stage access (testing, diagnostics, custom pipelines)
 * ------------------------------------------------------------------------ */

/* The index stage alone (pre-processing of Section 3.3.5): writes
 * nrow * nchan records, (row, channel) order, to `out` (device).  Each record
 * is computed in FP64 with the operation sequence
 *     s_c = f / c0 (once per channel);  u_lambda = u * s_c;  x = u_lambda * L + N/2;
 *     q = floor(beta * x + 0.5);  k = floor((q + beta/2) / beta);  o = q - k beta
 * (same for v), plane p = the number of thresholds
 * T_j = ((j - 1/2) / (P-1))^2 * w_max, j = 1 .. P-1, with T_j <= |w * s_c|
 * (the plane nearest in sqrt|w|, ties up, at most P-1; w * s_c must be finite),
 * every operation rounded to nearest with no fused multiply-add.  n_dropped
 * as for gw_grid_vis. */
gw_status gw_index_vis(gw_plan plan, const double* uvw_m, const double* freq_hz, int64_t nrow,
                       int32_t nchan, gw_index_rec* out, int64_t* n_dropped, void* cuda_stream);

/* Copy the plan's kernel tables to host memory as interleaved float32
 * complex, layout [plane][ov + beta/2][ou + beta/2][tv + h][tu + h]
 * (table_elems complex elements; `out` must hold 2 * table_elems floats).
 * plane_offsets (host, may be NULL) receives n_wplanes + 1 element offsets;
 * supports (host, may be NULL) receives n_wplanes supports.  Synchronous. */
gw_status gw_plan_copy_tables(gw_plan plan, float* out, int64_t* plane_offsets, int32_t* supports);

/* Copy the tables as stored (table_dtype elements: 8 bytes for GW_C64, 4
 * for the 16-bit kinds, scaled by 2^table_exp2), same layout and element
 * count as gw_plan_copy_tables.  Synchronous. */
gw_status gw_plan_copy_stored_tables(gw_plan plan, void* out);

/* Copy the corrector h(l_i), i = 0..N-1, to host memory (float64).  Synchronous. */
gw_status gw_plan_copy_corrector(gw_plan plan, double* out);

/* Run index + binning and copy the bins to host memory (tests).  Mode 0
 * ("footprint", the gridder's bins): tiles of grid_tile_u x grid_tile_v
 * pixels, each visibility listed once in every tile its footprint touches.
 * Mode 1 ("centre", the degridder's bins): degrid_tile^2 tiles, each
 * visibility listed once, in the tile of its centre pixel.  Tiles are
 * row-major (v rows); tile_offsets receives ntiles + 1 offsets, entries the
 * visibility ids.  Order within a tile is unspecified.
 * `capacity` is the size of `entries`; GW_EINVAL if too small.  Synchronous. */
gw_status gw_debug_bins(gw_plan plan, const double* uvw_m, const double* freq_hz, int64_t nrow,
                        int32_t nchan, int32_t mode, int64_t* tile_offsets, uint32_t* entries,
                        int64_t capacity, void* cuda_stream);

/* ------------------------------------------------------------------------
 * Tracing
 * ------------------------------------------------------------------------ */

/* Per-stage device time and work of the calls made since the last
 * gw_plan_timing_get (or since timing was enabled). */
typedef struct {
    double index_ms, bin_ms, grid_ms, degrid_ms;   /* summed CUDA-event durations */
    int64_t index_calls, bin_calls, grid_calls, degrid_calls;
    int64_t valid_vis;    /* visibilities that passed the index stage */
    int64_t taps;         /* sum over valid visibilities of S_p^2 (per polarisation) */
} gw_timing;

/* Enable (1) or disable (0) stage timing: when enabled every stage of
 * gw_grid_vis / gw_degrid_vis is bracketed by CUDA events recorded on the
 * call's stream.  Work counters (valid_vis, taps) are always kept. */
gw_status gw_plan_timing_enable(gw_plan plan, int32_t enable);

/* Wait for the recorded events, return the accumulated timings and work,
 * and reset them.  Synchronous. */
gw_status gw_plan_timing_get(gw_plan plan, gw_timing* out);

/* ------------------------------------------------------------------------
 * Misc
 * ------------------------------------------------------------------------ */

/* Measured FP32 FMA throughput of the current device (TFLOP/s, FMA = 2
 * FLOP) from a kernel of independent packed FMAs running `iters` iterations
 * on every SM: a cross-check of the nominal FP32 roofline.  Synchronous.
 * No thesis counterpart.  Errors: GW_EINVAL, GW_ECUDA. */
gw_status gw_ffma_peak(int32_t iters, double* tflops, void* cuda_stream);

/* Number of CUDA kernels this library has launched in this process. */
uint64_t gw_launch_count(void);

/* Static description of a status code. */
const char* gw_strerror(gw_status status);

/* Message describing the last error returned on the calling thread. */
const char* gw_last_error(void);

int32_t gw_api_version(void);

#ifdef __cplusplus
}
#endif

#endif /* GW_H */

/*
 * rick.h -- C ABI of librick, a single-GPU (sm_103a) w-stacking imager.
 *
 * The library computes the hot path of the w-stacking method of
 * arXiv 2601.19714 ("Accelerating radio astronomy imaging with RICK"):
 *   1. rick_grid:  convolutional gridding of visibilities onto the closest
 *                  of Nw w-planes (Sec. 2, Eq. 3; the binning of visibilities
 *                  into tiles is the GPU form of the bucket sort of Sec. 3.2,
 *                  with tile halos in the role of the ghost regions of Eq. 5);
 *   2. rick_fft_wplanes: a 2-D inverse FFT of every w-plane (Sec. 2, Sec. 3.4);
 *   3. rick_phase_correct_reduce: the w phase screen exp(+2 pi i w_k (n-1))
 *                  applied to each transformed plane and the sum over planes
 *                  (Eq. 2), normalised by the sum of weights (natural
 *                  weighting, Sec. 4.1.1) and by the gridding taper.
 *
 * Conventions shared by every call (the readings of the paper they fix are
 * listed in the repository's design notes):
 *   - u, v, w are in wavelengths at a reference frequency, stored [nrow][3]
 *     (FP64).  Channel c scales them by chan_scale[c] = nu_c / nu_ref.
 *   - Visibilities are complex64 interleaved (re, im), [nrow][C][2] floats;
 *     weights float32 [nrow][C]; flags uint8 [nrow][C] (non-zero = flagged)
 *     or NULL.  A visibility is skipped if flagged or if its weight is zero
 *     or not finite, and dropped (counted) if its support leaves the grid.
 *   - Grid cell i holds u = (i - N/2)/fov; a visibility at x = u fov + N/2
 *     covers the S cells x - S/2 < i <= x + S/2.  Plane k covers
 *     w in [w_min + k dw, w_min + (k+1) dw), dw = (w_max - w_min)/Nw, with
 *     k = floor((w - w_min) * (Nw/(w_max - w_min))) clamped to [0, Nw-1];
 *     its phase screen uses w_k = w_min + (k + 1/2) dw.
 *   - Grids are complex64 [planes][N][N] (row = v cell, column = u cell),
 *     stored with the checkerboard sign (-1)^(i+j) that centres the FFT.
 *   - Images are float32 [C][N][N] (row q = m, column p = l), pixel p at
 *     l = (p - N/2) fov/N.  Images ACCUMULATE (+=) so that plane groups can
 *     be streamed; the caller zeroes them once.
 *   - Unless a call says otherwise, array pointers are DEVICE pointers owned
 *     by the caller; the plan owns only its tables and scratch.  Calls are
 *     asynchronous and ordered on the given stream (a cudaStream_t passed as
 *     void*; NULL = the legacy default stream).
 *   - Every call returns a rick_status; RICK_OK = 0.  No C++ exception
 *     crosses the ABI.  rick_last_error() gives a message for the calling
 *     thread.  Errors found by a kernel (there are none by design; the
 *     status word exists for internal consistency checks) are reported by
 *     rick_plan_sync_status().
 *   - A plan may be used from one host thread at a time.
 */
#ifndef RICK_H
#define RICK_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    RICK_OK = 0,
    RICK_ERR_INVALID_ARG = 1, /* a size, pointer or configuration value is invalid */
    RICK_ERR_OOM = 2,         /* device or host allocation failed */
    RICK_ERR_CUDA = 3,        /* a CUDA runtime call or kernel launch failed */
    RICK_ERR_CUFFT = 4,       /* cuFFT plan creation or execution failed */
    RICK_ERR_TIMEOUT = 5,     /* reserved: a bounded device-side wait expired */
    RICK_ERR_UNSUPPORTED = 6, /* valid, but outside what this build supports */
    RICK_ERR_INTERNAL = 7,    /* a device-side consistency check failed */
    RICK_ERR_CAPACITY = 8     /* more visibilities than the plan's reservation */
} rick_status;

typedef enum {
    RICK_KERNEL_GAUSS = 0,          /* exp(-s^2/(2 sigma^2)), kernel_param = sigma in cells */
    RICK_KERNEL_KAISER_BESSEL = 1,  /* I0(beta sqrt(1-(2s/S)^2))/I0(beta), kernel_param = beta */
    RICK_KERNEL_TABLE = 2           /* learned support 4: the Kaiser-Bessel taps (beta =
                                       kernel_param) plus a correction table set by
                                       rick_set_kernel_table; the image is divided by the
                                       support-4 Kaiser-Bessel taper */
} rick_kernel_kind;

typedef enum {
    RICK_PREC_FP32_FP64IDX = 0, /* FP64 uvw->cell index and phase; FP32 accumulation (default) */
    RICK_PREC_ALL_FP32 = 1      /* index and phase in FP32 as well (precision study) */
} rick_precision;

/* Imaging weights.  The paper images with natural weighting (the data
 * weights W, Sec. 4.1.1).  Uniform and Briggs weighting replace W by W'
 * before gridding (and in the sum of weights): with D the density of the
 * channel's gridded visibilities -- the sum of their W on their nearest mesh
 * cell (floor(x + 1/2), floor(y + 1/2)), each counted there and at the cell
 * of its Hermitian partner ((N - i) mod N, (N - j) mod N) --
 *   uniform: W' = W / D(cell),
 *   Briggs:  W' = W / (1 + f^2 D(cell)),  f^2 = (5 10^-R)^2 sum D / sum D^2
 * over the cells of the channel, R = robust (R -> +inf: natural, R -> -inf:
 * proportional to uniform).  W' is stored in FP32. */
/* The 2-D DFT of the w-planes (rick_config.fft_impl). */
typedef enum {
    RICK_FFT_OWN = 0,   /* the library's own transform where it applies (the default) */
    RICK_FFT_CUFFT = 1  /* cuFFT */
} rick_fft_impl;

typedef enum {
    RICK_WEIGHT_NATURAL = 0,
    RICK_WEIGHT_UNIFORM = 1,
    RICK_WEIGHT_BRIGGS = 2
} rick_weighting;

typedef struct rick_config {
    int32_t N;            /* grid side = image side: power of two, 64..65536 */
    int32_t n_wplanes;    /* Nw >= 1 */
    int32_t support;      /* S: 1..16 (4 for RICK_KERNEL_TABLE), S <= tile */
    int32_t n_channels;   /* C >= 1 */
    double fov_rad;       /* field of view, direction cosines, 0 < fov < 1 */
    double w_min, w_max;  /* w range of the planes, wavelengths; w_max > w_min if Nw > 1 */
    double kernel_param;  /* see rick_kernel_kind */
    int32_t kernel_kind;  /* rick_kernel_kind */
    int32_t precision;    /* rick_precision */
    int32_t tile;         /* gridder tile side T: 16, 32 or 64 (0 = 32); T <= N; one warp
                           * grids one tile at a time, so T = 64 allows 128 grid_threads */
    int32_t grid_threads; /* gridder CTA size: 128, 256 or 512 (0 = 128) */
    int32_t fft_batch;    /* planes per cuFFT execution (0 = up to 4 GiB of planes) */
    int32_t tiles_per_grab; /* tiles a gridder warp takes from the work queue at once: 1..8 (0 = 4) */
    int64_t grid_budget_bytes; /* rick_dirty_image: device bytes for plane groups (0 = all) */
    /* Hermitian fold (0 = off).  The dirty image is the real part of the sum
     * over planes in Eq. 2, and Re(z) = Re(conj z), so a visibility V at
     * (u, v) on plane k contributes exactly what conj(V) at (-u, -v) on the
     * plane of w = -w_k contributes.  With the fold on, every record whose
     * plane k lies in the upper half (2k > Nt - 1, Nt the plane count: Nw, or
     * Nw + Sw with a w-kernel) is gridded as its conjugate on plane Nt - 1 - k
     * at the mirrored cells (N - i) mod N, (N - j) mod N, with the same kernel
     * taps and plane weight.  Only the lower ceil(Nt/2) planes are then
     * stored, transformed and reduced: every plane index, plane range and
     * grid array of the API counts stored planes, and the real image equals
     * the unfolded one up to FP32 rounding (the imaginary part of the
     * complex image is not the unfolded one).  The placement decisions (plane,
     * footprint, drop) are those of the unfolded visibility.  Requires
     * w_min == -w_max (so that plane Nt - 1 - k sits at -w_k) and a
     * point-symmetric kernel (Gaussian or Kaiser-Bessel, not TABLE). */
    int32_t hermitian_fold;
    /* w-direction kernel ("improved w-stacking"; 0 or 1 = off).  Eq. 3 writes
     * the gridding kernel as a function of (u, v, w); the paper's method puts
     * each visibility on its closest plane.  With an even w_support Sw in
     * [2, 8] each visibility is spread over Sw consecutive planes with
     * Kaiser-Bessel weights g_w(k - z) (beta = w_kernel_param, z the continuous
     * plane coordinate (w - w_min)/dw - 1/2, clamped to the w range), the
     * planes extend Sw/2 beyond [w_min, w_max] at each end (Nw + Sw planes
     * before the fold, plane k centred at w_min + (k - Sw/2 + 1/2) dw), and the
     * image is also divided by the kernel's transform C_w((n - 1) dw).  The
     * prediction uses the same weights and taper.  Gridding work and records
     * grow by Sw, and nrow * C * Sw must stay below 2^32 - 1 per plan call.
     * The plane spacing must keep the first zero of C_w outside the field:
     * pi Sw dw max|n - 1| < sqrt(beta^2 + pi^2), max over the field corners
     * (else RICK_ERR_INVALID_ARG; the method needs dw max|n - 1| well below
     * 1/2 anyway).
     * Not with a TABLE kernel nor in rick_grid_noalloc or the learned-kernel
     * trainer (RICK_ERR_INVALID_ARG / RICK_ERR_UNSUPPORTED). */
    int32_t w_support;
    double w_kernel_param;
    /* 2-D DFT of the w-planes, rick_fft_impl: RICK_FFT_OWN (0, the default) =
     * the library's own two-pass transform (columns, then rows; the imaging
     * path fuses the row pass with the phase screen and reduction) on a
     * power-of-two mesh 256 <= Ng <= 16384 (padded or not), cuFFT on any other
     * mesh; RICK_FFT_CUFFT (1) = cuFFT, batched (fft_batch planes per
     * execution). */
    int32_t fft_impl;
    int32_t weighting;    /* rick_weighting (0 = natural); imaging only, prediction ignores it */
    double robust;        /* Briggs robustness R (weighting = RICK_WEIGHT_BRIGGS) */
    /* Padded mesh (0 = N, the paper's mesh = image size).  A power of two
     * Ng = alpha N >= N: the visibilities are gridded on Ng x Ng cells of
     * 1/(alpha fov) (x = u fov alpha + Ng/2), every plane, plane range and
     * grid array of the API is Ng x Ng, and the image is the central N x N of
     * the transformed planes, divided by C(p) = int g(s) cos(2 pi s (p - N/2)/Ng)
     * ds (rick_plan_taper returns it).  Less aliasing at the field edge for
     * alpha^2 times the grid memory and FFT work.  Needs a Gaussian or
     * Kaiser-Bessel kernel; not in rick_grid_noalloc.  The weighting
     * density stays on the N x N mesh of cell 1/fov. */
    int32_t grid_size;
} rick_config;

/* Planes a plan stores for cfg: P = Nw, or Nw + Sw with a w-kernel; ceil(P / 2)
 * with the Hermitian fold; -1 if cfg is NULL. */
int32_t rick_stored_planes(const rick_config* cfg);

typedef struct rick_plan rick_plan;

/* ---- plan ------------------------------------------------------------ */

/* Validate cfg, build the kernel and taper tables (FP64 on the host) and the
 * cuFFT plans -- or, with the library's own transform (RICK_FFT_OWN), its
 * twiddle tables, the per-pixel table of the fused row passes (the phase of
 * stored plane 0 and the plane step as Q0.32 turns, and the imaging and model
 * scales: 16 bytes per image pixel, computed once in FP64 on the device) and
 * the occupancy masks used for pruning.  The current CUDA device is the
 * plan's device.  On failure *out is NULL and nothing is leaked. */
rick_status rick_plan_create(const rick_config* cfg, rick_plan** out);

/* Release the plan and everything it owns.  NULL is accepted. */
rick_status rick_plan_destroy(rick_plan* plan);

/* Pre-allocate binning scratch for up to max_rows rows (all channels), so
 * that later calls with nrow <= max_rows allocate nothing; required before a
 * sequence of calls is captured into a CUDA graph.  Without it, rick_bin
 * grows the scratch on demand (synchronously). */
rick_status rick_plan_reserve(rick_plan* plan, int64_t max_rows);

/* The taper C(p), p = 0..N-1, that rick_phase_correct_reduce divides by:
 * C(p) = integral_{-S/2}^{S/2} g(s) cos(2 pi s (p - N/2)/N) ds.  Host out. */
rick_status rick_plan_taper(const rick_plan* plan, double* taper_host);

/* Learned kernel: the correction taps[Nw][L+1][L+1][16] (device, float32,
 * copied into the plan) on an (L+1)x(L+1) lattice of fractional offsets
 * (dx, dy) in [0,1]^2 per w-plane; tap t = 4b + a weighs footprint cell
 * (i0 + a, j0 + b).  The gridder interpolates the correction bilinearly
 * between lattice points and adds it to the separable support-4
 * Kaiser-Bessel taps g(a + 1 - 2 - dx) g(b + 1 - 2 - dy), so an all-zero table
 * is exactly the Kaiser-Bessel kernel.  Only for plans with kernel_kind =
 * RICK_KERNEL_TABLE; 1 <= L <= 256.  The table is read by each gridding
 * call, so a table set after rick_bin applies to the next gridding call. */
rick_status rick_set_kernel_table(rick_plan* plan, const float* taps, int32_t lattice, void* stream);

/* ---- the hot path ---------------------------------------------------- */

/* Place and bin: for every visibility compute, in FP64 (FP32 under
 * RICK_PREC_ALL_FP32), its footprint start, fractional offset and w-plane,
 * then counting-sort the visibilities by (channel, plane, tile, halo class)
 * into plan scratch.  weight_sum[C] (device, out) receives the sum of the
 * weights of the gridded visibilities of each channel; counts[2] (device,
 * out, nullable) receives (gridded, dropped).  nrow * C < 2^32 - 1. */
rick_status rick_bin(rick_plan* plan, const double* uvw, const double* chan_scale,
                     const float* vis, const float* weight, const uint8_t* flag, int64_t nrow,
                     double* weight_sum, int64_t* counts, void* stream);

/* Grid the binned visibilities of channels [chan_begin, chan_end) onto
 * planes [plane_begin, plane_end) (Eq. 3).  grids is
 * [chan_end-chan_begin][plane_end-plane_begin][N][N] complex64; every cell
 * of it is written (cells no visibility touches are written as zero), so it
 * need not be cleared.  Requires a preceding rick_bin on the same plan. */
rick_status rick_grid_binned(rick_plan* plan, int32_t chan_begin, int32_t chan_end,
                             int32_t plane_begin, int32_t plane_end, float* grids, void* stream);

/* rick_grid_binned without the zero fill: the tiles (tile x tile cells) that
 * no binned visibility reaches are not written and keep whatever grids held.
 * Such planes are complete only for the calls that take them with
 * RICK_GRIDDED_BY_PLAN on a plan with the library's own transform, which
 * read every unreached tile as zero without touching it; pass them to
 * nothing else (cuFFT, rick_phase_correct_reduce and the plain transform
 * calls read every cell).  On the sparse coverage of a real array most tiles
 * of most planes are unreached, so this writes a fraction of the plane bytes.
 * RICK_ERR_UNSUPPORTED without the own transform; otherwise as
 * rick_grid_binned (Eq. 3). */
rick_status rick_grid_binned_sparse(rick_plan* plan, int32_t chan_begin, int32_t chan_end,
                                    int32_t plane_begin, int32_t plane_end, float* grids, void* stream);

/* The imaging weights W'[nrow][C] (device, f32) that rick_bin grids with:
 * the data weights for natural weighting, else uniform or Briggs weights of
 * the plan's configuration (see rick_weighting); visibilities that are not
 * gridded keep their weight.  Inputs as for rick_bin.  Uses plan-owned
 * scratch: a [C][N][N] FP64 density. */
rick_status rick_imaging_weights(rick_plan* plan, const double* uvw, const double* chan_scale,
                                 const float* weight, const uint8_t* flag, int64_t nrow,
                                 float* weight_out, void* stream);

/* rick_bin followed by rick_grid_binned for all channels and planes
 * [plane_begin, plane_end). */
rick_status rick_grid(rick_plan* plan, const double* uvw, const double* chan_scale,
                      const float* vis, const float* weight, const uint8_t* flag, int64_t nrow,
                      int32_t plane_begin, int32_t plane_end, float* grids, double* weight_sum,
                      int64_t* counts, void* stream);

/* In place, unnormalised 2-D inverse FFT (exponent +) of n_planes
 * consecutive N x N complex64 planes: the library's own transform (a column
 * pass and a row pass, 2 kernel launches) or cuFFT, see fft_impl. */
rick_status rick_fft_wplanes(rick_plan* plan, float* grids, int64_t n_planes, void* stream);

/* Phase screen and reduction over planes (Eq. 2): for channels
 * [chan_begin, chan_end) and transformed planes [plane_begin, plane_end)
 * (grids laid out as for rick_grid_binned),
 *   image[c][q][p] += (-1)^(p+q) n / (weight_sum[c] C(p) C(q))
 *                     * Re sum_k F_k[q][p] exp(+2 pi i w_k (n - 1)),
 * n = sqrt(1 - l^2 - m^2).  The phase is formed in FP64 per pixel (fixed
 * point per plane).  Precision of the plane sum (this call and the fused row
 * pass alike): per block of 8 planes the sum is taken by Horner's rule with
 * the FP32 rotation z = exp(-2 pi i dw (n - 1)), and the block's last plane
 * gets its exact phasor (formed from the Q0.32 turns); the FP32 powers of z
 * cost 6.6e-7 of the peak on 24 planes at N = 1024 (1.4e-6 without the
 * blocks), within the 1e-5 gate the full-size tests apply at 4096^2 x 16,
 * 8192^2 x 24 and 16384^2 x 16 stored planes.  weight_sum is indexed by
 * absolute channel.
 * image_real is [chan_end-chan_begin][N][N]; image_complex (nullable) the
 * same shape complex64 and receives the value before Re. */
rick_status rick_phase_correct_reduce(rick_plan* plan, const float* grids, int32_t chan_begin,
                                      int32_t chan_end, int32_t plane_begin, int32_t plane_end,
                                      const double* weight_sum, float* image_real,
                                      float* image_complex, void* stream);

/* rick_fft_wplanes followed by rick_phase_correct_reduce over channels
 * [chan_begin, chan_end) and planes [plane_begin, plane_end) of the gridded
 * (untransformed) planes in grids, with the same result up to FP32 rounding.
 * With the library's own transform the row pass is fused with the phase
 * screen and the reduction (2 kernel launches; the transformed planes are
 * never written): grids is left holding the column-transformed planes, not
 * the transformed ones.  With cuFFT it is exactly the two calls. */
rick_status rick_fft_phase_correct_reduce(rick_plan* plan, float* grids, int32_t chan_begin,
                                          int32_t chan_end, int32_t plane_begin, int32_t plane_end,
                                          const double* weight_sum, float* image_real,
                                          float* image_complex, int32_t flags, void* stream);

/* flags of the transform calls:
 * RICK_GRIDDED_BY_PLAN -- grids holds the planes [plane_begin, plane_end) of
 *   channels [chan_begin, chan_end) exactly as the preceding rick_grid_binned
 *   or rick_grid_binned_sparse of this plan's current binning wrote them.
 *   With the library's own transform the calls then prune: every tile that
 *   no visibility reached is taken as zero and never read; the column pass
 *   skips the tile columns (tile-wide bands of columns) that no visibility
 *   reached, the row pass the planes that no visibility reached and the
 *   unreached tile columns of the others (zeros transform to zeros).
 *   Ignored with cuFFT. */
#define RICK_GRIDDED_BY_PLAN 1

/* The two passes of rick_fft_phase_correct_reduce with the library's own
 * transform, as separate calls (RICK_ERR_UNSUPPORTED with cuFFT):
 * rick_fft_wplanes_columns: the length-N inverse DFT down every column of the
 *   planes [plane_begin, plane_end) of channels [chan_begin, chan_end)
 *   (grids laid out as for rick_grid_binned), in place (pass 1).  At N = 16384
 *   with tiles of 32 or more it runs as two four-step passes (whole 256-byte
 *   row segments) and leaves each plane's rows in the four-step order: the
 *   transform's row m is stored at row 128 (m mod 128) + m / 128 (as does
 *   rick_fft_phase_correct_reduce with grids);
 * rick_rows_phase_correct_reduce: the row DFTs of column-transformed planes
 *   (at N = 16384 with tiles of 32 or more, rows in the four-step order above)
 *   fused with the phase screen and reduction, arguments as for
 *   rick_phase_correct_reduce (pass 2; one launch; grids is only read).
 * flags as for rick_fft_phase_correct_reduce (with RICK_GRIDDED_BY_PLAN each
 * call first derives the occupancy from the bin offsets: one small launch). */
rick_status rick_fft_wplanes_columns(rick_plan* plan, float* grids, int32_t chan_begin, int32_t chan_end,
                                     int32_t plane_begin, int32_t plane_end, int32_t flags, void* stream);
rick_status rick_rows_phase_correct_reduce(rick_plan* plan, const float* grids, int32_t chan_begin,
                                           int32_t chan_end, int32_t plane_begin, int32_t plane_end,
                                           const double* weight_sum, float* image_real,
                                           float* image_complex, int32_t flags, void* stream);

/* The whole path on device buffers: bin, then for each group of channels and
 * planes that fits grid_budget_bytes grid, transform and reduce into
 * image_real[C][N][N] (+=) using plan-owned grid memory.  weight_sum[C] and
 * counts[2] as for rick_bin (both nullable). */
rick_status rick_dirty_image(rick_plan* plan, const double* uvw, const double* chan_scale,
                             const float* vis, const float* weight, const uint8_t* flag,
                             int64_t nrow, float* image_real, float* image_complex,
                             double* weight_sum, int64_t* counts, void* stream);

/* As rick_dirty_image, but every pointer is a HOST pointer: the inputs are
 * copied to plan-owned device memory, the image (overwritten, not
 * accumulated) and weight_sum/counts (nullable) are copied back, and the
 * call returns when they are in host memory.  Page-locked host buffers give
 * the fastest copies. */
rick_status rick_dirty_image_host(rick_plan* plan, const double* uvw, const double* chan_scale,
                                  const float* vis, const float* weight, const uint8_t* flag,
                                  int64_t nrow, float* image_real, double* weight_sum,
                                  int64_t* counts, void* stream);

/* ---- batched launch: graph capture and autotuning (pattern 2) -------- */

typedef struct rick_graph rick_graph;

/* Capture the whole path for ALL channels and planes of the plan into one
 * CUDA graph: zero image_real, rick_bin, one persistent rick_grid_binned over
 * every (channel, plane, tile), and rick_fft_phase_correct_reduce over every
 * plane.  Channels may have any (uneven, flagged)
 * visibility counts; the gridder's work queue spans all of them.  Pointers are
 * the device buffers the graph will use on every launch (their contents may
 * change between launches, their addresses may not): grids must hold
 * [C][Nw][N][N] complex64, image_real [C][N][N], weight_sum [C], counts[2]
 * (nullable).  With grids = NULL the graph instead streams channel/plane
 * groups through plan-owned grid memory of grid_budget_bytes (allocated
 * before the capture), exactly as rick_dirty_image does.  The plan must have
 * been reserved (rick_plan_reserve) for at
 * least nrow rows, else RICK_ERR_CAPACITY.  The graph references the plan,
 * which must outlive it. */
rick_status rick_graph_capture(rick_plan* plan, const double* uvw, const double* chan_scale,
                               const float* vis, const float* weight, const uint8_t* flag,
                               int64_t nrow, float* grids, double* weight_sum, float* image_real,
                               int64_t* counts, rick_graph** out);

/* Launch a captured graph on a stream (asynchronous). */
rick_status rick_graph_launch(rick_graph* graph, void* stream);

/* Destroy a captured graph.  NULL is accepted. */
rick_status rick_graph_destroy(rick_graph* graph);

typedef struct rick_tune_entry {
    int32_t tile, grid_threads, tiles_per_grab;
    float grid_ms; /* median time of rick_grid_binned over the timed region */
} rick_tune_entry;

/* Autotune the gridder for this data: for every valid tile side T (16, 32,
 * 64 with S <= T <= N), CTA size (128, 256, 512; those that fit shared
 * memory) and tiles per grab (1, 4, 8), bin the visibilities with T and time rick_grid_binned over channels
 * [chan_begin, chan_end) and planes [plane_begin, plane_end) (grids sized for
 * that region), reps times after one warm-up.  Writes up to max_results
 * entries to results (nullable), their number to *n_results, and the base
 * configuration with the fastest (tile, grid_threads, tiles_per_grab) to
 * *best.  Synchronous; allocates a plan per tile side. */
rick_status rick_autotune(const rick_config* base, const double* uvw, const double* chan_scale,
                          const float* vis, const float* weight, const uint8_t* flag,
                          int64_t nrow, int32_t chan_begin, int32_t chan_end,
                          int32_t plane_begin, int32_t plane_end, float* grids, int32_t reps,
                          rick_tune_entry* results, int32_t max_results, int32_t* n_results,
                          rick_config* best);

/* ---- prediction (degridding) ------------------------------------------
 *
 * The adjoint direction of the imaging path, for major cycles: a real model
 * image per channel to model visibilities.  The paper images only (Sec. 2);
 * the prediction is Eq. 1 discretised on the pixels,
 *   V(u, v, w) = sum_{p,q} J(p, q) / n exp(-2 pi i (u l + v m + w (n - 1))),
 * in w-stacking form with the readings of the imaging path (cell and pixel
 * maps, footprint, planes, checkerboard, taper):
 *   M_k = (-1)^(p+q) J exp(-2 pi i w_k (n - 1)) / (n C(p) C(q) C_w)   (per plane)
 *   F_k = forward 2-D DFT of M_k (cuFFT, exponent -)
 *   V   = sum over the footprint of g(i - x) g(j - y) (-1)^(i+j) F_k(i, j)
 * (C_w = 1 and the closest plane without a w-kernel; with one, V sums the Sw
 * planes' values times their weights g_w).
 * With the Hermitian fold, visibilities of the upper half of the planes are
 * predicted on the mirrored plane at the mirrored cells and conjugated (exact
 * for a real image).  Gaussian and Kaiser-Bessel kernels (not TABLE). */

/* Place and bin every visibility for prediction: the same selection as
 * rick_bin (flags, zero weights and footprints off the grid are skipped;
 * counts[2] (device, nullable) receives (predicted, dropped)).  Replaces any
 * binning of the plan made for gridding, and vice versa. */
rick_status rick_bin_predict(rick_plan* plan, const double* uvw, const double* chan_scale,
                             const float* weight, const uint8_t* flag, int64_t nrow, int64_t* counts,
                             void* stream);

/* M_k for channels [chan_begin, chan_end) and stored planes [plane_begin,
 * plane_end): image_real[chan_end-chan_begin][N][N] (device, f32, row q major)
 * to grids laid out as for rick_grid_binned; every cell is written. */
rick_status rick_model_to_wplanes(rick_plan* plan, const float* image_real, int32_t chan_begin,
                                  int32_t chan_end, int32_t plane_begin, int32_t plane_end,
                                  float* grids, void* stream);

/* In place, unnormalised 2-D forward FFT (exponent -) of n_planes planes. */
rick_status rick_fft_wplanes_forward(rick_plan* plan, float* grids, int64_t n_planes, void* stream);

/* rick_model_to_wplanes followed by rick_fft_wplanes_forward, fused, with the
 * library's own transform on a mesh of 256 to 8192 (RICK_ERR_UNSUPPORTED with
 * cuFFT or a 16384 mesh, where rick_predict forms the model planes and runs
 * the plain transform instead): each model row
 * M_k[q][.] is formed in registers and transformed along the row, so the
 * model planes are never written; then the column pass.  grids receives the
 * transformed planes, up to FP32 rounding those of the two calls.  flags:
 * RICK_GRIDDED_BY_PLAN -- prune to the plan's current prediction binning
 *   (rick_bin_predict): planes and tile columns that no binned visibility
 *   reaches are skipped and only the reached tiles of grids are written (the
 *   rest keep what they held); rick_degrid_binned of the same binning reads
 *   nothing else.  The adjoint of rick_fft_phase_correct_reduce. */
rick_status rick_model_fft_wplanes(rick_plan* plan, const float* image_real, int32_t chan_begin,
                                   int32_t chan_end, int32_t plane_begin, int32_t plane_end, float* grids,
                                   int32_t flags, void* stream);

/* V for every visibility binned by rick_bin_predict whose channel and plane lie
 * in the ranges, from the transformed planes `grids` (layout as for
 * rick_grid_binned): vis_out[nrow][C] complex64 (device) receives those
 * entries; the others are left untouched.  With a w-kernel a visibility has
 * Sw planes and each adds its share (+=), so the caller zeroes vis_out. */
rick_status rick_degrid_binned(rick_plan* plan, const float* grids, int32_t chan_begin,
                               int32_t chan_end, int32_t plane_begin, int32_t plane_end,
                               float* vis_out, void* stream);

/* The whole prediction: rick_bin_predict, then per plane group of the
 * plan-owned grid rick_model_to_wplanes + rick_fft_wplanes_forward +
 * rick_degrid_binned (with the own transform: rick_model_fft_wplanes pruned
 * to the binning + rick_degrid_binned).  vis_out[nrow][C] (device) is zeroed first, so skipped
 * visibilities read 0.  image_real[C][N][N] device f32. */
rick_status rick_predict(rick_plan* plan, const double* uvw, const double* chan_scale,
                         const float* weight, const uint8_t* flag, int64_t nrow,
                         const float* image_real, float* vis_out, int64_t* counts, void* stream);

/* ---- learned support-4 kernel (pattern 4) ---------------------------- */

/* A multilayer perceptron in[3] = (dx, dy, w-plane in [-1, 1]) -> H GELU ->
 * H GELU -> 16 outputs (output t = 4b + a for footprint cell (i0 + a, j0 + b)),
 * FP32, GELU in its tanh form.  Parameters are packed W1[H][3], b1[H],
 * W2[H][H], b2[H], W3[16][H], b3[16]; H is 16, 32 or 64.  The paper grids with
 * a Kaiser-Bessel kernel (Sec. 2, Eq. 3); the network's outputs are a
 * correction to its support-4 taps (the Kaiser-Bessel stays as the fallback
 * and as the untrained starting point), and the image is still divided by
 * the support-4 Kaiser-Bessel taper, so it stays linear in the taps. */
int64_t rick_mlp_param_count(int32_t hidden);

/* out[n][16] = mlp(in[n][3]).  work (nullable) receives [n][6H] saved values
 * for rick_mlp_backward.  All device pointers. */
rick_status rick_mlp_forward(const float* params, int32_t hidden, const float* in, int64_t n,
                             float* out, float* work, void* stream);

/* grad[P] += d(sum_i gout[i] . mlp(in[i]))/dparams for the n points
 * (forward recomputed).  work: [n][6H] floats, scratch: [n][16] floats. */
rick_status rick_mlp_backward(const float* params, int32_t hidden, const float* in, int64_t n,
                              const float* gout, float* grad, float* work, float* scratch,
                              void* stream);

/* One Adam update (Kingma & Ba 2015) of n parameters; step counts from 1. */
rick_status rick_adam_step(float* params, const float* grad, float* m, float* v, int64_t n,
                           float lr, float beta1, float beta2, float eps, int32_t step,
                           void* stream);

/* The inputs of the baked table: out[Nw][L+1][L+1][3] = (ix/L, iy/L, plane
 * coordinate (2k - (Nw-1))/(Nw-1)).  rick_mlp_forward on them gives the
 * correction table rick_set_kernel_table takes. */
rick_status rick_mlp_lattice_inputs(int32_t n_wplanes, int32_t lattice, float* out, void* stream);

typedef struct rick_learn rick_learn;

/* Training set-up: one channel of visibilities (uvw[nvis][3] in wavelengths
 * and weight[nvis], device) placed once with the plan rules of cfg
 * (kernel_kind RICK_KERNEL_TABLE, support 4, one channel, kernel_param = beta
 * of the support-4 Kaiser-Bessel taper) and sorted by w-plane.  The tap table
 * has lattice L (1..64). */
rick_status rick_learn_create(const rick_config* cfg, int32_t lattice, const double* uvw,
                              const float* weight, int64_t nvis, rick_learn** out);
rick_status rick_learn_destroy(rick_learn* learn);

/* Number of visibilities placed on the grid (the rest are skipped/dropped). */
int64_t rick_learn_placed(const rick_learn* learn);

/* One training field: sources[ns][3] = (p, q, flux), positions in pixels
 * anywhere in [0, N) (host, 1..64; p = N/2 is l = 0), probes[np][2] pixels
 * (host, 1..64).  Predicts the
 * field's visibilities (Eq. 1), evaluates at the probes the w-stacking image
 * that gridding with the tap table (device [Nw][L+1][L+1][16]) would give
 * (Eq. 2, 3) and the direct Fourier inversion, and writes the loss
 * sum_P (I_P - D_P)^2 / sum_P D_P^2 to loss[0] (device), grad_scale times
 * its gradient with respect to the table to table_grad (device, same shape;
 * overwritten, or added to if accumulate != 0, so that a batch of fields can
 * be summed; nullable) and (I_P, D_P) pairs to image_dft[np][2] (device,
 * nullable). */
rick_status rick_learn_field_grad(rick_learn* learn, const float* table, const float* sources,
                                  int32_t ns, const int32_t* probes, int32_t np,
                                  float* table_grad, int32_t accumulate, float grad_scale,
                                  float* loss, float* image_dft, void* stream);


/* ---- gridding without allocation ------------------------------------ */

/* rick_grid for callers that may not allocate device memory once they run:
 * for example a streaming pipeline that sizes all device memory at start-up
 * and must not stall on cudaMalloc/cudaFree while data arrives, or a host
 * framework that owns the device memory budget through its own pool.  Same
 * inputs, outputs and layout as rick_grid (all channels, planes
 * [plane_begin, plane_end)), but it takes the configuration directly instead
 * of a plan, and keeps its binning scratch in one fixed 32 MiB array in device
 * memory.  It calls no cudaMalloc, cudaFree or allocating library routine.
 *   - CUDA loads device code lazily by default, so the first call on each
 *     device loads the 32 MiB array and the kernels the call runs, which takes
 *     device memory (RICK_ERR_OOM if there is none left).  Make that first
 *     call at start-up, outside any stream capture, with the support and tile
 *     size that later calls use; later calls allocate nothing, and the array
 *     stays until the process exits.
 *   - The configuration is checked as by rick_plan_create.  Sizes whose scratch
 *     does not fit (about 40 bytes per visibility plus 8 bytes per (channel,
 *     plane, tile, class) bin) return RICK_ERR_CAPACITY; a table kernel, a
 *     w-kernel, a padded grid, non-natural weighting or a kernel too narrow for
 *     its support return RICK_ERR_UNSUPPORTED.  Every refusal is made before
 *     anything is launched or written.
 *   - Every call shares the one array and clears what must start at zero;
 *     calls whose work overlaps on the GPU (other streams or threads) race on
 *     it and must be serialised by the caller.
 * The paper has no counterpart: this is an integration variant only. */
rick_status rick_grid_noalloc(const rick_config* cfg, const double* uvw, const double* chan_scale,
                              const float* vis, const float* weight, const uint8_t* flag,
                              int64_t nrow, int32_t plane_begin, int32_t plane_end, float* grids,
                              double* weight_sum, int64_t* counts, void* stream);

/* ---- introspection --------------------------------------------------- */

/* Synchronise the plan's last stream and report device-side errors. */
rick_status rick_plan_sync_status(rick_plan* plan);

/* Number of this library's kernels the plan has launched so far. */
int64_t rick_plan_launch_count(const rick_plan* plan);

/* The 2-D DFT the plan runs: RICK_FFT_OWN (power-of-two mesh 256 <= Ng <=
 * 16384 with fft_impl = RICK_FFT_OWN) or RICK_FFT_CUFFT; -1 if plan is NULL. */
int32_t rick_plan_fft_impl(const rick_plan* plan);

/* The lengths of the gridder's three longest-first tile lists in the plan's
 * last rick_grid_binned / rick_grid_binned_sparse / rick_grid call: the
 * tiles reached by at least 64 T, 16 T and 4 T records (T the tile side).
 * The first two lists are the dense tiles that the gridder splits over the
 * warps of a CTA (the load balancing of Sec. 3.2 on one device); for tests.
 * Synchronous (waits for the plan's last stream). */
rick_status rick_plan_schedule_counts(rick_plan* plan, uint32_t counts[3]);

/* ---- failure handling (tests) ---------------------------------------
 *
 * The paper's pipeline has no failure handling; these hooks let a caller's
 * (and this library's) tests drive every error path without a GPU fault. */

typedef enum {
    RICK_INJECT_NONE = 0,
    RICK_INJECT_DEVICE_ALLOC = 1, /* a device allocation of a plan returns RICK_ERR_OOM */
    RICK_INJECT_CUFFT_PLAN = 2,   /* a cuFFT plan creation returns RICK_ERR_CUFFT */
    RICK_INJECT_LAUNCH = 3        /* a kernel launch is reported as failed (RICK_ERR_CUDA) */
} rick_inject_site;

/* Arm one failure: the countdown-th event of that kind from now (process
 * wide, any thread) fails once, then the site disarms.  RICK_INJECT_NONE or
 * countdown 0 disarms.  The call that fails returns its status and leaks
 * nothing (a failing rick_plan_create frees what it allocated; a failing
 * call on a plan leaves the plan's memory owned by the plan, and the plan
 * usable).  The launched kernel of an injected launch failure has run; only
 * its report is replaced.  The environment variable RICK_INJECT="site:n"
 * arms the same at the library's first check, unless this call came first. */
rick_status rick_debug_inject(int32_t site, int32_t countdown);

/* 1 in a RICK_DEBUG build of the library (device-side consistency checks:
 * a failed check records its code in the plan's status word, the guarded
 * access is skipped, and rick_plan_sync_status returns RICK_ERR_INTERNAL
 * and clears the word; no trap), else 0. */
int32_t rick_debug_build(void);

/* RICK_DEBUG builds only (else RICK_ERR_UNSUPPORTED): overwrite the first
 * footprint cell (tile-relative, 0..255) of binned record `index` of the
 * plan's current gridding binning, keeping its fractions, so that a test can
 * make the gridder's record check fail.  A cell outside the tile is also
 * harmless in a normal build (the gridder clips every cell to its tile).
 * Synchronous. */
rick_status rick_debug_poke_record(rick_plan* plan, int64_t index, int32_t cell_x, int32_t cell_y);

/* Copy the binning result of the last rick_bin to host memory, for tests:
 * offsets[n_keys + 1] (uint32, start of every (channel, plane, tile, class)
 * bin) and records[n_records][4] (uint32: W*V re and im as float bits, then
 * the packed x and y: first footprint cell relative to the tile in the top 8
 * bits, fractional offset * 2^24 in the low 24).  Pass NULL to query the
 * sizes only.  Synchronous. */
rick_status rick_plan_bins(rick_plan* plan, int64_t* n_keys, int64_t* n_records,
                           uint32_t* offsets, uint32_t* records);

const char* rick_status_string(rick_status status);
const char* rick_last_error(void);

#ifdef __cplusplus
}
#endif

#endif /* RICK_H */

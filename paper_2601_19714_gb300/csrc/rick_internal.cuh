// rick_internal.cuh -- types shared by the translation units of librick.
//
// Data layout in HBM (all device memory):
//   inputs   uvw[nrow][3] f64, chan_scale[C] f64, vis[nrow][C] complex64,
//            weight[nrow][C] f32, flag[nrow][C] u8
//   binning  key[nrec] u32, rank[nrec] u32, stage[nrec] VisRecord (unsorted),
//            hist[nkeys] u32, offsets[nkeys+1] u32, records[nrec] VisRecord
//            (sorted by key = (((c*Nw + k)*NT + ty)*NT + tx)*4 + halo class);
//            nrec = nvis, or nvis * Sw with a w-kernel (Sw records per
//            visibility, record s of visibility v at v * Sw + s before sorting)
//   grids    [channels][planes][N][N] complex64, checkerboard-signed
//   images   [channels][N][N] f32
#pragma once

#include <cuda_runtime.h>
#include <cufft.h>
#include <stdint.h>

#include <vector>

#include "rick.h"

namespace rick {

// One binned visibility: W*V (FP32) and, per axis, the first footprint cell
// relative to the anchor tile (top 8 bits) and the fractional offset
// f = (x - S/2) - floor(x - S/2) in units of 2^-24 (low 24 bits).  Records
// binned for prediction hold the visibility index in the bits of wv_re and
// the record's plane weight in wv_im (1, or the w-kernel tap), negative where
// the prediction is to be conjugated.
struct __align__(16) VisRecord {
    float wv_re, wv_im;
    uint32_t px, py;
};

constexpr uint32_t kInvalidKey = 0xFFFFFFFFu;
constexpr int kFracBits = 24;
constexpr uint32_t kFracMask = (1u << kFracBits) - 1u;

// Halo classes of a visibility relative to its anchor tile, ordered so that
// each neighbour reads one contiguous class range:
//   0 interior, 1 spills down only, 2 spills right and down, 3 spills right only.
// The tile to the right reads classes [2,4), the tile below [1,3), the
// diagonal tile [2,3).
__host__ __device__ inline int halo_class(bool right, bool down) {
    return right ? (down ? 2 : 3) : (down ? 1 : 0);
}

// Separable kernels are evaluated per footprint tap a from a polynomial in
// t = 2 f - 1 (f = fractional offset in [0, 1)): g(a + 1 - S/2 - f) ~= sum_k
// coef[a][k] t^k, degree kPolyDegree, fitted on the host in FP64 (Chebyshev
// interpolation) and checked there against g to 1e-6 (typically 6e-8).
constexpr int kMaxSupport = 16;
constexpr int kPolyDegree = 11;
constexpr int kMaxWSupport = 8;   // w-kernel support

struct PlaceParams {
    int N, S, Nw, C, T, NT;
    int precision;
    // Hermitian fold: visibilities on planes 2k > Nw - 1 go to plane Nw - 1 - k
    // as conj(V) at the mirrored footprint; the keys count Nw_store planes.
    int fold, Nw_store;
    // Prediction binning: records carry the visibility's index (bits of
    // wv_re) and its plane weight, negated if its prediction is to be
    // conjugated (set by the fold), in wv_im, instead of W V.
    int predict;
    // w-kernel (w_support >= 2): Sw records per visibility on planes k0 .. k0 +
    // Sw - 1 of the extended set of Nw_total = Nw + Sw planes (the first Sw/2
    // below w_min), weights from the fitted tap polynomials wcoef (t = 2 fw - 1).
    // Nw_total is also the plane count the fold mirrors.
    int w_support, Nw_total;
    float wcoef[kMaxWSupport][kPolyDegree + 1];
    double fov, half_n, half_s, w_min, w_scale;  // w_scale = Nw/(w_max - w_min), 0 if Nw == 1
    float fov_f, half_n_f, half_s_f, w_min_f, w_scale_f;
    // The mesh above has N = Ng cells of 1/(fov Ng/Ni) (fov is scaled); the
    // imaging-weight density uses the Ni x Ni mesh of cell 1/fov_i.
    int Ni;
    double fov_i, half_i;
    float fov_i_f, half_i_f;
};

// Device-side consistency checks of the RICK_DEBUG build: a failed check
// records its code in the plan's status word (the first failure wins), the
// access it guards is skipped, and rick_plan_sync_status returns
// RICK_ERR_INTERNAL.  No trap, no assert: the context stays usable.  The
// normal build compiles the checks away.
#ifdef RICK_DEBUG
#define RICK_DCHECK(cond, code, status)                                      \
    ((cond) ? true : ((status) != nullptr ? (atomicCAS((status), 0, (code)), false) : false))
#else
#define RICK_DCHECK(cond, code, status) true
#endif
constexpr int kCheckGridItem = 1;     // a gridder work item beyond the launch's tiles
constexpr int kCheckRecordCell = 2;   // a record's first footprint cell outside its tile

struct GridParams {
    int N, S, T, NT, Nw;  // Nw: stored planes (the bin keys' plane count)
    int c0, nc, k0, nk;
    uint32_t n_items;     // nc * nk * NT * NT tiles
    int kind;             // rick_kernel_kind
    const float* table;   // RICK_KERNEL_TABLE: [Nw][L+1][L+1][16]
    int lattice;
    uint32_t grab;        // tiles a warp takes from the work queue per atomic
    // Longest-first order (optional): three lists, list_cap entries each, of
    // the tiles with at least 64T, 16T and 4T records (own bins plus the
    // neighbours' spill), filled by a scheduling pass; work_counter[1..3]
    // hold their lengths.  The gridder takes those tiles first, heaviest list
    // first, then every other tile in natural order.  nullptr: natural order.
    uint32_t* lists;
    uint32_t list_cap;
    // Sparse mode (skip_empty) only, optional: every other reached tile (fewer
    // than 4T records, at least one), listed by the scheduling pass
    // (work_counter[5] holds the count); the gridder then visits the lists
    // only, never the unreached tiles.  light_cap >= the launch's tiles.
    uint32_t* light;
    uint32_t light_cap;
    int w_support;        // prediction: >= 2 accumulates the Sw partial predictions
    // 1: tiles that no record reaches are not written (the zero fill is left
    // out); the planes are then only valid where tile_reach() > 0
    int skip_empty;
    int* status;          // the plan's status word (RICK_DEBUG checks); may be null
    float coef[kMaxSupport][kPolyDegree + 1];
};

// Records that reach tile (ty, tx) of a plane, kplane = (channel * planes +
// plane) * NT (the plane's bin keys start at kplane * NT * 4, keys as in the
// layout above): those of the tile's own bins (every halo class) and the
// spilling classes of its left (2, 3), upper (1, 2) and upper-left (2)
// neighbours, which wrap around the mesh (only the Hermitian fold's mirrored
// footprints spill out of the last row or column).  These are the eight bin
// bounds the gridder reads for a tile; zero means the gridder finds no
// record for it.
__device__ __forceinline__ uint32_t tile_reach(const uint32_t* __restrict__ offsets, uint64_t kplane,
                                               int NT, int ty, int tx) {
    const int txl = tx > 0 ? tx - 1 : NT - 1, tyu = ty > 0 ? ty - 1 : NT - 1;
    const uint64_t own = ((kplane + ty) * NT + tx) * 4u, left = ((kplane + ty) * NT + txl) * 4u;
    const uint64_t up = ((kplane + tyu) * NT + tx) * 4u, ul = ((kplane + tyu) * NT + txl) * 4u;
    return (__ldg(offsets + own + 4) - __ldg(offsets + own)) +
           (__ldg(offsets + left + 4) - __ldg(offsets + left + 2)) +
           (__ldg(offsets + up + 3) - __ldg(offsets + up + 1)) +
           (__ldg(offsets + ul + 3) - __ldg(offsets + ul + 2));
}

// Entries per longest-first list for a plan binning up to max_vis
// visibilities with tile side T: a record is counted by at most 4 tiles (its
// own and 3 neighbours), so at most 4 max_vis / (4T) tiles reach 4T records.
inline uint32_t schedule_list_cap(int64_t max_vis, int T) {
    return (uint32_t)(max_vis / T + 64);
}

// Fit the tap polynomials of a Gaussian or Kaiser-Bessel kernel of support S
// (param = sigma or beta) into G.coef; returns the largest deviation from the
// kernel found on a fine grid with FP32 Horner evaluation.
double fit_tap_polynomials(int kind, double param, int S, GridParams& G);

struct PhaseParams {
    int N, nc, nk;        // N: mesh side of the planes (Ng)
    int Ni, off;          // image side and its offset in the planes (padding: (Ng - Ni)/2)
    double dl;            // fov / Ni
    double w_first;       // w of plane plane_begin (plane centre)
    int k_first;          // plane_begin (stored plane index)
    int rows_four;        // N = 16384: the planes' rows are in the four-step order
    double dw;            // plane spacing (0 if Nw == 1)
    int precision;
    // w-kernel (w_support >= 2): every pixel is also divided by the kernel's
    // transform C_w((n - 1) dw) (Kaiser-Bessel, beta = w_beta):
    //   C_w(nu) = w_c0 (beta / r) sinh(r) / sinh(beta),  r^2 = beta^2 - (pi Sw nu)^2 > 0
    //           = w_s_i0 sin(r) / r,                     r^2 = (pi Sw nu)^2 - beta^2 >= 0
    // with w_c0 = C_w(0) and w_s_i0 = Sw / I0(beta) from the host in FP64.
    int w_support;
    double w_beta;
    float w_c0, w_s_i0, w_exp2b;  // w_exp2b = exp(-2 beta)
};

// 1 / C_w(delta dw) for the Kaiser-Bessel w-kernel of support Sw (1 without
// one), from its closed-form transform
//   C_w(nu) = Sw sinh(r) / (r I0(beta)),  r = sqrt(beta^2 - (pi Sw nu)^2),
// (sin for r^2 < 0).  Inside the main lobe it is written relative to C_w(0):
//   C_w(nu) / C_w(0) = (beta / r) e^(-eps) (1 - e^(-2 r)) / (1 - e^(-2 beta)),
// eps = beta - r = a^2 / (beta + r), a = pi Sw nu, so that FP32 sees no
// large argument and no cancellation; r and eps come from FP64 once per pixel.
__device__ __forceinline__ float w_taper_inv(const PhaseParams& P, double delta) {
    if (P.w_support < 2) return 1.0f;
    const double a = 3.141592653589793 * P.w_support * (delta * P.dw);
    const double b = P.w_beta;
    const double x2 = b * b - a * a;
    if (x2 > 0.0) {
        const double r = sqrt(x2);
        const float eps = (float)(a * a / (b + r));
        const float ratio = (float)(b / r) * expf(-eps) * (1.0f - expf(-2.0f * (float)r)) /
                            (1.0f - P.w_exp2b);
        return 1.0f / (P.w_c0 * ratio);
    }
    const float r = (float)sqrt(-x2);
    const float h = r < 1e-4f ? 1.0f : sinf(r) / r;
    return 1.0f / (P.w_s_i0 * h);
}

// The configuration check of rick_plan_create (RICK_OK, or the status and a
// message for rick_last_error()).
rick_status validate_config(const rick_config* cfg);

// --- launchers (one per kernel family), all asynchronous on `stream` -------

// vis_base: index of the first visibility of this call in the whole binning
// (the pointers are offset to it; prediction records carry vis_base + index).
cudaError_t launch_place(const PlaceParams& P, const double* uvw, const double* chan_scale,
                         const float2* vis, const float* weight, const uint8_t* flag,
                         int64_t nvis, uint32_t* hist, uint32_t* key, uint32_t* rank,
                         VisRecord* stage, double* weight_sum, unsigned long long* counts,
                         int num_sms, cudaStream_t stream, int* launches, int64_t vis_base = 0);

// Imaging weights W' (uniform / Briggs) of every visibility into out[nvis];
// density [C][N][N] and moments [2C] are scratch (zeroed here).
cudaError_t launch_imaging_weights(const PlaceParams& P, const double* uvw, const double* chan_scale,
                                   const float* weight, const uint8_t* flag, int64_t nvis, int mode,
                                   double robust, double* density, double* moments, float* out,
                                   int num_sms, cudaStream_t stream, int* launches);

cudaError_t launch_scan(const uint32_t* in, uint32_t* out, uint32_t* partials, uint64_t n,
                        cudaStream_t stream, int* launches);

cudaError_t launch_scatter(const uint32_t* key, const uint32_t* rank, const VisRecord* stage,
                           const uint32_t* offsets, VisRecord* records, int64_t nvis,
                           int num_sms, cudaStream_t stream, int* launches);

// work_counter: 8 words, zero on entry (queue positions, list lengths).
cudaError_t launch_grid(const GridParams& G, const uint32_t* offsets, const VisRecord* records,
                        float2* grids, uint32_t* work_counter, int threads, int num_sms,
                        cudaStream_t stream, int* launches);

cudaError_t launch_phase_reduce(const PhaseParams& P, const float2* grids, const double* wsum,
                                const float* taper, float* image_real, float2* image_complex,
                                cudaStream_t stream, int* launches);

// prediction (degridding)
cudaError_t launch_model_planes(const PhaseParams& P, const float* image, const float* inv_taper,
                                float2* grids, cudaStream_t stream, int* launches);

// Gathers the prediction of every record binned for prediction whose
// (channel, plane) lies in G's range from the transformed planes `grids`
// (layout as for the gridder) into vis_out[index] (conjugated where flagged).
// work_counter: 1 word, zero on entry.
cudaError_t launch_degrid(const GridParams& G, const uint32_t* offsets, const VisRecord* records,
                          const float2* grids, float2* vis_out, uint32_t* work_counter, int threads,
                          int num_sms, cudaStream_t stream, int* launches);

uint64_t scan_partials_needed(uint64_t n);

// The library's own 2-D DFT of the w-planes (rick_fft.cu), 256 <= N <= 16384
// (powers of two).  twid: the table fft_twiddles(N) in device memory (for
// N = 16384 the 16384-point tables followed by the 8192-point ones).  The
// fused model row pass of the prediction (launch_model_rows) takes N <= 8192.
bool fft_supported(int N);
bool fft_fused_model_supported(int N);
void fft_twiddles(int N, std::vector<float2>& out);
// In place, unnormalised, over n_planes planes [N][N]: columns then rows.
cudaError_t launch_fft2d(float2* grids, int64_t n_planes, int N, bool inverse, const float2* twid,
                         cudaStream_t stream, int* launches);
// Occupancy of gridded planes, for pruning (plane p of the launch, tiles of
// side T = 1 << tshift, NT per side):
//   col[p * NT + tx] != 0 if tile column tx of plane p is reached by a record,
//   plane[p] != 0 if any tile of plane p is,
//   tile[(p * NT + ty) * words + tx / 32] bit tx % 32: tile (ty, tx) is reached
//   (words = ceil(NT / 32)).
// A tile no record reaches is zero in the gridder's output (or, with
// skip_empty, unwritten), so the transforms treat it as zero without reading
// it.  Null pointers: no pruning.
struct Occupancy {
    const uint8_t* col = nullptr;
    const uint8_t* plane = nullptr;
    const uint32_t* tile = nullptr;
    int tshift = 0, NT = 1, words = 1;
    // the reached tile columns of the launch as a list: list[0] entries
    // col index p * NT + tx in list[2 ..], list[1] the column pass's work
    // counter (zeroed with the list); nullptr: the column pass launches one
    // CTA per column and skips the unreached ones
    uint32_t* list = nullptr;
    // column pass: false -- the input's unreached tiles are zero (imaging);
    // true -- the input is dense and only the reached tiles of the output are
    // written (prediction)
    bool tiles_out = false;
};
// The three masks of the launch's planes (channels [c0, c0 + nc), stored
// planes [k0, k0 + nk)) from the bin offsets of the plan's binning.
cudaError_t launch_occupancy(const uint32_t* offsets, int c0, int nc, int k0, int nk, int Nw_store, int NT,
                             uint8_t* col, uint8_t* plane, uint32_t* tile, uint32_t* list,
                             cudaStream_t stream, int* launches);
// Pass 1 alone (the inverse DFT down every column), in place; with occ, the
// unreached column tiles are skipped and the unreached tiles of the others
// read as zeros.
// fourstep (N = 16384 only): the two four-step passes, which leave the rows
// of every plane in the four-step order (mesh row m at row 128 (m mod 128) +
// m / 128), the order the fused row pass reads with PhaseParams::rows_four.
cudaError_t launch_fft_columns(float2* grids, int64_t n_planes, int N, bool inverse, const float2* twid,
                               const Occupancy& occ, cudaStream_t stream, int* launches,
                               bool fourstep = false);
// Pass 2 fused with the phase screen and reduction: grids must hold the
// column-transformed planes [nc][nk][N][N]; image_real [nc][N][N] (+=).
// With occ, unreached planes are skipped and unreached tile columns read as
// zeros (the column pass left them untouched).  pix_turns / pix_scale: the
// plan's per-pixel table (launch_pixel_phase), P.k_first the launch's first
// stored plane.
cudaError_t launch_rows_phase_reduce(const PhaseParams& P, const float2* grids, const double* wsum,
                                     const uint2* pix_turns, const float* pix_scale, const float2* twid,
                                     float* image_real, float2* image_complex, const Occupancy& occ,
                                     cudaStream_t stream, int* launches);
// The per-pixel table of the fused row passes ([N][N] each): the phase of
// stored plane 0 and the plane step in Q0.32 turns, and the pixel's scale for
// imaging (checkerboard sign, n, tapers) and for the model of a prediction
// (sign, 1/n, tapers); P0 = the phase parameters of stored plane 0.
cudaError_t launch_pixel_phase(const PhaseParams& P0, const float* inv_taper, uint2* turns, float* scale,
                               float* model_scale, cudaStream_t stream);
// Prediction: the model rows of image[nc][N][N] for the launch's planes,
// transformed along the rows (forward), into grids[nc][nk][N][N]; with occ,
// unreached planes are skipped and only reached tile columns written.
cudaError_t launch_model_rows(const PhaseParams& P, const float* image, const uint2* pix_turns,
                              const float* pix_model_scale, const float2* twid, float2* grids,
                              const Occupancy& occ, cudaStream_t stream, int* launches);

// learned kernel network (rick_mlp.cu)
int64_t mlp_param_count(int H);
cudaError_t mlp_forward(const float* params, int H, const float* in, int64_t n, float* out,
                        float* work, cudaStream_t st);
cudaError_t mlp_backward(const float* params, int H, const float* in, int64_t n, const float* gout,
                         float* grad, float* work, float* scratch_out, cudaStream_t st);
cudaError_t adam_step(float* p, const float* g, float* m, float* v, int64_t n, float lr, float b1,
                      float b2, float eps, int step, cudaStream_t st);
cudaError_t lattice_inputs(int Nw, int L, float* out, cudaStream_t st);

}  // namespace rick

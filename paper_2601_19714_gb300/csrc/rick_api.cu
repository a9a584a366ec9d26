// rick_api.cu -- the C ABI of librick: plans, validation, scratch, cuFFT,
// and the host-side sequencing of the w-stacking path.
//
// Everything here is host code; the kernels live in rick_bin.cu (placement
// and binning), rick_grid.cu (gridding, Eq. 3) and rick_phase.cu (phase
// screen and reduction, Eq. 2).
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <algorithm>
#include <atomic>
#include <mutex>
#include <new>
#include <vector>

#include "rick_internal.cuh"

using namespace rick;

namespace {

thread_local char g_err[1024] = "";

void set_err(const char* fmt, ...) {
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(g_err, sizeof g_err, fmt, ap);
    va_end(ap);
}

#define RK_CUDA(expr)                                                                     \
    do {                                                                                  \
        cudaError_t e_ = (expr);                                                          \
        if (e_ != cudaSuccess) {                                                          \
            set_err("%s failed: %s (%s:%d)", #expr, cudaGetErrorString(e_), __FILE__,    \
                    __LINE__);                                                            \
            return e_ == cudaErrorMemoryAllocation ? RICK_ERR_OOM : RICK_ERR_CUDA;        \
        }                                                                                 \
    } while (0)

#define RK_TRY(expr)                          \
    do {                                      \
        rick_status s_ = (expr);              \
        if (s_ != RICK_OK) return s_;         \
    } while (0)

#define RK_ARG(cond, msg)                     \
    do {                                      \
        if (!(cond)) {                        \
            set_err("invalid argument: %s", msg); \
            return RICK_ERR_INVALID_ARG;      \
        }                                     \
    } while (0)

// ---- fault injection (tests of the error paths) ------------------------------
//
// rick_debug_inject arms one site: the countdown-th event of that kind from
// now fails once -- a device allocation of the library returns
// cudaErrorMemoryAllocation without allocating, a cuFFT plan creation
// returns an error, or a kernel launch is reported as failed (the kernel has
// been queued; the call returns RICK_ERR_CUDA as if the launch had failed).
// The environment variable RICK_INJECT="site:countdown" arms the same at the
// first check of a process.
std::atomic<int> g_inject_site{0}, g_inject_left{0};
std::once_flag g_inject_env;

void inject_init() {
    std::call_once(g_inject_env, [] {
        const char* e = std::getenv("RICK_INJECT");
        int a = 0, b = 0;
        if (e && std::sscanf(e, "%d:%d", &a, &b) == 2 && a > 0 && a <= RICK_INJECT_LAUNCH && b > 0) {
            g_inject_left.store(b);
            g_inject_site.store(a);
        }
    });
}

bool inject_fire(int site) {
    inject_init();
    if (site == RICK_INJECT_NONE || g_inject_site.load(std::memory_order_relaxed) != site) return false;
    if (g_inject_left.fetch_sub(1) == 1) {
        g_inject_site.store(0);
        return true;
    }
    return false;
}

// cudaMalloc for the plan's memory, with the injection point
template <class T>
cudaError_t dmalloc(T** p, size_t bytes) {
    if (inject_fire(RICK_INJECT_DEVICE_ALLOC)) {
        *p = nullptr;
        return cudaErrorMemoryAllocation;
    }
    return cudaMalloc(reinterpret_cast<void**>(p), bytes);
}

// ---- FP64 host math for the tables (independent of any other code) -------

double bessel_i0(double x) {
    // I0(x) = sum_k (x^2/4)^k / (k!)^2
    const double y = 0.25 * x * x;
    double term = 1.0, sum = 1.0;
    for (int k = 1; k < 400 && term > 1e-17 * sum; ++k) {
        term *= y / ((double)k * k);
        sum += term;
    }
    return sum;
}

double kernel_fn(int kind, double param, int S, double s) {
    if (std::fabs(s) > 0.5 * S) return 0.0;
    if (kind == RICK_KERNEL_GAUSS) return std::exp(-0.5 * s * s / (param * param));
    const double t = 2.0 * s / S;
    return bessel_i0(param * std::sqrt(std::fmax(0.0, 1.0 - t * t))) / bessel_i0(param);
}

// n-point Gauss-Legendre rule on [-1, 1] (Newton iteration on P_n).
void legendre_rule(int n, std::vector<double>& x, std::vector<double>& w) {
    x.assign(n, 0.0);
    w.assign(n, 0.0);
    const double pi = 3.14159265358979323846;
    for (int i = 0; i < (n + 1) / 2; ++i) {
        double z = std::cos(pi * (i + 0.75) / (n + 0.5)), dp = 1.0;
        for (int it = 0; it < 64; ++it) {
            double pm = 1.0, pc = z;
            for (int k = 2; k <= n; ++k) {
                const double pn = ((2 * k - 1) * z * pc - (k - 1) * pm) / k;
                pm = pc;
                pc = pn;
            }
            dp = n * (z * pc - pm) / (z * z - 1.0);
            const double dz = pc / dp;
            z -= dz;
            if (std::fabs(dz) < 1e-16) break;
        }
        x[i] = -z;
        x[n - 1 - i] = z;
        w[i] = w[n - 1 - i] = 2.0 / ((1.0 - z * z) * dp * dp);
    }
}

// C(p) = int_{-S/2}^{S/2} g(s) cos(2 pi s (p - N/2)/Ng) ds: the continuous
// Fourier transform of the kernel at image pixel p of a mesh of Ng cells
// (Ng = N without padding), by composite Gauss-Legendre quadrature (24 nodes
// per cell of the support).  C is even about N/2.
void make_taper(int kind, double param, int S, int N, int Ng, std::vector<double>& C) {
    std::vector<double> gx, gw;
    legendre_rule(24, gx, gw);
    std::vector<double> s, wg;
    for (int seg = 0; seg < S; ++seg) {
        const double a = -0.5 * S + seg;
        for (size_t i = 0; i < gx.size(); ++i) {
            const double si = a + 0.5 + 0.5 * gx[i];
            s.push_back(si);
            wg.push_back(0.5 * gw[i] * kernel_fn(kind, param, S, si));
        }
    }
    const double two_pi = 6.283185307179586476925;
    std::vector<double> val(N / 2 + 1);
    for (int d = 0; d <= N / 2; ++d) {
        double acc = 0.0;
        for (size_t i = 0; i < s.size(); ++i) acc += wg[i] * std::cos(two_pi * s[i] * d / Ng);
        val[d] = acc;
    }
    C.assign(N, 0.0);
    for (int p = 0; p < N; ++p) C[p] = val[p >= N / 2 ? p - N / 2 : N / 2 - p];
}

}  // namespace

// rick_dirty_image_host transforms and downloads the channels in this many
// chunks, and (natural weighting) uploads and places the rows in kInChunks
constexpr int kHostChunks = 8;
constexpr int kInChunks = 4;

struct rick_plan {
    rick_config cfg;
    int device = 0, num_sms = 0;
    int T = 64, NT = 0, threads = 256, grab = 8;
    int Ng = 0;      // mesh side (grid_size, or N without padding)
    int planes = 0;  // stored planes: ceil(Nt/2) with the Hermitian fold, else Nt
                     // (Nt = Nw, or Nw + Sw with a w-kernel)
    int nrec_per_vis = 1;  // records per visibility: Sw with a w-kernel, else 1
    uint64_t nkeys = 0;
    double w_scale = 0.0, dw = 0.0;
    std::vector<double> taper;
    float* d_inv_taper = nullptr;
    float* d_table = nullptr;
    int lattice = 0;
    // binning scratch, sized in records (visibilities x records per visibility)
    int64_t cap_vis = 0;
    uint32_t* d_key = nullptr;
    uint32_t* d_rank = nullptr;
    VisRecord* d_stage = nullptr;
    VisRecord* d_records = nullptr;
    uint32_t* d_hist = nullptr;
    uint32_t* d_offsets = nullptr;
    uint32_t* d_partials = nullptr;
    uint32_t* d_counter = nullptr;   // gridder queues and list lengths (8 words)
    uint32_t* d_lists = nullptr;     // longest-first tile lists, 3 x list_cap
    uint32_t list_cap = 0;
    uint32_t* d_light = nullptr;     // sparse gridding: the other reached tiles (one per tile of the plan)
    uint32_t light_cap = 0;
    unsigned long long* d_counts = nullptr;
    int* d_status = nullptr;
    double* d_wsum = nullptr;
    bool binned = false;
    bool binned_for_predict = false;  // records hold (index, signed weight) instead of W V
    // cuFFT: batch B and single-plane plans
    cufftHandle fft_b = 0, fft_1 = 0;
    bool have_b = false, have_1 = false;
    int fft_B = 1;
    // plan-owned grid and staging for rick_dirty_image(_host)
    float2* d_grid = nullptr;
    size_t grid_cap = 0;
    unsigned char* d_in = nullptr;
    size_t in_cap = 0;
    float* d_img = nullptr;
    size_t img_cap = 0;
    // rick_dirty_image_host: a copy stream and events for overlapping the image
    // download with the transform of later channels
    cudaStream_t copy_stream = nullptr;
    cudaEvent_t chunk_done[kHostChunks] = {};
    cudaEvent_t in_done[kInChunks] = {};
    int64_t launches = 0;
    cudaStream_t last_stream = nullptr;
    float tap_coef[kMaxSupport][kPolyDegree + 1] = {};
    double tap_fit_error = 0.0;
    // imaging weights (uniform / Briggs): density [C][N][N], moments [2C], W' [cap_w]
    double* d_density = nullptr;
    double* d_wmom = nullptr;
    float* d_wbuf = nullptr;
    int64_t cap_w = 0;
    // the library's own 2-D DFT (RICK_FFT_OWN, mesh 256 <= Ng <= 16384): twiddle tables
    bool own_fft = false;
    float2* d_twid = nullptr;
    uint8_t* d_colocc = nullptr;     // occupancy for pruning: [C][planes][NT] and [C][planes]
    uint8_t* d_planeocc = nullptr;
    uint32_t* d_tileocc = nullptr;   // [C][planes][NT][ceil(NT/32)] tile bits
    uint32_t* d_collist = nullptr;   // 2 + [C][planes][NT]: reached tile columns (Occupancy::list)
    uint2* d_pix_turns = nullptr;    // fused row passes: per-pixel turns and scales [N][N]
    float* d_pix_scale = nullptr;
    float* d_pix_model_scale = nullptr;
    // w-kernel: tap polynomials and the constants of its transform C_w
    float w_coef[kMaxWSupport][kPolyDegree + 1] = {};
    double w_c0 = 1.0, w_s_i0 = 1.0;
};

namespace {

PhaseParams phase_params(const rick_plan* P, int c0, int c1, int k0, int k1);


template <class T>
void dfree(T*& p) {
    if (p) cudaFree((void*)p);
    p = nullptr;
}

void release(rick_plan* P) {
    dfree(P->d_inv_taper);
    dfree(P->d_twid);
    dfree(P->d_colocc);
    dfree(P->d_planeocc);
    dfree(P->d_tileocc);
    dfree(P->d_collist);
    dfree(P->d_pix_turns);
    dfree(P->d_pix_scale);
    dfree(P->d_pix_model_scale);
    dfree(P->d_density);
    dfree(P->d_wmom);
    dfree(P->d_wbuf);
    dfree(P->d_table);
    dfree(P->d_key);
    dfree(P->d_rank);
    dfree(P->d_stage);
    dfree(P->d_records);
    dfree(P->d_hist);
    dfree(P->d_offsets);
    dfree(P->d_partials);
    dfree(P->d_counter);
    dfree(P->d_lists);
    dfree(P->d_light);
    dfree(P->d_counts);
    dfree(P->d_status);
    dfree(P->d_wsum);
    dfree(P->d_grid);
    dfree(P->d_in);
    dfree(P->d_img);
    for (auto& ev : P->chunk_done)
        if (ev) {
            cudaEventDestroy(ev);
            ev = nullptr;
        }
    for (auto& ev : P->in_done)
        if (ev) {
            cudaEventDestroy(ev);
            ev = nullptr;
        }
    if (P->copy_stream) {
        cudaStreamDestroy(P->copy_stream);
        P->copy_stream = nullptr;
    }
    if (P->have_b) cufftDestroy(P->fft_b);
    if (P->have_1) cufftDestroy(P->fft_1);
    P->have_b = P->have_1 = false;
}

int planes_total(const rick_config& c) { return c.n_wplanes + (c.w_support >= 2 ? c.w_support : 0); }

int stored_planes(const rick_config& c) {
    const int t = planes_total(c);
    return c.hermitian_fold ? (t + 1) / 2 : t;
}

rick_status validate(const rick_config* c) {
    RK_ARG(c != nullptr, "cfg is NULL");
    RK_ARG(c->N >= 64 && c->N <= 65536 && (c->N & (c->N - 1)) == 0,
           "N must be a power of two in [64, 65536]");
    const int T = c->tile ? c->tile : 32;
    RK_ARG(T == 16 || T == 32 || T == 64, "tile must be 16, 32 or 64");
    RK_ARG(T <= c->N, "tile must not exceed N");
    const int Ng = c->grid_size ? c->grid_size : c->N;
    RK_ARG(c->grid_size == 0 || (c->grid_size >= c->N && c->grid_size <= 65536 &&
                                 (c->grid_size & (c->grid_size - 1)) == 0),
           "grid_size must be 0 or a power of two in [N, 65536]");
    if (Ng != c->N) {
        RK_ARG(c->kernel_kind != RICK_KERNEL_TABLE, "a padded grid needs a Gaussian or Kaiser-Bessel kernel");
    }
    RK_ARG(c->n_wplanes >= 1, "n_wplanes must be >= 1");
    RK_ARG(c->n_channels >= 1, "n_channels must be >= 1");
    RK_ARG(c->support >= 1 && c->support <= 16 && c->support <= T, "support must be in [1, min(16, tile)]");
    RK_ARG(c->fov_rad > 0.0 && c->fov_rad < 1.0, "fov_rad must be in (0, 1)");
    RK_ARG(std::isfinite(c->w_min) && std::isfinite(c->w_max), "w range must be finite");
    RK_ARG(c->n_wplanes == 1 || c->w_max > c->w_min, "w_max must exceed w_min when n_wplanes > 1");
    RK_ARG(c->kernel_kind == RICK_KERNEL_GAUSS || c->kernel_kind == RICK_KERNEL_KAISER_BESSEL ||
               c->kernel_kind == RICK_KERNEL_TABLE,
           "unknown kernel_kind");
    RK_ARG(c->kernel_param > 0.0 && std::isfinite(c->kernel_param), "kernel_param must be > 0");
    RK_ARG(c->kernel_kind != RICK_KERNEL_TABLE || c->support == 4, "table kernels have support 4");
    RK_ARG(c->precision == RICK_PREC_FP32_FP64IDX || c->precision == RICK_PREC_ALL_FP32,
           "unknown precision");
    const int th = c->grid_threads ? c->grid_threads : 128;
    RK_ARG(th == 128 || th == 256 || th == 512, "grid_threads must be 128, 256 or 512");
    // every warp of a gridder CTA holds one T x (T + 8) complex tile in shared memory
    RK_ARG((size_t)(th / 32) * T * (T + 8) * 8 <= (size_t)160 * 1024,
           "tile 64 allows at most 128 grid_threads (one 37 KB shared tile per warp)");
    RK_ARG(c->fft_batch >= 0, "fft_batch must be >= 0");
    RK_ARG(c->tiles_per_grab >= 0 && c->tiles_per_grab <= 8, "tiles_per_grab must be in [0, 8]");
    RK_ARG(c->grid_budget_bytes >= 0, "grid_budget_bytes must be >= 0");
    RK_ARG(c->hermitian_fold == 0 || c->hermitian_fold == 1, "hermitian_fold must be 0 or 1");
    RK_ARG(c->fft_impl == RICK_FFT_OWN || c->fft_impl == RICK_FFT_CUFFT,
           "fft_impl must be 0 (own transform) or 1 (cuFFT)");
    RK_ARG(c->weighting >= RICK_WEIGHT_NATURAL && c->weighting <= RICK_WEIGHT_BRIGGS,
           "weighting must be 0 (natural), 1 (uniform) or 2 (Briggs)");
    RK_ARG(c->weighting != RICK_WEIGHT_BRIGGS || std::isfinite(c->robust), "robust must be finite");
    RK_ARG(c->w_support == 0 || c->w_support == 1 ||
               (c->w_support >= 2 && c->w_support <= 8 && (c->w_support & 1) == 0),
           "w_support must be 0, 1 or even in [2, 8]");
    if (c->w_support >= 2) {
        RK_ARG(c->n_wplanes >= 2, "a w-kernel needs n_wplanes >= 2");
        RK_ARG(c->kernel_kind != RICK_KERNEL_TABLE,
               "a w-kernel needs a Gaussian or Kaiser-Bessel uv kernel (not a table kernel)");
        RK_ARG(c->w_kernel_param > 0.0 && std::isfinite(c->w_kernel_param),
               "w_kernel_param must be > 0 with a w-kernel");
        // the image is divided by C_w((n - 1) dw); its first zero, at
        // pi Sw |nu| = sqrt(beta^2 + pi^2), must lie outside the field (the
        // field corner has the largest |n - 1|)
        const double half = 0.5 * c->fov_rad, r2 = 2.0 * half * half;
        const double delta = r2 / (1.0 + std::sqrt(1.0 - r2));
        const double dw = (c->w_max - c->w_min) / c->n_wplanes;
        const double pi = 3.141592653589793;
        const double b = c->w_kernel_param;
        RK_ARG(pi * c->w_support * dw * delta < std::sqrt(b * b + pi * pi),
               "w-kernel: the planes are too sparse for the field (C_w has a zero inside it); "
               "use more w-planes or a smaller w_support");
    }
    if (c->hermitian_fold) {
        RK_ARG(c->kernel_kind != RICK_KERNEL_TABLE,
               "hermitian_fold needs a point-symmetric kernel (Gaussian or Kaiser-Bessel)");
        RK_ARG(c->w_min == -c->w_max, "hermitian_fold needs w_min == -w_max");
    }
    // bins = C x stored planes x NT^2 x 4 halo classes, tested factor by factor
    // so that the product cannot wrap
    const uint64_t NT = (uint64_t)(Ng / T);
    const uint64_t per_plane = NT * NT * 4ull;   // <= 2^26
    const uint64_t limit = 0xFFFFFFFFull;
    const uint64_t cp = (uint64_t)c->n_channels * (uint64_t)stored_planes(*c);   // < 2^63
    if (cp >= limit || cp * per_plane >= limit) {
        set_err("channels x planes x tiles exceeds the 32-bit bin space; use a larger tile or "
                "fewer channels per plan");
        return RICK_ERR_UNSUPPORTED;
    }
    return RICK_OK;
}

rick_status ensure_vis_capacity(rick_plan* P, int64_t nvis) {
    if (nvis <= P->cap_vis) return RICK_OK;
    dfree(P->d_key);
    dfree(P->d_rank);
    dfree(P->d_stage);
    dfree(P->d_records);
    dfree(P->d_lists);
    P->cap_vis = 0;
    P->list_cap = 0;
    const size_t n = (size_t)nvis;
    RK_CUDA(dmalloc(&P->d_key, n * sizeof(uint32_t)));
    RK_CUDA(dmalloc(&P->d_rank, n * sizeof(uint32_t)));
    RK_CUDA(dmalloc(&P->d_stage, n * sizeof(VisRecord)));
    RK_CUDA(dmalloc(&P->d_records, n * sizeof(VisRecord)));
    const uint32_t cap = schedule_list_cap(nvis, P->T);
    RK_CUDA(dmalloc(&P->d_lists, 3 * (size_t)cap * sizeof(uint32_t)));
    P->list_cap = cap;
    P->cap_vis = nvis;
    return RICK_OK;
}

rick_status ensure_weight_capacity(rick_plan* P, int64_t nvis) {
    if (nvis <= P->cap_w) return RICK_OK;
    dfree(P->d_wbuf);
    P->cap_w = 0;
    RK_CUDA(dmalloc(&P->d_wbuf, sizeof(float) * (size_t)(nvis > 0 ? nvis : 1)));
    P->cap_w = nvis;
    return RICK_OK;
}

rick_status make_fft_plan(cufftHandle* h, bool* have, int N, int batch) {
    if (inject_fire(RICK_INJECT_CUFFT_PLAN)) {
        set_err("cuFFT plan creation failed (injected)");
        return RICK_ERR_CUFFT;
    }
    if (cufftCreate(h) != CUFFT_SUCCESS) {
        set_err("cufftCreate failed");
        return RICK_ERR_CUFFT;
    }
    *have = true;
    long long n[2] = {N, N};
    size_t work = 0;
    const long long dist = (long long)N * N;
    cufftResult r = cufftMakePlanMany64(*h, 2, n, nullptr, 1, dist, nullptr, 1, dist, CUFFT_C2C,
                                        batch, &work);
    if (r != CUFFT_SUCCESS) {
        set_err("cufftMakePlanMany64(N=%d, batch=%d) failed: %d", N, batch, (int)r);
        return r == CUFFT_ALLOC_FAILED ? RICK_ERR_OOM : RICK_ERR_CUFFT;
    }
    return RICK_OK;
}

rick_status plan_init(rick_plan* P, const rick_config* cfg) {
    P->cfg = *cfg;
    rick_config& c = P->cfg;
    P->T = c.tile ? c.tile : 32;
    c.tile = P->T;
    P->threads = c.grid_threads ? c.grid_threads : 128;
    c.grid_threads = P->threads;
    P->grab = c.tiles_per_grab ? c.tiles_per_grab : 4;
    c.tiles_per_grab = P->grab;
    P->Ng = c.grid_size ? c.grid_size : c.N;
    c.grid_size = P->Ng;
    P->NT = P->Ng / P->T;
    P->planes = stored_planes(c);
    P->nkeys = (uint64_t)c.n_channels * P->planes * (uint64_t)P->NT * P->NT * 4ull;
    if (c.n_wplanes > 1) {
        P->w_scale = (double)c.n_wplanes / (c.w_max - c.w_min);
        P->dw = (c.w_max - c.w_min) / c.n_wplanes;
    }
    RK_CUDA(cudaGetDevice(&P->device));
    RK_CUDA(cudaDeviceGetAttribute(&P->num_sms, cudaDevAttrMultiProcessorCount, P->device));

    {
        // a table kernel is a learned correction added to the Kaiser-Bessel taps
        const int fit_kind = c.kernel_kind == RICK_KERNEL_TABLE ? RICK_KERNEL_KAISER_BESSEL : c.kernel_kind;
        GridParams fit;
        P->tap_fit_error = fit_tap_polynomials(fit_kind, c.kernel_param, c.support, fit);
        std::memcpy(P->tap_coef, fit.coef, sizeof P->tap_coef);
        if (!(P->tap_fit_error <= 1e-6)) {
            set_err("kernel_param %g: the degree-%d tap polynomials reach only %.2e of the kernel "
                    "(limit 1e-6); the kernel is too narrow for this support",
                    c.kernel_param, kPolyDegree, P->tap_fit_error);
            return RICK_ERR_UNSUPPORTED;
        }
    }
    if (c.w_support >= 2) {
        // the w-kernel: Kaiser-Bessel of support Sw; its taps by the same
        // polynomial fit, and C_w(0) = Sw sinh(beta) / (beta I0(beta))
        GridParams fit;
        const double err = fit_tap_polynomials(RICK_KERNEL_KAISER_BESSEL, c.w_kernel_param, c.w_support, fit);
        if (!(err <= 1e-6)) {
            set_err("w_kernel_param %g: the w-kernel's tap polynomials reach only %.2e (limit 1e-6)",
                    c.w_kernel_param, err);
            return RICK_ERR_UNSUPPORTED;
        }
        for (int a = 0; a < c.w_support; ++a)
            for (int q = 0; q <= kPolyDegree; ++q) P->w_coef[a][q] = fit.coef[a][q];
        const double b = c.w_kernel_param;
        double term = 1.0, i0 = 1.0;
        for (int k = 1; k < 400 && term > 1e-17 * i0; ++k) {
            term *= 0.25 * b * b / ((double)k * k);
            i0 += term;
        }
        P->w_s_i0 = c.w_support / i0;
        P->w_c0 = P->w_s_i0 * std::sinh(b) / b;
        P->nrec_per_vis = c.w_support;
    }
    const int taper_kind = c.kernel_kind == RICK_KERNEL_TABLE ? RICK_KERNEL_KAISER_BESSEL : c.kernel_kind;
    make_taper(taper_kind, c.kernel_param, c.support, c.N, P->Ng, P->taper);
    std::vector<float> inv(c.N);
    for (int p = 0; p < c.N; ++p) inv[p] = (float)(1.0 / P->taper[p]);
    RK_CUDA(dmalloc(&P->d_inv_taper, sizeof(float) * c.N));
    RK_CUDA(cudaMemcpy(P->d_inv_taper, inv.data(), sizeof(float) * c.N, cudaMemcpyHostToDevice));

    RK_CUDA(dmalloc(&P->d_hist, sizeof(uint32_t) * P->nkeys));
    RK_CUDA(dmalloc(&P->d_offsets, sizeof(uint32_t) * (P->nkeys + 1)));
    RK_CUDA(dmalloc(&P->d_partials, sizeof(uint32_t) * scan_partials_needed(P->nkeys)));
    RK_CUDA(dmalloc(&P->d_counter, 8 * sizeof(uint32_t)));
    RK_CUDA(dmalloc(&P->d_counts, 2 * sizeof(unsigned long long)));
    RK_CUDA(dmalloc(&P->d_status, sizeof(int)));
    RK_CUDA(cudaMemset(P->d_status, 0, sizeof(int)));
    RK_CUDA(dmalloc(&P->d_wsum, sizeof(double) * c.n_channels));
    if (c.weighting != RICK_WEIGHT_NATURAL) {
        RK_CUDA(dmalloc(&P->d_density, sizeof(double) * (size_t)c.N * c.N * c.n_channels));
        RK_CUDA(dmalloc(&P->d_wmom, sizeof(double) * 2 * c.n_channels));
    }

    P->own_fft = c.fft_impl == RICK_FFT_OWN && fft_supported(P->Ng);
    if (P->own_fft) {
        std::vector<float2> tw;
        fft_twiddles(P->Ng, tw);   // the transforms run on the mesh
        RK_CUDA(dmalloc(&P->d_twid, sizeof(float2) * tw.size()));
        RK_CUDA(cudaMemcpy(P->d_twid, tw.data(), sizeof(float2) * tw.size(), cudaMemcpyHostToDevice));
        RK_CUDA(dmalloc(&P->d_colocc, (size_t)c.n_channels * P->planes * P->NT));
        RK_CUDA(dmalloc(&P->d_planeocc, (size_t)c.n_channels * P->planes));
        RK_CUDA(dmalloc(&P->d_tileocc, sizeof(uint32_t) * (size_t)c.n_channels * P->planes * P->NT *
                                              ((P->NT + 31) / 32)));
        RK_CUDA(dmalloc(&P->d_collist, sizeof(uint32_t) * (2 + (size_t)c.n_channels * P->planes * P->NT)));
        const size_t NN = (size_t)c.N * c.N;
        // the sparse gridder's list of light tiles: room for every tile of the plan
        P->light_cap = (uint32_t)(P->nkeys / 4);
        RK_CUDA(dmalloc(&P->d_light, sizeof(uint32_t) * (size_t)P->light_cap));
        RK_CUDA(dmalloc(&P->d_pix_turns, sizeof(uint2) * NN));
        RK_CUDA(dmalloc(&P->d_pix_scale, sizeof(float) * NN));
        RK_CUDA(dmalloc(&P->d_pix_model_scale, sizeof(float) * NN));
        RK_CUDA(launch_pixel_phase(phase_params(P, 0, 1, 0, 1), P->d_inv_taper, P->d_pix_turns, P->d_pix_scale,
                                   P->d_pix_model_scale, nullptr));
        RK_CUDA(cudaDeviceSynchronize());
        return RICK_OK;   // no cuFFT plans
    }
    const size_t plane_bytes = (size_t)P->Ng * P->Ng * sizeof(float2);
    int B = c.fft_batch;
    if (B <= 0) {
        const size_t cap = (size_t)4 << 30;
        B = (int)(cap / plane_bytes);
        const long long total = (long long)P->planes * c.n_channels;
        if (B > total) B = (int)total;
        if (B < 1) B = 1;
    }
    P->fft_B = B;
    c.fft_batch = B;
    RK_TRY(make_fft_plan(&P->fft_1, &P->have_1, P->Ng, 1));
    if (B > 1) RK_TRY(make_fft_plan(&P->fft_b, &P->have_b, P->Ng, B));
    return RICK_OK;
}

inline cudaStream_t as_stream(void* s) { return reinterpret_cast<cudaStream_t>(s); }

rick_status check_launch(cudaError_t e, const char* what) {
    if (e == cudaSuccess && inject_fire(RICK_INJECT_LAUNCH)) e = cudaErrorLaunchFailure;
    if (e != cudaSuccess) {
        set_err("%s: %s", what, cudaGetErrorString(e));
        return RICK_ERR_CUDA;
    }
    return RICK_OK;
}

// Placement parameters of the plan (binning for gridding or for prediction).
PlaceParams place_params(const rick_plan* P, bool predict) {
    const rick_config& c = P->cfg;
    PlaceParams pp;
    pp.N = P->Ng;
    pp.S = c.support;
    pp.Nw = c.n_wplanes;
    pp.C = c.n_channels;
    pp.T = P->T;
    pp.NT = P->NT;
    pp.precision = c.precision;
    pp.fold = c.hermitian_fold;
    pp.Nw_store = P->planes;
    pp.predict = predict ? 1 : 0;
    pp.w_support = c.w_support >= 2 ? c.w_support : 0;
    pp.Nw_total = planes_total(c);
    std::memcpy(pp.wcoef, P->w_coef, sizeof pp.wcoef);
    // x = u fov Ng/N + Ng/2 (exact scaling: powers of two); the weighting
    // density's mesh is the N x N mesh of cell 1/fov
    pp.fov = c.fov_rad * (double)P->Ng / (double)c.N;
    pp.half_n = 0.5 * P->Ng;
    pp.Ni = c.N;
    pp.fov_i = c.fov_rad;
    pp.half_i = 0.5 * c.N;
    pp.fov_i_f = (float)c.fov_rad;
    pp.half_i_f = (float)(0.5 * c.N);
    pp.half_s = 0.5 * c.support;
    pp.w_min = c.w_min;
    pp.w_scale = P->w_scale;
    pp.fov_f = (float)pp.fov;
    pp.half_n_f = (float)pp.half_n;
    pp.half_s_f = (float)pp.half_s;
    pp.w_min_f = (float)c.w_min;
    pp.w_scale_f = (float)P->w_scale;
    return pp;
}

// The first part of a binning: checks, scratch capacity, zeroed counters.
rick_status bin_begin(rick_plan* P, int64_t nrow, double* weight_sum, bool predict, cudaStream_t st,
                      int64_t* nrec_out) {
    const rick_config& c = P->cfg;
    RK_ARG(nrow >= 0, "nrow must be >= 0");
    RK_ARG(weight_sum != nullptr, "weight_sum is NULL");
    const int64_t nvis = nrow * (int64_t)c.n_channels;
    RK_ARG(nrow == 0 || nvis / nrow == c.n_channels, "nrow * C overflows");
    const int64_t nrec = nvis * P->nrec_per_vis;
    if (nrec >= (int64_t)0xFFFFFFFFLL) {
        set_err("nrow * C%s = %lld exceeds 2^32 - 2 records per plan call",
                P->nrec_per_vis > 1 ? " * w_support" : "", (long long)nrec);
        return RICK_ERR_UNSUPPORTED;
    }
    RK_TRY(ensure_vis_capacity(P, nrec));
    if (!predict && c.weighting != RICK_WEIGHT_NATURAL) RK_TRY(ensure_weight_capacity(P, nvis));
    P->last_stream = st;
    RK_CUDA(cudaMemsetAsync(P->d_hist, 0, sizeof(uint32_t) * P->nkeys, st));
    RK_CUDA(cudaMemsetAsync(weight_sum, 0, sizeof(double) * c.n_channels, st));
    RK_CUDA(cudaMemsetAsync(P->d_counts, 0, 2 * sizeof(unsigned long long), st));
    *nrec_out = nrec;
    return RICK_OK;
}

// The last part: the scan of the bin counts and the scatter into bins.
rick_status bin_end(rick_plan* P, int64_t nrec, int64_t* counts, bool predict, cudaStream_t st) {
    int launches = 0;
    rick_status s = check_launch(launch_scan(P->d_hist, P->d_offsets, P->d_partials, P->nkeys, st, &launches),
                                 "scan kernels");
    if (s == RICK_OK)
        s = check_launch(launch_scatter(P->d_key, P->d_rank, P->d_stage, P->d_offsets,
                                        P->d_records, nrec, P->num_sms, st, &launches),
                         "scatter kernel");
    P->launches += launches;
    RK_TRY(s);
    if (counts)
        RK_CUDA(cudaMemcpyAsync(counts, P->d_counts, 2 * sizeof(int64_t), cudaMemcpyDeviceToDevice, st));
    P->binned = true;
    P->binned_for_predict = predict;
    return RICK_OK;
}

rick_status bin_impl(rick_plan* P, const double* uvw, const double* chan_scale, const float* vis,
                     const float* weight, const uint8_t* flag, int64_t nrow, double* weight_sum,
                     int64_t* counts, cudaStream_t st, bool predict = false) {
    const rick_config& c = P->cfg;
    if (nrow > 0) {
        RK_ARG(uvw && chan_scale && (vis || predict) && weight,
               "uvw, chan_scale, vis and weight are required");
    }
    int64_t nrec = 0;
    RK_TRY(bin_begin(P, nrow, weight_sum, predict, st, &nrec));
    const int64_t nvis = nrow * (int64_t)c.n_channels;
    int launches = 0;
    const PlaceParams pp = place_params(P, predict);
    rick_status s = RICK_OK;
    if (!predict && c.weighting != RICK_WEIGHT_NATURAL && nvis > 0) {
        // imaging weights W' into the plan's buffer, gridded in place of W
        s = check_launch(launch_imaging_weights(pp, uvw, chan_scale, weight, flag, nvis, c.weighting,
                                                c.robust, P->d_density, P->d_wmom, P->d_wbuf,
                                                P->num_sms, st, &launches),
                         "imaging weight kernels");
        weight = P->d_wbuf;
    }
    if (s == RICK_OK) s = check_launch(
        launch_place(pp, uvw, chan_scale, reinterpret_cast<const float2*>(vis), weight, flag, nvis,
                     P->d_hist, P->d_key, P->d_rank, P->d_stage, weight_sum, P->d_counts,
                     P->num_sms, st, &launches),
        "placement kernel");
    P->launches += launches;
    RK_TRY(s);
    return bin_end(P, nrec, counts, predict, st);
}

// Imaging binning from host inputs (natural weighting): the rows arrive in
// kInChunks chunks on the copy stream, and each chunk is placed on st as soon
// as it is in device memory, so the upload overlaps the placement.  d_* are
// the device copies (the same layout as the host arrays).
rick_status bin_from_host(rick_plan* P, const double* uvw, const double* chan_scale, const float* vis,
                          const float* weight, const uint8_t* flag, int64_t nrow, double* d_uvw,
                          double* d_sc, float* d_vis, float* d_w, uint8_t* d_f, double* weight_sum,
                          int64_t* counts, cudaStream_t st) {
    const rick_config& c = P->cfg;
    const int64_t C = c.n_channels;
    int64_t nrec = 0;
    RK_TRY(bin_begin(P, nrow, weight_sum, false, st, &nrec));
    if (!P->copy_stream) RK_CUDA(cudaStreamCreateWithFlags(&P->copy_stream, cudaStreamNonBlocking));
    for (auto& ev : P->in_done)
        if (!ev) RK_CUDA(cudaEventCreateWithFlags(&ev, cudaEventDisableTiming));
    // the copies must not overtake earlier work of st on the input buffers
    RK_CUDA(cudaEventRecord(P->in_done[0], st));
    RK_CUDA(cudaStreamWaitEvent(P->copy_stream, P->in_done[0], 0));
    RK_CUDA(cudaMemcpyAsync(d_sc, chan_scale, C * sizeof(double), cudaMemcpyHostToDevice, P->copy_stream));
    const PlaceParams pp = place_params(P, false);
    const int64_t nr = P->nrec_per_vis;
    int launches = 0;
    rick_status s = RICK_OK;
    for (int i = 0; i < kInChunks && s == RICK_OK; ++i) {
        const int64_t r0 = nrow * i / kInChunks, r1 = nrow * (i + 1) / kInChunks;
        if (r1 == r0) continue;
        const int64_t n = r1 - r0, v0 = r0 * C;
        RK_CUDA(cudaMemcpyAsync(d_uvw + 3 * r0, uvw + 3 * r0, n * 3 * sizeof(double), cudaMemcpyHostToDevice,
                                P->copy_stream));
        RK_CUDA(cudaMemcpyAsync(d_vis + 2 * v0, vis + 2 * v0, n * C * 2 * sizeof(float), cudaMemcpyHostToDevice,
                                P->copy_stream));
        RK_CUDA(cudaMemcpyAsync(d_w + v0, weight + v0, n * C * sizeof(float), cudaMemcpyHostToDevice,
                                P->copy_stream));
        if (flag)
            RK_CUDA(cudaMemcpyAsync(d_f + v0, flag + v0, n * C, cudaMemcpyHostToDevice, P->copy_stream));
        RK_CUDA(cudaEventRecord(P->in_done[i], P->copy_stream));
        RK_CUDA(cudaStreamWaitEvent(st, P->in_done[i], 0));
        s = check_launch(launch_place(pp, d_uvw + 3 * r0, d_sc, reinterpret_cast<const float2*>(d_vis + 2 * v0),
                                      d_w + v0, flag ? d_f + v0 : nullptr, n * C, P->d_hist, P->d_key + v0 * nr,
                                      P->d_rank + v0 * nr, P->d_stage + v0 * nr, weight_sum, P->d_counts,
                                      P->num_sms, st, &launches, v0),
                         "placement kernel");
    }
    P->launches += launches;
    RK_TRY(s);
    return bin_end(P, nrec, counts, false, st);
}

// sparse: tiles no record reaches are not written (only for the pruned own
// transform, which never reads them)
rick_status grid_impl(rick_plan* P, int c0, int c1, int k0, int k1, float* grids, cudaStream_t st,
                      bool sparse = false) {
    const rick_config& c = P->cfg;
    RK_ARG(P->binned && !P->binned_for_predict, "rick_bin must precede gridding");
    RK_ARG(0 <= c0 && c0 < c1 && c1 <= c.n_channels, "channel range");
    RK_ARG(0 <= k0 && k0 < k1 && k1 <= P->planes, "plane range");
    RK_ARG(grids != nullptr, "grids is NULL");
    RK_ARG(((uintptr_t)grids & 15u) == 0, "grids must be 16-byte aligned");
    if (c.kernel_kind == RICK_KERNEL_TABLE && !P->d_table) {
        set_err("table kernel: call rick_set_kernel_table first");
        return RICK_ERR_INVALID_ARG;
    }
    const uint64_t items = (uint64_t)(c1 - c0) * (k1 - k0) * (uint64_t)P->NT * P->NT;
    RK_ARG(items < 0xFFFFFFFFull, "too many tiles in one call");
    GridParams G;
    std::memset(&G, 0, sizeof G);
    G.N = P->Ng;
    G.S = c.support;
    G.T = P->T;
    G.NT = P->NT;
    G.Nw = P->planes;
    G.c0 = c0;
    G.nc = c1 - c0;
    G.k0 = k0;
    G.nk = k1 - k0;
    G.n_items = (uint32_t)items;
    G.kind = c.kernel_kind;
    std::memcpy(G.coef, P->tap_coef, sizeof G.coef);
    G.table = P->d_table;
    G.lattice = P->lattice;
    G.grab = (uint32_t)P->grab;
    G.lists = P->d_lists;
    G.list_cap = P->list_cap;
    G.w_support = 0;
    G.skip_empty = sparse ? 1 : 0;
    if (sparse && P->d_light) {
        G.light = P->d_light;
        G.light_cap = P->light_cap;
    }
    G.status = P->d_status;
    P->last_stream = st;
    RK_CUDA(cudaMemsetAsync(P->d_counter, 0, 8 * sizeof(uint32_t), st));
    int launches = 0;
    rick_status s = check_launch(launch_grid(G, P->d_offsets, P->d_records,
                                             reinterpret_cast<float2*>(grids), P->d_counter,
                                             P->threads, P->num_sms, st, &launches),
                                 "gridding kernel");
    P->launches += launches;
    return s;
}

rick_status fft_impl(rick_plan* P, float* grids, int64_t n_planes, cudaStream_t st,
                     int direction = CUFFT_INVERSE) {
    RK_ARG(n_planes >= 0, "n_planes must be >= 0");
    RK_ARG(n_planes == 0 || grids != nullptr, "grids is NULL");
    const size_t NN = (size_t)P->Ng * P->Ng;
    P->last_stream = st;
    if (P->own_fft) {
        RK_ARG(((uintptr_t)grids & 15u) == 0, "grids must be 16-byte aligned");
        int launches = 0;
        rick_status s = check_launch(launch_fft2d(reinterpret_cast<float2*>(grids), n_planes, P->Ng,
                                                  direction == CUFFT_INVERSE, P->d_twid, st, &launches),
                                     "FFT kernels");
        P->launches += launches;
        return s;
    }
    cufftComplex* g = reinterpret_cast<cufftComplex*>(grids);
    int64_t done = 0;
    if (P->have_b) {
        if (cufftSetStream(P->fft_b, st) != CUFFT_SUCCESS) {
            set_err("cufftSetStream failed");
            return RICK_ERR_CUFFT;
        }
        for (; done + P->fft_B <= n_planes; done += P->fft_B) {
            cufftComplex* d = g + (size_t)done * NN;
            const cufftResult r = cufftExecC2C(P->fft_b, d, d, direction);
            if (r != CUFFT_SUCCESS) {
                set_err("cufftExecC2C (batch) failed: %d", (int)r);
                return RICK_ERR_CUFFT;
            }
        }
    }
    if (done < n_planes) {
        if (cufftSetStream(P->fft_1, st) != CUFFT_SUCCESS) {
            set_err("cufftSetStream failed");
            return RICK_ERR_CUFFT;
        }
        for (; done < n_planes; ++done) {
            cufftComplex* d = g + (size_t)done * NN;
            const cufftResult r = cufftExecC2C(P->fft_1, d, d, direction);
            if (r != CUFFT_SUCCESS) {
                set_err("cufftExecC2C failed: %d", (int)r);
                return RICK_ERR_CUFFT;
            }
        }
    }
    return RICK_OK;
}

// Phase-screen parameters of planes [k0, k1) (stored indices) of channels
// [c0, c1): plane k is centred at w_min + (k - off + 1/2) dw, off = Sw/2 with
// a w-kernel (its extended plane set starts below w_min), else 0.
// At N = 16384 with tiles of at least 32, the column pass of the imaging calls
// is the four-step pair (two passes of whole 256-byte row segments) and
// leaves the rows in the four-step order, which the fused row pass reads.
bool fourstep_layout(const rick_plan* P) { return P->own_fft && P->Ng == 16384 && P->T >= 32; }

PhaseParams phase_params(const rick_plan* P, int c0, int c1, int k0, int k1) {
    const rick_config& c = P->cfg;
    PhaseParams pp;
    pp.N = P->Ng;
    pp.Ni = c.N;
    pp.off = (P->Ng - c.N) / 2;
    pp.nc = c1 - c0;
    pp.nk = k1 - k0;
    pp.dl = c.fov_rad / c.N;
    pp.dw = c.n_wplanes > 1 ? P->dw : 0.0;
    const int off = c.w_support >= 2 ? c.w_support / 2 : 0;
    pp.w_first = c.n_wplanes > 1 ? c.w_min + (k0 - off + 0.5) * P->dw : 0.5 * (c.w_min + c.w_max);
    pp.k_first = k0;
    pp.rows_four = fourstep_layout(P) ? 1 : 0;
    pp.precision = c.precision;
    pp.w_support = c.w_support >= 2 && c.n_wplanes > 1 ? c.w_support : 0;
    pp.w_beta = c.w_kernel_param;
    pp.w_c0 = (float)P->w_c0;
    pp.w_s_i0 = (float)P->w_s_i0;
    pp.w_exp2b = (float)std::exp(-2.0 * c.w_kernel_param);
    return pp;
}

rick_status phase_impl(rick_plan* P, const float* grids, int c0, int c1, int k0, int k1,
                       const double* weight_sum, float* image_real, float* image_complex,
                       cudaStream_t st) {
    const rick_config& c = P->cfg;
    RK_ARG(0 <= c0 && c0 < c1 && c1 <= c.n_channels, "channel range");
    RK_ARG(0 <= k0 && k0 < k1 && k1 <= P->planes, "plane range");
    RK_ARG(grids && weight_sum && image_real, "grids, weight_sum and image_real are required");
    RK_ARG(((uintptr_t)grids & 15u) == 0 && ((uintptr_t)image_real & 7u) == 0 &&
               ((uintptr_t)image_complex & 15u) == 0,
           "grids/image_complex must be 16-byte and image_real 8-byte aligned");
    const PhaseParams pp = phase_params(P, c0, c1, k0, k1);
    P->last_stream = st;
    int launches = 0;
    rick_status s = check_launch(
        launch_phase_reduce(pp, reinterpret_cast<const float2*>(grids), weight_sum + c0,
                            P->d_inv_taper, image_real, reinterpret_cast<float2*>(image_complex),
                            st, &launches),
        "phase kernel");
    P->launches += launches;
    return s;
}

// Occupancy of the planes [k0, k1) of channels [c0, c1) from the current
// binning (for pruning the own transform): the gridding binning, or with
// predict the prediction binning.
rick_status occupancy_impl(rick_plan* P, int c0, int c1, int k0, int k1, cudaStream_t st,
                           bool predict = false) {
    if (predict)
        RK_ARG(P->binned && P->binned_for_predict,
               "RICK_GRIDDED_BY_PLAN on the model needs the plan's binning for prediction (rick_bin_predict)");
    else
        RK_ARG(P->binned && !P->binned_for_predict,
               "RICK_GRIDDED_BY_PLAN needs the plan's binning for gridding (rick_bin)");
    int launches = 0;
    rick_status s = check_launch(launch_occupancy(P->d_offsets, c0, c1 - c0, k0, k1 - k0, P->planes, P->NT,
                                                  P->d_colocc, P->d_planeocc, P->d_tileocc, P->d_collist,
                                                  st, &launches),
                                 "occupancy kernel");
    P->launches += launches;
    return s;
}

// The occupancy masks of the last occupancy_impl.
Occupancy plan_occupancy(const rick_plan* P) {
    Occupancy o;
    o.col = P->d_colocc;
    o.plane = P->d_planeocc;
    o.tile = P->d_tileocc;
    o.list = P->d_collist;
    int sh = 0;
    while ((1 << sh) < P->T) ++sh;
    o.tshift = sh;
    o.NT = P->NT;
    o.words = (P->NT + 31) / 32;
    return o;
}

// Pass 1 of the own transform (inverse DFT down every column), in place.
rick_status columns_impl(rick_plan* P, float* grids, int c0, int c1, int k0, int k1, int32_t flags,
                         cudaStream_t st) {
    const rick_config& c = P->cfg;
    if (!P->own_fft) {
        set_err("the column pass needs the library's own transform (RICK_FFT_OWN, a mesh of 256 to 16384)");
        return RICK_ERR_UNSUPPORTED;
    }
    RK_ARG(0 <= c0 && c0 < c1 && c1 <= c.n_channels, "channel range");
    RK_ARG(0 <= k0 && k0 < k1 && k1 <= P->planes, "plane range");
    RK_ARG(grids != nullptr, "grids is NULL");
    RK_ARG(((uintptr_t)grids & 15u) == 0, "grids must be 16-byte aligned");
    P->last_stream = st;
    Occupancy occ;
    if (flags & RICK_GRIDDED_BY_PLAN) {
        RK_TRY(occupancy_impl(P, c0, c1, k0, k1, st));
        occ = plan_occupancy(P);
    }
    int launches = 0;
    rick_status s = check_launch(launch_fft_columns(reinterpret_cast<float2*>(grids),
                                                    (int64_t)(c1 - c0) * (k1 - k0), P->Ng, true,
                                                    P->d_twid, occ, st, &launches, fourstep_layout(P)),
                                 "FFT column kernel");
    P->launches += launches;
    return s;
}

// Pass 2 fused with the phase screen and reduction, on column-transformed planes.
rick_status rows_phase_impl(rick_plan* P, const float* grids, int c0, int c1, int k0, int k1,
                            const double* weight_sum, float* image_real, float* image_complex,
                            int32_t flags, cudaStream_t st, bool occ_ready = false) {
    const rick_config& c = P->cfg;
    if (!P->own_fft) {
        set_err("the fused row pass needs the library's own transform (RICK_FFT_OWN, a mesh of 256 to 16384)");
        return RICK_ERR_UNSUPPORTED;
    }
    RK_ARG(0 <= c0 && c0 < c1 && c1 <= c.n_channels, "channel range");
    RK_ARG(0 <= k0 && k0 < k1 && k1 <= P->planes, "plane range");
    RK_ARG(grids && weight_sum && image_real, "grids, weight_sum and image_real are required");
    RK_ARG(((uintptr_t)grids & 15u) == 0 && ((uintptr_t)image_real & 3u) == 0 &&
               ((uintptr_t)image_complex & 7u) == 0,
           "grids must be 16-byte, image_real 4-byte and image_complex 8-byte aligned");
    P->last_stream = st;
    if ((flags & RICK_GRIDDED_BY_PLAN) && !occ_ready) RK_TRY(occupancy_impl(P, c0, c1, k0, k1, st));
    int launches = 0;
    rick_status s = check_launch(launch_rows_phase_reduce(phase_params(P, c0, c1, k0, k1),
                                                          reinterpret_cast<const float2*>(grids),
                                                          weight_sum + c0, P->d_pix_turns, P->d_pix_scale,
                                                          P->d_twid,
                                                          image_real,
                                                          reinterpret_cast<float2*>(image_complex),
                                                          (flags & RICK_GRIDDED_BY_PLAN) ? plan_occupancy(P) : Occupancy{},
                                                          st, &launches),
                                 "fused row FFT / phase kernel");
    P->launches += launches;
    return s;
}

// Transform + phase screen + reduction of gridded planes [k0, k1) of channels
// [c0, c1): with the own transform, the column pass and the fused row pass.
rick_status fft_phase_impl(rick_plan* P, float* grids, int c0, int c1, int k0, int k1,
                           const double* weight_sum, float* image_real, float* image_complex,
                           cudaStream_t st, int32_t flags = 0) {
    const rick_config& c = P->cfg;
    if (!P->own_fft) {
        RK_ARG(0 <= c0 && c0 < c1 && c1 <= c.n_channels, "channel range");
        RK_ARG(0 <= k0 && k0 < k1 && k1 <= P->planes, "plane range");
        RK_TRY(fft_impl(P, grids, (int64_t)(c1 - c0) * (k1 - k0), st));
        return phase_impl(P, grids, c0, c1, k0, k1, weight_sum, image_real, image_complex, st);
    }
    RK_ARG(0 <= c0 && c0 < c1 && c1 <= c.n_channels, "channel range");
    RK_ARG(0 <= k0 && k0 < k1 && k1 <= P->planes, "plane range");
    RK_TRY(columns_impl(P, grids, c0, c1, k0, k1, flags, st));
    // the occupancy computed by the column pass serves the row pass too
    return rows_phase_impl(P, grids, c0, c1, k0, k1, weight_sum, image_real, image_complex, flags, st, true);
}

rick_status model_impl(rick_plan* P, const float* image, int c0, int c1, int k0, int k1, float* grids,
                       cudaStream_t st) {
    const rick_config& c = P->cfg;
    RK_ARG(0 <= c0 && c0 < c1 && c1 <= c.n_channels, "channel range");
    RK_ARG(0 <= k0 && k0 < k1 && k1 <= P->planes, "plane range");
    RK_ARG(image && grids, "image and grids are required");
    RK_ARG(((uintptr_t)grids & 15u) == 0 && ((uintptr_t)image & 7u) == 0,
           "grids must be 16-byte and image 8-byte aligned");
    P->last_stream = st;
    int launches = 0;
    rick_status s = check_launch(
        launch_model_planes(phase_params(P, c0, c1, k0, k1), image, P->d_inv_taper,
                            reinterpret_cast<float2*>(grids), st, &launches),
        "model kernel");
    P->launches += launches;
    return s;
}

// Prediction's model planes and their forward 2-D DFT with the own transform:
// the model rows are formed and transformed in one pass (never written as
// model planes), then the column pass.  With RICK_GRIDDED_BY_PLAN (the plan's
// prediction binning) unreached planes and tile columns are skipped and only
// the reached tiles of the result are written.
rick_status model_fft_impl(rick_plan* P, const float* image, int c0, int c1, int k0, int k1, float* grids,
                           int32_t flags, cudaStream_t st) {
    const rick_config& c = P->cfg;
    if (!P->own_fft || !fft_fused_model_supported(P->Ng)) {
        set_err("the fused model pass needs the library's own transform on a mesh of 256 to 8192 "
                "(RICK_FFT_OWN); use rick_model_to_wplanes + rick_fft_wplanes_forward");
        return RICK_ERR_UNSUPPORTED;
    }
    RK_ARG(0 <= c0 && c0 < c1 && c1 <= c.n_channels, "channel range");
    RK_ARG(0 <= k0 && k0 < k1 && k1 <= P->planes, "plane range");
    RK_ARG(image && grids, "image and grids are required");
    RK_ARG(((uintptr_t)grids & 15u) == 0 && ((uintptr_t)image & 3u) == 0,
           "grids must be 16-byte and image 4-byte aligned");
    P->last_stream = st;
    Occupancy occ;
    if (flags & RICK_GRIDDED_BY_PLAN) {
        RK_TRY(occupancy_impl(P, c0, c1, k0, k1, st, true));
        occ = plan_occupancy(P);
        occ.tiles_out = true;
    }
    int launches = 0;
    rick_status s = check_launch(launch_model_rows(phase_params(P, c0, c1, k0, k1), image, P->d_pix_turns,
                                                   P->d_pix_model_scale, P->d_twid,
                                                   reinterpret_cast<float2*>(grids), occ, st, &launches),
                                 "fused model / row kernel");
    if (s == RICK_OK)
        s = check_launch(launch_fft_columns(reinterpret_cast<float2*>(grids), (int64_t)(c1 - c0) * (k1 - k0),
                                            P->Ng, false, P->d_twid, occ, st, &launches),
                         "FFT column kernel");
    P->launches += launches;
    return s;
}

rick_status degrid_impl(rick_plan* P, const float* grids, int c0, int c1, int k0, int k1,
                        float* vis_out, cudaStream_t st) {
    const rick_config& c = P->cfg;
    RK_ARG(P->binned && P->binned_for_predict, "rick_bin_predict must precede degridding");
    RK_ARG(0 <= c0 && c0 < c1 && c1 <= c.n_channels, "channel range");
    RK_ARG(0 <= k0 && k0 < k1 && k1 <= P->planes, "plane range");
    RK_ARG(grids && vis_out, "grids and vis_out are required");
    RK_ARG(((uintptr_t)grids & 15u) == 0 && ((uintptr_t)vis_out & 7u) == 0,
           "grids must be 16-byte and vis_out 8-byte aligned");
    const uint64_t items = (uint64_t)(c1 - c0) * (k1 - k0) * (uint64_t)P->NT * P->NT;
    RK_ARG(items < 0xFFFFFFFFull, "too many tiles in one call");
    GridParams G;
    std::memset(&G, 0, sizeof G);
    G.N = P->Ng;
    G.S = c.support;
    G.T = P->T;
    G.NT = P->NT;
    G.Nw = P->planes;
    G.c0 = c0;
    G.nc = c1 - c0;
    G.k0 = k0;
    G.nk = k1 - k0;
    G.n_items = (uint32_t)items;
    G.kind = c.kernel_kind;
    G.w_support = c.w_support >= 2 ? c.w_support : 0;
    G.status = P->d_status;
    std::memcpy(G.coef, P->tap_coef, sizeof G.coef);
    P->last_stream = st;
    RK_CUDA(cudaMemsetAsync(P->d_counter, 0, sizeof(uint32_t), st));
    int launches = 0;
    rick_status s = check_launch(
        launch_degrid(G, P->d_offsets, P->d_records, reinterpret_cast<const float2*>(grids),
                      reinterpret_cast<float2*>(vis_out), P->d_counter, 128, P->num_sms, st, &launches),
        "degridding kernel");
    P->launches += launches;
    return s;
}

// Plane groups for the plan-owned grid: all channels x all planes if they fit
// the budget, else whole channels, else planes of one channel.
void plan_groups(const rick_plan* P, int* gc, int* gk) {
    const rick_config& c = P->cfg;
    const size_t plane = (size_t)P->Ng * P->Ng * sizeof(float2);
    const size_t budget = c.grid_budget_bytes > 0 ? (size_t)c.grid_budget_bytes : (size_t)-1;
    const size_t per_chan = plane * P->planes;
    if (budget / per_chan >= (size_t)c.n_channels) {
        *gc = c.n_channels;
        *gk = P->planes;
    } else if (budget >= per_chan) {
        *gc = (int)(budget / per_chan);
        *gk = P->planes;
    } else {
        *gc = 1;
        size_t k = budget / plane;
        *gk = k < 1 ? 1 : (int)k;
    }
}

rick_status ensure_group_grid(rick_plan* P) {
    const rick_config& c = P->cfg;
    int gc, gk;
    plan_groups(P, &gc, &gk);
    const size_t need = (size_t)gc * gk * (size_t)P->Ng * P->Ng * sizeof(float2);
    if (need > P->grid_cap) {
        dfree(P->d_grid);
        P->grid_cap = 0;
        RK_CUDA(dmalloc(&P->d_grid, need));
        P->grid_cap = need;
    }
    return RICK_OK;
}

// The plane and channel groups of the binned visibilities, gridded,
// transformed and reduced into image_real (device).  host_out (optional):
// each channel group's images are copied to host_out on the plan's copy
// stream as soon as the group's last plane group is reduced, overlapped with
// the next group's gridding and transforms; the caller synchronises the copy
// stream.
rick_status image_groups_impl(rick_plan* P, float* image_real, float* image_complex, double* ws,
                              cudaStream_t st, float* host_out = nullptr) {
    const rick_config& c = P->cfg;
    int gc, gk;
    plan_groups(P, &gc, &gk);
    const size_t NN = (size_t)c.N * c.N;
    RK_TRY(ensure_group_grid(P));
    float* g = reinterpret_cast<float*>(P->d_grid);
    for (int c0 = 0; c0 < c.n_channels; c0 += gc) {
        const int c1 = c0 + gc < c.n_channels ? c0 + gc : c.n_channels;
        for (int k0 = 0; k0 < P->planes; k0 += gk) {
            const int k1 = k0 + gk < P->planes ? k0 + gk : P->planes;
            RK_TRY(grid_impl(P, c0, c1, k0, k1, g, st, P->own_fft));
            RK_TRY(fft_phase_impl(P, g, c0, c1, k0, k1, ws, image_real + (size_t)c0 * NN,
                                  image_complex ? image_complex + 2 * (size_t)c0 * NN : nullptr, st,
                                  RICK_GRIDDED_BY_PLAN));
        }
        if (host_out) {
            // the wait takes the event's latest record, so one event serves every group
            RK_CUDA(cudaEventRecord(P->chunk_done[0], st));
            RK_CUDA(cudaStreamWaitEvent(P->copy_stream, P->chunk_done[0], 0));
            RK_CUDA(cudaMemcpyAsync(host_out + (size_t)c0 * NN, image_real + (size_t)c0 * NN,
                                    (size_t)(c1 - c0) * NN * sizeof(float), cudaMemcpyDeviceToHost,
                                    P->copy_stream));
        }
    }
    return RICK_OK;
}

rick_status dirty_image_impl(rick_plan* P, const double* uvw, const double* chan_scale,
                             const float* vis, const float* weight, const uint8_t* flag,
                             int64_t nrow, float* image_real, float* image_complex,
                             double* weight_sum, int64_t* counts, cudaStream_t st) {
    RK_ARG(image_real != nullptr, "image_real is NULL");
    double* ws = weight_sum ? weight_sum : P->d_wsum;
    RK_TRY(bin_impl(P, uvw, chan_scale, vis, weight, flag, nrow, ws, counts, st));
    return image_groups_impl(P, image_real, image_complex, ws, st);
}

rick_status predict_impl(rick_plan* P, const double* uvw, const double* chan_scale,
                         const float* weight, const uint8_t* flag, int64_t nrow, const float* image,
                         float* vis_out, int64_t* counts, cudaStream_t st) {
    const rick_config& c = P->cfg;
    RK_ARG(image != nullptr && vis_out != nullptr, "image and vis_out are required");
    RK_TRY(bin_impl(P, uvw, chan_scale, nullptr, weight, flag, nrow, P->d_wsum, counts, st, true));
    if (nrow > 0)
        RK_CUDA(cudaMemsetAsync(vis_out, 0, sizeof(float2) * (size_t)nrow * c.n_channels, st));
    int gc, gk;
    plan_groups(P, &gc, &gk);
    const size_t NN = (size_t)c.N * c.N;
    RK_TRY(ensure_group_grid(P));
    float* g = reinterpret_cast<float*>(P->d_grid);
    for (int c0 = 0; c0 < c.n_channels; c0 += gc) {
        const int c1 = c0 + gc < c.n_channels ? c0 + gc : c.n_channels;
        for (int k0 = 0; k0 < P->planes; k0 += gk) {
            const int k1 = k0 + gk < P->planes ? k0 + gk : P->planes;
            if (P->own_fft && fft_fused_model_supported(P->Ng)) {   // fused model rows + pruned column pass
                RK_TRY(model_fft_impl(P, image + (size_t)c0 * NN, c0, c1, k0, k1, g, RICK_GRIDDED_BY_PLAN, st));
            } else {
                RK_TRY(model_impl(P, image + (size_t)c0 * NN, c0, c1, k0, k1, g, st));
                RK_TRY(fft_impl(P, g, (int64_t)(c1 - c0) * (k1 - k0), st, CUFFT_FORWARD));
            }
            RK_TRY(degrid_impl(P, g, c0, c1, k0, k1, vis_out, st));
        }
    }
    return RICK_OK;
}

}  // namespace

namespace rick {
// Lets other translation units of the library report a message through
// rick_last_error().
void set_error_message(const char* msg) { set_err("%s", msg); }
// The configuration check of rick_plan_create, for entry points without a plan.
rick_status validate_config(const rick_config* cfg) { return validate(cfg); }
}  // namespace rick

// ===========================================================================
// C ABI
// ===========================================================================

extern "C" {

rick_status rick_plan_create(const rick_config* cfg, rick_plan** out) {
    if (!out) {
        set_err("invalid argument: out is NULL");
        return RICK_ERR_INVALID_ARG;
    }
    *out = nullptr;
    RK_TRY(validate(cfg));
    rick_plan* P = new (std::nothrow) rick_plan();
    if (!P) {
        set_err("host allocation failed");
        return RICK_ERR_OOM;
    }
    rick_status s = plan_init(P, cfg);
    if (s != RICK_OK) {
        release(P);
        delete P;
        return s;
    }
    *out = P;
    return RICK_OK;
}

rick_status rick_plan_destroy(rick_plan* plan) {
    if (!plan) return RICK_OK;
    release(plan);
    delete plan;
    return RICK_OK;
}

rick_status rick_plan_reserve(rick_plan* plan, int64_t max_rows) {
    RK_ARG(plan != nullptr, "plan is NULL");
    RK_ARG(max_rows >= 0, "max_rows must be >= 0");
    const int64_t nvis = max_rows * (int64_t)plan->cfg.n_channels * plan->nrec_per_vis;
    RK_ARG(max_rows == 0 || nvis / max_rows == (int64_t)plan->cfg.n_channels * plan->nrec_per_vis,
           "overflow");
    if (nvis >= (int64_t)0xFFFFFFFFLL) {
        set_err("reservation exceeds 2^32 - 2 records");
        return RICK_ERR_UNSUPPORTED;
    }
    if (plan->cfg.weighting != RICK_WEIGHT_NATURAL)
        RK_TRY(ensure_weight_capacity(plan, max_rows * (int64_t)plan->cfg.n_channels));
    return ensure_vis_capacity(plan, nvis);
}

rick_status rick_plan_taper(const rick_plan* plan, double* taper_host) {
    RK_ARG(plan && taper_host, "plan and taper_host are required");
    std::memcpy(taper_host, plan->taper.data(), sizeof(double) * plan->cfg.N);
    return RICK_OK;
}

rick_status rick_set_kernel_table(rick_plan* plan, const float* taps, int32_t lattice, void* stream) {
    RK_ARG(plan && taps, "plan and taps are required");
    RK_ARG(plan->cfg.kernel_kind == RICK_KERNEL_TABLE, "plan does not use a table kernel");
    RK_ARG(lattice >= 1 && lattice <= 256, "lattice must be in [1, 256]");
    const size_t n = (size_t)plan->cfg.n_wplanes * (lattice + 1) * (lattice + 1) * 16;
    if (n >= ((size_t)1 << 31)) {
        set_err("kernel table of %zu floats exceeds the gridder's 32-bit table index", n);
        return RICK_ERR_UNSUPPORTED;
    }
    if (lattice != plan->lattice) {
        dfree(plan->d_table);
        plan->lattice = 0;
        RK_CUDA(dmalloc(&plan->d_table, n * sizeof(float)));
        plan->lattice = lattice;
    }
    RK_CUDA(cudaMemcpyAsync(plan->d_table, taps, n * sizeof(float), cudaMemcpyDeviceToDevice,
                            as_stream(stream)));
    return RICK_OK;
}

rick_status rick_bin(rick_plan* plan, const double* uvw, const double* chan_scale, const float* vis,
                     const float* weight, const uint8_t* flag, int64_t nrow, double* weight_sum,
                     int64_t* counts, void* stream) {
    RK_ARG(plan != nullptr, "plan is NULL");
    return bin_impl(plan, uvw, chan_scale, vis, weight, flag, nrow, weight_sum, counts,
                    as_stream(stream));
}

rick_status rick_grid_binned(rick_plan* plan, int32_t chan_begin, int32_t chan_end,
                             int32_t plane_begin, int32_t plane_end, float* grids, void* stream) {
    RK_ARG(plan != nullptr, "plan is NULL");
    return grid_impl(plan, chan_begin, chan_end, plane_begin, plane_end, grids, as_stream(stream));
}

rick_status rick_grid_binned_sparse(rick_plan* plan, int32_t chan_begin, int32_t chan_end,
                                    int32_t plane_begin, int32_t plane_end, float* grids, void* stream) {
    RK_ARG(plan != nullptr, "plan is NULL");
    if (!plan->own_fft) {
        set_err("sparse gridding is only read by the library's own transform (RICK_FFT_OWN, a mesh of 256 to 16384)");
        return RICK_ERR_UNSUPPORTED;
    }
    return grid_impl(plan, chan_begin, chan_end, plane_begin, plane_end, grids, as_stream(stream), true);
}

rick_status rick_grid(rick_plan* plan, const double* uvw, const double* chan_scale, const float* vis,
                      const float* weight, const uint8_t* flag, int64_t nrow, int32_t plane_begin,
                      int32_t plane_end, float* grids, double* weight_sum, int64_t* counts,
                      void* stream) {
    RK_ARG(plan != nullptr, "plan is NULL");
    RK_TRY(bin_impl(plan, uvw, chan_scale, vis, weight, flag, nrow, weight_sum, counts,
                    as_stream(stream)));
    return grid_impl(plan, 0, plan->cfg.n_channels, plane_begin, plane_end, grids,
                     as_stream(stream));
}

rick_status rick_imaging_weights(rick_plan* plan, const double* uvw, const double* chan_scale,
                                 const float* weight, const uint8_t* flag, int64_t nrow,
                                 float* weight_out, void* stream) {
    RK_ARG(plan != nullptr, "plan is NULL");
    const rick_config& c = plan->cfg;
    RK_ARG(nrow >= 0, "nrow must be >= 0");
    const int64_t nvis = nrow * (int64_t)c.n_channels;
    if (nvis == 0) return RICK_OK;
    RK_ARG(uvw && chan_scale && weight && weight_out, "uvw, chan_scale, weight and weight_out are required");
    cudaStream_t st = as_stream(stream);
    plan->last_stream = st;
    if (c.weighting == RICK_WEIGHT_NATURAL) {
        RK_CUDA(cudaMemcpyAsync(weight_out, weight, sizeof(float) * (size_t)nvis, cudaMemcpyDeviceToDevice, st));
        return RICK_OK;
    }
    int launches = 0;
    rick_status s = check_launch(
        launch_imaging_weights(place_params(plan, false), uvw, chan_scale, weight, flag, nvis,
                               c.weighting, c.robust, plan->d_density, plan->d_wmom, weight_out,
                               plan->num_sms, st, &launches),
        "imaging weight kernels");
    plan->launches += launches;
    return s;
}

rick_status rick_fft_wplanes(rick_plan* plan, float* grids, int64_t n_planes, void* stream) {
    RK_ARG(plan != nullptr, "plan is NULL");
    return fft_impl(plan, grids, n_planes, as_stream(stream));
}

rick_status rick_phase_correct_reduce(rick_plan* plan, const float* grids, int32_t chan_begin,
                                      int32_t chan_end, int32_t plane_begin, int32_t plane_end,
                                      const double* weight_sum, float* image_real,
                                      float* image_complex, void* stream) {
    RK_ARG(plan != nullptr, "plan is NULL");
    return phase_impl(plan, grids, chan_begin, chan_end, plane_begin, plane_end, weight_sum,
                      image_real, image_complex, as_stream(stream));
}

rick_status rick_fft_phase_correct_reduce(rick_plan* plan, float* grids, int32_t chan_begin,
                                          int32_t chan_end, int32_t plane_begin, int32_t plane_end,
                                          const double* weight_sum, float* image_real,
                                          float* image_complex, int32_t flags, void* stream) {
    RK_ARG(plan != nullptr, "plan is NULL");
    return fft_phase_impl(plan, grids, chan_begin, chan_end, plane_begin, plane_end, weight_sum,
                          image_real, image_complex, as_stream(stream), flags);
}

rick_status rick_fft_wplanes_columns(rick_plan* plan, float* grids, int32_t chan_begin, int32_t chan_end,
                                     int32_t plane_begin, int32_t plane_end, int32_t flags, void* stream) {
    RK_ARG(plan != nullptr, "plan is NULL");
    return columns_impl(plan, grids, chan_begin, chan_end, plane_begin, plane_end, flags, as_stream(stream));
}

rick_status rick_rows_phase_correct_reduce(rick_plan* plan, const float* grids, int32_t chan_begin,
                                           int32_t chan_end, int32_t plane_begin, int32_t plane_end,
                                           const double* weight_sum, float* image_real,
                                           float* image_complex, int32_t flags, void* stream) {
    RK_ARG(plan != nullptr, "plan is NULL");
    return rows_phase_impl(plan, grids, chan_begin, chan_end, plane_begin, plane_end, weight_sum,
                           image_real, image_complex, flags, as_stream(stream));
}

rick_status rick_dirty_image(rick_plan* plan, const double* uvw, const double* chan_scale,
                             const float* vis, const float* weight, const uint8_t* flag,
                             int64_t nrow, float* image_real, float* image_complex,
                             double* weight_sum, int64_t* counts, void* stream) {
    RK_ARG(plan != nullptr, "plan is NULL");
    return dirty_image_impl(plan, uvw, chan_scale, vis, weight, flag, nrow, image_real,
                            image_complex, weight_sum, counts, as_stream(stream));
}

rick_status rick_dirty_image_host(rick_plan* plan, const double* uvw, const double* chan_scale,
                                  const float* vis, const float* weight, const uint8_t* flag,
                                  int64_t nrow, float* image_real, double* weight_sum,
                                  int64_t* counts, void* stream) {
    RK_ARG(plan != nullptr, "plan is NULL");
    RK_ARG(nrow >= 0 && image_real != nullptr, "nrow >= 0 and image_real are required");
    const rick_config& c = plan->cfg;
    const size_t C = (size_t)c.n_channels, R = (size_t)nrow;
    auto up = [](size_t x) { return (x + 255) & ~(size_t)255; };
    const size_t b_uvw = up(R * 3 * sizeof(double)), b_sc = up(C * sizeof(double));
    const size_t b_vis = up(R * C * 2 * sizeof(float)), b_w = up(R * C * sizeof(float));
    const size_t b_f = flag ? up(R * C) : 0, b_ws = up(C * sizeof(double)), b_cnt = 256;
    const size_t need = b_uvw + b_sc + b_vis + b_w + b_f + b_ws + b_cnt;
    if (need > plan->in_cap) {
        dfree(plan->d_in);
        plan->in_cap = 0;
        RK_CUDA(dmalloc(&plan->d_in, need));
        plan->in_cap = need;
    }
    const size_t NN = (size_t)c.N * c.N, img_bytes = C * NN * sizeof(float);
    if (img_bytes > plan->img_cap) {
        dfree(plan->d_img);
        plan->img_cap = 0;
        RK_CUDA(dmalloc(&plan->d_img, img_bytes));
        plan->img_cap = img_bytes;
    }
    unsigned char* b = plan->d_in;
    double* d_uvw = reinterpret_cast<double*>(b);
    double* d_sc = reinterpret_cast<double*>(b + b_uvw);
    float* d_vis = reinterpret_cast<float*>(b + b_uvw + b_sc);
    float* d_w = reinterpret_cast<float*>(b + b_uvw + b_sc + b_vis);
    uint8_t* d_f = flag ? b + b_uvw + b_sc + b_vis + b_w : nullptr;
    double* d_ws = reinterpret_cast<double*>(b + b_uvw + b_sc + b_vis + b_w + b_f);
    int64_t* d_cnt = reinterpret_cast<int64_t*>(b + b_uvw + b_sc + b_vis + b_w + b_f + b_ws);
    cudaStream_t st = as_stream(stream);
    int gc, gk;
    plan_groups(plan, &gc, &gk);
    const bool whole = gc == c.n_channels && gk == plan->planes && c.n_channels > 1;
    // upload overlapped with placement: natural weighting (the other weightings
    // need every visibility's density before any placement)
    const bool overlap_in = R > 0 && c.weighting == RICK_WEIGHT_NATURAL;
    if (R) RK_ARG(uvw && chan_scale && vis && weight, "uvw, chan_scale, vis and weight are required");
    if (R && !overlap_in) {
        RK_CUDA(cudaMemcpyAsync(d_uvw, uvw, R * 3 * sizeof(double), cudaMemcpyHostToDevice, st));
        RK_CUDA(cudaMemcpyAsync(d_vis, vis, R * C * 2 * sizeof(float), cudaMemcpyHostToDevice, st));
        RK_CUDA(cudaMemcpyAsync(d_w, weight, R * C * sizeof(float), cudaMemcpyHostToDevice, st));
        if (flag) RK_CUDA(cudaMemcpyAsync(d_f, flag, R * C, cudaMemcpyHostToDevice, st));
    }
    if (chan_scale && !overlap_in)
        RK_CUDA(cudaMemcpyAsync(d_sc, chan_scale, C * sizeof(double), cudaMemcpyHostToDevice, st));
    RK_CUDA(cudaMemsetAsync(plan->d_img, 0, img_bytes, st));
    if (whole) {
        // the whole grid fits: grid every channel, then transform and reduce in
        // channel chunks, each chunk's images downloaded on the copy stream
        // while the next chunk is transformed
        if (!plan->copy_stream) RK_CUDA(cudaStreamCreateWithFlags(&plan->copy_stream, cudaStreamNonBlocking));
        for (auto& ev : plan->chunk_done)
            if (!ev) RK_CUDA(cudaEventCreateWithFlags(&ev, cudaEventDisableTiming));
        if (overlap_in)
            RK_TRY(bin_from_host(plan, uvw, chan_scale, vis, weight, flag, nrow, d_uvw, d_sc, d_vis, d_w, d_f,
                                 d_ws, d_cnt, st));
        else
            RK_TRY(bin_impl(plan, d_uvw, d_sc, d_vis, d_w, d_f, nrow, d_ws, d_cnt, st));
        RK_TRY(ensure_group_grid(plan));
        float* g = reinterpret_cast<float*>(plan->d_grid);
        RK_TRY(grid_impl(plan, 0, c.n_channels, 0, plan->planes, g, st, plan->own_fft));
        const int nch = c.n_channels < kHostChunks ? c.n_channels : kHostChunks;
        const size_t plane_floats = 2 * (size_t)plan->Ng * plan->Ng;
        for (int i = 0; i < nch; ++i) {
            const int c0 = (int)((int64_t)c.n_channels * i / nch), c1 = (int)((int64_t)c.n_channels * (i + 1) / nch);
            float* gi = g + (size_t)c0 * plan->planes * plane_floats;
            RK_TRY(fft_phase_impl(plan, gi, c0, c1, 0, plan->planes, d_ws, plan->d_img + (size_t)c0 * NN,
                                  nullptr, st, RICK_GRIDDED_BY_PLAN));
            RK_CUDA(cudaEventRecord(plan->chunk_done[i], st));
            RK_CUDA(cudaStreamWaitEvent(plan->copy_stream, plan->chunk_done[i], 0));
            RK_CUDA(cudaMemcpyAsync(image_real + (size_t)c0 * NN, plan->d_img + (size_t)c0 * NN,
                                    (size_t)(c1 - c0) * NN * sizeof(float), cudaMemcpyDeviceToHost,
                                    plan->copy_stream));
        }
        RK_CUDA(cudaStreamSynchronize(plan->copy_stream));
    } else {
        // streamed groups: each channel group's images go to the host while the
        // next group is gridded and transformed
        if (!plan->copy_stream) RK_CUDA(cudaStreamCreateWithFlags(&plan->copy_stream, cudaStreamNonBlocking));
        if (!plan->chunk_done[0]) RK_CUDA(cudaEventCreateWithFlags(&plan->chunk_done[0], cudaEventDisableTiming));
        rick_status s = overlap_in ? bin_from_host(plan, uvw, chan_scale, vis, weight, flag, nrow, d_uvw, d_sc,
                                                   d_vis, d_w, d_f, d_ws, d_cnt, st)
                                   : bin_impl(plan, d_uvw, d_sc, d_vis, d_w, d_f, nrow, d_ws, d_cnt, st);
        if (s == RICK_OK) s = image_groups_impl(plan, plan->d_img, nullptr, d_ws, st, image_real);
        RK_CUDA(cudaStreamSynchronize(plan->copy_stream));   // also after a failure: no copy left in flight
        RK_TRY(s);
    }
    if (weight_sum)
        RK_CUDA(cudaMemcpyAsync(weight_sum, d_ws, C * sizeof(double), cudaMemcpyDeviceToHost, st));
    if (counts)
        RK_CUDA(cudaMemcpyAsync(counts, d_cnt, 2 * sizeof(int64_t), cudaMemcpyDeviceToHost, st));
    RK_CUDA(cudaStreamSynchronize(st));
    return RICK_OK;
}

rick_status rick_plan_sync_status(rick_plan* plan) {
    RK_ARG(plan != nullptr, "plan is NULL");
    RK_CUDA(cudaStreamSynchronize(plan->last_stream));
    int st = 0;
    RK_CUDA(cudaMemcpy(&st, plan->d_status, sizeof(int), cudaMemcpyDeviceToHost));
    if (st != 0) {
        set_err("device-side check failed (code %d: %s)", st,
                st == kCheckGridItem ? "a gridder work item beyond the launch's tiles"
                : st == kCheckRecordCell ? "a record's first footprint cell outside its tile"
                                         : "unknown");
        RK_CUDA(cudaMemset(plan->d_status, 0, sizeof(int)));   // reported once
        return RICK_ERR_INTERNAL;
    }
    return RICK_OK;
}

int64_t rick_plan_launch_count(const rick_plan* plan) { return plan ? plan->launches : -1; }

rick_status rick_debug_inject(int32_t site, int32_t countdown) {
    RK_ARG(site >= RICK_INJECT_NONE && site <= RICK_INJECT_LAUNCH, "unknown injection site");
    RK_ARG(countdown >= 0, "countdown must be >= 0");
    inject_init();   // reads RICK_INJECT once, so that it cannot override this call
    g_inject_site.store(0);
    if (site != RICK_INJECT_NONE && countdown > 0) {
        g_inject_left.store(countdown);
        g_inject_site.store(site);
    }
    return RICK_OK;
}

int32_t rick_debug_build(void) {
#ifdef RICK_DEBUG
    return 1;
#else
    return 0;
#endif
}

rick_status rick_debug_poke_record(rick_plan* plan, int64_t index, int32_t cell_x, int32_t cell_y) {
#ifdef RICK_DEBUG
    RK_ARG(plan != nullptr, "plan is NULL");
    RK_ARG(plan->binned && !plan->binned_for_predict, "nothing binned for gridding");
    RK_ARG(cell_x >= 0 && cell_x < 256 && cell_y >= 0 && cell_y < 256, "cells are 8-bit fields");
    RK_CUDA(cudaStreamSynchronize(plan->last_stream));
    uint32_t total = 0;
    RK_CUDA(cudaMemcpy(&total, plan->d_offsets + plan->nkeys, sizeof(uint32_t), cudaMemcpyDeviceToHost));
    RK_ARG(index >= 0 && index < (int64_t)total, "record index out of range");
    VisRecord r;
    RK_CUDA(cudaMemcpy(&r, plan->d_records + index, sizeof r, cudaMemcpyDeviceToHost));
    r.px = (r.px & kFracMask) | ((uint32_t)cell_x << kFracBits);
    r.py = (r.py & kFracMask) | ((uint32_t)cell_y << kFracBits);
    RK_CUDA(cudaMemcpy(plan->d_records + index, &r, sizeof r, cudaMemcpyHostToDevice));
    return RICK_OK;
#else
    (void)plan;
    (void)index;
    (void)cell_x;
    (void)cell_y;
    set_err("rick_debug_poke_record exists only in RICK_DEBUG builds");
    return RICK_ERR_UNSUPPORTED;
#endif
}

int32_t rick_plan_fft_impl(const rick_plan* plan) {
    return plan ? (plan->own_fft ? RICK_FFT_OWN : RICK_FFT_CUFFT) : -1;
}

rick_status rick_plan_schedule_counts(rick_plan* plan, uint32_t counts[3]) {
    RK_ARG(plan && counts, "plan and counts are required");
    RK_ARG(plan->binned && !plan->binned_for_predict, "nothing gridded yet");
    RK_CUDA(cudaStreamSynchronize(plan->last_stream));
    // the gridder's counter words 1..3 hold the list lengths
    RK_CUDA(cudaMemcpy(counts, plan->d_counter + 1, 3 * sizeof(uint32_t), cudaMemcpyDeviceToHost));
    return RICK_OK;
}

rick_status rick_plan_bins(rick_plan* plan, int64_t* n_keys, int64_t* n_records, uint32_t* offsets,
                           uint32_t* records) {
    RK_ARG(plan && n_keys && n_records, "plan, n_keys and n_records are required");
    RK_ARG(plan->binned, "nothing binned yet");
    RK_CUDA(cudaStreamSynchronize(plan->last_stream));
    uint32_t total = 0;
    RK_CUDA(cudaMemcpy(&total, plan->d_offsets + plan->nkeys, sizeof(uint32_t), cudaMemcpyDeviceToHost));
    *n_keys = (int64_t)plan->nkeys;
    *n_records = total;
    if (offsets)
        RK_CUDA(cudaMemcpy(offsets, plan->d_offsets, sizeof(uint32_t) * (plan->nkeys + 1),
                           cudaMemcpyDeviceToHost));
    if (records && total)
        RK_CUDA(cudaMemcpy(records, plan->d_records, sizeof(VisRecord) * total, cudaMemcpyDeviceToHost));
    return RICK_OK;
}

struct rick_graph {
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    rick_plan* plan = nullptr;
    int64_t kernels = 0;  // this library's kernels per launch
};

rick_status rick_graph_capture(rick_plan* plan, const double* uvw, const double* chan_scale,
                               const float* vis, const float* weight, const uint8_t* flag,
                               int64_t nrow, float* grids, double* weight_sum, float* image_real,
                               int64_t* counts, rick_graph** out) {
    RK_ARG(plan && out && weight_sum && image_real, "plan, out, weight_sum and image_real are required");
    *out = nullptr;
    const rick_config& c = plan->cfg;
    const int64_t nvis = nrow * (int64_t)c.n_channels * plan->nrec_per_vis;
    RK_ARG(nrow >= 0, "nrow must be >= 0");
    if (nvis > plan->cap_vis) {
        set_err("graph capture: the plan is reserved for %lld records, %lld requested; call "
                "rick_plan_reserve first (nothing may allocate during capture)",
                (long long)plan->cap_vis, (long long)nvis);
        return RICK_ERR_CAPACITY;
    }
    if (!grids) RK_TRY(ensure_group_grid(plan));  // nothing may allocate during capture
    cudaStream_t st = nullptr;
    RK_CUDA(cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking));
    cudaError_t e = cudaStreamBeginCapture(st, cudaStreamCaptureModeThreadLocal);
    if (e != cudaSuccess) {
        cudaStreamDestroy(st);
        set_err("cudaStreamBeginCapture: %s", cudaGetErrorString(e));
        return RICK_ERR_CUDA;
    }
    const size_t NN = (size_t)c.N * c.N;
    const int64_t launches_before = plan->launches;
    rick_status s = RICK_OK;
    if (cudaMemsetAsync(image_real, 0, sizeof(float) * NN * c.n_channels, st) != cudaSuccess) {
        set_err("cudaMemsetAsync of the image during capture failed");
        s = RICK_ERR_CUDA;
    }
    if (grids) {
        if (s == RICK_OK) s = bin_impl(plan, uvw, chan_scale, vis, weight, flag, nrow, weight_sum, counts, st);
        if (s == RICK_OK) s = grid_impl(plan, 0, c.n_channels, 0, plan->planes, grids, st);
        if (s == RICK_OK)
            s = fft_phase_impl(plan, grids, 0, c.n_channels, 0, plan->planes, weight_sum, image_real,
                               nullptr, st, RICK_GRIDDED_BY_PLAN);
    } else if (s == RICK_OK) {
        s = dirty_image_impl(plan, uvw, chan_scale, vis, weight, flag, nrow, image_real, nullptr,
                             weight_sum, counts, st);
    }
    cudaGraph_t g = nullptr;
    e = cudaStreamEndCapture(st, &g);
    cudaStreamDestroy(st);
    if (s != RICK_OK) {
        if (g) cudaGraphDestroy(g);
        return s;
    }
    if (e != cudaSuccess || !g) {
        if (g) cudaGraphDestroy(g);
        set_err("cudaStreamEndCapture: %s", cudaGetErrorString(e));
        return RICK_ERR_CUDA;
    }
    rick_graph* G = new (std::nothrow) rick_graph();
    if (!G) {
        cudaGraphDestroy(g);
        set_err("host allocation failed");
        return RICK_ERR_OOM;
    }
    G->graph = g;
    G->plan = plan;
    G->kernels = plan->launches - launches_before;
    plan->launches = launches_before;  // capturing launches nothing
    e = cudaGraphInstantiate(&G->exec, g, 0);
    if (e != cudaSuccess) {
        cudaGraphDestroy(g);
        delete G;
        set_err("cudaGraphInstantiate: %s", cudaGetErrorString(e));
        return RICK_ERR_CUDA;
    }
    *out = G;
    return RICK_OK;
}

rick_status rick_graph_launch(rick_graph* graph, void* stream) {
    RK_ARG(graph != nullptr, "graph is NULL");
    RK_CUDA(cudaGraphLaunch(graph->exec, as_stream(stream)));
    graph->plan->last_stream = as_stream(stream);
    graph->plan->launches += graph->kernels;
    return RICK_OK;
}

rick_status rick_graph_destroy(rick_graph* graph) {
    if (!graph) return RICK_OK;
    if (graph->exec) cudaGraphExecDestroy(graph->exec);
    if (graph->graph) cudaGraphDestroy(graph->graph);
    delete graph;
    return RICK_OK;
}

rick_status rick_autotune(const rick_config* base, const double* uvw, const double* chan_scale,
                          const float* vis, const float* weight, const uint8_t* flag,
                          int64_t nrow, int32_t chan_begin, int32_t chan_end,
                          int32_t plane_begin, int32_t plane_end, float* grids, int32_t reps,
                          rick_tune_entry* results, int32_t max_results, int32_t* n_results,
                          rick_config* best) {
    RK_TRY(validate(base));
    RK_ARG(n_results && best && grids, "n_results, best and grids are required");
    RK_ARG(reps >= 1 && reps <= 100, "reps must be in [1, 100]");
    RK_ARG(0 <= chan_begin && chan_begin < chan_end && chan_end <= base->n_channels, "channel range");
    RK_ARG(0 <= plane_begin && plane_begin < plane_end && plane_end <= stored_planes(*base),
           "plane range");
    *n_results = 0;
    *best = *base;
    float best_ms = 1e30f;
    const int tiles[3] = {16, 32, 64};
    const int threads[3] = {128, 256, 512};
    const int grabs[3] = {1, 4, 8};
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    RK_CUDA(cudaEventCreate(&e0));
    RK_CUDA(cudaEventCreate(&e1));
    rick_status result = RICK_OK;
    double* wsum = nullptr;
    if (cudaMalloc(&wsum, sizeof(double) * base->n_channels) != cudaSuccess) {
        cudaEventDestroy(e0);
        cudaEventDestroy(e1);
        set_err("autotune: allocation failed");
        return RICK_ERR_OOM;
    }
    for (int ti = 0; ti < 3 && result == RICK_OK; ++ti) {
        rick_config cfg = *base;
        cfg.tile = tiles[ti];
        if (cfg.tile > cfg.N || cfg.support > cfg.tile) continue;
        if (validate(&cfg) != RICK_OK) continue;  // e.g. bin space too large for this tile
        rick_plan* P = nullptr;
        result = rick_plan_create(&cfg, &P);
        if (result != RICK_OK) break;
        result = bin_impl(P, uvw, chan_scale, vis, weight, flag, nrow, wsum, nullptr, nullptr);
        for (int hi = 0; hi < 3 && result == RICK_OK; ++hi) {
            for (int gi = 0; gi < 3 && result == RICK_OK; ++gi) {
                {
                    rick_config shape = cfg;
                    shape.grid_threads = threads[hi];
                    if (validate(&shape) != RICK_OK) continue;  // too much shared memory
                }
                P->threads = threads[hi];
                P->grab = grabs[gi];
                std::vector<float> ms;
                for (int r = 0; r <= reps && result == RICK_OK; ++r) {
                    cudaEventRecord(e0, nullptr);
                    result = grid_impl(P, chan_begin, chan_end, plane_begin, plane_end, grids, nullptr);
                    cudaEventRecord(e1, nullptr);
                    if (cudaEventSynchronize(e1) != cudaSuccess) {
                        set_err("autotune: a timed launch failed");
                        result = RICK_ERR_CUDA;
                    }
                    float t = 0.f;
                    cudaEventElapsedTime(&t, e0, e1);
                    if (r > 0) ms.push_back(t);  // the first launch is the warm-up
                }
                if (result != RICK_OK) break;
                std::sort(ms.begin(), ms.end());
                const float med = ms[ms.size() / 2];
                if (results && *n_results < max_results)
                    results[*n_results] = rick_tune_entry{tiles[ti], threads[hi], grabs[gi], med};
                ++*n_results;
                if (med < best_ms) {
                    best_ms = med;
                    best->tile = tiles[ti];
                    best->grid_threads = threads[hi];
                    best->tiles_per_grab = grabs[gi];
                }
            }
        }
        rick_plan_destroy(P);
    }
    cudaFree(wsum);
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    return result;
}

rick_status rick_bin_predict(rick_plan* plan, const double* uvw, const double* chan_scale,
                             const float* weight, const uint8_t* flag, int64_t nrow, int64_t* counts,
                             void* stream) {
    RK_ARG(plan != nullptr, "plan is NULL");
    if (plan->cfg.kernel_kind == RICK_KERNEL_TABLE) {
        set_err("prediction supports the Gaussian and Kaiser-Bessel kernels");
        return RICK_ERR_UNSUPPORTED;
    }
    return bin_impl(plan, uvw, chan_scale, nullptr, weight, flag, nrow, plan->d_wsum, counts,
                    as_stream(stream), true);
}

rick_status rick_model_to_wplanes(rick_plan* plan, const float* image_real, int32_t chan_begin,
                                  int32_t chan_end, int32_t plane_begin, int32_t plane_end,
                                  float* grids, void* stream) {
    RK_ARG(plan != nullptr, "plan is NULL");
    return model_impl(plan, image_real, chan_begin, chan_end, plane_begin, plane_end, grids,
                      as_stream(stream));
}

rick_status rick_model_fft_wplanes(rick_plan* plan, const float* image_real, int32_t chan_begin,
                                   int32_t chan_end, int32_t plane_begin, int32_t plane_end, float* grids,
                                   int32_t flags, void* stream) {
    RK_ARG(plan != nullptr, "plan is NULL");
    return model_fft_impl(plan, image_real, chan_begin, chan_end, plane_begin, plane_end, grids, flags,
                          as_stream(stream));
}

rick_status rick_fft_wplanes_forward(rick_plan* plan, float* grids, int64_t n_planes, void* stream) {
    RK_ARG(plan != nullptr, "plan is NULL");
    return fft_impl(plan, grids, n_planes, as_stream(stream), CUFFT_FORWARD);
}

rick_status rick_degrid_binned(rick_plan* plan, const float* grids, int32_t chan_begin,
                               int32_t chan_end, int32_t plane_begin, int32_t plane_end,
                               float* vis_out, void* stream) {
    RK_ARG(plan != nullptr, "plan is NULL");
    return degrid_impl(plan, grids, chan_begin, chan_end, plane_begin, plane_end, vis_out,
                       as_stream(stream));
}

rick_status rick_predict(rick_plan* plan, const double* uvw, const double* chan_scale,
                         const float* weight, const uint8_t* flag, int64_t nrow,
                         const float* image_real, float* vis_out, int64_t* counts, void* stream) {
    RK_ARG(plan != nullptr, "plan is NULL");
    if (plan->cfg.kernel_kind == RICK_KERNEL_TABLE) {
        set_err("prediction supports the Gaussian and Kaiser-Bessel kernels");
        return RICK_ERR_UNSUPPORTED;
    }
    return predict_impl(plan, uvw, chan_scale, weight, flag, nrow, image_real, vis_out, counts,
                        as_stream(stream));
}

const char* rick_status_string(rick_status s) {
    switch (s) {
        case RICK_OK: return "RICK_OK";
        case RICK_ERR_INVALID_ARG: return "RICK_ERR_INVALID_ARG";
        case RICK_ERR_OOM: return "RICK_ERR_OOM";
        case RICK_ERR_CUDA: return "RICK_ERR_CUDA";
        case RICK_ERR_CUFFT: return "RICK_ERR_CUFFT";
        case RICK_ERR_TIMEOUT: return "RICK_ERR_TIMEOUT";
        case RICK_ERR_UNSUPPORTED: return "RICK_ERR_UNSUPPORTED";
        case RICK_ERR_INTERNAL: return "RICK_ERR_INTERNAL";
        case RICK_ERR_CAPACITY: return "RICK_ERR_CAPACITY";
    }
    return "unknown rick_status";
}

const char* rick_last_error(void) { return g_err; }

int32_t rick_stored_planes(const rick_config* cfg) { return cfg ? stored_planes(*cfg) : -1; }

}  // extern "C"

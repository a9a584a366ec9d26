// rick_noalloc.cu -- rick_grid_noalloc: binning + gridding with no device
// allocation at all.
//
// Who needs this: code that must not call cudaMalloc/cudaFree once it is
// running.  Examples are a real-time pipeline (a correlator or beamformer back
// end) that sizes all device memory at start-up and may not stall on the
// allocator while data streams in, and host frameworks that own the device's
// memory budget through their own pool, where a library that allocates behind
// their back breaks the accounting.  rick_grid needs a plan, and creating a
// plan allocates tables, scratch and cuFFT work areas; this entry point takes
// the configuration directly and keeps its scratch in one fixed array in device
// memory.
//
// The array is kNoallocScratchBytes (32 MiB).  CUDA loads a library's device
// code lazily by default: the array and the kernels this call runs are loaded,
// and take device memory, on the first call on each device (the address lookup
// below loads the array's module; the first launch of each kernel loads that
// kernel).  After that first call -- make it at start-up, outside any stream
// capture, with the support and tile size that later calls use -- calls
// allocate nothing, and the array stays until the process exits.  A call whose
// binning scratch does not fit (roughly 40 bytes per visibility plus 8 bytes
// per bin) is rejected with RICK_ERR_CAPACITY, and every other refusal is made
// too, before anything is launched.  All calls share the array: each call
// clears what must start at zero, and calls whose work overlaps on the GPU
// (different streams, or different host threads) race on it -- serialise them.
#include <cmath>
#include <cstdio>
#include <cstring>
#include <mutex>

#include "rick_internal.cuh"

namespace rick {
void set_error_message(const char* msg);
}

using namespace rick;

namespace {

constexpr size_t kNoallocScratchBytes = size_t(32) << 20;
constexpr int kMaxDevices = 64;

// The scratch itself.  In host code this name only stands in for the symbol;
// its device address comes from cudaGetSymbolAddress below.
static __device__ __align__(256) unsigned char rick_noalloc_scratch[kNoallocScratchBytes];

std::mutex g_mutex;
void* g_scratch_addr[kMaxDevices] = {};

rick_status fail(rick_status s, const char* msg) {
    set_error_message(msg);
    return s;
}

// Device address of the scratch on the current device, looked up once per
// device (the first call on a device does this; make it before any capture).
rick_status scratch_address(unsigned char** out) {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return fail(RICK_ERR_CUDA, "rick_grid_noalloc: cudaGetDevice failed");
    if (dev < 0 || dev >= kMaxDevices)
        return fail(RICK_ERR_UNSUPPORTED, "rick_grid_noalloc: device ordinal out of range");
    std::lock_guard<std::mutex> lock(g_mutex);
    if (!g_scratch_addr[dev]) {
        void* p = nullptr;
        e = cudaGetSymbolAddress(&p, rick_noalloc_scratch);
        if (e == cudaErrorMemoryAllocation)   // loading the array's module needs its 32 MiB
            return fail(RICK_ERR_OOM,
                        "rick_grid_noalloc: no device memory left to load the 32 MiB scratch on its first "
                        "call on this device; make the first call at start-up");
        if (e != cudaSuccess || p == nullptr)
            return fail(RICK_ERR_CUDA, "rick_grid_noalloc: cudaGetSymbolAddress of the scratch failed");
        g_scratch_addr[dev] = p;
    }
    *out = static_cast<unsigned char*>(g_scratch_addr[dev]);
    return RICK_OK;
}

size_t up256(size_t x) { return (x + 255) & ~size_t(255); }

}  // namespace

extern "C" rick_status rick_grid_noalloc(const rick_config* cfg, const double* uvw,
                                         const double* chan_scale, const float* vis,
                                         const float* weight, const uint8_t* flag, int64_t nrow,
                                         int32_t plane_begin, int32_t plane_end, float* grids,
                                         double* weight_sum, int64_t* counts, void* stream) {
    if (!cfg) return fail(RICK_ERR_INVALID_ARG, "invalid argument: cfg is NULL");
    // the same configuration check as rick_plan_create, then what needs a plan
    const rick_status valid = validate_config(cfg);
    if (valid != RICK_OK) return valid;
    const rick_config& c = *cfg;
    const int T = c.tile ? c.tile : 32;
    const int threads = c.grid_threads ? c.grid_threads : 128;
    const int planes = rick_stored_planes(cfg);
    if (c.kernel_kind != RICK_KERNEL_GAUSS && c.kernel_kind != RICK_KERNEL_KAISER_BESSEL)
        return fail(RICK_ERR_UNSUPPORTED,
                    "rick_grid_noalloc: only Gaussian and Kaiser-Bessel kernels (a table kernel needs a plan)");
    if (c.grid_size != 0 && c.grid_size != c.N)
        return fail(RICK_ERR_UNSUPPORTED, "rick_grid_noalloc: a padded grid (grid_size != N) needs a plan");
    if (c.weighting != RICK_WEIGHT_NATURAL)
        return fail(RICK_ERR_UNSUPPORTED,
                    "rick_grid_noalloc: uniform or Briggs weighting needs a plan (a density grid)");
    if (c.w_support >= 2)
        return fail(RICK_ERR_UNSUPPORTED,
                    "rick_grid_noalloc: a w-kernel (w_support >= 2) needs a plan (Sw records per visibility)");
    if (nrow < 0 || !weight_sum || !grids || (nrow > 0 && !(uvw && chan_scale && vis && weight)))
        return fail(RICK_ERR_INVALID_ARG, "invalid argument: inputs");
    if (!(0 <= plane_begin && plane_begin < plane_end && plane_end <= planes))
        return fail(RICK_ERR_INVALID_ARG, "invalid argument: plane range");
    if (((uintptr_t)grids & 15u) != 0)
        return fail(RICK_ERR_INVALID_ARG, "invalid argument: grids must be 16-byte aligned");

    // sizes, each product tested before it is formed (validate_config bounds
    // the bins below 2^32)
    const int NT = c.N / T;
    const uint64_t nkeys = (uint64_t)c.n_channels * planes * (uint64_t)NT * NT * 4ull;
    const uint64_t limit = 0xFFFFFFFFull;
    const bool vis_fit = (uint64_t)nrow < limit / (uint64_t)c.n_channels;
    const uint64_t nvis = vis_fit ? (uint64_t)nrow * (uint64_t)c.n_channels : limit;
    const uint64_t items = (uint64_t)c.n_channels * (plane_end - plane_begin) * (uint64_t)NT * NT;
    // scratch layout: hist, offsets, scan partials, key, rank, stage, records, counter, counts
    const size_t b_hist = up256(nkeys * 4), b_off = up256((nkeys + 1) * 4);
    const size_t b_part = up256(scan_partials_needed(nkeys) * 4);
    const size_t b_key = up256(nvis * 4), b_rec = up256(nvis * sizeof(VisRecord));
    const size_t need = b_hist + b_off + b_part + 2 * b_key + 2 * b_rec + 256 + 256;
    if (!vis_fit || nkeys >= limit || items >= limit || need > kNoallocScratchBytes) {
        char msg[256];
        snprintf(msg, sizeof msg,
                 "rick_grid_noalloc: needs %llu bytes of scratch (%lld rows x %d channels, %llu bins); "
                 "the fixed scratch holds %llu bytes -- use rick_grid with a plan",
                 vis_fit ? (unsigned long long)need : ~0ull, (long long)nrow, c.n_channels,
                 (unsigned long long)nkeys, (unsigned long long)kNoallocScratchBytes);
        return fail(RICK_ERR_CAPACITY, msg);
    }

    GridParams G;
    std::memset(&G, 0, sizeof G);
    if (!(fit_tap_polynomials(c.kernel_kind, c.kernel_param, c.support, G) <= 1e-6))
        return fail(RICK_ERR_UNSUPPORTED, "rick_grid_noalloc: kernel too narrow for its support");

    unsigned char* base = nullptr;
    rick_status s = scratch_address(&base);
    if (s != RICK_OK) return s;
    uint32_t* hist = reinterpret_cast<uint32_t*>(base);
    uint32_t* offsets = reinterpret_cast<uint32_t*>(base + b_hist);
    uint32_t* partials = reinterpret_cast<uint32_t*>(base + b_hist + b_off);
    uint32_t* key = reinterpret_cast<uint32_t*>(base + b_hist + b_off + b_part);
    uint32_t* rank = reinterpret_cast<uint32_t*>(base + b_hist + b_off + b_part + b_key);
    VisRecord* stage = reinterpret_cast<VisRecord*>(base + b_hist + b_off + b_part + 2 * b_key);
    VisRecord* records = reinterpret_cast<VisRecord*>(base + b_hist + b_off + b_part + 2 * b_key + b_rec);
    uint32_t* counter = reinterpret_cast<uint32_t*>(base + b_hist + b_off + b_part + 2 * b_key + 2 * b_rec);
    unsigned long long* cnt = reinterpret_cast<unsigned long long*>(
        base + b_hist + b_off + b_part + 2 * b_key + 2 * b_rec + 256);

    cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
    int dev = 0, num_sms = 0;
    if (cudaGetDevice(&dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&num_sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
        return fail(RICK_ERR_CUDA, "rick_grid_noalloc: device query failed");

    // the array keeps the previous call's contents: clear what must start at zero
    if (cudaMemsetAsync(hist, 0, nkeys * 4, st) != cudaSuccess ||
        cudaMemsetAsync(cnt, 0, 2 * sizeof(unsigned long long), st) != cudaSuccess ||
        cudaMemsetAsync(counter, 0, 8 * sizeof(uint32_t), st) != cudaSuccess ||
        cudaMemsetAsync(weight_sum, 0, sizeof(double) * c.n_channels, st) != cudaSuccess)
        return fail(RICK_ERR_CUDA, "rick_grid_noalloc: cudaMemsetAsync failed");

    PlaceParams pp;
    pp.N = c.N;
    pp.S = c.support;
    pp.Nw = c.n_wplanes;
    pp.C = c.n_channels;
    pp.T = T;
    pp.NT = NT;
    pp.precision = c.precision;
    pp.fold = c.hermitian_fold;
    pp.Nw_store = planes;
    pp.predict = 0;
    pp.w_support = 0;
    pp.Nw_total = c.n_wplanes;
    pp.Ni = c.N;
    pp.fov_i = c.fov_rad;
    pp.half_i = 0.5 * c.N;
    pp.fov_i_f = (float)c.fov_rad;
    pp.half_i_f = (float)(0.5 * c.N);
    pp.fov = c.fov_rad;
    pp.half_n = 0.5 * c.N;
    pp.half_s = 0.5 * c.support;
    pp.w_min = c.w_min;
    pp.w_scale = c.n_wplanes > 1 ? (double)c.n_wplanes / (c.w_max - c.w_min) : 0.0;
    pp.fov_f = (float)c.fov_rad;
    pp.half_n_f = (float)pp.half_n;
    pp.half_s_f = (float)pp.half_s;
    pp.w_min_f = (float)c.w_min;
    pp.w_scale_f = (float)pp.w_scale;
    int launches = 0;
    cudaError_t e = launch_place(pp, uvw, chan_scale, reinterpret_cast<const float2*>(vis), weight,
                                 flag, (int64_t)nvis, hist, key, rank, stage, weight_sum, cnt,
                                 num_sms, st, &launches);
    if (e == cudaSuccess) e = launch_scan(hist, offsets, partials, nkeys, st, &launches);
    if (e == cudaSuccess)
        e = launch_scatter(key, rank, stage, offsets, records, (int64_t)nvis, num_sms, st, &launches);
    if (e == cudaSuccess) {
        G.N = c.N;
        G.S = c.support;
        G.T = T;
        G.NT = NT;
        G.Nw = planes;
        G.c0 = 0;
        G.nc = c.n_channels;
        G.k0 = plane_begin;
        G.nk = plane_end - plane_begin;
        G.n_items = (uint32_t)items;
        G.kind = c.kernel_kind;
        G.table = nullptr;
        G.lattice = 0;
        G.lists = nullptr;  // natural tile order (no scheduling scratch)
        G.list_cap = 0;
        G.w_support = 0;
        G.skip_empty = 0;
        G.grab = c.tiles_per_grab > 0 ? (uint32_t)c.tiles_per_grab : 4u;   // validated: 0..8
        e = launch_grid(G, offsets, records, reinterpret_cast<float2*>(grids), counter, threads,
                        num_sms, st, &launches);
    }
    if (e == cudaSuccess && counts)
        e = cudaMemcpyAsync(counts, cnt, 2 * sizeof(int64_t), cudaMemcpyDeviceToDevice, st);
    if (e != cudaSuccess) {
        char msg[256];
        snprintf(msg, sizeof msg, "rick_grid_noalloc: %s", cudaGetErrorString(e));
        return fail(RICK_ERR_CUDA, msg);
    }
    return RICK_OK;
}

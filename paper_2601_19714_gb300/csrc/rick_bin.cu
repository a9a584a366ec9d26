// rick_bin.cu -- placement and binning of visibilities (the "a0" step).
//
// The paper's bucket sort assigns visibilities to v-slabs and widens each
// slab by a ghost region of half the kernel (Sec. 3.2, Eq. 5).  On one GPU the
// same idea becomes a counting sort of the visibilities into square tiles of
// every (channel, w-plane): each visibility is stored once, in the tile that
// holds the first cell of its footprint, together with a halo class saying
// whether the footprint spills into the tile to the right and/or below.  The
// gridder of a tile then reads its own bins plus the spilling classes of its
// left, upper and upper-left neighbours.
//
// Kernels:
//   k_place    per visibility: FP64 cell position, plane, tile, class; rank in
//              its bin from a warp-aggregated atomicAdd on the histogram
//              (__match_any_sync groups lanes with the same key); partial sums
//              of the weights per channel.
//   k_scan_*   exclusive scan of the histogram -> bin offsets.
//   k_scatter  record -> offsets[key] + rank.
#include <cmath>

#include "rick_internal.cuh"

namespace rick {

namespace {

constexpr int kPlaceThreads = 256;

struct Placed {
    uint32_t key;
    VisRecord rec;
    int status;  // 1 gridded, 0 skipped, -1 dropped
};

// Placement of one visibility before its records are formed: footprint start,
// 24-bit fractions, first plane (of the extended set with a w-kernel) and the
// w fraction.
struct Base {
    int status;  // 1 placed, 0 skipped, -1 dropped
    int i0, j0, k;
    uint32_t fqx, fqy;
    float fw;
};

// The record and bin key of a placed visibility: plane k, footprint start
// (i0, j0) and fractional offsets fq = round(f * 2^24) in [0, 2^24].
//
// Hermitian fold: a visibility of the upper half of the planes (2k > Nw - 1)
// is stored as conj(W V) on plane Nw - 1 - k.  Its footprint, mirrored
// through cell i -> N - i, starts at N - i0 - S + 1 with offset 1 - f: tap a
// of the mirrored footprint sits at distance (a + 1 - S/2 - (1 - f)) =
// -(S - 1 - a + 1 - S/2 - f) from the mirrored centre, the distance of tap
// S - 1 - a of the original, so a symmetric kernel gives it the same weight.
// If i0 = 0 the last mirrored cell is N, which is cell 0 on the periodic
// mesh; it spills out of the last tile column and the gridder of tile column
// 0 picks it up as a halo (likewise for rows).
__device__ __forceinline__ void finish_record(const PlaceParams& P, int c, int k, int i0, int j0,
                                              uint32_t fqx, uint32_t fqy, float W, float2 V,
                                              float gw, uint32_t vidx, Placed& out) {
    const float Wg = W * gw;
    float wv_im = Wg * V.y;
    bool folded = false;
    if (P.fold && 2 * k > P.Nw_total - 1) {
        folded = true;
        k = P.Nw_total - 1 - k;
        i0 = P.N - i0 - P.S + 1;  // in [1, N - S + 1]; N only for S = 1, i0 = 0
        j0 = P.N - j0 - P.S + 1;
        if (i0 == P.N) i0 = 0;
        if (j0 == P.N) j0 = 0;
        fqx = (1u << kFracBits) - fqx;
        fqy = (1u << kFracBits) - fqy;
        wv_im = -wv_im;
    }
    fqx = min(fqx, kFracMask);
    fqy = min(fqy, kFracMask);
    const int tx = i0 / P.T, ty = j0 / P.T;
    const int il = i0 - tx * P.T, jl = j0 - ty * P.T;
    const int cls = halo_class(il + P.S - 1 >= P.T, jl + P.S - 1 >= P.T);
    const uint64_t key =
        ((((uint64_t)c * P.Nw_store + k) * P.NT + ty) * P.NT + tx) * 4u + (uint64_t)cls;
    out.key = (uint32_t)key;
    out.rec.wv_re = P.predict ? __uint_as_float(vidx) : Wg * V.x;
    out.rec.wv_im = P.predict ? (folded ? -gw : gw) : wv_im;
    out.rec.px = ((uint32_t)il << kFracBits) | fqx;
    out.rec.py = ((uint32_t)jl << kFracBits) | fqy;
    out.status = 1;
}

// floor(s) and round-half-even((s - floor(s)) 2^24) of an FP64 value s >= 0,
// read exactly from its bits with integer operations: s = m 2^(e-52), so
// s 2^24 = m 2^(e-28) is m shifted, and the bits shifted out decide the
// rounding.  These equal the FP64 results of floor, s - floor(s) (exact) and
// __double2uint_rn((s - floor(s)) * 2^24).  False if s is not finite or s >= 2^30.
__device__ __forceinline__ bool split_cell(double s, int& fl, uint32_t& fq) {
    const unsigned long long b = (unsigned long long)__double_as_longlong(s);
    const int be = (int)((b >> 52) & 0x7ffu);
    if (be == 0x7ff) return false;
    const int e = be - 1023;
    if (e >= 30) return false;
    if (be == 0) {  // zero or subnormal: below 2^-1022, rounds to 0
        fl = 0;
        fq = 0;
        return true;
    }
    const unsigned long long m = (b & 0xFFFFFFFFFFFFFull) | (1ull << 52);
    unsigned long long qf, qr;
    if (e >= 28) {
        qf = qr = m << (e - 28);
    } else if (28 - e >= 64) {
        qf = qr = 0;  // s 2^24 < 2^53 2^-64 < 1/2
    } else {
        const int sh = 28 - e;
        qf = m >> sh;
        const unsigned long long rem = m & ((1ull << sh) - 1ull), half = 1ull << (sh - 1);
        qr = qf + ((rem > half || (rem == half && (qf & 1ull))) ? 1ull : 0ull);
    }
    fl = (int)(qf >> 24);
    fq = (uint32_t)(qr - ((unsigned long long)(uint32_t)fl << 24));
    return true;
}

__device__ __forceinline__ bool finite_bits(double s) {
    return (((unsigned long long)__double_as_longlong(s) >> 52) & 0x7ffu) != 0x7ffu;
}

// One axis of the placement from sx = x - S/2: footprint start i0 and 24-bit
// fraction; false if the visibility leaves the grid or sx is not finite.
// sx >= 0 (all but footprints starting at cell 0) takes the integer path;
// sx < 0 the FP64 operations floor, subtraction and conversion.
__device__ __forceinline__ bool place_axis(const PlaceParams& P, double sx, int& i0, uint32_t& fq) {
    int fl;
    if (!(__double_as_longlong(sx) < 0)) {
        if (!split_cell(sx, fl, fq)) return false;
    } else {
        if (!finite_bits(sx)) return false;
        const double f = floor(sx);
        if (f < -1.0) return false;
        fl = (int)f;
        fq = __double2uint_rn(__dsub_rn(sx, f) * 16777216.0);
    }
    if (fl + P.S > P.N - 1) return false;
    i0 = fl + 1;
    return true;
}

// FP64 placement.  The FP64 operations and their order are fixed (no
// contraction) so that the footprint start, fraction and plane index are the
// IEEE results of
//   u = uvw * s;  x = u * fov + N/2;  sx = x - S/2;  i0 = floor(sx) + 1
//   k = floor((w - w_min) * (Nw / (w_max - w_min)))   (clamped)
// Only the multiplications and additions run on the FP64 pipe (11 per
// visibility, GB300's FP64 rate being a small fraction of its FP32 rate); the
// floors, fractions, 24-bit rounding, range and finiteness tests are read from
// the bit patterns with integer operations (exactly the same results).
__device__ __forceinline__ Base place_fp64(const PlaceParams& P, double u0, double v0, double w0,
                                           double sc) {
    Base out;
    out.status = -1;
    out.fw = 0.f;
    const double u = __dmul_rn(u0, sc), v = __dmul_rn(v0, sc), w = __dmul_rn(w0, sc);
    const double x = __dadd_rn(__dmul_rn(u, P.fov), P.half_n);
    const double y = __dadd_rn(__dmul_rn(v, P.fov), P.half_n);
    if (!finite_bits(w)) return out;
    int i0, j0;
    uint32_t fqx, fqy;
    if (!place_axis(P, __dsub_rn(x, P.half_s), i0, fqx)) return out;
    if (!place_axis(P, __dsub_rn(y, P.half_s), j0, fqy)) return out;
    int k = 0;
    if (P.Nw > 1 && P.w_support >= 2) {
        // w-kernel: plane coordinate z = t - 1/2 clamped to the w range, first
        // plane floor(z - Sw/2) + 1 (+ Sw/2 in the extended set), fraction fw
        const double t = __dmul_rn(__dsub_rn(w, P.w_min), P.w_scale);
        double z = __dsub_rn(t, 0.5);
        if (z < -0.5) z = -0.5;
        if (z > P.Nw - 0.5) z = P.Nw - 0.5;
        const double sz = __dsub_rn(z, 0.5 * P.w_support);
        const double fl = floor(sz);
        k = min(max((int)fl + 1 + P.w_support / 2, 0), P.Nw);  // in [0, Nw] by the clamp
        out.fw = (float)__dsub_rn(sz, fl);
    } else if (P.Nw > 1) {
        const double t = __dmul_rn(__dsub_rn(w, P.w_min), P.w_scale);
        const unsigned long long tb = (unsigned long long)__double_as_longlong(t);
        int fl;
        uint32_t unused;
        if (tb >> 63) k = 0;                                        // t < 0 or -0: clamp low
        else if ((tb & 0x7FFFFFFFFFFFFFFFull) > 0x7FF0000000000000ull) k = 0;  // NaN: fmax gives 0
        else if (!split_cell(t, fl, unused)) k = P.Nw - 1;          // +inf or >= 2^30: clamp high
        else k = min(fl, P.Nw - 1);
    }
    out.status = 1;
    out.i0 = i0;
    out.j0 = j0;
    out.k = k;
    out.fqx = fqx;
    out.fqy = fqy;
    return out;
}

// All-FP32 placement (precision study): same steps in single precision.
__device__ __forceinline__ Base place_fp32(const PlaceParams& P, double u0, double v0, double w0,
                                           double sc) {
    Base out;
    out.status = 0;
    out.fw = 0.f;
    const float s = (float)sc;
    const float u = (float)u0 * s, v = (float)v0 * s, w = (float)w0 * s;
    const float x = u * P.fov_f + P.half_n_f, y = v * P.fov_f + P.half_n_f;
    if (!isfinite(x) || !isfinite(y) || !isfinite(w)) {
        out.status = -1;
        return out;
    }
    const float sx = x - P.half_s_f, sy = y - P.half_s_f;
    const float flx = floorf(sx), fly = floorf(sy);
    if (flx < -1.0f || fly < -1.0f || flx + P.S > P.N - 1 || fly + P.S > P.N - 1) {
        out.status = -1;
        return out;
    }
    const int i0 = (int)flx + 1, j0 = (int)fly + 1;
    const float fx = sx - flx, fy = sy - fly;
    int k = 0;
    if (P.Nw > 1 && P.w_support >= 2) {
        float z = (w - P.w_min_f) * P.w_scale_f - 0.5f;
        z = fminf(fmaxf(z, -0.5f), (float)P.Nw - 0.5f);
        const float sz = z - 0.5f * P.w_support;
        const float fl = floorf(sz);
        k = min(max((int)fl + 1 + P.w_support / 2, 0), P.Nw);
        out.fw = sz - fl;
    } else if (P.Nw > 1) {
        float kf = floorf((w - P.w_min_f) * P.w_scale_f);
        kf = fminf(fmaxf(kf, 0.0f), (float)(P.Nw - 1));
        k = (int)kf;
    }
    out.status = 1;
    out.i0 = i0;
    out.j0 = j0;
    out.k = k;
    out.fqx = __float2uint_rn(fx * 16777216.0f);
    out.fqy = __float2uint_rn(fy * 16777216.0f);
    return out;
}

// One thread per visibility (grid-stride).  The launch makes the stride a
// multiple of C, so every thread sees one channel only and can keep a private
// FP64 partial sum of that channel's weights.
template <int PREC>
__global__ void __launch_bounds__(kPlaceThreads)
k_place(PlaceParams P, const double* __restrict__ uvw, const double* __restrict__ chan_scale,
        const float2* __restrict__ vis, const float* __restrict__ weight,
        const uint8_t* __restrict__ flag, int64_t nvis, uint32_t* __restrict__ hist,
        uint32_t* __restrict__ key_out, uint32_t* __restrict__ rank_out,
        VisRecord* __restrict__ stage, double* __restrict__ weight_sum,
        unsigned long long* __restrict__ counts, int64_t vis_base) {
    __shared__ double s_wsum[kPlaceThreads];
    __shared__ unsigned long long s_cnt[2];
    const int lane = threadIdx.x & 31;
    const int64_t tid0 = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    const int c = (int)(tid0 % P.C);
    const double sc = chan_scale[c];
    s_wsum[threadIdx.x] = 0.0;
    if (threadIdx.x < 2) s_cnt[threadIdx.x] = 0ull;
    __syncthreads();

    double my_wsum = 0.0;
    uint32_t n_grid = 0, n_drop = 0;
    const int nrec = P.w_support >= 2 ? P.w_support : 1;   // records per visibility
    for (int64_t base = tid0 - lane; base < nvis; base += stride) {
        const int64_t idx = base + lane;
        Base b;
        b.status = 0;
        float W = 0.f;
        float2 V = make_float2(0.f, 0.f);
        if (idx < nvis) {
            const bool flagged = flag != nullptr && flag[idx] != 0;
            W = weight[idx];
            if (!flagged && W != 0.0f && isfinite(W)) {
                const int64_t r = idx / P.C;
                const double u0 = uvw[3 * r], v0 = uvw[3 * r + 1], w0 = uvw[3 * r + 2];
                if (vis != nullptr) V = vis[idx];
                b = PREC == RICK_PREC_ALL_FP32 ? place_fp32(P, u0, v0, w0, sc)
                                               : place_fp64(P, u0, v0, w0, sc);
                if (b.status == 1) {
                    my_wsum += (double)W;
                    ++n_grid;
                } else if (b.status == -1) {
                    ++n_drop;
                }
            }
        }
        const float tw = fmaf(2.0f, b.fw, -1.0f);
        for (int sw = 0; sw < nrec; ++sw) {
            Placed pl;
            pl.key = kInvalidKey;
            if (b.status == 1) {
                float gw = 1.0f;
                if (P.w_support >= 2) {
                    gw = P.wcoef[sw][kPolyDegree];
#pragma unroll
                    for (int q = kPolyDegree - 1; q >= 0; --q) gw = fmaf(gw, tw, P.wcoef[sw][q]);
                }
                finish_record(P, c, b.k + sw, b.i0, b.j0, b.fqx, b.fqy, W, V, gw, (uint32_t)(vis_base + idx), pl);
            }
            // rank within the bin: one atomic per distinct key in the warp
            const unsigned peers = __match_any_sync(0xffffffffu, pl.key);
            const int leader = __ffs(peers) - 1;
            uint32_t first = 0;
            if (lane == leader && pl.key != kInvalidKey) first = atomicAdd(&hist[pl.key], __popc(peers));
            first = __shfl_sync(0xffffffffu, first, leader);
            if (idx < nvis) {
                const int64_t o = idx * nrec + sw;
                key_out[o] = pl.key;
                if (pl.key != kInvalidKey) {
                    rank_out[o] = first + __popc(peers & ((1u << lane) - 1u));
                    stage[o] = pl.rec;
                }
            }
        }
    }

    // per-channel weight sums: block reduction in shared memory, then global
    if (P.C <= kPlaceThreads) {
        if (my_wsum != 0.0) atomicAdd(&s_wsum[c], my_wsum);
    } else if (my_wsum != 0.0) {
        atomicAdd(&weight_sum[c], my_wsum);
    }
    const unsigned g = __reduce_add_sync(0xffffffffu, n_grid);
    const unsigned d = __reduce_add_sync(0xffffffffu, n_drop);
    if (lane == 0) {
        if (g) atomicAdd(&s_cnt[0], (unsigned long long)g);
        if (d) atomicAdd(&s_cnt[1], (unsigned long long)d);
    }
    __syncthreads();
    if (P.C <= kPlaceThreads && threadIdx.x < P.C && s_wsum[threadIdx.x] != 0.0)
        atomicAdd(&weight_sum[threadIdx.x], s_wsum[threadIdx.x]);
    if (threadIdx.x < 2 && s_cnt[threadIdx.x]) atomicAdd(&counts[threadIdx.x], s_cnt[threadIdx.x]);
}

// ---- exclusive scan (three kernels) ---------------------------------------

constexpr int kScanThreads = 256;
constexpr int kScanItems = 16;
constexpr int kScanChunk = kScanThreads * kScanItems;

__device__ __forceinline__ uint32_t block_exclusive_scan(uint32_t v, uint32_t* total) {
    __shared__ uint32_t s_warp[32];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    uint32_t x = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const uint32_t y = __shfl_up_sync(0xffffffffu, x, o);
        if (lane >= o) x += y;
    }
    if (lane == 31) s_warp[warp] = x;
    __syncthreads();
    const int nw = blockDim.x >> 5;
    if (warp == 0) {
        uint32_t w = lane < nw ? s_warp[lane] : 0u;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const uint32_t y = __shfl_up_sync(0xffffffffu, w, o);
            if (lane >= o) w += y;
        }
        s_warp[lane] = w;  // inclusive warp prefix
    }
    __syncthreads();
    const uint32_t warp_excl = warp ? s_warp[warp - 1] : 0u;
    *total = s_warp[nw - 1];
    const uint32_t r = warp_excl + x - v;
    __syncthreads();  // s_warp reusable
    return r;
}

__device__ __forceinline__ void load_items(const uint32_t* in, uint64_t n, uint64_t first,
                                           uint32_t v[kScanItems]) {
    if (first + kScanItems <= n) {
        const uint4* p = reinterpret_cast<const uint4*>(in + first);
#pragma unroll
        for (int q = 0; q < kScanItems / 4; ++q) {
            const uint4 t = p[q];
            v[4 * q] = t.x;
            v[4 * q + 1] = t.y;
            v[4 * q + 2] = t.z;
            v[4 * q + 3] = t.w;
        }
    } else {
#pragma unroll
        for (int q = 0; q < kScanItems; ++q) v[q] = first + q < n ? in[first + q] : 0u;
    }
}

__global__ void __launch_bounds__(kScanThreads)
k_scan_reduce(const uint32_t* __restrict__ in, uint64_t n, uint32_t* __restrict__ partials) {
    const uint64_t first = (uint64_t)blockIdx.x * kScanChunk + (uint64_t)threadIdx.x * kScanItems;
    uint32_t v[kScanItems];
    load_items(in, n, first, v);
    uint32_t s = 0;
#pragma unroll
    for (int q = 0; q < kScanItems; ++q) s += v[q];
    uint32_t total;
    block_exclusive_scan(s, &total);
    if (threadIdx.x == 0) partials[blockIdx.x] = total;
}

// Single block: exclusive scan of the block totals in place.
__global__ void __launch_bounds__(1024) k_scan_partials(uint32_t* partials, uint64_t nb) {
    uint32_t carry = 0;
    for (uint64_t base = 0; base < nb; base += blockDim.x) {
        const uint64_t i = base + threadIdx.x;
        const uint32_t v = i < nb ? partials[i] : 0u;
        uint32_t total;
        const uint32_t ex = block_exclusive_scan(v, &total);
        if (i < nb) partials[i] = carry + ex;
        carry += total;
    }
}

__global__ void __launch_bounds__(kScanThreads)
k_scan_apply(const uint32_t* __restrict__ in, uint32_t* __restrict__ out, uint64_t n,
             const uint32_t* __restrict__ partials) {
    const uint64_t first = (uint64_t)blockIdx.x * kScanChunk + (uint64_t)threadIdx.x * kScanItems;
    uint32_t v[kScanItems];
    load_items(in, n, first, v);
    uint32_t s = 0;
#pragma unroll
    for (int q = 0; q < kScanItems; ++q) s += v[q];
    uint32_t total;
    uint32_t run = partials[blockIdx.x] + block_exclusive_scan(s, &total);
#pragma unroll
    for (int q = 0; q < kScanItems; ++q) {
        const uint64_t i = first + q;
        if (i < n) out[i] = run;
        run += v[q];
        if (i + 1 == n) out[n] = run;  // offsets[n] = total number of records
    }
}

__global__ void __launch_bounds__(256)
k_scatter(const uint32_t* __restrict__ key, const uint32_t* __restrict__ rank,
          const VisRecord* __restrict__ stage, const uint32_t* __restrict__ offsets,
          VisRecord* __restrict__ records, int64_t nvis) {
    // four visibilities per thread and step, their loads issued together: the
    // key -> offset -> store chain is latency-bound, so this keeps 4x more
    // requests in flight
    constexpr int kU = 4;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x * kU;
    for (int64_t base = ((int64_t)blockIdx.x * blockDim.x) * kU + threadIdx.x; base < nvis;
         base += stride) {
        uint32_t k[kU], r[kU], o[kU];
        VisRecord v[kU];
#pragma unroll
        for (int u = 0; u < kU; ++u) {
            const int64_t i = base + (int64_t)u * blockDim.x;
            k[u] = i < nvis ? key[i] : kInvalidKey;
        }
#pragma unroll
        for (int u = 0; u < kU; ++u) {
            const int64_t i = base + (int64_t)u * blockDim.x;
            if (k[u] != kInvalidKey) {
                o[u] = offsets[k[u]];
                r[u] = rank[i];
                v[u] = stage[i];
            }
        }
#pragma unroll
        for (int u = 0; u < kU; ++u)
            if (k[u] != kInvalidKey) records[o[u] + r[u]] = v[u];
    }
}

// ---- imaging weights (uniform / Briggs) ------------------------------------
//
// The density of a channel is the sum of the weights of its gridded
// visibilities on their nearest mesh cell (floor(x + 1/2), floor(y + 1/2)),
// each added there and at the cell of its Hermitian partner ((N - i) mod N,
// (N - j) mod N).  Uniform: W' = W / D(cell); Briggs: W' = W / (1 + f^2 D),
// f^2 = (5 10^-R)^2 sum D / sum D^2.  Same skip and drop decisions as the
// placement; the cell is taken in the placement's precision.

// True if visibility idx is gridded; its cell and the mirrored cell (flat
// indices into the channel's N x N density) and its weight.
template <int PREC>
__device__ __forceinline__ bool weight_cell(const PlaceParams& P, const double* __restrict__ uvw,
                                            const double* __restrict__ chan_scale,
                                            const float* __restrict__ weight,
                                            const uint8_t* __restrict__ flag, int64_t idx, int& cell,
                                            int& mcell, float& W) {
    if (flag != nullptr && flag[idx] != 0) return false;
    W = weight[idx];
    if (!(W != 0.0f) || !isfinite(W)) return false;
    const int64_t r = idx / P.C;
    const int c = (int)(idx - r * P.C);
    const double sc = chan_scale[c];
    const double u0 = uvw[3 * r], v0 = uvw[3 * r + 1], w0 = uvw[3 * r + 2];
    const Base b = PREC == RICK_PREC_ALL_FP32 ? place_fp32(P, u0, v0, w0, sc) : place_fp64(P, u0, v0, w0, sc);
    if (b.status != 1) return false;
    // nearest cell of the Ni x Ni mesh of cell 1/fov (the image mesh, also
    // with a padded grid), taken mod Ni
    int i, j;
    if (PREC == RICK_PREC_ALL_FP32) {
        const float s = (float)sc;
        const float x = (float)u0 * s * P.fov_i_f + P.half_i_f, y = (float)v0 * s * P.fov_i_f + P.half_i_f;
        i = (int)floorf(x + 0.5f);
        j = (int)floorf(y + 0.5f);
    } else {
        const double x = __dadd_rn(__dmul_rn(__dmul_rn(u0, sc), P.fov_i), P.half_i);
        const double y = __dadd_rn(__dmul_rn(__dmul_rn(v0, sc), P.fov_i), P.half_i);
        i = (int)floor(__dadd_rn(x, 0.5));
        j = (int)floor(__dadd_rn(y, 0.5));
    }
    const int Ni = P.Ni;
    i = ((i % Ni) + Ni) % Ni;
    j = ((j % Ni) + Ni) % Ni;
    cell = j * Ni + i;
    mcell = ((Ni - j) % Ni) * Ni + (Ni - i) % Ni;
    return true;
}

template <int PREC>
__global__ void __launch_bounds__(256)
k_density(PlaceParams P, const double* __restrict__ uvw, const double* __restrict__ chan_scale,
          const float* __restrict__ weight, const uint8_t* __restrict__ flag, int64_t nvis,
          double* __restrict__ D) {
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; idx < nvis; idx += stride) {
        int cell, mcell;
        float W;
        if (!weight_cell<PREC>(P, uvw, chan_scale, weight, flag, idx, cell, mcell, W)) continue;
        double* Dc = D + (size_t)(idx % P.C) * P.Ni * P.Ni;
        atomicAdd(Dc + cell, (double)W);
        atomicAdd(Dc + mcell, (double)W);
    }
}

// mom[2c] += sum D, mom[2c+1] += sum D^2 over channel c = blockIdx.y
__global__ void __launch_bounds__(256)
k_density_moments(const double* __restrict__ D, int64_t cells, double* __restrict__ mom) {
    __shared__ double s1[8], s2[8];
    const double* Dc = D + (size_t)blockIdx.y * cells;
    double a = 0.0, b = 0.0;
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < cells;
         e += (int64_t)gridDim.x * blockDim.x) {
        const double d = Dc[e];
        a += d;
        b += d * d;
    }
    for (int o = 16; o > 0; o >>= 1) {
        a += __shfl_xor_sync(0xffffffffu, a, o);
        b += __shfl_xor_sync(0xffffffffu, b, o);
    }
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    if (lane == 0) {
        s1[warp] = a;
        s2[warp] = b;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        a = b = 0.0;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) {
            a += s1[w];
            b += s2[w];
        }
        atomicAdd(mom + 2 * blockIdx.y, a);
        atomicAdd(mom + 2 * blockIdx.y + 1, b);
    }
}

template <int PREC>
__global__ void __launch_bounds__(256)
k_reweight(PlaceParams P, const double* __restrict__ uvw, const double* __restrict__ chan_scale,
           const float* __restrict__ weight, const uint8_t* __restrict__ flag, int64_t nvis,
           const double* __restrict__ D, const double* __restrict__ mom, int mode, double a2,
           float* __restrict__ out) {
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; idx < nvis; idx += stride) {
        int cell, mcell;
        float W;
        if (!weight_cell<PREC>(P, uvw, chan_scale, weight, flag, idx, cell, mcell, W)) {
            out[idx] = weight[idx];
            continue;
        }
        const int c = (int)(idx % P.C);
        const double d = D[(size_t)c * P.Ni * P.Ni + cell];
        if (mode == RICK_WEIGHT_UNIFORM) {
            out[idx] = (float)((double)W / d);
        } else {
            const double s1 = mom[2 * c], s2 = mom[2 * c + 1];
            const double f2 = s2 > 0.0 ? a2 * s1 / s2 : 0.0;
            out[idx] = (float)((double)W / (1.0 + f2 * d));
        }
    }
}

}  // namespace

cudaError_t launch_imaging_weights(const PlaceParams& P, const double* uvw, const double* chan_scale,
                                   const float* weight, const uint8_t* flag, int64_t nvis, int mode,
                                   double robust, double* density, double* moments, float* out,
                                   int num_sms, cudaStream_t stream, int* launches) {
    if (nvis <= 0) return cudaSuccess;
    const size_t cells = (size_t)P.Ni * P.Ni;
    cudaError_t e = cudaMemsetAsync(density, 0, sizeof(double) * cells * P.C, stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(moments, 0, sizeof(double) * 2 * P.C, stream);
    if (e != cudaSuccess) return e;
    int64_t blocks = (nvis + 255) / 256;
    if (blocks > (int64_t)num_sms * 16) blocks = (int64_t)num_sms * 16;
    const bool f32 = P.precision == RICK_PREC_ALL_FP32;
    if (f32)
        k_density<RICK_PREC_ALL_FP32><<<(unsigned)blocks, 256, 0, stream>>>(P, uvw, chan_scale, weight, flag, nvis, density);
    else
        k_density<RICK_PREC_FP32_FP64IDX><<<(unsigned)blocks, 256, 0, stream>>>(P, uvw, chan_scale, weight, flag, nvis, density);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    ++*launches;
    double a2 = 0.0;
    if (mode == RICK_WEIGHT_BRIGGS) {
        int64_t mb = ((int64_t)cells + 255) / 256;
        if (mb > num_sms * 4) mb = num_sms * 4;
        k_density_moments<<<dim3((unsigned)mb, (unsigned)P.C), 256, 0, stream>>>(density, (int64_t)cells, moments);
        if ((e = cudaGetLastError()) != cudaSuccess) return e;
        ++*launches;
        const double a = 5.0 * std::pow(10.0, -robust);
        a2 = a * a;
    }
    if (f32)
        k_reweight<RICK_PREC_ALL_FP32><<<(unsigned)blocks, 256, 0, stream>>>(P, uvw, chan_scale, weight, flag, nvis, density, moments, mode, a2, out);
    else
        k_reweight<RICK_PREC_FP32_FP64IDX><<<(unsigned)blocks, 256, 0, stream>>>(P, uvw, chan_scale, weight, flag, nvis, density, moments, mode, a2, out);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    ++*launches;
    return cudaSuccess;
}

cudaError_t launch_place(const PlaceParams& P, const double* uvw, const double* chan_scale,
                         const float2* vis, const float* weight, const uint8_t* flag,
                         int64_t nvis, uint32_t* hist, uint32_t* key, uint32_t* rank,
                         VisRecord* stage, double* weight_sum, unsigned long long* counts,
                         int num_sms, cudaStream_t stream, int* launches, int64_t vis_base) {
    if (nvis <= 0) return cudaSuccess;
    // grid: a multiple of C blocks (so that the stride is a multiple of C),
    // about 8 blocks per SM, never more than the work needs
    const int64_t per_block = kPlaceThreads;
    int64_t want = (nvis + per_block - 1) / per_block;
    int64_t target = (int64_t)num_sms * 8;
    if (want < target) target = want;
    int64_t mult = (target + P.C - 1) / P.C;
    if (mult < 1) mult = 1;
    const int64_t blocks = mult * P.C;
    if (blocks > 0x7fffffffLL) return cudaErrorInvalidConfiguration;
    if (P.precision == RICK_PREC_ALL_FP32)
        k_place<RICK_PREC_ALL_FP32><<<(unsigned)blocks, kPlaceThreads, 0, stream>>>(
            P, uvw, chan_scale, vis, weight, flag, nvis, hist, key, rank, stage, weight_sum,
            counts, vis_base);
    else
        k_place<RICK_PREC_FP32_FP64IDX><<<(unsigned)blocks, kPlaceThreads, 0, stream>>>(
            P, uvw, chan_scale, vis, weight, flag, nvis, hist, key, rank, stage, weight_sum,
            counts, vis_base);
    ++*launches;
    return cudaGetLastError();
}

cudaError_t launch_scan(const uint32_t* in, uint32_t* out, uint32_t* partials, uint64_t n,
                        cudaStream_t stream, int* launches) {
    if (n == 0) return cudaSuccess;
    const uint64_t nb = (n + kScanChunk - 1) / kScanChunk;
    if (nb > 0x7fffffffULL) return cudaErrorInvalidConfiguration;
    k_scan_reduce<<<(unsigned)nb, kScanThreads, 0, stream>>>(in, n, partials);
    k_scan_partials<<<1, 1024, 0, stream>>>(partials, nb);
    k_scan_apply<<<(unsigned)nb, kScanThreads, 0, stream>>>(in, out, n, partials);
    *launches += 3;
    return cudaGetLastError();
}

uint64_t scan_partials_needed(uint64_t n) { return (n + kScanChunk - 1) / kScanChunk + 1; }

cudaError_t launch_scatter(const uint32_t* key, const uint32_t* rank, const VisRecord* stage,
                           const uint32_t* offsets, VisRecord* records, int64_t nvis,
                           int num_sms, cudaStream_t stream, int* launches) {
    if (nvis <= 0) return cudaSuccess;
    int64_t blocks = (nvis + 1023) / 1024;
    const int64_t cap = (int64_t)num_sms * 8;
    if (blocks > cap) blocks = cap;
    k_scatter<<<(unsigned)blocks, 256, 0, stream>>>(key, rank, stage, offsets, records, nvis);
    ++*launches;
    return cudaGetLastError();
}

}  // namespace rick

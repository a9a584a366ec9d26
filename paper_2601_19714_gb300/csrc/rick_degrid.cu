// rick_degrid.cu -- prediction (degridding): transformed w-planes -> visibilities.
//
// The adjoint direction of Eq. 3: for every visibility binned for prediction,
//   V = sum_{a,b} g(i0 + a - x) g(j0 + b - y) (-1)^(i+j) F_k(i0 + a, j0 + b),
// where F_k is the forward transform of the model planes built by
// k_model_planes (so that (-1)^(i+j) F_k is the plane of the w-stacking
// prediction), times the record's plane weight and conjugated for records
// that the Hermitian fold mapped onto the mirrored plane.  Without a w-kernel
// a visibility has one record and its prediction is stored; with one
// (improved w-stacking) its Sw records each add their plane's part.
//
// One warp per tile of one (channel, plane): the warp copies the tile's
// (T + S - 1)^2 region of the plane (rows and columns taken mod N, which only
// the fold's footprints ending on cell N use) into its shared buffer with
// coalesced loads, then predicts the records anchored in that tile, one record
// per lane, 32 at a time: 2S tap polynomials (the tap index is the same in all
// lanes, so the coefficients are read once for the warp) and S^2 products with
// the buffered cells.  Every record is read once and every prediction written
// once; the plane is read only where records are.
#include "rick_internal.cuh"

namespace rick {

namespace {

constexpr unsigned kFull = 0xffffffffu;
constexpr int kDegridGrab = 4;

// g(a + 1 - S/2 - f) for footprint tap a (warp-uniform), by Horner in t = 2 f - 1.
__device__ __forceinline__ float tap_poly_uniform(const GridParams& G, int a, float t) {
    float acc = G.coef[a][kPolyDegree];
#pragma unroll
    for (int k = kPolyDegree - 1; k >= 0; --k) acc = fmaf(acc, t, G.coef[a][k]);
    return acc;
}

template <int SS>
__global__ void k_degrid(GridParams G, const uint32_t* __restrict__ offsets,
                         const VisRecord* __restrict__ records, const float2* __restrict__ grids,
                         float2* __restrict__ vis_out, uint32_t* __restrict__ work_counter) {
    extern __shared__ __align__(16) float smem[];
    constexpr int kS = SS > 0 ? SS : kMaxSupport;
    const int S = SS > 0 ? SS : G.S;
    const int T = G.T, N = G.N, NT = G.NT;
    const int R = T + S - 1, RP = R + 1;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    float2* region = reinterpret_cast<float2*>(smem) + (size_t)warp * R * RP;
    const uint32_t tiles = (uint32_t)NT * NT;
    constexpr float kInvFrac = 1.0f / 16777216.0f;

    for (;;) {
        uint32_t first = 0;
        if (lane == 0) first = atomicAdd(work_counter, (uint32_t)kDegridGrab);
        first = __shfl_sync(kFull, first, 0);
        if (first >= G.n_items) break;
        const uint32_t last = min(first + (uint32_t)kDegridGrab, G.n_items);
        for (uint32_t item = first; item < last; ++item) {
            const uint32_t plane = item / tiles, tile = item - plane * tiles;
            const int kk = (int)(plane % G.nk), cc = (int)(plane / G.nk);
            const int ty = (int)(tile / NT), tx = (int)(tile - (uint32_t)ty * NT);
            const uint64_t key = ((((uint64_t)(G.c0 + cc) * G.Nw + (G.k0 + kk)) * NT + ty) * NT + tx) * 4u;
            const uint32_t rb = __ldg(offsets + key), re = __ldg(offsets + key + 4);
            if (rb == re) continue;
            // the tile's region of the plane, rows and columns mod N
            const float2* src = grids + (size_t)plane * N * N;
            for (int e = lane; e < R * R; e += 32) {
                const int rr = e / R, col = e - rr * R;
                const int gy = (ty * T + rr) & (N - 1), gx = (tx * T + col) & (N - 1);
                region[rr * RP + col] = __ldg(src + (size_t)gy * N + gx);
            }
            __syncwarp();
            for (uint32_t base = rb; base < re; base += 32u) {
                const uint32_t r = base + lane;
                if (r < re) {
                    const VisRecord rec = records[r];
                    const int il = (int)(rec.px >> kFracBits), jl = (int)(rec.py >> kFracBits);
                    const float tx2 = fmaf(2.0f, (float)(rec.px & kFracMask) * kInvFrac, -1.0f);
                    const float ty2 = fmaf(2.0f, (float)(rec.py & kFracMask) * kInvFrac, -1.0f);
                    // 1-D taps with the checkerboard folded in: (-1)^a, (-1)^b
                    float gx[kS], gy[kS];
#pragma unroll
                    for (int a = 0; a < kS; ++a) {
                        if (a < S) {
                            const float sa = (a & 1) ? -1.f : 1.f;
                            gx[a] = sa * tap_poly_uniform(G, a, tx2);
                            gy[a] = sa * tap_poly_uniform(G, a, ty2);
                        }
                    }
                    float2 acc = make_float2(0.f, 0.f);
                    const float2* row = region + jl * RP + il;
#pragma unroll
                    for (int b = 0; b < kS; ++b) {
                        if (b < S) {
                            float2 rs = make_float2(0.f, 0.f);
#pragma unroll
                            for (int a = 0; a < kS; ++a) {
                                if (a < S) {
                                    const float2 f = row[b * RP + a];
                                    rs.x = fmaf(gx[a], f.x, rs.x);
                                    rs.y = fmaf(gx[a], f.y, rs.y);
                                }
                            }
                            acc.x = fmaf(gy[b], rs.x, acc.x);
                            acc.y = fmaf(gy[b], rs.y, acc.y);
                        }
                    }
                    // (-1)^(i0 + j0) of the footprint's first cell (T is even),
                    // the plane weight, and its sign bit: conjugate
                    const float s0 = ((il + jl) & 1) ? -1.f : 1.f;
                    const float gw = s0 * fabsf(rec.wv_im);
                    const float2 out = make_float2(gw * acc.x, signbit(rec.wv_im) ? -gw * acc.y : gw * acc.y);
                    float2* dst = vis_out + __float_as_uint(rec.wv_re);
                    if (G.w_support >= 2) atomicAdd(dst, out);
                    else *dst = out;
                }
            }
            __syncwarp();  // the region is rewritten for the next tile
        }
    }
}

template <int SS>
cudaError_t launch_degrid_one(const GridParams& G, const uint32_t* offsets, const VisRecord* records,
                              const float2* grids, float2* vis_out, uint32_t* counter, int threads,
                              int num_sms, cudaStream_t stream) {
    const int R = G.T + G.S - 1;
    const size_t smem = (size_t)(threads / 32) * R * (R + 1) * sizeof(float2);
    auto fn = k_degrid<SS>;
    cudaError_t e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    int per_sm = 0;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, fn, threads, smem);
    if (e != cudaSuccess) return e;
    if (per_sm < 1) return cudaErrorInvalidConfiguration;
    uint64_t blocks = (uint64_t)per_sm * num_sms;
    const uint64_t need = (G.n_items + (uint64_t)kDegridGrab * (threads / 32) - 1) /
                          ((uint64_t)kDegridGrab * (threads / 32));
    if (blocks > need) blocks = need;
    if (blocks < 1) blocks = 1;
    fn<<<(unsigned)blocks, threads, smem, stream>>>(G, offsets, records, grids, vis_out, counter);
    return cudaGetLastError();
}

}  // namespace

cudaError_t launch_degrid(const GridParams& G, const uint32_t* offsets, const VisRecord* records,
                          const float2* grids, float2* vis_out, uint32_t* work_counter, int threads,
                          int num_sms, cudaStream_t stream, int* launches) {
    if (G.n_items == 0) return cudaSuccess;
    if (G.kind == RICK_KERNEL_TABLE) return cudaErrorInvalidValue;
    cudaError_t e;
    switch (G.S) {
        case 4: e = launch_degrid_one<4>(G, offsets, records, grids, vis_out, work_counter, threads, num_sms, stream); break;
        case 7: e = launch_degrid_one<7>(G, offsets, records, grids, vis_out, work_counter, threads, num_sms, stream); break;
        case 8: e = launch_degrid_one<8>(G, offsets, records, grids, vis_out, work_counter, threads, num_sms, stream); break;
        default: e = launch_degrid_one<0>(G, offsets, records, grids, vis_out, work_counter, threads, num_sms, stream); break;
    }
    if (e == cudaSuccess) ++*launches;
    return e;
}

}  // namespace rick

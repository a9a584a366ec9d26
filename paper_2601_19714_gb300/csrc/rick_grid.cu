// rick_grid.cu -- convolutional gridding onto w-planes (Eq. 3), the "a1" step.
//
// Design (one GB300, HBM-bound): the unit of work is one T x T tile of one
// (channel, w-plane).  A persistent CTA takes tiles from a global counter in
// chunks ("grabs"), loads the bin offsets of the whole chunk at once, and for
// each tile
//   * accumulates every visibility that touches the tile into a shared-memory
//     tile of interleaved complex cells (row pitch T + 8 cells, so that the
//     re and im words of 8 consecutive cells of two rows hit 32 distinct
//     banks), with the checkerboard sign (-1)^(i+j) folded into the weight;
//   * hands the finished rows to the bulk-copy engine (cp.async.bulk, shared
//     -> global, one 8T-byte copy per row) and moves on: the threads never
//     hold the tile's output in registers and HBM writes overlap the next
//     tile's work;
//   * for a tile no visibility touches, copies one shared zero row T times
//     (or, with skip_empty, writes nothing: the library's pruned transforms
//     never read such a tile).
// So every grid cell is written exactly once (the zero fill is fused into
// the gridder) and no global atomics are needed: a tile is owned by one CTA,
// and the halo of neighbouring tiles is read, not written -- the binning
// stores each visibility once with its halo class.
//
// Records of the tile's own bins and of the three neighbour bins that spill
// into it form one index range.  Each warp owns a band of tile rows and is
// the only writer of its cells, so accumulation is plain FP32 load-add-store
// in a fixed order (no shared-memory atomics, which for FP32 are
// compare-and-swap loops, and a result that does not depend on scheduling).
// A warp loads 32 records at once (one per lane), keeps those that reach its
// band and walks them one by one: lanes 0..S-1 and 16..16+S-1 evaluate the 2S
// one-dimensional taps (fitted polynomials), and the footprint cells inside
// the band are covered 16 per instruction, an even/odd lane pair adding the
// re/im parts of one cell.  The learned support-4 kernel adds a non-separable
// correction interpolated from a per-plane lattice table.
#include <algorithm>
#include <cmath>

#include "rick_internal.cuh"

namespace rick {

namespace {

constexpr unsigned kFull = 0xffffffffu;
constexpr int kMaxWarpGrab = 8;  // tiles a warp takes from the queue at once

// g(a + 1 - S/2 - f) for footprint tap a, by Horner in t = 2 f - 1, from the
// tap's coefficients held in registers (a lane evaluates the same tap a for
// the whole kernel, so its coefficients are loaded once: indexing the kernel
// parameter by a lane-dependent a would serialise the constant-bank reads).
__device__ __forceinline__ float tap_poly(const float (&cf)[kPolyDegree + 1], float t) {
    float acc = cf[kPolyDegree];
#pragma unroll
    for (int k = kPolyDegree - 1; k >= 0; --k) acc = fmaf(acc, t, cf[k]);
    return acc;
}

// Learned correction taps c = 4b + a of one record: bilinear interpolation
// of the plane's (L+1)^2 x 16 lattice table at (fx, fy), written to out[0..15].
__device__ __forceinline__ void table_taps(const GridParams& G, int k, float fx, float fy,
                                           float* out) {
    const int L = G.lattice;
    const float X = fx * L, Y = fy * L;
    const int ix = min((int)X, L - 1), iy = min((int)Y, L - 1);
    const float ax = X - ix, ay = Y - iy;
    const size_t row = (size_t)(L + 1);
    const float4* t00 = reinterpret_cast<const float4*>(G.table + (((size_t)k * row + iy) * row + ix) * 16);
    const float4* t10 = t00 + 4;
    const float4* t01 = t00 + row * 4;
    const float4* t11 = t01 + 4;
    const float w00 = (1.f - ax) * (1.f - ay), w10 = ax * (1.f - ay), w01 = (1.f - ax) * ay,
                w11 = ax * ay;
#pragma unroll
    for (int q = 0; q < 4; ++q) {
        const float4 a = __ldg(t00 + q), b = __ldg(t10 + q), c = __ldg(t01 + q), d = __ldg(t11 + q);
        out[4 * q + 0] = w00 * a.x + w10 * b.x + w01 * c.x + w11 * d.x;
        out[4 * q + 1] = w00 * a.y + w10 * b.y + w01 * c.y + w11 * d.y;
        out[4 * q + 2] = w00 * a.z + w10 * b.z + w01 * c.z + w11 * d.z;
        out[4 * q + 3] = w00 * a.w + w10 * b.w + w01 * c.w + w11 * d.w;
    }
}

// --- bulk copies shared -> global (sm_90+ PTX) ------------------------------

__device__ __forceinline__ void bulk_row_store(void* gdst, const void* ssrc, uint32_t bytes) {
    const uint32_t s = (uint32_t)__cvta_generic_to_shared(ssrc);
    asm volatile("cp.async.bulk.global.shared::cta.bulk_group [%0], [%1], %2;\n"
                 :: "l"(gdst), "r"(s), "r"(bytes) : "memory");
}
__device__ __forceinline__ void bulk_commit() { asm volatile("cp.async.bulk.commit_group;\n" ::: "memory"); }
// the shared sources of every committed group have been read
__device__ __forceinline__ void bulk_wait_read() { asm volatile("cp.async.bulk.wait_group.read 0;\n" ::: "memory"); }
// every committed group has completed
__device__ __forceinline__ void bulk_wait_all() { asm volatile("cp.async.bulk.wait_group 0;\n" ::: "memory"); }
// order this thread's generic-proxy shared writes before later async-proxy reads
__device__ __forceinline__ void fence_async_shared() {
    asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory");
}

// Bin bound q (0..7) of tile `item`: own bins [0,1) all classes, left
// neighbour [2,3) classes 2-3, upper [4,5) classes 1-2, upper-left [6,7)
// class 2.  Neighbours wrap around the mesh: only the Hermitian fold puts
// records in the spill classes of the last tile row or column (footprints
// ending on cell N = cell 0); without it those bins are empty.
__device__ __forceinline__ uint32_t tile_bound(const GridParams& G, const uint32_t* __restrict__ offsets,
                                               uint32_t item, uint32_t q) {
    const int NT = G.NT;
    const uint32_t tiles = (uint32_t)NT * NT;
    const uint32_t plane = item / tiles, tile = item - plane * tiles;
    const int kk = (int)(plane % G.nk), cc = (int)(plane / G.nk);
    const uint64_t kplane = ((uint64_t)(G.c0 + cc) * G.Nw + (G.k0 + kk)) * NT;
    const int ty = (int)(tile / NT), tx = (int)(tile - (uint32_t)ty * NT);
    const int txl = tx > 0 ? tx - 1 : NT - 1, tyu = ty > 0 ? ty - 1 : NT - 1;
    uint64_t key;
    int cls;
    if (q < 2) {
        key = ((kplane + ty) * NT + tx) * 4u;
        cls = q == 0 ? 0 : 4;
    } else if (q < 4) {
        key = ((kplane + ty) * NT + txl) * 4u;
        cls = q == 2 ? 2 : 4;
    } else if (q < 6) {
        key = ((kplane + tyu) * NT + tx) * 4u;
        cls = q == 4 ? 1 : 3;
    } else {
        key = ((kplane + tyu) * NT + txl) * 4u;
        cls = q == 6 ? 2 : 3;
    }
    return __ldg(offsets + key + cls);
}

// Scheduling pass: the record count of every tile, and the tiles with at
// least 64T, 16T, 4T records appended to the three lists (warp-aggregated
// atomics on the list lengths counts[0..2]); with G.light, every other tile
// with a record to the light list (length counts[4]).
__global__ void k_schedule(GridParams G, const uint32_t* __restrict__ offsets,
                           uint32_t* __restrict__ counts) {
    const int lane = threadIdx.x & 31;
    const uint32_t th3 = 4u * G.T, th2 = 16u * G.T, th1 = 64u * G.T;
    const uint32_t stride = gridDim.x * blockDim.x;
    for (uint32_t base = blockIdx.x * blockDim.x + (threadIdx.x & ~31u); base < G.n_items;
         base += stride) {
        const uint32_t item = base + lane;
        int level = 3;
        if (item < G.n_items) {
            uint32_t b[8];
#pragma unroll
            for (int q = 0; q < 8; ++q) b[q] = tile_bound(G, offsets, item, q);
            const uint32_t R = (b[1] - b[0]) + (b[3] - b[2]) + (b[5] - b[4]) + (b[7] - b[6]);
            level = R >= th1 ? 0 : R >= th2 ? 1 : R >= th3 ? 2 : R > 0 ? 3 : 4;
        }
#pragma unroll
        for (int lv = 0; lv < 4; ++lv) {
            if (lv == 3 && G.light == nullptr) break;
            const unsigned m = __ballot_sync(kFull, level == lv);
            if (m == 0u) continue;
            const int leader = __ffs(m) - 1;
            uint32_t* cnt = lv < 3 ? &counts[lv] : &counts[4];
            uint32_t at = 0;
            if (lane == leader) at = atomicAdd(cnt, (uint32_t)__popc(m));
            at = __shfl_sync(kFull, at, leader);
            if (level == lv) {
                const uint32_t pos = at + (uint32_t)__popc(m & ((1u << lane) - 1u));
                if (lv < 3) {
                    if (pos < G.list_cap) G.lists[(size_t)lv * G.list_cap + pos] = item;
                } else if (pos < G.light_cap) {
                    G.light[pos] = item;
                }
            }
        }
    }
}

// Row pitch (in cells) of a warp's tile buffer: a pass covers 16 footprint
// cells, i.e. 16 / S rows of S cells, each cell as an even/odd lane pair
// (re, im); the pitch puts those rows on disjoint bank ranges (S = 8: two
// rows 16 banks apart; S = 4: four rows 8 banks apart).
__host__ __device__ constexpr int tile_pitch(int T, int S) { return S == 4 ? T + 4 : T + 8; }

// Accumulate records [beg, end) of one tile's record range into buf
// (interleaved re/im floats, row pitch P cells), by one warp that is the only
// writer of buf: plain FP32 load-add-store in bin order, so no atomics and a
// fixed order of additions.  rng: the tile's bin bounds -- own [0,1) all
// classes, left [2,3), up [4,5), up-left [6,7); a neighbour's records are
// relative to its origin (dx, dy = -T).  The warp stages 32 records at a time
// in shared memory (fractions, W V, footprint start) and walks them: lanes
// 0..S-1 / 16..16+S-1 evaluate the 2S 1-D taps, and the footprint is covered
// 16 cells per instruction, an even/odd lane pair holding the re/im words of
// one cell.
template <bool TABLE, int SS>
__device__ __forceinline__ void accumulate_range(const GridParams& G,
                                                 const VisRecord* __restrict__ records,
                                                 const uint32_t (&rng)[8], uint32_t beg,
                                                 uint32_t end, int k, float* buf, int P,
                                                 const float (&cf)[kPolyDegree + 1],
                                                 float4* stg4, int* stg_ij, float* stg_corr) {
    const int S = SS > 0 ? SS : G.S;
    const int T = G.T;
    constexpr float kInvFrac = 1.0f / 16777216.0f;
    const int lane = threadIdx.x & 31;
    const uint32_t n0 = rng[1] - rng[0], n1 = rng[3] - rng[2], n2 = rng[5] - rng[4];
    const int comp = lane & 1, cl = lane >> 1;       // cell slot 0..15 of a pass
    // tap groups: 32 / 2S records share one tap evaluation; lane (m, q)
    const int S2 = 2 * S, RG = 32 / S2;
    const int m = lane / S2, q = lane - m * S2;
    for (uint32_t base = beg; base < end; base += 32u) {
        const uint32_t g = base + lane;
        if (g < end) {
            uint32_t src;
            int dx = 0, dy = 0;
            if (g < n0) {
                src = rng[0] + g;
            } else if (g < n0 + n1) {
                src = rng[2] + (g - n0);
                dx = -T;
            } else if (g < n0 + n1 + n2) {
                src = rng[4] + (g - n0 - n1);
                dy = -T;
            } else {
                src = rng[6] + (g - n0 - n1 - n2);
                dx = -T;
                dy = -T;
            }
            VisRecord rec = records[src];
            // RICK_DEBUG: the first footprint cell lies in the record's own tile
            // (a corrupt record is dropped; the cell clipping below keeps every
            // access inside the tile in any build)
            if (!RICK_DCHECK((int)(rec.px >> kFracBits) < T && (int)(rec.py >> kFracBits) < T,
                             kCheckRecordCell, G.status)) {
                rec.wv_re = rec.wv_im = 0.f;
                rec.px = rec.py = 0;
            }
            const int i0 = (int)(rec.px >> kFracBits) + dx, j0 = (int)(rec.py >> kFracBits) + dy;
            stg4[lane] = make_float4((float)(rec.px & kFracMask) * kInvFrac,
                                     (float)(rec.py & kFracMask) * kInvFrac, rec.wv_re, rec.wv_im);
            stg_ij[lane] = (i0 + 256) | ((j0 + 256) << 16);
            if (TABLE) {
                // the record's 16 correction taps, interpolated by its own lane:
                // 16 independent 16-byte loads per lane, the 32 records of the
                // batch in parallel (one round trip per batch); row stride 20
                float corr[16];
                table_taps(G, k, (float)(rec.px & kFracMask) * kInvFrac,
                           (float)(rec.py & kFracMask) * kInvFrac, corr);
#pragma unroll
                for (int t = 0; t < 16; t += 4)
                    *reinterpret_cast<float4*>(stg_corr + lane * 20 + t) =
                        make_float4(corr[t], corr[t + 1], corr[t + 2], corr[t + 3]);
            }
        }
        __syncwarp();
        const int cnt = (int)min(32u, end - base);
        // 1-D taps of records r0 .. r0 + RG - 1 in one go: lane (m, q) holds
        // tap q of record r0 + m (x taps q < S, y taps q - S).  The taps of
        // the next group are evaluated while the current group is
        // accumulated, so the Horner chain's latency overlaps that work.
        auto group_taps = [&](int r0) {
            float t = 0.f;
            if (m < RG && r0 + m < cnt) {
                const float4 fm = stg4[r0 + m];
                t = tap_poly(cf, fmaf(2.0f, q < S ? fm.x : fm.y, -1.0f));
            }
            return t;
        };
        float tap_next = group_taps(0);
        for (int r0 = 0; r0 < cnt; r0 += RG) {
            const float tap = tap_next;
            if (r0 + RG < cnt) tap_next = group_taps(r0 + RG);
            const int nr = min(RG, cnt - r0);
            if constexpr (SS == 4) {
                // two records per pass, 16 lanes each (lane = cell 4b + a, both
                // words), when their footprints do not overlap; else one by one
                const int h = lane >> 4, c = lane & 15, a = c & 3, b = c >> 2;
                for (int mm = 0; mm < nr; mm += 2) {
                    const bool pair = mm + 1 < nr;
                    const int ijA = stg_ij[r0 + mm], ijB = pair ? stg_ij[r0 + mm + 1] : ijA;
                    const int dxi = (ijA & 0xffff) - (ijB & 0xffff), dyj = (ijA >> 16) - (ijB >> 16);
                    const bool apart = pair && (dxi >= 4 || dxi <= -4 || dyj >= 4 || dyj <= -4);
                    for (int step = 0; step < 2; ++step) {
                        // step 0: record mm (half 0) and, if apart, mm + 1 (half 1);
                        // step 1: record mm + 1 alone when the two overlap
                        if (step == 1 && (!pair || apart)) break;
                        const int mine = step == 0 ? mm + h : mm + 1;
                        const bool act = step == 0 ? (h == 0 || apart) : h == 1;
                        const int r = r0 + mine;
                        const float4 f = stg4[min(r, cnt - 1)];
                        const int ij = h == 0 ? (step == 0 ? ijA : ijB) : ijB;
                        const int i0 = (ij & 0xffff) - 256, j0 = (ij >> 16) - 256;
                        const float ga = __shfl_sync(kFull, tap, min(mine, RG - 1) * S2 + a);
                        const float gb = __shfl_sync(kFull, tap, min(mine, RG - 1) * S2 + 4 + b);
                        const int i = i0 + a, j = j0 + b;
                        if (act && (unsigned)i < (unsigned)T && (unsigned)j < (unsigned)T) {
                            float g = ga * gb;
                            if (TABLE) g += stg_corr[r * 20 + c];
                            if ((i + j) & 1) g = -g;
                            float2* cp = reinterpret_cast<float2*>(buf) + j * P + i;
                            float2 v = *cp;
                            v.x = fmaf(f.z, g, v.x);
                            v.y = fmaf(f.w, g, v.y);
                            *cp = v;
                        }
                        __syncwarp();
                    }
                }
            } else {
            for (int mm = 0; mm < nr; ++mm) {
                const int r = r0 + mm, tb = mm * S2;
                const float4 f = stg4[r];
                const int ij = stg_ij[r];
                const int i0 = (ij & 0xffff) - 256, j0 = (ij >> 16) - 256;
                if constexpr (SS == 8 && !TABLE) {
                    // a lane owns both words of cell (a, rl + 4 pp), pp = 0, 1:
                    // rows step by 4, so its checkerboard sign and x tap are
                    // fixed for the record; rows rl, rl + 1 are 16 banks apart
                    const int a = lane & 7, rl = lane >> 3;
                    const int i = i0 + a;
                    const bool col_in = (unsigned)i < (unsigned)T;
                    const float ga = __shfl_sync(kFull, tap, tb + a);
                    const float sg = ((i + j0 + rl) & 1) ? -ga : ga;
                    const float gre = sg * f.z, gim = sg * f.w;
                    float2* cell = reinterpret_cast<float2*>(buf) + (j0 + rl) * P + i;
#pragma unroll
                    for (int pp = 0; pp < 2; ++pp) {
                        const int b = rl + 4 * pp;
                        const float gb = __shfl_sync(kFull, tap, tb + 8 + b);
                        if (col_in && (unsigned)(j0 + b) < (unsigned)T) {
                            float2* c = cell + 4 * P * pp;
                            float2 v = *c;
                            v.x = fmaf(gre, gb, v.x);
                            v.y = fmaf(gim, gb, v.y);
                            *c = v;
                        }
                    }
                } else if constexpr (SS == 4 || SS == 8) {
                    // a lane keeps column a and steps kRows (even) rows per pass,
                    // so its checkerboard sign and x tap are fixed for the record
                    constexpr int kRows = 16 / SS;
                    const int a = cl % SS, rl = cl / SS;
                    const int i = i0 + a;
                    const bool col_in = (unsigned)i < (unsigned)T;
                    const float wv = comp ? f.w : f.z;
                    const float ga = __shfl_sync(kFull, tap, tb + a);
                    const float sw = ((i + j0 + rl) & 1) ? -wv : wv;
                    const float gw = sw * ga;
                    float* cell = buf + 2 * ((j0 + rl) * P + i) + comp;
#pragma unroll
                    for (int pp = 0; pp < SS / kRows; ++pp) {
                        const int b = rl + kRows * pp;
                        const float gb = __shfl_sync(kFull, tap, tb + SS + b);
                        if (col_in && (unsigned)(j0 + b) < (unsigned)T) {
                            float* c = cell + 2 * kRows * P * pp;
                            if (TABLE)
                                *c = fmaf(sw, fmaf(ga, gb, stg_corr[r * 20 + 4 * b + a]), *c);
                            else
                                *c = fmaf(gw, gb, *c);
                        }
                    }
                } else {
                    const float wv = comp ? f.w : f.z;
                    const int n16 = (S * S + 15) & ~15;
                    for (int c = cl; c < n16; c += 16) {
                        const int a = c % S, b = min(c / S, S - 1);
                        const float ga = __shfl_sync(kFull, tap, tb + a);
                        const float gb = __shfl_sync(kFull, tap, tb + S + b);
                        const int i = i0 + a, j = j0 + c / S;
                        if (c < S * S && (unsigned)i < (unsigned)T && (unsigned)j < (unsigned)T) {
                            float* cell = buf + 2 * (j * P + i) + comp;
                            *cell = fmaf(((i + j) & 1) ? -wv : wv, ga * gb, *cell);
                        }
                    }
                }
                __syncwarp();
            }
            }
        }
    }
}

// Shared memory of a gridder CTA of nw warps (bytes): one zero row, one
// T x P complex tile per warp, per-warp record staging and chunk bounds.
__host__ __device__ inline size_t grid_smem_bytes(int T, int P, int nw, int grab_max, bool table) {
    return sizeof(float) * (2 * (size_t)T + (size_t)nw * 2 * T * P) +
           (size_t)nw * 32 * (sizeof(float4) + sizeof(int)) +
           sizeof(uint32_t) * (size_t)nw * 9 * grab_max +
           (table ? (size_t)nw * 32 * 20 * sizeof(float) : 0);
}

// The gridder.  work_counter: [0] dense-tile queue, [1..3] list lengths,
// [4] tile queue.
//  Phase 1 -- dense tiles (the first two longest-first lists, >= 16T
//  records), one per CTA: the tile's records are split evenly over the warps,
//  each accumulates its share into its own tile buffer, the buffers are summed
//  in warp order (a fixed order), and the CTA hands the rows to the bulk-copy
//  engine.
//  Phase 2 -- every other tile, one warp per tile: a warp takes `grab` queue
//  positions (the third list, then all tiles in natural order, skipping those
//  already done), accumulates into its own buffer, hands the rows to the
//  bulk-copy engine, waits until the engine has read them and clears the
//  buffer; tiles without records are written from a shared zero row.  No
//  CTA-wide barrier in this phase, so a tile delays only its own warp.
template <bool TABLE, int SS>
__global__ void k_grid(GridParams G, const uint32_t* __restrict__ offsets,
                       const VisRecord* __restrict__ records, float2* __restrict__ grids,
                       uint32_t* __restrict__ work_counter) {
    extern __shared__ __align__(128) float smem[];
    __shared__ uint32_t s_heavy;
    __shared__ uint32_t s_hrng[8];
    const int T = G.T, P = tile_pitch(G.T, SS > 0 ? SS : G.S), N = G.N, NT = G.NT;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    const size_t tile_f = 2 * (size_t)T * P;                       // floats per warp tile
    float2* zrow = reinterpret_cast<float2*>(smem);                 // T zero cells
    float* bufs = smem + 2 * T;
    float* buf = bufs + warp * tile_f;                              // this warp's tile
    float4* stg4_all = reinterpret_cast<float4*>(bufs + nw * tile_f);
    float4* stg4 = stg4_all + warp * 32;
    int* stg_ij = reinterpret_cast<int*>(stg4_all + nw * 32) + warp * 32;
    uint32_t* rng_all = reinterpret_cast<uint32_t*>(reinterpret_cast<int*>(stg4_all + nw * 32) + nw * 32) +
                        warp * 9 * kMaxWarpGrab;
    uint32_t* items = rng_all + 8 * kMaxWarpGrab;
    // learned-kernel staging; 16-byte aligned (the tiles, the zero row and
    // the 928 bytes per warp of record staging and chunk bounds before it are
    // all multiples of 16 bytes), so rows of 20 floats take float4 stores
    float* tbl_base = reinterpret_cast<float*>(rng_all - warp * 9 * kMaxWarpGrab + nw * 9 * kMaxWarpGrab);
    float* stg_corr = TABLE ? tbl_base + warp * 32 * 20 : nullptr;
    const uint32_t tiles = (uint32_t)NT * NT;
    const uint32_t row_bytes = (uint32_t)T * sizeof(float2);
    // this lane's tap polynomial: lane (m, q) of a tap group of 2S lanes
    // evaluates tap q mod S (x taps q < S, y taps q >= S); zero beyond the groups
    float cf[kPolyDegree + 1];
    {
        const int S = SS > 0 ? SS : G.S;
        const int S2 = 2 * S, m = lane / S2, ta = (lane - m * S2) % S;
#pragma unroll
        for (int q = 0; q <= kPolyDegree; ++q) cf[q] = m < 32 / S2 ? G.coef[ta][q] : 0.0f;
    }
    for (int e = threadIdx.x; e < 2 * T; e += blockDim.x) smem[e] = 0.f;
    {
        float4* b4 = reinterpret_cast<float4*>(buf);
        for (int e = lane; e < (int)(tile_f / 4); e += 32) b4[e] = make_float4(0.f, 0.f, 0.f, 0.f);
    }
    fence_async_shared();
    __syncthreads();

    // longest-first lists (if any): their lengths, capped; an overflow (which
    // the capacity bound excludes) falls back to natural order for all tiles
    uint32_t n1 = 0, n2 = 0, n3 = 0, th3 = 0xffffffffu;
    uint32_t n_light = 0;
    bool light = false;   // phase 2 visits the lists only (sparse mode)
    if (G.lists) {
        n1 = __ldg(work_counter + 1);
        n2 = __ldg(work_counter + 2);
        n3 = __ldg(work_counter + 3);
        if (n1 > G.list_cap || n2 > G.list_cap || n3 > G.list_cap) {
            n1 = n2 = n3 = 0;
        } else {
            th3 = 4u * T;
            if (G.light != nullptr && G.skip_empty) {
                n_light = __ldg(work_counter + 5);
                light = n_light <= G.light_cap;
            }
        }
    }

    // ---- phase 1: dense tiles, one per CTA --------------------------------
    const uint32_t nH = n1 + n2;
    auto dense_tiles = [&]() {
    for (;;) {
        if (threadIdx.x == 0) s_heavy = atomicAdd(work_counter, 1u);
        __syncthreads();
        const uint32_t h = s_heavy;
        if (h >= nH) break;
        const uint32_t item = h < n1 ? G.lists[h] : G.lists[G.list_cap + (h - n1)];
        if (!RICK_DCHECK(item < G.n_items, kCheckGridItem, G.status)) {   // uniform over the CTA
            __syncthreads();   // everyone has read s_heavy before thread 0 rewrites it
            continue;
        }
        if (threadIdx.x < 8) s_hrng[threadIdx.x] = tile_bound(G, offsets, item, threadIdx.x);
        __syncthreads();
        uint32_t rng[8];
#pragma unroll
        for (int q = 0; q < 8; ++q) rng[q] = s_hrng[q];
        const uint32_t R = (rng[1] - rng[0]) + (rng[3] - rng[2]) + (rng[5] - rng[4]) + (rng[7] - rng[6]);
        const uint32_t beg = (uint32_t)((uint64_t)R * warp / nw);
        const uint32_t end = (uint32_t)((uint64_t)R * (warp + 1) / nw);
        const uint32_t plane = item / tiles, tile = item - plane * tiles;
        const int kk = (int)(plane % G.nk);
        const int ty = (int)(tile / NT), tx = (int)(tile - (uint32_t)ty * NT);
        float2* out = grids + ((uint64_t)plane * N + (uint64_t)ty * T) * N + (uint64_t)tx * T;
        accumulate_range<TABLE, SS>(G, records, rng, beg, end, G.k0 + kk, buf, P, cf, stg4, stg_ij, stg_corr);
        __syncthreads();
        // sum the warps' tiles into warp 0's in warp order, clearing the others
        {
            float4* t0 = reinterpret_cast<float4*>(bufs);
            for (int e = threadIdx.x; e < (int)(tile_f / 4); e += blockDim.x) {
                float4 acc = t0[e];
                for (int w = 1; w < nw; ++w) {
                    float4* tw = reinterpret_cast<float4*>(bufs + w * tile_f) + e;
                    const float4 v = *tw;
                    acc.x += v.x;
                    acc.y += v.y;
                    acc.z += v.z;
                    acc.w += v.w;
                    *tw = make_float4(0.f, 0.f, 0.f, 0.f);
                }
                t0[e] = acc;
            }
        }
        fence_async_shared();
        __syncthreads();
        for (int r = threadIdx.x; r < T; r += blockDim.x)
            bulk_row_store(out + (size_t)r * N, bufs + 2 * r * P, row_bytes);
        bulk_commit();
        bulk_wait_read();
        __syncthreads();
        {
            float4* t0 = reinterpret_cast<float4*>(bufs);
            for (int e = threadIdx.x; e < (int)(tile_f / 4); e += blockDim.x) t0[e] = make_float4(0.f, 0.f, 0.f, 0.f);
        }
        __syncthreads();
    }
    };

    // ---- phase 2: every other tile, one warp per tile ---------------------
    const uint32_t n_pos = n3 + (light ? n_light : G.n_items);
    auto other_tiles = [&]() {
    for (;;) {
        uint32_t first = 0;
        if (lane == 0) first = atomicAdd(work_counter + 4, G.grab);
        first = __shfl_sync(kFull, first, 0);
        if (first >= n_pos) break;
        const uint32_t n = min(G.grab, n_pos - first);
        // queue positions -> tiles: the third list, then the light list (sparse
        // mode) or every tile in natural order
        if (lane < (int)n) {
            const uint32_t pos = first + lane;
            items[lane] = pos < n3 ? G.lists[2 * (size_t)G.list_cap + pos]
                          : light  ? G.light[pos - n3]
                                   : pos - n3;
        }
        __syncwarp();
        for (uint32_t e = lane; e < 8 * n; e += 32) rng_all[e] = tile_bound(G, offsets, items[e >> 3], e & 7);
        __syncwarp();
        for (uint32_t t = 0; t < n; ++t) {
            const uint32_t item = items[t];
            const uint32_t plane = item / tiles, tile = item - plane * tiles;
            const int kk = (int)(plane % G.nk);
            const int ty = (int)(tile / NT), tx = (int)(tile - (uint32_t)ty * NT);
            float2* out = grids + ((uint64_t)plane * N + (uint64_t)ty * T) * N + (uint64_t)tx * T;
            uint32_t rng[8];
#pragma unroll
            for (int q = 0; q < 8; ++q) rng[q] = rng_all[8 * t + q];
            const uint32_t total = (rng[1] - rng[0]) + (rng[3] - rng[2]) + (rng[5] - rng[4]) +
                                   (rng[7] - rng[6]);
            if (!light && first + t >= n3 && total >= th3) continue;  // taken from a list earlier
            if (total == 0) {
                if (!G.skip_empty) {
                    for (int r = lane; r < T; r += 32) bulk_row_store(out + (size_t)r * N, zrow, row_bytes);
                    bulk_commit();
                }
                continue;
            }
            accumulate_range<TABLE, SS>(G, records, rng, 0u, total, G.k0 + kk, buf, P, cf, stg4, stg_ij, stg_corr);
            fence_async_shared();
            __syncwarp();
            for (int r = lane; r < T; r += 32)
                bulk_row_store(out + (size_t)r * N, buf + 2 * r * P, row_bytes);
            bulk_commit();
            bulk_wait_read();
            __syncwarp();
            // clear the tile for the next one (its rows have been read)
            float4* b4 = reinterpret_cast<float4*>(buf);
            for (int e = lane; e < (int)(tile_f / 4); e += 32) b4[e] = make_float4(0.f, 0.f, 0.f, 0.f);
            __syncwarp();
        }
        __syncwarp();  // rng_all and items are rewritten by the next chunk
    }
    };

    // Half of the CTAs start on the dense tiles and half on the others, so
    // that compute-heavy and store-heavy tiles overlap; each half then helps
    // with the other queue.  Every tile is taken exactly once either way.
    if (blockIdx.x & 1) {
        other_tiles();
        __syncthreads();
        dense_tiles();
    } else {
        dense_tiles();
        other_tiles();
    }
    bulk_wait_all();
}

template <bool TABLE, int SS>
cudaError_t launch_one(const GridParams& G, const uint32_t* offsets, const VisRecord* records,
                       float2* grids, uint32_t* counter, int threads, int num_sms,
                       cudaStream_t stream) {
    const int P = tile_pitch(G.T, SS > 0 ? SS : G.S);
    const int nw = threads / 32;
    const size_t smem = grid_smem_bytes(G.T, P, nw, kMaxWarpGrab, TABLE);
    auto fn = k_grid<TABLE, SS>;
    cudaError_t e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    int per_sm = 0;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, fn, threads, smem);
    if (e != cudaSuccess) return e;
    if (per_sm < 1) return cudaErrorInvalidConfiguration;
    uint64_t blocks = (uint64_t)per_sm * num_sms;
    const uint64_t need = (2ull * G.n_items + (uint64_t)G.grab * nw - 1) / ((uint64_t)G.grab * nw);
    if (blocks > need) blocks = need;
    if (blocks < 1) blocks = 1;
    fn<<<(unsigned)blocks, threads, smem, stream>>>(G, offsets, records, grids, counter);
    return cudaGetLastError();
}

}  // namespace

double fit_tap_polynomials(int kind, double param, int S, GridParams& G) {
    // g(s) for the separable kernels (FP64)
    auto i0 = [](double x) {
        const double y = 0.25 * x * x;
        double term = 1.0, sum = 1.0;
        for (int k = 1; k < 400 && term > 1e-17 * sum; ++k) {
            term *= y / ((double)k * k);
            sum += term;
        }
        return sum;
    };
    const double inv_i0b = kind == RICK_KERNEL_KAISER_BESSEL ? 1.0 / i0(param) : 0.0;
    auto g = [&](double s) {
        if (std::fabs(s) > 0.5 * S) return 0.0;
        if (kind == RICK_KERNEL_GAUSS) return std::exp(-0.5 * s * s / (param * param));
        const double t = 2.0 * s / S;
        return i0(param * std::sqrt(std::fmax(0.0, 1.0 - t * t))) * inv_i0b;
    };
    const double pi = 3.14159265358979323846;
    const int n = kPolyDegree + 1;
    double worst = 0.0;
    for (int a = 0; a < kMaxSupport; ++a)
        for (int k = 0; k <= kPolyDegree; ++k) G.coef[a][k] = 0.0f;
    for (int a = 0; a < S; ++a) {
        // h(t) = g(a + 1 - S/2 - (t + 1)/2), t in [-1, 1]: Chebyshev interpolation at
        // the n Chebyshev points, then conversion to the monomial basis in t.
        auto h = [&](double t) { return g(a + 1 - 0.5 * S - 0.5 * (t + 1.0)); };
        double c[kPolyDegree + 1];
        for (int k = 0; k < n; ++k) {
            double acc = 0.0;
            for (int j = 0; j < n; ++j) {
                const double th = pi * (j + 0.5) / n;
                acc += h(std::cos(th)) * std::cos(k * th);
            }
            c[k] = (k == 0 ? 1.0 : 2.0) * acc / n;
        }
        double mono[kPolyDegree + 1] = {0.0}, tkm1[kPolyDegree + 2] = {0.0},
               tk[kPolyDegree + 2] = {0.0}, tkp1[kPolyDegree + 2];
        tkm1[0] = 1.0;  // T0
        tk[1] = 1.0;    // T1
        mono[0] += c[0];
        if (n > 1) mono[1] += c[1];
        for (int k = 2; k < n; ++k) {
            for (int i = 0; i <= kPolyDegree + 1; ++i) tkp1[i] = -tkm1[i] + (i > 0 ? 2.0 * tk[i - 1] : 0.0);
            for (int i = 0; i <= kPolyDegree; ++i) mono[i] += c[k] * tkp1[i];
            for (int i = 0; i <= kPolyDegree + 1; ++i) {
                tkm1[i] = tk[i];
                tk[i] = tkp1[i];
            }
        }
        for (int k = 0; k <= kPolyDegree; ++k) G.coef[a][k] = (float)mono[k];
        for (int q = 0; q <= 2000; ++q) {
            const float t = (float)(-1.0 + q / 1000.0);
            float acc = G.coef[a][kPolyDegree];
            for (int k = kPolyDegree - 1; k >= 0; --k) acc = std::fmaf(acc, t, G.coef[a][k]);
            worst = std::fmax(worst, std::fabs((double)acc - h((double)t)));
        }
    }
    return worst;
}

cudaError_t launch_grid(const GridParams& G, const uint32_t* offsets, const VisRecord* records,
                        float2* grids, uint32_t* work_counter, int threads, int num_sms,
                        cudaStream_t stream, int* launches) {
    if (G.n_items == 0) return cudaSuccess;
    if (G.grab < 1 || G.grab > (uint32_t)kMaxWarpGrab) return cudaErrorInvalidValue;
    cudaError_t e;
    if (G.lists) {
        const unsigned blocks = (unsigned)std::min<uint64_t>((G.n_items + 255) / 256, (uint64_t)num_sms * 8);
        k_schedule<<<blocks, 256, 0, stream>>>(G, offsets, work_counter + 1);
        e = cudaGetLastError();
        if (e != cudaSuccess) return e;
        ++*launches;
    }
    if (G.kind == RICK_KERNEL_TABLE) {
        e = launch_one<true, 4>(G, offsets, records, grids, work_counter, threads, num_sms, stream);
    } else {
        switch (G.S) {
            case 4: e = launch_one<false, 4>(G, offsets, records, grids, work_counter, threads, num_sms, stream); break;
            case 7: e = launch_one<false, 7>(G, offsets, records, grids, work_counter, threads, num_sms, stream); break;
            case 8: e = launch_one<false, 8>(G, offsets, records, grids, work_counter, threads, num_sms, stream); break;
            default: e = launch_one<false, 0>(G, offsets, records, grids, work_counter, threads, num_sms, stream); break;
        }
    }
    if (e == cudaSuccess) ++*launches;
    return e;
}

}  // namespace rick

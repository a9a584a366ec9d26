// rick_grid.cu -- convolutional gridding onto w-planes (Eq. 3), the "a1" step.
//
// Design (one GB300, HBM-bound): the unit of work is one T x T tile of one
// (channel, w-plane).  A persistent CTA takes tiles from a global counter
// (in chunks), accumulates every visibility that touches the tile into a
// shared-memory subgrid (separate re/im planes with a padded pitch so that
// the S x S footprint of one visibility, spread over the 32 lanes of a warp,
// hits 32 distinct banks), then writes the whole tile to HBM once with
// coalesced 16-byte streaming stores, applying the checkerboard sign.  Tiles
// that no visibility touches are written as zeros without touching shared
// memory.  So every grid cell is written exactly once: the zero fill is fused
// into the gridder and no global atomics are needed, because a tile is owned
// by exactly one CTA (the halo of neighbouring tiles is read, not written --
// the binning stores each visibility once with its halo class).
//
// Kernel taps: separable g(i - x) g(j - y) (Gaussian, Kaiser-Bessel), or the
// learned support-4 kernel: Kaiser-Bessel taps plus a non-separable 4x4
// correction interpolated from a per-plane table.  Each
// lane evaluates the 2S (or 16) taps of one record into a warp-private
// staging area; then the warp walks the 32 records, lanes spread over the
// footprint cells, and adds into shared memory (red.shared.add.f32).
#include <cmath>

#include "rick_internal.cuh"

namespace rick {

namespace {

// g(a + 1 - S/2 - f) for footprint tap a, by Horner in t = 2 f - 1.
template <int SS>
__device__ __forceinline__ float tap_poly(const GridParams& G, int a, float t) {
    float acc = G.coef[a][kPolyDegree];
#pragma unroll
    for (int k = kPolyDegree - 1; k >= 0; --k) acc = fmaf(acc, t, G.coef[a][k]);
    return acc;
}

// Learned taps: bilinear interpolation of the plane's (L+1)^2 x 16 table.
__device__ __forceinline__ void table_taps(const GridParams& G, int k, float fx, float fy,
                                           float* out /* 16, stride 1 */) {
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

// Accumulate records [rb, re) whose coordinates are relative to a tile at
// offset (dx, dy) from this one (0 or -T per axis).
//
// Per warp and batch of 32 records: every lane decodes one record and
// evaluates its 2S separable taps (or its 16 learned taps) into the warp's
// staging area, together with the record's W*V and first cell; then the warp
// walks the batch record by record, each lane owning fixed footprint cells
// (offsets precomputed once), and adds W*V*g into the shared subgrid.  Records
// whose footprint lies inside the tile skip the bounds test.
template <int KIND, int SS>
__device__ __forceinline__ void accumulate_range(const GridParams& G,
                                                 const VisRecord* __restrict__ records,
                                                 uint32_t rb, uint32_t re, int dx, int dy, int k,
                                                 float* s_re, float* s_im, int pitch,
                                                 float* wstage, float4* wmeta, int stg) {
    const int S = SS > 0 ? SS : G.S;
    const int T = G.T;
    const int lane = threadIdx.x & 31;
    const int warp = threadIdx.x >> 5, nwarps = blockDim.x >> 5;
    constexpr float kInvFrac = 1.0f / 16777216.0f;
    constexpr int kTaps = SS * SS;
    constexpr int kPer = SS > 0 ? (kTaps + 31) / 32 : 1;
    // footprint cells owned by this lane (compile-time support only)
    int ta[kPer], tb[kPer], toff[kPer];
    bool tact[kPer];
    if (SS > 0 && kTaps > 16) {
#pragma unroll
        for (int m = 0; m < kPer; ++m) {
            const int t = lane + 32 * m;
            tact[m] = t < kTaps;
            ta[m] = tact[m] ? t % (SS > 0 ? SS : 1) : 0;
            tb[m] = tact[m] ? t / (SS > 0 ? SS : 1) : 0;
            toff[m] = tb[m] * pitch + ta[m];
        }
    }
    for (uint32_t base = rb + 32u * warp; base < re; base += 32u * nwarps) {
        const uint32_t idx = base + lane;
        VisRecord rec = {0.f, 0.f, 0u, 0u};
        if (idx < re) rec = records[idx];
        const int i0 = (int)(rec.px >> kFracBits) + dx;
        const int j0 = (int)(rec.py >> kFracBits) + dy;
        const float fx = (float)(rec.px & kFracMask) * kInvFrac;
        const float fy = (float)(rec.py & kFracMask) * kInvFrac;
        float* my = wstage + lane * stg;
        if (KIND == RICK_KERNEL_TABLE) {
            // learned kernel: Kaiser-Bessel support-4 taps plus the network's
            // correction, interpolated from the plane's lattice
            table_taps(G, k, fx, fy, my);
            const float tx = fmaf(2.0f, fx, -1.0f), ty = fmaf(2.0f, fy, -1.0f);
            float gx[4], gy[4];
#pragma unroll
            for (int a = 0; a < 4; ++a) {
                gx[a] = tap_poly<4>(G, a, tx);
                gy[a] = tap_poly<4>(G, a, ty);
            }
#pragma unroll
            for (int b = 0; b < 4; ++b)
#pragma unroll
                for (int a = 0; a < 4; ++a) my[4 * b + a] += gx[a] * gy[b];
        } else {
            const float tx = fmaf(2.0f, fx, -1.0f), ty = fmaf(2.0f, fy, -1.0f);
#pragma unroll
            for (int a = 0; a < (SS > 0 ? SS : kMaxSupport); ++a) {
                if (SS == 0 && a >= S) break;
                my[a] = tap_poly<SS>(G, a, tx);
                my[S + a] = tap_poly<SS>(G, a, ty);
            }
        }
        const bool inside = i0 >= 0 && j0 >= 0 && i0 + S <= T && j0 + S <= T;
        wmeta[lane] = make_float4(rec.wv_re, rec.wv_im, __int_as_float(j0 * pitch + i0),
                                  __int_as_float((inside ? 1 : 0) | ((i0 + 256) << 1) | ((j0 + 256) << 12)));
        __syncwarp();
        const int n = (int)min(32u, re - base);
        if (SS > 0 && kTaps <= 16) {
            // two records per pass: lanes 0-15 take record r, lanes 16-31 record r+1
            const int t = lane & 15;
            const int a = t % (SS > 0 ? SS : 1), b = t / (SS > 0 ? SS : 1);
            const int off = b * pitch + a;
            for (int r0 = 0; r0 < n; r0 += 2) {
                const int r = r0 + (lane >> 4);
                if (r < n && t < kTaps) {
                    const float4 m4 = wmeta[r];
                    const int cell = __float_as_int(m4.z), bits = __float_as_int(m4.w);
                    const int ri = ((bits >> 1) & 2047) - 256 + a, rj = ((bits >> 12) & 2047) - 256 + b;
                    if ((bits & 1) || ((unsigned)ri < (unsigned)T && (unsigned)rj < (unsigned)T)) {
                        const float* st = wstage + r * stg;
                        const float g = KIND == RICK_KERNEL_TABLE ? st[t] : st[a] * st[SS + b];
                        atomicAdd(&s_re[cell + off], m4.x * g);
                        atomicAdd(&s_im[cell + off], m4.y * g);
                    }
                }
            }
        } else if (SS > 0) {
            for (int r = 0; r < n; ++r) {
                const float4 m4 = wmeta[r];
                const int cell = __float_as_int(m4.z), bits = __float_as_int(m4.w);
                const float* st = wstage + r * stg;
                if (bits & 1) {
#pragma unroll
                    for (int m = 0; m < kPer; ++m) {
                        if (tact[m]) {
                            const float g = st[ta[m]] * st[SS + tb[m]];
                            atomicAdd(&s_re[cell + toff[m]], m4.x * g);
                            atomicAdd(&s_im[cell + toff[m]], m4.y * g);
                        }
                    }
                } else {
                    const int ri0 = ((bits >> 1) & 2047) - 256, rj0 = ((bits >> 12) & 2047) - 256;
#pragma unroll
                    for (int m = 0; m < kPer; ++m) {
                        const int i = ri0 + ta[m], j = rj0 + tb[m];
                        if (tact[m] && (unsigned)i < (unsigned)T && (unsigned)j < (unsigned)T) {
                            const float g = st[ta[m]] * st[SS + tb[m]];
                            atomicAdd(&s_re[cell + toff[m]], m4.x * g);
                            atomicAdd(&s_im[cell + toff[m]], m4.y * g);
                        }
                    }
                }
            }
        } else {
            // runtime support (any S <= 16)
            const int taps = S * S;
            for (int r = 0; r < n; ++r) {
                const float4 m4 = wmeta[r];
                const int bits = __float_as_int(m4.w);
                const int ri0 = ((bits >> 1) & 2047) - 256, rj0 = ((bits >> 12) & 2047) - 256;
                const float* st = wstage + r * stg;
                for (int t = lane; t < taps; t += 32) {
                    const int a = t % S, b = t / S;
                    const int i = ri0 + a, j = rj0 + b;
                    if ((unsigned)i < (unsigned)T && (unsigned)j < (unsigned)T) {
                        const float g = st[a] * st[S + b];
                        atomicAdd(&s_re[j * pitch + i], m4.x * g);
                        atomicAdd(&s_im[j * pitch + i], m4.y * g);
                    }
                }
            }
        }
        __syncwarp();
    }
}

template <int KIND, int SS>
__global__ void k_grid(GridParams G, const uint32_t* __restrict__ offsets,
                       const VisRecord* __restrict__ records, float2* __restrict__ grids,
                       uint32_t* __restrict__ work_counter) {
    extern __shared__ __align__(16) float smem[];
    __shared__ uint32_t s_first;
    const int T = G.T, pitch = T + 8, N = G.N, NT = G.NT;
    float* s_re = smem;
    float* s_im = smem + T * pitch;
    const int stg = KIND == RICK_KERNEL_TABLE ? 17 : 2 * (SS > 0 ? SS : G.S) + 1;
    const int nwarps = blockDim.x >> 5;
    float4* wmeta = reinterpret_cast<float4*>(smem + 2 * T * pitch) + (threadIdx.x >> 5) * 32;
    float* wstage = smem + 2 * T * pitch + 4 * 32 * nwarps + (threadIdx.x >> 5) * 32 * stg;
    const uint32_t tiles = (uint32_t)NT * NT;
    const int half = T / 2;
    const int half_log2 = 31 - __clz(half);  // T is a power of two

    for (;;) {
        if (threadIdx.x == 0) s_first = atomicAdd(work_counter, G.grab);
        __syncthreads();
        const uint32_t first = s_first;
        __syncthreads();
        if (first >= G.n_items) break;
        const uint32_t last = min(first + G.grab, G.n_items);
        for (uint32_t item = first; item < last; ++item) {
            const uint32_t plane = item / tiles, tile = item - plane * tiles;
            const int kk = (int)(plane % G.nk), cc = (int)(plane / G.nk);
            const int c = G.c0 + cc, k = G.k0 + kk;
            const int ty = (int)(tile / NT), tx = (int)(tile - (uint32_t)ty * NT);
            const uint64_t kplane = ((uint64_t)c * G.Nw + k) * NT;
            const uint64_t key = ((kplane + ty) * NT + tx) * 4u;
            // own bins (all classes), left (classes 2-3), up (1-2), up-left (2).
            // Neighbours wrap around the mesh: only the Hermitian fold puts
            // records in the spill classes of the last tile row or column
            // (footprints ending on cell N = cell 0); without it those bins
            // are empty.
            const int txl = tx > 0 ? tx - 1 : NT - 1, tyu = ty > 0 ? ty - 1 : NT - 1;
            const uint64_t kl = ((kplane + ty) * NT + txl) * 4u;
            const uint64_t ku = ((kplane + tyu) * NT + tx) * 4u;
            const uint64_t kd = ((kplane + tyu) * NT + txl) * 4u;
            const uint32_t o0 = __ldg(offsets + key), o4 = __ldg(offsets + key + 4);
            const uint32_t l2 = __ldg(offsets + kl + 2), l4 = __ldg(offsets + kl + 4);
            const uint32_t u1 = __ldg(offsets + ku + 1), u3 = __ldg(offsets + ku + 3);
            const uint32_t d2 = __ldg(offsets + kd + 2), d3 = __ldg(offsets + kd + 3);
            const uint32_t total = (o4 - o0) + (l4 - l2) + (u3 - u1) + (d3 - d2);
            float2* out = grids + ((uint64_t)plane * N + (uint64_t)ty * T) * N + (uint64_t)tx * T;
            if (total == 0) {
                const float4 z = make_float4(0.f, 0.f, 0.f, 0.f);
                for (int e = threadIdx.x; e < T * half; e += blockDim.x) {
                    const int j = e >> half_log2, i = (e & (half - 1)) << 1;
                    __stcs(reinterpret_cast<float4*>(out + (size_t)j * N + i), z);
                }
                continue;
            }
            {
                float4* s4 = reinterpret_cast<float4*>(smem);
                const int n4 = (2 * T * pitch) / 4;
                const float4 z = make_float4(0.f, 0.f, 0.f, 0.f);
                for (int e = threadIdx.x; e < n4; e += blockDim.x) s4[e] = z;
            }
            __syncthreads();
            accumulate_range<KIND, SS>(G, records, o0, o4, 0, 0, k, s_re, s_im, pitch, wstage, wmeta, stg);
            if (l4 > l2)
                accumulate_range<KIND, SS>(G, records, l2, l4, -T, 0, k, s_re, s_im, pitch, wstage, wmeta, stg);
            if (u3 > u1)
                accumulate_range<KIND, SS>(G, records, u1, u3, 0, -T, k, s_re, s_im, pitch, wstage, wmeta, stg);
            if (d3 > d2)
                accumulate_range<KIND, SS>(G, records, d2, d3, -T, -T, k, s_re, s_im, pitch, wstage, wmeta, stg);
            __syncthreads();
            for (int e = threadIdx.x; e < T * half; e += blockDim.x) {
                const int j = e >> half_log2, i = (e & (half - 1)) << 1;
                const float2 re = *reinterpret_cast<const float2*>(s_re + j * pitch + i);
                const float2 im = *reinterpret_cast<const float2*>(s_im + j * pitch + i);
                const float sg = (j & 1) ? -1.f : 1.f;  // (-1)^(i+j), i even, T even
                __stcs(reinterpret_cast<float4*>(out + (size_t)j * N + i),
                       make_float4(sg * re.x, sg * im.x, -sg * re.y, -sg * im.y));
            }
            __syncthreads();
        }
    }
}

template <int KIND, int SS>
cudaError_t launch_one(const GridParams& G, const uint32_t* offsets, const VisRecord* records,
                       float2* grids, uint32_t* counter, int threads, int num_sms,
                       cudaStream_t stream) {
    const int stg = KIND == RICK_KERNEL_TABLE ? 17 : 2 * (SS > 0 ? SS : G.S) + 1;
    const size_t smem =
        sizeof(float) * ((size_t)2 * G.T * (G.T + 8) + (size_t)(threads / 32) * 32 * (stg + 4));
    auto fn = k_grid<KIND, SS>;
    cudaError_t e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    int per_sm = 0;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, fn, threads, smem);
    if (e != cudaSuccess) return e;
    if (per_sm < 1) return cudaErrorInvalidConfiguration;
    uint64_t blocks = (uint64_t)per_sm * num_sms;
    const uint64_t need = (G.n_items + G.grab - 1) / G.grab;
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
    cudaError_t e;
    if (G.kind == RICK_KERNEL_TABLE) {
        e = launch_one<RICK_KERNEL_TABLE, 4>(G, offsets, records, grids, work_counter, threads,
                                             num_sms, stream);
    } else if (G.kind == RICK_KERNEL_GAUSS) {
        switch (G.S) {
            case 4: e = launch_one<RICK_KERNEL_GAUSS, 4>(G, offsets, records, grids, work_counter, threads, num_sms, stream); break;
            case 7: e = launch_one<RICK_KERNEL_GAUSS, 7>(G, offsets, records, grids, work_counter, threads, num_sms, stream); break;
            case 8: e = launch_one<RICK_KERNEL_GAUSS, 8>(G, offsets, records, grids, work_counter, threads, num_sms, stream); break;
            default: e = launch_one<RICK_KERNEL_GAUSS, 0>(G, offsets, records, grids, work_counter, threads, num_sms, stream); break;
        }
    } else {
        switch (G.S) {
            case 4: e = launch_one<RICK_KERNEL_KAISER_BESSEL, 4>(G, offsets, records, grids, work_counter, threads, num_sms, stream); break;
            case 7: e = launch_one<RICK_KERNEL_KAISER_BESSEL, 7>(G, offsets, records, grids, work_counter, threads, num_sms, stream); break;
            case 8: e = launch_one<RICK_KERNEL_KAISER_BESSEL, 8>(G, offsets, records, grids, work_counter, threads, num_sms, stream); break;
            default: e = launch_one<RICK_KERNEL_KAISER_BESSEL, 0>(G, offsets, records, grids, work_counter, threads, num_sms, stream); break;
        }
    }
    if (e == cudaSuccess) ++*launches;
    return e;
}

}  // namespace rick

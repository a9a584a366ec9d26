// rick_fft.cu -- the 2-D DFTs of the w-planes in two passes over HBM.
//
// Eq. 2 needs, per plane, F_k[q][p] = sum_{i,j} G_k[j][i] e^{+2 pi i (i p + j q)/N}
// (unnormalised); the prediction needs the same with e^{-...}.  The 2-D DFT is
// a length-N DFT down every column followed by one along every row:
//   pass 1 (k_fft_columns): one CTA transforms COLS adjacent columns of a plane
//     in shared memory (rows of COLS x 8 bytes are read and written back);
//   pass 2 (k_fft_rows): one CTA transforms one row, in place; or, for imaging,
//     k_rows_phase_reduce: one CTA owns one image row q, transforms that row of
//     every plane of every channel of the launch, applies the phase screen
//     exp(+2 pi i w_k (n - 1)) and sums the planes in registers, so that the
//     transformed planes are never written back (Eq. 2's reduction fused into
//     the transform).
// Every plane is therefore read twice and written once (24 B per cell) on the
// imaging path, against one read and one write per pass of a generic 2-D FFT
// plus the reduction's read.
//
// The length-N DFT (N = 2^m, 256 <= N <= 8192) is a Stockham decimation-in-
// frequency transform with radix-16 stages and, where m is not a multiple of
// 4, one last stage of radix 2, 4 or 8.  With M the product of the radices of
// the previous stages and L = N/M, a radix-R stage takes butterfly u = t1 M + g
// (t1 < L/R, g < M) from positions u + (N/R) t2, t2 < R, computes the length-R
// DFT, multiplies output f0 by W_L^(t1 f0) = W_N^(t1 f0 M), W_N = e^(+-2 pi i/N),
// and stores it at t1 M R + g + M f0; after the last stage the array is in
// natural order.  N/16 threads transform one array: one radix-16 butterfly per
// thread per stage (16/R butterflies of the last radix-R stage).  Thread b
// therefore ends with the outputs b + (N/16) j, j < 16, in registers.
//
// Pruning: planes made by the library's gridder are zero in every column tile
// that no visibility reached and in every plane no visibility reached.  Given
// the occupancy of the current binning (launch_occupancy: per plane and tile
// column, from the bin offsets), the column pass skips the empty column tiles
// (their DFT is zero, and they already hold zeros) and the fused row pass skips
// the empty planes (they add nothing) -- the same result with less work.
//
// Shared arrays are indexed through skew(a) = a + a/16, which spreads the
// stride-16 stores of the first stages over all banks.  Twiddles come from two
// tables of e^(+2 pi i e/N) rounded from FP64 on the host, e = 64 eh + el:
// W = T_hi[eh] T_lo[el] (conjugated for the forward transform).
#include <cmath>
#include <vector>

#include "rick_internal.cuh"

namespace rick {

namespace {

// cos(2 pi k / 32) for 0 <= k <= 8, from the values of cos(pi k / 16)
__host__ __device__ constexpr float quarter32(int k) {
    return k == 0 ? 1.0f
         : k == 1 ? 0.98078528040323044913f
         : k == 2 ? 0.92387953251128675613f
         : k == 3 ? 0.83146961230254523708f
         : k == 4 ? 0.70710678118654752440f
         : k == 5 ? 0.55557023301960222474f
         : k == 6 ? 0.38268343236508977173f
         : k == 7 ? 0.19509032201612826785f
         : 0.0f;
}

__host__ __device__ constexpr float cos32(int k) {
    return (k & 31) <= 8    ? quarter32(k & 31)
         : (k & 31) <= 16 ? -quarter32(16 - (k & 31))
         : (k & 31) <= 24 ? -quarter32((k & 31) - 16)
                            : quarter32(32 - (k & 31));
}

__host__ __device__ constexpr float sin32(int k) { return cos32(k - 8); }

__device__ __forceinline__ float2 cadd(float2 a, float2 b) { return make_float2(a.x + b.x, a.y + b.y); }
__device__ __forceinline__ float2 csub(float2 a, float2 b) { return make_float2(a.x - b.x, a.y - b.y); }
__device__ __forceinline__ float2 cmulf(float2 a, float2 b) {
    return make_float2(fmaf(a.x, b.x, -a.y * b.y), fmaf(a.x, b.y, a.y * b.x));
}
// a * (s i), s = +1 (INV) or -1
template <bool INV>
__device__ __forceinline__ float2 mul_si(float2 a) {
    return INV ? make_float2(-a.y, a.x) : make_float2(a.y, -a.x);
}

// v * e^(s 2 pi i e / R) for compile-time e and R <= 32 (after unrolling), s = +1 (INV) or -1
template <bool INV>
__device__ __forceinline__ float2 twiddle_const(float2 v, int e, int R) {
    const int k = (e * (32 / R)) & 31;   // in 32nds of a turn
    if (k == 0) return v;
    if (k == 8) return mul_si<INV>(v);
    if (k == 16) return make_float2(-v.x, -v.y);
    if (k == 24) return mul_si<!INV>(v);
    const float c = cos32(k), s = INV ? sin32(k) : -sin32(k);
    return make_float2(fmaf(v.x, c, -v.y * s), fmaf(v.x, s, v.y * c));
}

// In-register length-R DFT, X[f] = sum_t a[t] e^(s 2 pi i t f / R), natural order.
template <int R, bool INV>
struct Dft;

template <bool INV>
struct Dft<2, INV> {
    static __device__ __forceinline__ void run(float2* a) {
        const float2 x = a[0], y = a[1];
        a[0] = cadd(x, y);
        a[1] = csub(x, y);
    }
};

template <bool INV>
struct Dft<4, INV> {
    static __device__ __forceinline__ void run(float2* a) {
        const float2 t0 = cadd(a[0], a[2]), t1 = csub(a[0], a[2]);
        const float2 t2 = cadd(a[1], a[3]), t3 = mul_si<INV>(csub(a[1], a[3]));
        a[0] = cadd(t0, t2);
        a[2] = csub(t0, t2);
        a[1] = cadd(t1, t3);
        a[3] = csub(t1, t3);
    }
};

// R = 4 S: X[f0 + 4 f1] = sum_{t1 < S} W_S^(t1 f1) [W_R^(t1 f0) sum_{t2 < 4} a[t1 + S t2] W_4^(t2 f0)]
template <int R, bool INV>
struct Dft {
    static_assert(R == 8 || R == 16 || R == 32, "radix");
    static constexpr int S = R / 4;
    static __device__ __forceinline__ void run(float2* a) {
        float2 y[R];  // y[f0 S + t1]
#pragma unroll
        for (int t1 = 0; t1 < S; ++t1) {
            float2 b[4] = {a[t1], a[t1 + S], a[t1 + 2 * S], a[t1 + 3 * S]};
            Dft<4, INV>::run(b);
#pragma unroll
            for (int f0 = 0; f0 < 4; ++f0) y[f0 * S + t1] = twiddle_const<INV>(b[f0], t1 * f0, R);
        }
#pragma unroll
        for (int f0 = 0; f0 < 4; ++f0) {
            Dft<S, INV>::run(y + f0 * S);
#pragma unroll
            for (int f1 = 0; f1 < S; ++f1) a[f0 + 4 * f1] = y[f0 * S + f1];
        }
    }
};

__device__ __forceinline__ int skew(int a) { return a + (a >> 4); }

template <int LOG2N>
struct Shape {
    static constexpr int N = 1 << LOG2N;
    static constexpr int T = N / 16;                 // threads per transform
    static constexpr int kR16 = LOG2N / 4;            // radix-16 stages
    static constexpr int kLastR = 1 << (LOG2N % 4);   // 1: the last stage is radix 16
    static constexpr int kArray = N + N / 16;         // skewed array length
    static constexpr int kHi = N / 64;                // twiddle tables
    static constexpr int kTw = kHi + 64;
    static_assert(LOG2N >= 8 && LOG2N <= 13, "256 <= N <= 8192");
};

// W_N^e (e < N) from the two tables, conjugated for the forward transform
template <bool INV>
__device__ __forceinline__ float2 twiddle(const float2* th, const float2* tl, int e) {
    float2 w = cmulf(th[e >> 6], tl[e & 63]);
    if (!INV) w.y = -w.y;
    return w;
}

// Radix-16 stage with M = 2^log2M (not the last stage): a holds the butterfly's
// inputs u + (N/16) t2 for u = b; the DFT, twiddles W_N^(t1 f0 M) and the
// stores t1 16 M + g + M f0 into buf.
template <int LOG2N, bool INV>
__device__ __forceinline__ void radix16_out(float2 (&a)[16], int b, int log2M, float2* buf,
                                            const float2* th, const float2* tl) {
    Dft<16, INV>::run(a);
    const int M = 1 << log2M;
    const int t1 = b >> log2M, g = b & (M - 1);
    const int base = (t1 << (log2M + 4)) + g;
    buf[skew(base)] = a[0];
    if (t1 == 0) {
#pragma unroll
        for (int f0 = 1; f0 < 16; ++f0) buf[skew(base + M * f0)] = a[f0];
    } else {
        const int e1 = t1 << log2M;
#pragma unroll
        for (int f0 = 1; f0 < 16; ++f0)
            buf[skew(base + M * f0)] = cmulf(a[f0], twiddle<INV>(th, tl, e1 * f0));
    }
}

// The middle radix-16 stages (all but the first, which starts from registers,
// and the last) on buf, in place: loads, barrier, compute and stores, barrier.
template <int LOG2N, bool INV>
__device__ __forceinline__ void middle_stages(float2* buf, int b, const float2* th, const float2* tl) {
    using Sh = Shape<LOG2N>;
    constexpr int kMiddle = Sh::kLastR == 1 ? Sh::kR16 - 2 : Sh::kR16 - 1;
#pragma unroll
    for (int s = 1; s <= kMiddle; ++s) {
        float2 a[16];
#pragma unroll
        for (int t2 = 0; t2 < 16; ++t2) a[t2] = buf[skew(b + Sh::T * t2)];
        __syncthreads();
        radix16_out<LOG2N, INV>(a, b, 4 * s, buf, th, tl);
        __syncthreads();
    }
}

// The last stage (radix kLastR, or 16), M = N/R, no twiddles: x[j] = X[b + (N/16) j].
template <int LOG2N, bool INV>
__device__ __forceinline__ void last_stage(const float2* buf, int b, float2 (&x)[16]) {
    using Sh = Shape<LOG2N>;
    constexpr int R = Sh::kLastR == 1 ? 16 : Sh::kLastR;
    constexpr int NB = 16 / R;          // butterflies per thread
    constexpr int M = Sh::N / R;
#pragma unroll
    for (int i = 0; i < NB; ++i) {
        float2 a[R];
        const int u = b + Sh::T * i;
#pragma unroll
        for (int t2 = 0; t2 < R; ++t2) a[t2] = buf[skew(u + M * t2)];
        Dft<R, INV>::run(a);
        // output u + M f0 = b + T (i + NB f0)
#pragma unroll
        for (int f0 = 0; f0 < R; ++f0) x[i + NB * f0] = a[f0];
    }
}

// One whole transform of the array whose first stage inputs a[t2] = x[b + T t2]
// are in registers; on return x[j] = X[b + T j].  buf is free on entry and
// holds the last stage's input on return (a barrier is needed before reuse).
template <int LOG2N, bool INV>
__device__ __forceinline__ void transform(float2 (&a)[16], float2* buf, int b, const float2* th,
                                          const float2* tl, float2 (&x)[16]) {
    radix16_out<LOG2N, INV>(a, b, 0, buf, th, tl);
    __syncthreads();
    middle_stages<LOG2N, INV>(buf, b, th, tl);
    last_stage<LOG2N, INV>(buf, b, x);
}

template <int LOG2N>
__device__ __forceinline__ void load_tables(const float2* __restrict__ twid, float2* th, int tid, int nthreads) {
    for (int i = tid; i < Shape<LOG2N>::kTw; i += nthreads) th[i] = __ldg(twid + i);
}

// ---- pass 1: columns ----------------------------------------------------------

// COLS adjacent columns of one plane per CTA (COLS * N/16 threads); rows of
// COLS * 8 bytes are read with 16-byte loads into COLS skewed arrays,
// transformed, and written back the same way.
template <int LOG2N, int COLS, bool INV>
__global__ void __launch_bounds__(COLS * (1 << LOG2N) / 16)
k_fft_columns(float2* __restrict__ grids, const float2* __restrict__ twid, OccMask occ, int64_t plane0) {
    using Sh = Shape<LOG2N>;
    constexpr int N = Sh::N, T = Sh::T;
    // a column tile that no visibility reached is zero: skip it
    if (occ.col != nullptr &&
        occ.col[(plane0 + blockIdx.y) * occ.NT + (int)(blockIdx.x * COLS) / occ.T] == 0)
        return;
    constexpr int kThreads = COLS * T;
    constexpr int kVec = COLS / 2;   // 16-byte pieces per row
    extern __shared__ __align__(16) float2 fsm[];
    float2* th = fsm;
    float2* tl = th + Sh::kHi;
    float2* arrays = fsm + Sh::kTw;
    const int tid = threadIdx.x;
    const int c = tid / T, b = tid - c * T;
    float2* buf = arrays + c * Sh::kArray;
    float2* plane = grids + (size_t)blockIdx.y * N * N + (size_t)blockIdx.x * COLS;
    load_tables<LOG2N>(twid, th, tid, kThreads);
#pragma unroll 4
    for (int e = tid; e < N * kVec; e += kThreads) {
        const int row = e / kVec, piece = e - row * kVec;
        const float4 v = __ldcs(reinterpret_cast<const float4*>(plane + (size_t)row * N) + piece);
        arrays[(2 * piece) * Sh::kArray + skew(row)] = make_float2(v.x, v.y);
        arrays[(2 * piece + 1) * Sh::kArray + skew(row)] = make_float2(v.z, v.w);
    }
    __syncthreads();
    float2 a[16], x[16];
#pragma unroll
    for (int t2 = 0; t2 < 16; ++t2) a[t2] = buf[skew(b + T * t2)];
    __syncthreads();
    transform<LOG2N, INV>(a, buf, b, th, tl, x);
    __syncthreads();
#pragma unroll
    for (int j = 0; j < 16; ++j) buf[skew(b + T * j)] = x[j];
    __syncthreads();
#pragma unroll 4
    for (int e = tid; e < N * kVec; e += kThreads) {
        const int row = e / kVec, piece = e - row * kVec;
        const float2 lo = arrays[(2 * piece) * Sh::kArray + skew(row)];
        const float2 hi = arrays[(2 * piece + 1) * Sh::kArray + skew(row)];
        __stcs(reinterpret_cast<float4*>(plane + (size_t)row * N) + piece, make_float4(lo.x, lo.y, hi.x, hi.y));
    }
}

// ---- pass 2: rows ---------------------------------------------------------------

// One row (blockIdx.x) of one plane (blockIdx.y) per CTA, in place.
template <int LOG2N, bool INV>
__global__ void __launch_bounds__((1 << LOG2N) / 16)
k_fft_rows(float2* __restrict__ grids, const float2* __restrict__ twid) {
    using Sh = Shape<LOG2N>;
    constexpr int N = Sh::N, T = Sh::T;
    extern __shared__ __align__(16) float2 fsm[];
    float2* th = fsm;
    float2* tl = th + Sh::kHi;
    float2* buf = fsm + Sh::kTw;
    const int b = threadIdx.x;
    float2* row = grids + (size_t)blockIdx.y * N * N + (size_t)blockIdx.x * N;
    load_tables<LOG2N>(twid, th, b, T);
    float2 a[16], x[16];
#pragma unroll
    for (int t2 = 0; t2 < 16; ++t2) a[t2] = __ldcs(row + b + T * t2);
    __syncthreads();
    transform<LOG2N, INV>(a, buf, b, th, tl, x);
#pragma unroll
    for (int j = 0; j < 16; ++j) __stcs(row + b + T * j, x[j]);
}

__device__ __forceinline__ uint32_t turns_q32(double t) {
    const double f = t - floor(t);  // [0, 1)
    return (uint32_t)__double2ull_rz(f * 4294967296.0);
}

__device__ __forceinline__ uint32_t turns_q32f(float t) {
    const float f = t - floorf(t);
    return (uint32_t)__float2ull_rz(f * 4294967296.0f);
}

// Imaging, pass 2 fused with Eq. 2's phase screen and reduction: image row q
// (blockIdx.x) of every channel of the launch,
//   image[c][q][p] += (-1)^(p+q) n C_w^-1 / (sum W_c C(p) C(q))
//                     * Re sum_k F_k[q][p] exp(+2 pi i w_k (n - 1)),
// where F_k[q][.] is the row DFT of the column-transformed plane k.  Thread b
// owns pixels p = b + (N/16) j; their phases t_k = w_k (n - 1) in turns are
// Q0.32 fixed point (FP64 once per pixel for t_0 and dt, kept in shared
// memory, then t_0 + k dt exact mod one turn), one sincospi per pixel and
// plane.  The next row is loaded into registers while the current one is
// transformed.  Two CTAs per SM for N <= 4096 (at most 128 registers).
template <int LOG2N, int PREC, bool COMPLEX_OUT>
__global__ void __launch_bounds__((1 << LOG2N) / 16, LOG2N <= 12 ? 2 : 1)
k_rows_phase_reduce(PhaseParams P, const float2* __restrict__ grids, const double* __restrict__ wsum,
                    const float* __restrict__ inv_taper, const float2* __restrict__ twid,
                    float* __restrict__ image_real, float2* __restrict__ image_complex,
                    const uint8_t* __restrict__ plane_occ) {
    using Sh = Shape<LOG2N>;
    constexpr int N = Sh::N, T = Sh::T;
    extern __shared__ __align__(16) float2 fsm[];
    float2* th = fsm;
    float2* tl = th + Sh::kHi;
    float2* buf = fsm + Sh::kTw;
    uint2* phase = reinterpret_cast<uint2*>(buf + Sh::kArray);   // (t_0, dt) per pixel
    float* scl = reinterpret_cast<float*>(phase + N);
    const int b = threadIdx.x, q = blockIdx.x;
    const int halfN = N / 2;
    load_tables<LOG2N>(twid, th, b, T);

#pragma unroll 1
    for (int j = 0; j < 16; ++j) {
        const int p = b + T * j;
        const double l = (double)(p - halfN) * P.dl, m = (double)(q - halfN) * P.dl;
        const double r2 = l * l + m * m;
        const double n = sqrt(1.0 - r2);
        const double delta = -r2 / (1.0 + n);
        if (PREC == RICK_PREC_ALL_FP32) {
            const float lf = (float)(p - halfN) * (float)P.dl, mf = (float)(q - halfN) * (float)P.dl;
            const float r2f = lf * lf + mf * mf;
            const float df = -r2f / (1.0f + sqrtf(1.0f - r2f));
            phase[p] = make_uint2(turns_q32f((float)P.w_first * df), turns_q32f((float)P.dw * df));
        } else {
            phase[p] = make_uint2(turns_q32(P.w_first * delta), turns_q32(P.dw * delta));
        }
        const float sg = ((p + q) & 1) ? -1.f : 1.f;
        scl[p] = sg * (float)n * inv_taper[p] * inv_taper[q] * w_taper_inv(P, delta);
    }

    const size_t NN = (size_t)N * N;
    const int n_rows = P.nc * P.nk;
    // planes no visibility reached (plane_occ == 0) are skipped
    auto next_row = [&](int r) {
        if (plane_occ != nullptr)
            while (r < n_rows && plane_occ[r] == 0) ++r;
        return r;
    };
    float2 a[16], x[16];
    int r = next_row(0);
    if (r < n_rows) {
        const float2* row = grids + (size_t)r * NN + (size_t)q * N;
#pragma unroll
        for (int t2 = 0; t2 < 16; ++t2) a[t2] = __ldcs(row + b + T * t2);
    }
    __syncthreads();
    for (int cc = 0; cc < P.nc; ++cc) {
        float acc[16], acci[16];
#pragma unroll
        for (int j = 0; j < 16; ++j) acc[j] = acci[j] = 0.f;
        for (int kk = 0; kk < P.nk; ++kk) {
            if (cc * P.nk + kk != r) continue;   // an empty plane
            radix16_out<LOG2N, true>(a, b, 0, buf, th, tl);
            const int rn = next_row(r + 1);
            if (rn < n_rows) {
                const float2* row = grids + (size_t)rn * NN + (size_t)q * N;
#pragma unroll
                for (int t2 = 0; t2 < 16; ++t2) a[t2] = __ldcs(row + b + T * t2);
            }
            r = rn;
            __syncthreads();
            middle_stages<LOG2N, true>(buf, b, th, tl);
            last_stage<LOG2N, true>(buf, b, x);
            __syncthreads();   // buf is rewritten by the next row's first stage
#pragma unroll
            for (int j = 0; j < 16; ++j) {
                const uint2 ph = phase[b + T * j];
                const uint32_t tk = ph.x + (uint32_t)kk * ph.y;
                float s, c;
                sincospif((float)(int32_t)tk * 4.656612873077392578125e-10f /* 2^-31 */, &s, &c);
                acc[j] = fmaf(x[j].x, c, fmaf(-x[j].y, s, acc[j]));
                if (COMPLEX_OUT) acci[j] = fmaf(x[j].x, s, fmaf(x[j].y, c, acci[j]));
            }
        }
        const double ws = wsum[cc];
        const float inv_ws = ws != 0.0 ? (float)(1.0 / ws) : 0.0f;
        float* ir = image_real + (size_t)cc * NN + (size_t)q * N;
#pragma unroll
        for (int j = 0; j < 16; ++j) {
            const int p = b + T * j;
            const float s = scl[p] * inv_ws;
            ir[p] += s * acc[j];
            if (COMPLEX_OUT) {
                float2* ic = image_complex + (size_t)cc * NN + (size_t)q * N + p;
                float2 v = *ic;
                v.x += s * acc[j];
                v.y += s * acci[j];
                *ic = v;
            }
        }
    }
}

constexpr int kCols = 2;   // columns per CTA in pass 1

// occupancy of plane p (p = cc nk + kk of the launch) and its tile columns
// from the bin offsets: a tile column is reached if any of its tiles holds a
// record, or a tile to its left holds a record that spills right (halo classes
// 2 and 3; the column after the last wraps to column 0, which only the
// Hermitian fold's mirrored footprints reach).
__global__ void k_occupancy(const uint32_t* __restrict__ offsets, int c0, int nc, int k0, int nk,
                            int Nw_store, int NT, uint8_t* __restrict__ col, uint8_t* __restrict__ plane) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= (int64_t)nc * nk * NT) return;
    const int tx = (int)(i % NT);
    const int64_t p = i / NT;
    const int cc = (int)(p / nk), kk = (int)(p - (int64_t)cc * nk);
    const int txl = (tx + NT - 1) % NT;
    const uint64_t pk = ((uint64_t)(c0 + cc) * Nw_store + (k0 + kk)) * NT;
    uint32_t any = 0;
    for (int ty = 0; ty < NT && !any; ++ty) {
        const uint64_t own = ((pk + ty) * NT + tx) * 4, left = ((pk + ty) * NT + txl) * 4;
        any |= __ldg(offsets + own + 4) - __ldg(offsets + own);     // all classes of the tile
        any |= __ldg(offsets + left + 4) - __ldg(offsets + left + 2);  // classes 2, 3 of the left tile
    }
    col[i] = any ? 1 : 0;
    if (any) plane[p] = 1;
}

template <int LOG2N, bool INV>
cudaError_t columns_one(float2* grids, int64_t n_planes, const float2* twid, OccMask occ, cudaStream_t st) {
    using Sh = Shape<LOG2N>;
    auto fn = k_fft_columns<LOG2N, kCols, INV>;
    const size_t smem = (size_t)(Sh::kTw + kCols * Sh::kArray) * sizeof(float2);
    cudaError_t e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    for (int64_t p0 = 0; p0 < n_planes; p0 += 65535) {
        const unsigned np = (unsigned)(n_planes - p0 < 65535 ? n_planes - p0 : 65535);
        fn<<<dim3(Sh::N / kCols, np), kCols * Sh::T, smem, st>>>(grids + p0 * Sh::N * Sh::N, twid, occ, p0);
        if ((e = cudaGetLastError()) != cudaSuccess) return e;
    }
    return cudaSuccess;
}

template <int LOG2N, bool INV>
cudaError_t rows_one(float2* grids, int64_t n_planes, const float2* twid, cudaStream_t st) {
    using Sh = Shape<LOG2N>;
    auto fn = k_fft_rows<LOG2N, INV>;
    const size_t smem = (size_t)(Sh::kTw + Sh::kArray) * sizeof(float2);
    cudaError_t e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    for (int64_t p0 = 0; p0 < n_planes; p0 += 65535) {
        const unsigned np = (unsigned)(n_planes - p0 < 65535 ? n_planes - p0 : 65535);
        fn<<<dim3(Sh::N, np), Sh::T, smem, st>>>(grids + p0 * Sh::N * Sh::N, twid);
        if ((e = cudaGetLastError()) != cudaSuccess) return e;
    }
    return cudaSuccess;
}

template <int LOG2N, int PREC, bool CPLX>
cudaError_t fused_one(const PhaseParams& P, const float2* grids, const double* wsum, const float* inv_taper,
                      const float2* twid, float* image_real, float2* image_complex, const uint8_t* pocc,
                      cudaStream_t st) {
    using Sh = Shape<LOG2N>;
    auto fn = k_rows_phase_reduce<LOG2N, PREC, CPLX>;
    const size_t smem = (size_t)(Sh::kTw + Sh::kArray) * sizeof(float2) +
                        (size_t)Sh::N * (sizeof(uint2) + sizeof(float));
    cudaError_t e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    fn<<<Sh::N, Sh::T, smem, st>>>(P, grids, wsum, inv_taper, twid, image_real, image_complex, pocc);
    return cudaGetLastError();
}

template <int LOG2N>
cudaError_t fused_n(const PhaseParams& P, const float2* grids, const double* wsum, const float* inv_taper,
                    const float2* twid, float* image_real, float2* image_complex, const uint8_t* pocc,
                    cudaStream_t st) {
    const bool c = image_complex != nullptr;
    if (P.precision == RICK_PREC_ALL_FP32)
        return c ? fused_one<LOG2N, RICK_PREC_ALL_FP32, true>(P, grids, wsum, inv_taper, twid, image_real, image_complex, pocc, st)
                 : fused_one<LOG2N, RICK_PREC_ALL_FP32, false>(P, grids, wsum, inv_taper, twid, image_real, image_complex, pocc, st);
    return c ? fused_one<LOG2N, RICK_PREC_FP32_FP64IDX, true>(P, grids, wsum, inv_taper, twid, image_real, image_complex, pocc, st)
             : fused_one<LOG2N, RICK_PREC_FP32_FP64IDX, false>(P, grids, wsum, inv_taper, twid, image_real, image_complex, pocc, st);
}

int log2_exact(int N) {
    int m = 0;
    while ((1 << m) < N) ++m;
    return (1 << m) == N ? m : -1;
}

}  // namespace

bool fft_supported(int N) {
    const int m = log2_exact(N);
    return m >= 8 && m <= 13;
}

void fft_twiddles(int N, std::vector<float2>& out) {
    const int hi = N / 64;
    out.resize((size_t)hi + 64);
    const double two_pi = 6.283185307179586476925;
    for (int i = 0; i < hi; ++i) {
        const double a = two_pi * (64.0 * i) / N;
        out[i] = make_float2((float)std::cos(a), (float)std::sin(a));
    }
    for (int i = 0; i < 64; ++i) {
        const double a = two_pi * i / N;
        out[hi + i] = make_float2((float)std::cos(a), (float)std::sin(a));
    }
}

cudaError_t launch_fft2d(float2* grids, int64_t n_planes, int N, bool inverse, const float2* twid,
                         cudaStream_t st, int* launches) {
    if (n_planes <= 0) return cudaSuccess;
    cudaError_t e = cudaErrorInvalidValue;
#define RICK_FFT_CASE(LG)                                                                   \
    case LG:                                                                                \
        e = inverse ? columns_one<LG, true>(grids, n_planes, twid, OccMask{}, st)           \
                    : columns_one<LG, false>(grids, n_planes, twid, OccMask{}, st);         \
        if (e == cudaSuccess)                                                               \
            e = inverse ? rows_one<LG, true>(grids, n_planes, twid, st)                     \
                        : rows_one<LG, false>(grids, n_planes, twid, st);                   \
        break;
    switch (log2_exact(N)) {
        RICK_FFT_CASE(8)
        RICK_FFT_CASE(9)
        RICK_FFT_CASE(10)
        RICK_FFT_CASE(11)
        RICK_FFT_CASE(12)
        RICK_FFT_CASE(13)
        default: break;
    }
#undef RICK_FFT_CASE
    if (e == cudaSuccess) *launches += 2 * (int)((n_planes + 65534) / 65535);
    return e;
}

cudaError_t launch_fft_columns(float2* grids, int64_t n_planes, int N, bool inverse, const float2* twid,
                               OccMask occ, cudaStream_t st, int* launches) {
    if (n_planes <= 0) return cudaSuccess;
    cudaError_t e = cudaErrorInvalidValue;
#define RICK_FFT_CASE(LG)                                                                   \
    case LG:                                                                                \
        e = inverse ? columns_one<LG, true>(grids, n_planes, twid, occ, st)                 \
                    : columns_one<LG, false>(grids, n_planes, twid, occ, st);               \
        break;
    switch (log2_exact(N)) {
        RICK_FFT_CASE(8)
        RICK_FFT_CASE(9)
        RICK_FFT_CASE(10)
        RICK_FFT_CASE(11)
        RICK_FFT_CASE(12)
        RICK_FFT_CASE(13)
        default: break;
    }
#undef RICK_FFT_CASE
    if (e == cudaSuccess) *launches += (int)((n_planes + 65534) / 65535);
    return e;
}

cudaError_t launch_rows_phase_reduce(const PhaseParams& P, const float2* grids, const double* wsum,
                                     const float* inv_taper, const float2* twid, float* image_real,
                                     float2* image_complex, const uint8_t* plane_occ, cudaStream_t st,
                                     int* launches) {
    cudaError_t e = cudaErrorInvalidValue;
    switch (log2_exact(P.N)) {
        case 8: e = fused_n<8>(P, grids, wsum, inv_taper, twid, image_real, image_complex, plane_occ, st); break;
        case 9: e = fused_n<9>(P, grids, wsum, inv_taper, twid, image_real, image_complex, plane_occ, st); break;
        case 10: e = fused_n<10>(P, grids, wsum, inv_taper, twid, image_real, image_complex, plane_occ, st); break;
        case 11: e = fused_n<11>(P, grids, wsum, inv_taper, twid, image_real, image_complex, plane_occ, st); break;
        case 12: e = fused_n<12>(P, grids, wsum, inv_taper, twid, image_real, image_complex, plane_occ, st); break;
        case 13: e = fused_n<13>(P, grids, wsum, inv_taper, twid, image_real, image_complex, plane_occ, st); break;
        default: break;
    }
    if (e == cudaSuccess) ++*launches;
    return e;
}

cudaError_t launch_occupancy(const uint32_t* offsets, int c0, int nc, int k0, int nk, int Nw_store, int NT,
                             uint8_t* col, uint8_t* plane, cudaStream_t st, int* launches) {
    const int64_t n = (int64_t)nc * nk * NT;
    if (n <= 0) return cudaSuccess;
    cudaError_t e = cudaMemsetAsync(plane, 0, (size_t)nc * nk, st);
    if (e != cudaSuccess) return e;
    k_occupancy<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(offsets, c0, nc, k0, nk, Nw_store, NT, col, plane);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    ++*launches;
    return cudaSuccess;
}

}  // namespace rick

// rick_fft.cu -- the 2-D DFTs of the w-planes in two passes over HBM.
//
// Eq. 2 needs, per plane, F_k[q][p] = sum_{i,j} G_k[j][i] e^{+2 pi i (i p + j q)/N}
// (unnormalised); the prediction needs the same with e^{-...}.  The 2-D DFT is
// a length-N DFT down every column followed by one along every row:
//   pass 1 (k_fft_columns): one CTA transforms COLS adjacent columns of a plane,
//     each warp reading and writing rows of COLS x 8 bytes straight from and to
//     registers;
//   pass 2 (k_fft_rows): one CTA transforms one row, in place; or, for imaging,
//     k_rows_phase_reduce: one CTA owns one image row q, transforms that row of
//     every plane of every channel of the launch, applies the phase screen
//     exp(+2 pi i w_k (n - 1)) and sums the planes in registers, so that the
//     transformed planes are never written back (Eq. 2's reduction fused into
//     the transform).
// Every plane is therefore read twice and written once (24 B per cell) on the
// imaging path, against one read and one write per pass of a generic 2-D FFT
// plus the reduction's read.  The prediction runs the same passes the other
// way: k_model_rows forms each model row from the image (the phase screen
// exp(-2 pi i w_k (n - 1)) and the scales) and transforms it along the row,
// so the model planes are never written, then the column pass.
//
// The length-N DFT (N = 2^m, 256 <= N <= 16384) is a Stockham decimation-in-
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
// N = 16384: a row of 128 KB fills most of an SM's shared memory, which leaves
// no room for the fused row pass's per-pixel state.  That pass therefore
// splits each row DFT between four CTAs by one radix-4 decimation-in-frequency
// step (k_rows_phase_reduce_split): with M = N/4,
//   X[4k + r] = sum_{n<M} y_r[n] W_M^(n k),
//   y_r[n] = W_N^(r n) sum_{t<4} x[n + t M] W_4^(r t),
// so CTA r transforms y_r with the 4096-point transform (two CTAs per SM) and
// owns the pixels 4k + r.  The plain column and row passes take one
// 16384-point transform per CTA (1024 threads); the imaging column pass (tiles
// of at least 32) is instead two four-step passes of 128-point transforms over
// groups of 32 columns (k_cols_four), which leave the rows in the four-step
// order that the split row pass reads.
//
// Pruning: planes made by the library's gridder are zero in every tile that no
// visibility reached (or, when the gridder skipped the zero fill, unwritten
// there).  Given the occupancy of the current binning (launch_occupancy: per
// plane, tile column and tile, from the bin offsets), the column pass skips
// the unreached tile columns (their DFT is zero) and reads the unreached tiles
// of the others as zeros, and the fused row pass skips the unreached planes
// and reads the unreached tile columns as zeros (the column pass left them
// untouched) -- the same result as the full transform of the zero-filled
// planes, with less work, and no read of a cell the gridder may have skipped.
// For the prediction the occupancy of its binning prunes the outputs instead:
// unreached planes and tile columns are not transformed, and the column pass
// writes only the reached tiles (the degridder reads nothing else).
//
// Shared arrays are indexed through skew(a) = a + a/16, which spreads the
// stride-16 stores of the first stages over all banks.  Twiddles: a radix-16
// stage with M = 16^s needs W^(e f0), f0 = 1..15, e = t1 M, for the thread's
// butterfly t1.  Per-stage tables, rounded from FP64 on the host
// (e^(+2 pi i e/N); conjugated for the forward transform), hold for stage 0,
// whose t1 takes N/16 values, W^e, W^2e, W^4e and W^8e -- the other eleven
// powers are products of at most three of them (W^7e = W^4e W^2e W^e, W^15e =
// W^8e W^7e) -- and for the later stages, whose t1 takes at most N/256 values,
// all fifteen.  A CTA copies the tables into shared memory once.
#include <cmath>
#include <type_traits>
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

// cos(2 pi k / 64) for 0 <= k <= 16 (cos(pi k / 32), from the FP64 values)
__host__ __device__ constexpr float quarter64(int k) {
    return k == 0 ? 1.0f
         : k == 1 ? 0.99518472667219692873f
         : k == 2 ? 0.98078528040323043058f
         : k == 3 ? 0.95694033573220882438f
         : k == 4 ? 0.92387953251128673848f
         : k == 5 ? 0.88192126434835504956f
         : k == 6 ? 0.83146961230254523567f
         : k == 7 ? 0.77301045336273699338f
         : k == 8 ? 0.70710678118654757274f
         : k == 9 ? 0.63439328416364548779f
         : k == 10 ? 0.55557023301960228867f
         : k == 11 ? 0.47139673682599780857f
         : k == 12 ? 0.38268343236508983729f
         : k == 13 ? 0.29028467725446233105f
         : k == 14 ? 0.19509032201612833135f
         : k == 15 ? 0.09801714032956077016f
         : 0.0f;
}

__host__ __device__ constexpr float cos64(int k) {
    return (k & 63) <= 16   ? quarter64(k & 63)
         : (k & 63) <= 32 ? -quarter64(32 - (k & 63))
         : (k & 63) <= 48 ? -quarter64((k & 63) - 32)
                            : quarter64(64 - (k & 63));
}

__host__ __device__ constexpr float sin64(int k) { return cos64(k - 16); }

// Complex add and subtract as one packed two-lane FP32 instruction each
// (add/sub.rn.f32x2, sm_100 and later): the same IEEE round-to-nearest results
// as two scalar instructions, half the issue slots -- the butterflies are
// mostly adds, and the transform kernels are issue-bound.
__device__ __forceinline__ float2 cadd(float2 a, float2 b) {
    uint64_t ra = *reinterpret_cast<uint64_t*>(&a), rb = *reinterpret_cast<uint64_t*>(&b), rd;
    asm("add.rn.f32x2 %0, %1, %2;" : "=l"(rd) : "l"(ra), "l"(rb));
    return *reinterpret_cast<float2*>(&rd);
}
__device__ __forceinline__ float2 csub(float2 a, float2 b) {
    uint64_t ra = *reinterpret_cast<uint64_t*>(&a), rb = *reinterpret_cast<uint64_t*>(&b), rd;
    asm("sub.rn.f32x2 %0, %1, %2;" : "=l"(rd) : "l"(ra), "l"(rb));
    return *reinterpret_cast<float2*>(&rd);
}
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

// v * e^(s 2 pi i k / 64) for compile-time k (after unrolling), s = +1 (INV) or -1
template <bool INV>
__device__ __forceinline__ float2 twiddle64(float2 v, int k) {
    k &= 63;
    if (k == 0) return v;
    if (k == 16) return mul_si<INV>(v);
    if (k == 32) return make_float2(-v.x, -v.y);
    if (k == 48) return mul_si<!INV>(v);
    const float c = cos64(k), s = INV ? sin64(k) : -sin64(k);
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
// skew(a + 16 k) = skew(a) + 17 k: an offset that is a multiple of 16 becomes
// a constant added to the skewed base, so unrolled accesses at base + 16 k
// need no address arithmetic of their own
__host__ __device__ constexpr int skew16(int k16) { return k16 + k16 / 16; }

template <int LOG2N>
struct Shape {
    static constexpr int N = 1 << LOG2N;
    static constexpr int T = N / 16;                 // threads per transform
    static constexpr int kR16 = LOG2N / 4;            // radix-16 stages
    static constexpr int kLastR = 1 << (LOG2N % 4);   // 1: the last stage is radix 16
    static constexpr int kArray = N + N / 16;         // skewed array length
    // radix-16 stages with twiddles (all but a last radix-16 stage)
    static constexpr int kTwStages = kLastR == 1 ? kR16 - 1 : kR16;
    // butterfly groups t1 of stage s, table entries per t1 (stage 0: 4 powers,
    // the others: all 15), and the offset of the stage's table
    __host__ __device__ static constexpr int stage_cnt(int s) { return (N / 16) >> (4 * s); }
    __host__ __device__ static constexpr int stage_per(int s) { return s == 0 ? 4 : 15; }
    __host__ __device__ static constexpr int stage_off(int s) {
        int o = 0;
        for (int i = 0; i < s; ++i) o += stage_per(i) * stage_cnt(i);
        return o;
    }
    static constexpr int kTw = stage_off(kTwStages);  // twiddle table entries
    // 128 (LOG2N = 7) only for the four-step column pass at N = 16384
    static_assert(LOG2N >= 7 && LOG2N <= 14, "128 <= N <= 16384");
};

// Radix-16 stage s (M = 16^s, not the last stage): a holds the butterfly's
// inputs u + (N/16) t2 for u = b; the DFT, the twiddles W_N^(t1 f0 M) from the
// stage's table sw (stage 0: sw[j cnt + t1] = W^(2^j t1 M), j < 4, the other
// powers formed from them; later stages, whose t1 takes few values, hold all
// fifteen: sw[(f0 - 1) cnt + t1] = W^(t1 f0 M)) and the stores t1 16 M + g +
// M f0 into buf.
template <int LOG2N, bool INV>
__device__ __forceinline__ void radix16_out(float2 (&a)[16], int b, int s, float2* buf,
                                            const float2* tw) {
    using Sh = Shape<LOG2N>;
    Dft<16, INV>::run(a);
    const int log2M = 4 * s;
    const int M = 1 << log2M;
    const int t1 = b >> log2M, g = b & (M - 1);
    const int base = (t1 << (log2M + 4)) + g;
    // output f0 goes to base + M f0: for M >= 16 (M f0 a multiple of 16) and
    // for M = 1 (base a multiple of 16, f0 < 16) its skewed index is
    // skew(base) plus a constant
    float2* out = buf + skew(base);
    auto at = [&](int f0) -> float2& { return M == 1 ? out[f0] : out[skew16(M * f0)]; };
    // t1 = 0: the table holds W^0 = 1 exactly, and a * 1 = a exactly
    const int cnt = Sh::stage_cnt(s);
    const float2* sw = tw + Sh::stage_off(s) + t1;
    if (Sh::stage_per(s) == 15) {
        at(0) = a[0];
#pragma unroll
        for (int f0 = 1; f0 < 16; ++f0) {
            float2 w = sw[(f0 - 1) * cnt];
            if (!INV) w.y = -w.y;
            at(f0) = cmulf(a[f0], w);
        }
        return;
    }
    float2 w[16];
    w[1] = sw[0];
    w[2] = sw[cnt];
    w[4] = sw[2 * cnt];
    w[8] = sw[3 * cnt];
    if (!INV) {
        w[1].y = -w[1].y;
        w[2].y = -w[2].y;
        w[4].y = -w[4].y;
        w[8].y = -w[8].y;
    }
    w[3] = cmulf(w[2], w[1]);
    w[5] = cmulf(w[4], w[1]);
    w[6] = cmulf(w[4], w[2]);
    w[7] = cmulf(w[4], w[3]);
#pragma unroll
    for (int f0 = 9; f0 < 16; ++f0) w[f0] = cmulf(w[8], w[f0 - 8]);
    at(0) = a[0];
#pragma unroll
    for (int f0 = 1; f0 < 16; ++f0) at(f0) = cmulf(a[f0], w[f0]);
}

// Stage 0 (M = 1) of the inverse transform whose 16 inputs of thread b all
// carry one more factor sc (the split row pass's e^(+2 pi i r b / N)): the
// factor is moved past the butterfly, so output f0 is multiplied by
// sc W^(b f0) -- the products formed from sc and the stage's four table
// powers -- instead of every input by sc (31 complex multiplies instead of 42).
template <int LOG2N>
__device__ __forceinline__ void radix16_first_scaled(float2 (&a)[16], int b, float2* buf, const float2* tw,
                                                     float2 sc) {
    using Sh = Shape<LOG2N>;
    Dft<16, true>::run(a);
    const int cnt = Sh::stage_cnt(0);
    const float2* sw = tw + Sh::stage_off(0) + b;   // t1 = b
    const float2 w1 = sw[0], w2 = sw[cnt], w4 = sw[2 * cnt], w8 = sw[3 * cnt];
    float2 w[16];
    w[0] = sc;
    w[1] = cmulf(sc, w1);
    w[2] = cmulf(sc, w2);
    w[3] = cmulf(w[1], w2);
    w[4] = cmulf(sc, w4);
#pragma unroll
    for (int f0 = 5; f0 < 8; ++f0) w[f0] = cmulf(w[f0 - 4], w4);
    w[8] = cmulf(sc, w8);
#pragma unroll
    for (int f0 = 9; f0 < 16; ++f0) w[f0] = cmulf(w[f0 - 8], w8);
    float2* out = buf + skew(16 * b);   // outputs 16 b + f0
#pragma unroll
    for (int f0 = 0; f0 < 16; ++f0) out[f0] = cmulf(a[f0], w[f0]);
}

// The middle radix-16 stages (all but the first, which starts from registers,
// and the last) on buf, in place: loads, barrier, compute and stores, barrier.
template <int LOG2N, bool INV>
__device__ __forceinline__ void middle_stages(float2* buf, int b, const float2* tw) {
    using Sh = Shape<LOG2N>;
    constexpr int kMiddle = Sh::kTwStages - 1;
    const float2* in = buf + skew(b);   // inputs b + T t2, T a multiple of 16
#pragma unroll
    for (int s = 1; s <= kMiddle; ++s) {
        float2 a[16];
#pragma unroll
        for (int t2 = 0; t2 < 16; ++t2) a[t2] = in[skew16(Sh::T * t2)];
        __syncthreads();
        radix16_out<LOG2N, INV>(a, b, s, buf, tw);
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
    const float2* in = buf + skew(b);   // T i + M t2 is a multiple of 16
#pragma unroll
    for (int i = 0; i < NB; ++i) {
        float2 a[R];
#pragma unroll
        for (int t2 = 0; t2 < R; ++t2) a[t2] = in[skew16(Sh::T * i + M * t2)];
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
__device__ __forceinline__ void transform(float2 (&a)[16], float2* buf, int b, const float2* tw,
                                          float2 (&x)[16]) {
    radix16_out<LOG2N, INV>(a, b, 0, buf, tw);
    __syncthreads();
    middle_stages<LOG2N, INV>(buf, b, tw);
    last_stage<LOG2N, INV>(buf, b, x);
}

template <int LOG2N>
__device__ __forceinline__ void load_tables(const float2* __restrict__ twid, float2* tw, int tid, int nthreads) {
    for (int i = tid; i < Shape<LOG2N>::kTw; i += nthreads) tw[i] = __ldg(twid + i);
}

// ---- pass 1: columns ----------------------------------------------------------

// COLS adjacent columns of one plane per CTA (COLS * N/16 threads), the
// threads of a column interleaved: thread (b, c) = COLS b + c, so a warp holds
// COLS columns x 32/COLS butterflies.  The first stage's inputs b + (N/16) t2
// are read straight into registers and the last stage's outputs written
// straight back: each warp access covers 32/COLS rows of COLS * 8 bytes (whole
// 32-byte sectors for COLS = 4), with no staging through shared memory.  Column
// c's skewed array is offset by 32/COLS banks from column c - 1's, so the
// COLS arrays a half-warp touches in every stage fall on distinct banks.
template <int LOG2N, int COLS, bool INV>
__global__ void __launch_bounds__(COLS * (1 << LOG2N) / 16)
k_fft_columns(float2* __restrict__ grids, const float2* __restrict__ twid, Occupancy occ, int64_t plane0) {
    using Sh = Shape<LOG2N>;
    constexpr int N = Sh::N, T = Sh::T;
    constexpr int kStride = Sh::kArray + 16 / COLS;   // float2 per column array
    __shared__ uint8_t s_live[N / 16];
    const int64_t pl = plane0 + blockIdx.y;
    const int tcol = (int)(blockIdx.x * COLS) >> occ.tshift;
    if (occ.col != nullptr && occ.col[pl * occ.NT + tcol] == 0) return;
    constexpr int kThreads = COLS * T;
    extern __shared__ __align__(16) float2 fsm[];
    float2* tw = fsm;
    const int tid = threadIdx.x;
    const int c = tid % COLS, b = tid / COLS;
    float2* buf = fsm + Sh::kTw + c * kStride;
    float2* col = grids + (size_t)blockIdx.y * N * N + (size_t)blockIdx.x * COLS + c;
    load_tables<LOG2N>(twid, tw, tid, kThreads);
    if (occ.tile != nullptr)
        for (int ty = tid; ty < occ.NT; ty += kThreads)
            s_live[ty] = (uint8_t)((occ.tile[(pl * occ.NT + ty) * occ.words + (tcol >> 5)] >> (tcol & 31)) & 1u);
    __syncthreads();
    const bool in_mask = occ.tile != nullptr && !occ.tiles_out, out_mask = occ.tile != nullptr && occ.tiles_out;
    float2 a[16], x[16];
#pragma unroll
    for (int t2 = 0; t2 < 16; ++t2) {
        const int row = b + T * t2;
        // an unreached tile is zero (and possibly unwritten): not read
        a[t2] = (!in_mask || s_live[row >> occ.tshift]) ? __ldcs(col + (size_t)row * N) : make_float2(0.f, 0.f);
    }
    transform<LOG2N, INV>(a, buf, b, tw, x);
    // with tiles_out, only the reached tiles of the result are written
#pragma unroll
    for (int j = 0; j < 16; ++j) {
        const int row = b + T * j;
        if (!out_mask || s_live[row >> occ.tshift]) __stcs(col + (size_t)row * N, x[j]);
    }
}

// The column pass over the reached tile columns only (occ.list): a persistent
// CTA (one or two per SM) loads the twiddle tables once, then takes COLS
// adjacent columns at a time from the list -- tile column entry e = p NT + tx
// gives columns (tx << tshift) + COLS j of plane p -- with an atomic work
// counter, and transforms them as k_fft_columns does.  The unreached tile
// columns cost nothing: with one CTA per column most CTAs of a sparse launch
// only looked up their mask byte and exited, and at N = 16384 (180 KB of
// shared memory, one CTA per SM at a time) those empty CTAs took most of the
// pass.
template <int LOG2N, int COLS, bool INV>
__global__ void __launch_bounds__(COLS * (1 << LOG2N) / 16)
k_fft_columns_list(float2* __restrict__ grids, const float2* __restrict__ twid, Occupancy occ) {
    using Sh = Shape<LOG2N>;
    constexpr int N = Sh::N, T = Sh::T;
    constexpr int kStride = Sh::kArray + 16 / COLS;
    constexpr int kThreads = COLS * T;
    __shared__ uint8_t s_live[N / 16];
    __shared__ uint32_t s_item;
    extern __shared__ __align__(16) float2 fsm[];
    float2* tw = fsm;
    const int tid = threadIdx.x;
    const int c = tid % COLS, b = tid / COLS;
    float2* buf = fsm + Sh::kTw + c * kStride;
    load_tables<LOG2N>(twid, tw, tid, kThreads);
    const uint32_t per = (1u << occ.tshift) / COLS;          // CTA items per tile column
    const uint64_t total = (uint64_t)__ldg(occ.list) * per;
    const bool in_mask = !occ.tiles_out, out_mask = occ.tiles_out;
    // thread 0 takes the next item while the current one is transformed
    uint32_t next = tid == 0 ? atomicAdd(occ.list + 1, 1u) : 0u;
    for (;;) {
        if (tid == 0) s_item = next;
        __syncthreads();   // also: the previous item's last stage has read buf
        const uint32_t item = s_item;
        if (item >= total) break;
        if (tid == 0) next = atomicAdd(occ.list + 1, 1u);
        const uint32_t e = __ldg(occ.list + 2 + item / per);
        const int64_t pl = e / (uint32_t)occ.NT;
        const int tcol = (int)(e - (uint32_t)pl * occ.NT);
        const int x0 = (tcol << occ.tshift) + (int)(item % per) * COLS;
        for (int ty = tid; ty < occ.NT; ty += kThreads)
            s_live[ty] = (uint8_t)((occ.tile[(pl * occ.NT + ty) * occ.words + (tcol >> 5)] >> (tcol & 31)) & 1u);
        __syncthreads();
        float2* col = grids + (size_t)pl * N * N + x0 + c;
        float2 a[16], x[16];
#pragma unroll
        for (int t2 = 0; t2 < 16; ++t2) {
            const int row = b + T * t2;
            a[t2] = (!in_mask || s_live[row >> occ.tshift]) ? __ldcs(col + (size_t)row * N) : make_float2(0.f, 0.f);
        }
        transform<LOG2N, INV>(a, buf, b, tw, x);
#pragma unroll
        for (int j = 0; j < 16; ++j) {
            const int row = b + T * j;
            if (!out_mask || s_live[row >> occ.tshift]) __stcs(col + (size_t)row * N, x[j]);
        }
    }
}

// The column pass at N = 16384 (tiles of at least 32 cells) in two four-step
// passes over groups of 32 adjacent columns, so that every global access is a
// whole 256-byte row segment of a group (one 16384-point column per CTA
// moves 8-byte pieces, one sector per row).  With L = 128 and rows
// n = n1 + L n2, output k = k2 + L k1:
//   pass A: for each n1, Y[n1 + L k2] = W_N^(n1 k2) sum_{n2} x[n1 + L n2] W_L^(n2 k2),
//   pass B: for each k2, X[k2 + L k1] = sum_{n1} Y[n1 + L k2] W_L^(n1 k1),
// both in place: pass A over the rows {n1 + L n2} of an n1, pass B over the
// contiguous block {L k2 + n1} of a k2, whose result X[k2 + L k1] it stores
// at row L k2 + k1 -- the column-transformed plane with its rows in the
// four-step order, which the fused row pass reads as such (mesh row m at
// row L (m mod L) + m / L).  W_N^m, m = n1 k2 < N, is the product of two
// 128-entry tables (e^(2 pi i mh / L) and e^(2 pi i ml / N), m = L mh + ml).
// A CTA of 256 threads holds the 32 columns' 128-point transforms (8 threads
// each, interleaved: thread (b, c) = 32 b + c, so a warp is one row of the
// group); persistent CTAs take (group, n1) or (group, k2) items in a fixed
// round robin.  PRUNED: the groups of the listed reached tile columns, and in
// pass A the unreached tiles read as zeros; else every group of n_planes
// planes.
constexpr int kFourL = 128;

__device__ __forceinline__ float2 four_twiddle(const float2* thi, const float2* tlo, uint32_t m, bool inv) {
    float2 w = cmulf(thi[m >> 7], tlo[m & 127u]);
    if (!inv) w.y = -w.y;
    return w;
}

template <bool INV, bool PRUNED, bool PASS_B>
__global__ void __launch_bounds__(256, 4)
k_cols_four(float2* __restrict__ grids, const float2* __restrict__ t4, Occupancy occ, uint32_t n_planes) {
    using Sh = Shape<7>;
    constexpr int N = 16384, L = kFourL, COLS = 32, T = Sh::T;   // T = 8 threads per transform
    constexpr int kStride = Sh::kArray + 1;   // odd: the 32 column arrays spread over the banks
    __shared__ uint8_t s_live[N / 32];        // tile-row liveness of the group's tile column
    __shared__ float2 s_thi[L], s_tlo[L];
    extern __shared__ __align__(16) float2 fsm[];
    float2* tw = fsm;
    const int tid = threadIdx.x, c = tid % COLS, b = tid / COLS;
    float2* buf = fsm + Sh::kTw + c * kStride;
    load_tables<7>(t4, tw, tid, 256);
    for (int i = tid; i < L; i += 256) {
        s_thi[i] = __ldg(t4 + Sh::kTw + i);
        s_tlo[i] = __ldg(t4 + Sh::kTw + L + i);
    }
    // groups of 32 columns: per listed tile column 2^gs of them
    const uint32_t gs = PRUNED ? (uint32_t)occ.tshift - 5u : 0u;
    const uint32_t n_groups = PRUNED ? (__ldg(occ.list) << gs) : n_planes * (uint32_t)(N / COLS);
    const uint32_t total = n_groups * L;   // below 2^32: checked at launch
    __syncthreads();
    for (uint32_t item = blockIdx.x; item < total; item += gridDim.x) {
        const uint32_t g = item / L, i1 = item % L;   // i1: n1 (pass A) or k2 (pass B)
        uint32_t pl;
        int x0, tcol = 0;
        if (PRUNED) {
            const uint32_t e = __ldg(occ.list + 2 + (g >> gs));
            pl = e / (uint32_t)occ.NT;
            tcol = (int)(e - pl * (uint32_t)occ.NT);
            x0 = (tcol << occ.tshift) + (int)(g & ((1u << gs) - 1u)) * COLS;
        } else {
            pl = g / (uint32_t)(N / COLS);
            x0 = (int)(g % (uint32_t)(N / COLS)) * COLS;
        }
        __syncthreads();   // the previous item has read buf and s_live
        if (PRUNED && !PASS_B)
            for (int ty = tid; ty < occ.NT; ty += 256)
                s_live[ty] = (uint8_t)((occ.tile[((size_t)pl * occ.NT + ty) * occ.words + (tcol >> 5)] >>
                                        (tcol & 31)) & 1u);
        __syncthreads();
        float2* col = grids + (size_t)pl * N * N + x0 + c;
        float2 a[16], x[16];
#pragma unroll
        for (int t2 = 0; t2 < 16; ++t2) {
            const int j = b + T * t2;                       // n2 (pass A) or n1 (pass B)
            const int row = PASS_B ? L * (int)i1 + j : (int)i1 + L * j;
            a[t2] = (!PRUNED || PASS_B || s_live[row >> occ.tshift]) ? __ldcs(col + (size_t)row * N)
                                                                     : make_float2(0.f, 0.f);
        }
        transform<7, INV>(a, buf, b, tw, x);                // x[j] = output b + T j
#pragma unroll
        for (int j = 0; j < 16; ++j) {
            const int k = b + T * j;                        // k2 (pass A) or k1 (pass B)
            if (PASS_B) {
                __stcs(col + (size_t)(L * (int)i1 + k) * N, x[j]);
            } else {
                const float2 w = four_twiddle(s_thi, s_tlo, i1 * (uint32_t)k, INV);
                __stcs(col + (size_t)((int)i1 + L * k) * N, cmulf(x[j], w));
            }
        }
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
    float2* tw = fsm;
    float2* buf = fsm + Sh::kTw;
    const int b = threadIdx.x;
    float2* row = grids + (size_t)blockIdx.y * N * N + (size_t)blockIdx.x * N;
    load_tables<LOG2N>(twid, tw, b, T);
    float2 a[16], x[16];
#pragma unroll
    for (int t2 = 0; t2 < 16; ++t2) a[t2] = __ldcs(row + b + T * t2);
    __syncthreads();
    transform<LOG2N, INV>(a, buf, b, tw, x);
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

// Per-pixel constants of the fused row pass, once per plan (they depend only
// on the mesh, the plane spacing and the tapers): for pixel (p, q),
//   turns[q N + p] = (t_0, dt), the phase w_0 (n - 1) of stored plane 0 and
//     the plane step dw (n - 1) in turns, Q0.32 fixed point (FP64 -- or FP32
//     under RICK_PREC_ALL_FP32 -- from n - 1 = -(l^2 + m^2)/(1 + n)), so that
//     plane k's phase is t_0 + k dt, exact modulo one turn;
//   scale[q N + p] = (-1)^(p+q) n / (C(p) C(q) C_w) (imaging),
//   model_scale[q N + p] = (-1)^(p+q) / (n C(p) C(q) C_w) (prediction).
// P describes stored plane 0 (w_first = its w).
__global__ void k_pixel_phase(PhaseParams P, const float* __restrict__ inv_taper, uint2* __restrict__ turns,
                              float* __restrict__ scale, float* __restrict__ model_scale) {
    const int N = P.Ni, halfN = N / 2;   // image pixels (the central Ni x Ni of a padded mesh)
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= (int64_t)N * N) return;
    const int q = (int)(i / N), p = (int)(i - (int64_t)q * N);
    const double l = (double)(p - halfN) * P.dl, m = (double)(q - halfN) * P.dl;
    const double r2 = l * l + m * m;
    const double n = sqrt(1.0 - r2);
    const double delta = -r2 / (1.0 + n);
    if (P.precision == RICK_PREC_ALL_FP32) {
        const float lf = (float)(p - halfN) * (float)P.dl, mf = (float)(q - halfN) * (float)P.dl;
        const float r2f = lf * lf + mf * mf;
        const float df = -r2f / (1.0f + sqrtf(1.0f - r2f));
        turns[i] = make_uint2(turns_q32f((float)P.w_first * df), turns_q32f((float)P.dw * df));
    } else {
        turns[i] = make_uint2(turns_q32(P.w_first * delta), turns_q32(P.dw * delta));
    }
    const float sg = ((p + q) & 1) ? -1.f : 1.f;
    const float c = sg * inv_taper[p] * inv_taper[q] * w_taper_inv(P, delta);
    scale[i] = c * (float)n;
    model_scale[i] = c / (float)n;
}

// Imaging, pass 2 fused with Eq. 2's phase screen and reduction: image row q
// (blockIdx.x) of every channel of the launch,
//   image[c][q][p] += (-1)^(p+q) n C_w^-1 / (sum W_c C(p) C(q))
//                     * Re sum_k F_k[q][p] exp(+2 pi i w_k (n - 1)),
// where F_k[q][.] is the row DFT of the column-transformed plane k.  Thread b
// owns pixels p = b + (N/16) j.  With t_k = t_0 + k dt the phase of plane k
// (turns), the sum over a block of planes k = k0..k1 is
//   e^(2 pi i t_k1) sum_k F_k z^(k1-k),  z = e^(-2 pi i dt),
// taken by Horner's rule: acc <- acc z + F_k, one complex multiply-add per
// pixel and plane (z per pixel in shared memory); the exact phasor of the
// block's last plane, from the Q0.32 turns, multiplies the result, which is
// summed per pixel in shared memory and added to the image at the channel's
// end (one read-modify-write of the image row per channel; the variant with
// the complex output adds every block to the images instead).  Blocks of
// kHornerBlock planes bound the rounding that
// the powers of the FP32 z carry (each rotation adds about one unit of FP32
// rounding in angle and modulus).  An unreached plane still rotates acc
// (acc z + 0), so pruning does not change the arithmetic.
// The per-pixel turns and scale come from the plan's table (k_pixel_phase).
// The next row is loaded into registers while the current one is transformed.
// Two CTAs per SM for N <= 4096 (at most 128 registers).
constexpr int kHornerBlock = 8;   // planes per Horner block of the fused row pass

template <int LOG2N, bool COMPLEX_OUT, bool PADDED>
__global__ void __launch_bounds__((1 << LOG2N) / 16, LOG2N <= 12 ? 2 : 1)
k_rows_phase_reduce(PhaseParams P, const float2* __restrict__ grids, const double* __restrict__ wsum,
                    const uint2* __restrict__ pix_turns, const float* __restrict__ pix_scale,
                    const float2* __restrict__ twid, float* __restrict__ image_real,
                    float2* __restrict__ image_complex, Occupancy occ) {
    using Sh = Shape<LOG2N>;
    constexpr int N = Sh::N, T = Sh::T;
    extern __shared__ __align__(16) float2 fsm[];
    float2* tw = fsm;
    float2* buf = fsm + Sh::kTw;
    float2* turn256 = buf + Sh::kArray;                          // e^(2 pi i j / 256)
    float2* zrot = turn256 + 256;                                // z = e^(-2 pi i dt) per pixel
    // the channel's finished blocks per pixel: Re of the phased sums
    float* part = reinterpret_cast<float*>(zrot + N);
    // image row q (blockIdx.x) is row q + off of the mesh; mesh pixel pm is
    // image pixel pm - off (a padded mesh keeps its central Ni x Ni; without
    // padding, off = 0 and Ni = N at compile time)
    const int Ni = PADDED ? P.Ni : N, off = PADDED ? P.off : 0;
    const int b = threadIdx.x, q = blockIdx.x;
    const float* scl = pix_scale + (size_t)q * Ni;               // per-pixel scale (read once per channel)
    const uint2* turns = pix_turns + (size_t)q * Ni;
    load_tables<LOG2N>(twid, tw, b, T);
    for (int j = b; j < 256; j += T) turn256[j] = __ldg(twid + Sh::kTw + j);
#pragma unroll 4
    for (int j = 0; j < 16; ++j) {
        const int pm = b + T * j, p = pm - off;
        float s = 0.f, c = 1.f;
        if (!PADDED || (unsigned)p < (unsigned)Ni)
            sincospif((float)(int32_t)__ldg(&turns[p].y) * 4.656612873077392578125e-10f /* 2^-31 */, &s, &c);
        zrot[pm] = make_float2(c, -s);
        if (!COMPLEX_OUT) part[pm] = 0.f;
    }

    const size_t NN = (size_t)N * N, NNi = (size_t)Ni * Ni;
    const int n_rows = P.nc * P.nk;
    // planes no visibility reached are not transformed
    auto next_row = [&](int r) {
        if (occ.plane != nullptr)
            while (r < n_rows && occ.plane[r] == 0) ++r;
        return r;
    };
    // row q of plane r: the inputs b + T t2 of this thread; the unreached tile
    // columns are zero (the column pass did not touch them): not read
    // With tiles of at least 32 columns (and N/16 >= 32) the tile column of
    // input b + T t2 is the same for a whole warp: lanes 0..15 read the 16
    // mask bytes and a ballot hands every lane the 16 bits.
    const bool warp_mask = occ.tshift >= 5 && T >= 32;
    auto load_row = [&](int r, float2 (&v)[16]) {
        const float2* row = grids + (size_t)r * NN + (size_t)(q + off) * N;
        if (occ.col != nullptr) {
            const uint8_t* cm = occ.col + (size_t)r * occ.NT;
            uint32_t live = 0;
            if (warp_mask) {
                const int lane = b & 31;
                const bool on = lane < 16 && __ldg(cm + (((b & ~31) + T * lane) >> occ.tshift)) != 0;
                live = __ballot_sync(0xffffffffu, on);
            } else {
#pragma unroll
                for (int t2 = 0; t2 < 16; ++t2)
                    live |= (__ldg(cm + ((b + T * t2) >> occ.tshift)) != 0 ? 1u : 0u) << t2;
            }
#pragma unroll
            for (int t2 = 0; t2 < 16; ++t2)
                v[t2] = (live >> t2) & 1u ? __ldcs(row + b + T * t2) : make_float2(0.f, 0.f);
        } else {
#pragma unroll
            for (int t2 = 0; t2 < 16; ++t2) v[t2] = __ldcs(row + b + T * t2);
        }
    };
    float2 a[16], x[16];
    int r = next_row(0);
    if (r < n_rows) load_row(r, a);
    __syncthreads();
    for (int cc = 0; cc < P.nc; ++cc) {
        float2 acc[16];
#pragma unroll
        for (int j = 0; j < 16; ++j) acc[j] = make_float2(0.f, 0.f);
        for (int kk = 0; kk < P.nk; ++kk) {
            if (cc * P.nk + kk != r) {   // an unreached plane: F_k = 0
#pragma unroll
                for (int j = 0; j < 16; ++j) {
                    const float2 z = zrot[b + T * j];
                    acc[j] = make_float2(fmaf(acc[j].x, z.x, -acc[j].y * z.y), fmaf(acc[j].x, z.y, acc[j].y * z.x));
                }
            } else {
                radix16_out<LOG2N, true>(a, b, 0, buf, tw);
                const int rn = next_row(r + 1);
                if (rn < n_rows) load_row(rn, a);
                r = rn;
                __syncthreads();
                middle_stages<LOG2N, true>(buf, b, tw);
                last_stage<LOG2N, true>(buf, b, x);
                __syncthreads();   // buf is rewritten by the next row's first stage
#pragma unroll
                for (int j = 0; j < 16; ++j) {
                    const float2 z = zrot[b + T * j];
                    acc[j] = make_float2(fmaf(acc[j].x, z.x, fmaf(-acc[j].y, z.y, x[j].x)),
                                         fmaf(acc[j].x, z.y, fmaf(acc[j].y, z.x, x[j].y)));
                }
            }
            const bool last = kk == P.nk - 1;
            if (kk % kHornerBlock != kHornerBlock - 1 && !last) continue;
            // end of a block: times the exact phasor of its last plane; at the
            // channel's end, scaled into the image
            const uint32_t k_end = (uint32_t)(P.k_first + kk);
            float inv_ws = 0.f;
            if (last || COMPLEX_OUT) {
                const double ws = wsum[cc];
                inv_ws = ws != 0.0 ? (float)(1.0 / ws) : 0.0f;
            }
#pragma unroll
            for (int j = 0; j < 16; ++j) {
                // pixels outside the image (a padded mesh) are computed from a
                // valid index and not stored, so that every load is unconditional
                const int pm = b + T * j, p = pm - off;
                const bool in_img = !PADDED || (unsigned)p < (unsigned)Ni;
                const int pc = in_img ? p : 0;
                // e^(2 pi i t) for t = tk 2^-32 turns, table-driven: the
                // nearest 1/256 of a turn from the table, the rest
                // (|theta| <= pi / 256) from its Taylor series to theta^3
                const uint2 ph = __ldg(&turns[pc]);
                const uint32_t tk = ph.x + k_end * ph.y;
                const uint32_t j8 = (tk + 0x800000u) >> 24;
                const float th = (float)(int32_t)(tk - (j8 << 24)) * 1.46291807926715968e-9f;  // 2 pi 2^-32
                const float t2 = th * th;
                const float c = fmaf(-0.5f, t2, 1.0f), sg = th * fmaf(t2, -0.16666667f, 1.0f);
                const float2 w = turn256[j8 & 255u];
                const float cs = fmaf(w.x, c, -w.y * sg), sn = fmaf(w.y, c, w.x * sg);
                const float re = fmaf(acc[j].x, cs, -acc[j].y * sn);
                const float im = fmaf(acc[j].x, sn, acc[j].y * cs);
                acc[j] = make_float2(0.f, 0.f);
                float* ir = image_real + (size_t)cc * NNi + (size_t)q * Ni + pc;
                if (COMPLEX_OUT) {
                    const float s = __ldg(scl + pc) * inv_ws;
                    float2* ic = image_complex + (size_t)cc * NNi + (size_t)q * Ni + pc;
                    const float r0 = *ir;
                    float2 v = *ic;
                    v.x += s * re;
                    v.y += s * im;
                    if (in_img) {
                        *ir = r0 + s * re;
                        *ic = v;
                    }
                } else if (!last) {
                    part[pm] += re;
                } else {
                    const float out = *ir + __ldg(scl + pc) * inv_ws * (part[pm] + re);
                    if (in_img) *ir = out;
                    part[pm] = 0.f;
                }
            }
        }
    }
}

// k_rows_phase_reduce with every image row q split between SPLIT CTAs (for
// N = 16384: SPLIT = 4, each running the 4096-point transform, two CTAs per
// SM), blockIdx.x = SPLIT q + r (the CTAs of a row run side by side and share
// its cache lines).  One decimation-in-frequency step of radix SPLIT: with
// M = N / SPLIT,
//   X[SPLIT k + r] = sum_{n<M} y_r[n] e^(+2 pi i n k / M),
//   y_r[n] = e^(+2 pi i r n / N) sum_{t<SPLIT} x[n + t M] e^(+2 pi i r t / SPLIT),
// so CTA r transforms y_r with the M-point transform and owns the pixels
// SPLIT k + r, to which it applies the phase screen and the plane sum of
// Eq. 2 exactly as k_rows_phase_reduce does (Horner blocks of kHornerBlock
// planes, exact phasor at each block's end).  The twiddle of y_r is
// e^(2 pi i r t2 / (16 SPLIT)) (a constant of the unrolled code,
// n = b + (M/16) t2) times e^(2 pi i r b / N) (per thread, from a table
// rounded from FP64), which is the same for the thread's 16 inputs and is
// applied with the first stage's output twiddles (radix16_first_scaled).  With pruning, the
// unreached tile columns of the row are not read; the prefetch of the next
// row holds one value per position n (its first reached part t), and the
// other reached parts of the same position (none on a centred uv coverage
// narrower than M) are read when the row is consumed.  Pruning also cuts the
// arithmetic: N log2(M) butterfly work per row instead of N log2(N).  Unlike
// the unsplit pass, an unreached plane rotates acc only once its block has a
// reached plane (before that acc is zero and stays zero), and a block with no
// reached plane takes no phasor -- the zeros the unpruned pass computes, so
// the pruned result is still the unpruned one.  (In the unsplit pass the same
// change measured 9 % slower at 4096^2 and is not made.)
template <int LOG2SUB, int SPLIT, bool COMPLEX_OUT, bool PADDED>
__global__ void __launch_bounds__((1 << LOG2SUB) / 16, LOG2SUB <= 12 ? 2 : 1)
k_rows_phase_reduce_split(PhaseParams P, const float2* __restrict__ grids, const double* __restrict__ wsum,
                          const uint2* __restrict__ pix_turns, const float* __restrict__ pix_scale,
                          const float2* __restrict__ twid_sub, float* __restrict__ image_real,
                          float2* __restrict__ image_complex, Occupancy occ) {
    // the split twiddle table (fft_twiddles) is built for N = 4 x 4096
    static_assert(SPLIT == 4 && LOG2SUB == 12, "split");
    using Sh = Shape<LOG2SUB>;
    constexpr int M = Sh::N, T = Sh::T;     // sub-transform: points, threads
    constexpr int N = SPLIT * M;
    extern __shared__ __align__(16) float2 fsm[];
    float2* tw = fsm;
    float2* buf = fsm + Sh::kTw;
    float2* turn256 = buf + Sh::kArray;                          // e^(2 pi i j / 256)
    float2* zrot = turn256 + 256;                                // z per owned pixel
    float* part = reinterpret_cast<float*>(zrot + M);
    // image row q is mesh row q + off; mesh pixel SPLIT k + r is image pixel
    // SPLIT k + r - off (a padded mesh keeps its central Ni x Ni; without
    // padding, off = 0 and Ni = N at compile time)
    const int Ni = PADDED ? P.Ni : N, off = PADDED ? P.off : 0;
    const int b = threadIdx.x, q = blockIdx.x / SPLIT, par = blockIdx.x % SPLIT;
    const float* scl = pix_scale + (size_t)q * Ni;
    const uint2* turns = pix_turns + (size_t)q * Ni;
    load_tables<LOG2SUB>(twid_sub, tw, b, T);
    for (int j = b; j < 256; j += T) turn256[j] = __ldg(twid_sub + Sh::kTw + SPLIT * T + j);
#pragma unroll 4
    for (int j = 0; j < 16; ++j) {
        const int k = b + T * j, p = SPLIT * k + par - off;
        float s = 0.f, c = 1.f;
        if (!PADDED || (unsigned)p < (unsigned)Ni)
            sincospif((float)(int32_t)__ldg(&turns[p].y) * 4.656612873077392578125e-10f /* 2^-31 */, &s, &c);
        zrot[k] = make_float2(c, -s);
        if (!COMPLEX_OUT) part[k] = 0.f;
    }
    // e^(+2 pi i r b / N) for this CTA's twiddles, rounded from FP64 on the
    // host (the table after the sub-transform's stage tables)
    const float2 wb = __ldg(twid_sub + Sh::kTw + par * T + b);

    const size_t NN = (size_t)N * N, NNi = (size_t)Ni * Ni;
    const int n_rows = P.nc * P.nk;
    // liveness of the inputs b + T t2 + t M of row (plane) r: bit 16 t + t2.
    // With tiles of at least 32 columns (T >= 32) every warp reads one tile
    // column per (t, t2): lane (t2 = lane % 16, t = lane / 16 + 2 h) reads one
    // mask byte and ballots hand every lane the bits
    const bool warp_mask = occ.tshift >= 5 && T >= 32;
    const int lane = b & 31;
    auto live_bits = [&](int r) -> uint64_t {
        if (occ.col == nullptr) return ~0ull >> (64 - 16 * SPLIT);
        const uint8_t* cm = occ.col + (size_t)r * occ.NT;
        uint64_t live = 0;
        if (warp_mask) {
#pragma unroll
            for (int h = 0; h < SPLIT / 2; ++h) {
                const int pos = (b & ~31) + T * (lane & 15) + ((lane >> 4) + 2 * h) * M;
                live |= (uint64_t)__ballot_sync(0xffffffffu, __ldg(cm + (pos >> occ.tshift)) != 0) << (32 * h);
            }
            return live;
        }
#pragma unroll
        for (int t = 0; t < SPLIT; ++t)
#pragma unroll
            for (int t2 = 0; t2 < 16; ++t2)
                live |= (uint64_t)(__ldg(cm + ((b + T * t2 + t * M) >> occ.tshift)) != 0 ? 1u : 0u) << (16 * t + t2);
        return live;
    };
    auto next_row = [&](int r) {
        if (occ.plane != nullptr)
            while (r < n_rows && occ.plane[r] == 0) ++r;
        return r;
    };
    // prefetch: the lowest reached part of each position; pf_first (2 bits per
    // position) says which, and pf_single that no position of this thread has
    // a second reached part (the usual case: a centred uv coverage narrower
    // than M), so that the combination needs no further load or test
    uint64_t pf_live = 0;
    uint32_t pf_first = 0;
    bool pf_single = true;
    const float2* pf_row = grids;
    auto load_row = [&](int r, float2 (&v)[16]) {
        // mesh row m = q + off; after the four-step column pass it is stored at
        // row 128 (m mod 128) + m / 128
        const int m = q + off;
        pf_row = grids + (size_t)r * NN + (size_t)(P.rows_four ? ((m & 127) << 7) + (m >> 7) : m) * N;
        pf_live = live_bits(r);
        pf_first = 0;
#pragma unroll
        for (int t2 = 0; t2 < 16; ++t2) {
            int first = -1;
#pragma unroll
            for (int t = SPLIT - 1; t >= 0; --t)
                if ((pf_live >> (16 * t + t2)) & 1u) first = t;
            pf_first |= (uint32_t)(first < 0 ? 0 : first) << (2 * t2);
            v[t2] = first >= 0 ? __ldcs(pf_row + b + T * t2 + first * M) : make_float2(0.f, 0.f);
        }
        const uint32_t l0 = (uint32_t)pf_live & 0xffffu, l1 = (uint32_t)(pf_live >> 16) & 0xffffu,
                       l2 = (uint32_t)(pf_live >> 32) & 0xffffu, l3 = (uint32_t)(pf_live >> 48) & 0xffffu;
        pf_single = ((l0 & (l1 | l2 | l3)) | (l1 & (l2 | l3)) | (l2 & l3)) == 0u;
    };
    // y * i^k for a runtime k in 0..3 (the quarter turns e^(2 pi i R t / 4))
    auto quarter = [](float2 y, int k) {
        const float re = (k & 1) ? y.y : y.x, im = (k & 1) ? y.x : y.y;
        return make_float2(((k + 1) & 2) ? -re : re, (k & 2) ? -im : im);
    };
    // y_r from the prefetched values (compile-time r)
    auto combine_r = [&](float2 (&v)[16], auto rc) {
        constexpr int R = decltype(rc)::value;
        if (pf_single) {
            if constexpr (R != 0) {   // (y_0[n] = x[n + first M])
#pragma unroll
                for (int t2 = 0; t2 < 16; ++t2) {
                    const int first = (int)((pf_first >> (2 * t2)) & 3u);
                    v[t2] = twiddle64<true>(quarter(v[t2], (R * first) & 3), R * t2);
                }
            }
            return;
        }
#pragma unroll
        for (int t2 = 0; t2 < 16; ++t2) {
            const int first = (int)((pf_first >> (2 * t2)) & 3u);
            // e^(2 pi i R first / 4) times the prefetched part (zero if none),
            // plus the other reached parts (above first)
            float2 y = quarter(v[t2], (R * first) & 3);
#pragma unroll
            for (int t = 1; t < SPLIT; ++t)
                if (t > first && ((pf_live >> (16 * t + t2)) & 1u)) {
                    const float2 u = __ldcs(pf_row + b + T * t2 + t * M);
                    y = cadd(y, twiddle_const<true>(u, R * t, SPLIT));
                }
            v[t2] = R == 0 ? y : twiddle64<true>(y, R * t2);
        }
    };
    auto combine = [&](float2 (&v)[16]) {
        if (par == 0) combine_r(v, std::integral_constant<int, 0>{});
        else if (par == 1) combine_r(v, std::integral_constant<int, 1>{});
        else if (SPLIT == 4 && par == 2) combine_r(v, std::integral_constant<int, 2>{});
        else if (SPLIT == 4) combine_r(v, std::integral_constant<int, 3>{});
    };
    float2 a[16], x[16];
    int r = next_row(0);
    if (r < n_rows) load_row(r, a);
    __syncthreads();
    for (int cc = 0; cc < P.nc; ++cc) {
        float2 acc[16];
#pragma unroll
        for (int j = 0; j < 16; ++j) acc[j] = make_float2(0.f, 0.f);
        // filled: the current block has a reached plane; any: the channel has
        bool filled = false, any = false;
        for (int kk = 0; kk < P.nk; ++kk) {
            if (cc * P.nk + kk != r) {   // an unreached plane: F_k = 0
                // acc z + 0; while the block has no reached plane acc is zero
                // and stays zero, so there is nothing to rotate
                if (filled) {
#pragma unroll
                    for (int j = 0; j < 16; ++j) {
                        const float2 z = zrot[b + T * j];
                        acc[j] = make_float2(fmaf(acc[j].x, z.x, -acc[j].y * z.y),
                                             fmaf(acc[j].x, z.y, acc[j].y * z.x));
                    }
                }
            } else {
                combine(a);
                // e^(2 pi i r b / N), common to the thread's inputs, enters
                // with the first stage's twiddles
                if (par == 0)
                    radix16_out<LOG2SUB, true>(a, b, 0, buf, tw);
                else
                    radix16_first_scaled<LOG2SUB>(a, b, buf, tw, wb);
                const int rn = next_row(r + 1);
                if (rn < n_rows) load_row(rn, a);
                r = rn;
                __syncthreads();
                middle_stages<LOG2SUB, true>(buf, b, tw);
                last_stage<LOG2SUB, true>(buf, b, x);
                __syncthreads();   // buf is rewritten by the next row's first stage
#pragma unroll
                for (int j = 0; j < 16; ++j) {
                    const float2 z = zrot[b + T * j];
                    acc[j] = make_float2(fmaf(acc[j].x, z.x, fmaf(-acc[j].y, z.y, x[j].x)),
                                         fmaf(acc[j].x, z.y, fmaf(acc[j].y, z.x, x[j].y)));
                }
                filled = any = true;
            }
            const bool last = kk == P.nk - 1;
            if (kk % kHornerBlock != kHornerBlock - 1 && !last) continue;
            // a block without a reached plane adds zero: nothing to do, except
            // at the channel's end, where the image takes the earlier blocks
            const bool empty = !filled;
            filled = false;
            if (empty && (COMPLEX_OUT || !last || !any)) continue;
            const uint32_t k_end = (uint32_t)(P.k_first + kk);
            float inv_ws = 0.f;
            if (last || COMPLEX_OUT) {
                const double ws = wsum[cc];
                inv_ws = ws != 0.0 ? (float)(1.0 / ws) : 0.0f;
            }
#pragma unroll
            for (int j = 0; j < 16; ++j) {
                // pixels outside the image (a padded mesh) are computed from a
                // valid index and not stored, so that every load is unconditional
                const int k = b + T * j, p = SPLIT * k + par - off;
                const bool in_img = !PADDED || (unsigned)p < (unsigned)Ni;
                const int pc = in_img ? p : 0;
                float sn = 0.f, cs = 1.f;   // acc is zero in an empty block
                if (!empty) {
                    // e^(2 pi i t) for t = tk 2^-32 turns, table-driven: the
                    // nearest 1/256 of a turn from the table, the rest
                    // (|theta| <= pi / 256) from its Taylor series to theta^3
                    // (truncation below 1e-9)
                    const uint2 ph = __ldg(&turns[pc]);
                    const uint32_t tk = ph.x + k_end * ph.y;
                    const uint32_t j8 = (tk + 0x800000u) >> 24;
                    const float th = (float)(int32_t)(tk - (j8 << 24)) * 1.46291807926715968e-9f;  // 2 pi 2^-32
                    const float t2 = th * th;
                    const float c = fmaf(-0.5f, t2, 1.0f), s = th * fmaf(t2, -0.16666667f, 1.0f);
                    const float2 w = turn256[j8 & 255u];
                    cs = fmaf(w.x, c, -w.y * s);
                    sn = fmaf(w.y, c, w.x * s);
                }
                const float re = fmaf(acc[j].x, cs, -acc[j].y * sn);
                const float im = fmaf(acc[j].x, sn, acc[j].y * cs);
                acc[j] = make_float2(0.f, 0.f);
                float* ir = image_real + (size_t)cc * NNi + (size_t)q * Ni + pc;
                if (COMPLEX_OUT) {
                    const float s = __ldg(scl + pc) * inv_ws;
                    float2* ic = image_complex + (size_t)cc * NNi + (size_t)q * Ni + pc;
                    const float r0 = *ir;
                    float2 v = *ic;
                    v.x += s * re;
                    v.y += s * im;
                    if (in_img) {
                        *ir = r0 + s * re;
                        *ic = v;
                    }
                } else if (!last) {
                    part[k] += re;
                } else {
                    const float out = *ir + __ldg(scl + pc) * inv_ws * (part[k] + re);
                    if (in_img) *ir = out;
                    part[k] = 0.f;
                }
            }
        }
    }
}

// Prediction, the row pass run backwards (the adjoint of k_rows_phase_reduce):
// for image row q (blockIdx.x) of every channel and plane of the launch, the
// model row M_k[q][p] = J_c[q][p] (-1)^(p+q) exp(-2 pi i w_k (n - 1)) /
// (n C(p) C(q) C_w) is formed in registers and transformed along the row
// (exponent -), and the result is written to row q of plane k -- the first
// pass of the forward 2-D DFT of the model plane, which is never written.
// Thread b owns pixels p = b + (N/16) t2, the first stage's inputs.  The phase
// of plane k, ph = exp(-2 pi i t_k), is advanced from plane to plane by
// ph <- ph z, z = exp(-2 pi i dt) (in shared memory), and formed exactly from
// the Q0.32 turns t_0 + k dt of the plan's table at the first plane of every
// block of 8, which bounds the FP32 rounding of the powers of z as in the
// imaging pass.  With occ, unreached planes are skipped and only the
// reached tile columns are written (the column pass reads nothing else, and
// the degridder only the reached tiles).
template <int LOG2N>
__global__ void __launch_bounds__((1 << LOG2N) / 16, LOG2N <= 12 ? 2 : 1)
k_model_rows(PhaseParams P, const float* __restrict__ image, const uint2* __restrict__ pix_turns,
             const float* __restrict__ pix_model_scale, const float2* __restrict__ twid,
             float2* __restrict__ grids, Occupancy occ) {
    using Sh = Shape<LOG2N>;
    constexpr int N = Sh::N, T = Sh::T;
    extern __shared__ __align__(16) float2 fsm[];
    float2* tw = fsm;
    float2* buf = fsm + Sh::kTw;
    float2* zrot = buf + Sh::kArray;                            // z = e^(-2 pi i dt) per pixel
    float* js = reinterpret_cast<float*>(zrot + N);             // J_c(p) times the pixel's scale
    // mesh row q (blockIdx.x) is image row q - off and mesh pixel pm image
    // pixel pm - off (a padded mesh holds the image in its central Ni x Ni;
    // the model is zero elsewhere)
    const int Ni = P.Ni, off = P.off;
    const int b = threadIdx.x, q = blockIdx.x, qi = q - off;
    const size_t NN = (size_t)N * N, NNi = (size_t)Ni * Ni;
    const bool warp_mask = occ.tshift >= 5 && T >= 32;
    const int lane = b & 31;
    // the tile columns of plane r that the column pass reads
    auto live_cols = [&](int r) -> uint32_t {
        uint32_t live = 0xffffu;
        if (occ.col != nullptr) {
            const uint8_t* cm = occ.col + (size_t)r * occ.NT;
            if (warp_mask) {
                const bool on = lane < 16 && __ldg(cm + (((b & ~31) + T * lane) >> occ.tshift)) != 0;
                live = __ballot_sync(0xffffffffu, on);
            } else {
                live = 0;
#pragma unroll
                for (int t2 = 0; t2 < 16; ++t2)
                    live |= (__ldg(cm + ((b + T * t2) >> occ.tshift)) != 0 ? 1u : 0u) << t2;
            }
        }
        return live;
    };
    if ((unsigned)qi >= (unsigned)Ni) {
        // a row of the padding: its transform is zero, written where it is read
        for (int r = 0; r < P.nc * P.nk; ++r) {
            if (occ.plane != nullptr && occ.plane[r] == 0) continue;
            const uint32_t live = live_cols(r);
            float2* row = grids + (size_t)r * NN + (size_t)q * N;
#pragma unroll
            for (int j = 0; j < 16; ++j)
                if ((live >> j) & 1u) __stcs(row + b + T * j, make_float2(0.f, 0.f));
        }
        return;
    }
    const uint2* turns = pix_turns + (size_t)qi * Ni;
    load_tables<LOG2N>(twid, tw, b, T);
#pragma unroll 4
    for (int t2 = 0; t2 < 16; ++t2) {
        const int pm = b + T * t2, p = pm - off;
        float s = 0.f, c = 1.f;
        if ((unsigned)p < (unsigned)Ni)
            sincospif((float)(int32_t)__ldg(&turns[p].y) * 4.656612873077392578125e-10f /* 2^-31 */, &s, &c);
        zrot[pm] = make_float2(c, -s);
    }
    for (int cc = 0; cc < P.nc; ++cc) {
        const float* jr = image + (size_t)cc * NNi + (size_t)qi * Ni;
        const float* ms = pix_model_scale + (size_t)qi * Ni;
        __syncthreads();   // the previous channel's js reads are done
#pragma unroll 4
        for (int t2 = 0; t2 < 16; ++t2) {
            const int pm = b + T * t2, p = pm - off;
            js[pm] = (unsigned)p < (unsigned)Ni ? __ldg(jr + p) * __ldg(ms + p) : 0.f;
        }
        // ph holds the phase of plane kcur; it is formed exactly at the first
        // plane of each block of kHornerBlock planes and advanced plane by plane
        // -- across skipped planes too, so that pruning does not change the
        // arithmetic
        float2 ph[16];
        int kcur = 0, block = -1;
        for (int kk = 0; kk < P.nk; ++kk) {
            const int r = cc * P.nk + kk;
            if (occ.plane != nullptr && occ.plane[r] == 0) continue;   // no record on this plane
            if (kk / kHornerBlock != block) {
                block = kk / kHornerBlock;
                kcur = block * kHornerBlock;
                const uint32_t k = (uint32_t)(P.k_first + kcur);
#pragma unroll
                for (int t2 = 0; t2 < 16; ++t2) {
                    const int p = b + T * t2 - off;
                    const uint2 t = (unsigned)p < (unsigned)Ni ? __ldg(&turns[p]) : make_uint2(0u, 0u);
                    float sn, cs;
                    sincospif((float)(int32_t)(t.x + k * t.y) * 4.656612873077392578125e-10f /* 2^-31 */, &sn, &cs);
                    ph[t2] = make_float2(cs, -sn);
                }
            }
            for (; kcur < kk; ++kcur) {   // over skipped planes
#pragma unroll
                for (int t2 = 0; t2 < 16; ++t2) {
                    const float2 z = zrot[b + T * t2];
                    ph[t2] = make_float2(fmaf(ph[t2].x, z.x, -ph[t2].y * z.y), fmaf(ph[t2].x, z.y, ph[t2].y * z.x));
                }
            }
            float2 a[16], x[16];
#pragma unroll
            for (int t2 = 0; t2 < 16; ++t2) {
                const int p = b + T * t2;
                const float j = js[p];
                const float2 z = zrot[p];
                a[t2] = make_float2(j * ph[t2].x, j * ph[t2].y);
                ph[t2] = make_float2(fmaf(ph[t2].x, z.x, -ph[t2].y * z.y), fmaf(ph[t2].x, z.y, ph[t2].y * z.x));
            }
            kcur = kk + 1;
            transform<LOG2N, false>(a, buf, b, tw, x);
            const uint32_t live = live_cols(r);
            float2* row = grids + (size_t)r * NN + (size_t)q * N;
#pragma unroll
            for (int j = 0; j < 16; ++j)
                if ((live >> j) & 1u) __stcs(row + b + T * j, x[j]);
            __syncthreads();   // buf is rewritten by the next plane's first stage
        }
    }
}

// columns per CTA in pass 1: warp accesses of 32-byte row pieces (whole DRAM
// sectors) where 4 N/16 threads fit a CTA, else 16 bytes
template <int LOG2N>
constexpr int kCols = LOG2N <= 12 ? 4 : LOG2N == 13 ? 2 : 1;

// Occupancy of the planes p = cc nk + kk of the launch from the bin offsets:
// one thread per tile (tx fastest), reached iff tile_reach() > 0 -- the
// gridder's own test for an empty tile.  A warp's ballot is a word of the
// tile bits (NT >= 32) or holds whole tile rows (NT < 32); col and plane are
// zeroed beforehand and set where a tile is reached.
__global__ void k_occupancy(const uint32_t* __restrict__ offsets, int c0, int nc, int k0, int nk,
                            int Nw_store, int NT, int words, uint8_t* __restrict__ col,
                            uint8_t* __restrict__ plane, uint32_t* __restrict__ tile) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int64_t n = (int64_t)nc * nk * NT * NT;
    const int lane = threadIdx.x & 31;
    bool reached = false;
    int tx = 0;
    int64_t prow = 0;   // p * NT + ty
    if (i < n) {
        tx = (int)(i % NT);
        prow = i / NT;
        const int ty = (int)(prow % NT);
        const int64_t p = prow / NT;
        const int cc = (int)(p / nk), kk = (int)(p - (int64_t)cc * nk);
        const uint64_t kplane = ((uint64_t)(c0 + cc) * Nw_store + (k0 + kk)) * NT;
        reached = tile_reach(offsets, kplane, NT, ty, tx) != 0;
        if (reached) {
            col[(p * NT) + tx] = 1;
            plane[p] = 1;
        }
    }
    const unsigned m = __ballot_sync(0xffffffffu, reached);
    if (i < n) {
        if (NT >= 32) {
            if (lane == 0) tile[prow * words + (tx >> 5)] = m;
        } else if (tx == 0) {
            tile[prow] = (m >> lane) & ((1u << NT) - 1u);
        }
    }
}

// The reached tile columns (col bytes set) appended to list[2 ..], their
// count in list[0] (zeroed beforehand); warp-aggregated atomics, so the order
// is arbitrary (each column's transform does not depend on it).
__global__ void k_col_list(const uint8_t* __restrict__ col, int64_t n, uint32_t* __restrict__ list) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const bool on = i < n && col[i] != 0;
    const unsigned m = __ballot_sync(0xffffffffu, on);
    if (m == 0) return;
    const int lane = threadIdx.x & 31;
    uint32_t base = 0;
    if (lane == 0) base = atomicAdd(list, (uint32_t)__popc(m));
    base = __shfl_sync(0xffffffffu, base, 0);
    if (on) list[2 + base + __popc(m & ((1u << lane) - 1u))] = (uint32_t)i;
}

// The two four-step passes at N = 16384 (k_cols_four); t4: the plan's tables
// of the 128-point transform and of W_N^m after the split row pass's tables.
template <bool INV, bool PRUNED>
cudaError_t columns_four(float2* grids, int64_t n_planes, const float2* t4, const Occupancy& occ,
                         cudaStream_t st) {
    using Sh = Shape<7>;
    const size_t smem = (size_t)(Sh::kTw + 32 * (Sh::kArray + 1)) * sizeof(float2);
    auto fa = k_cols_four<INV, PRUNED, false>;
    auto fb = k_cols_four<INV, PRUNED, true>;
    cudaError_t e = cudaFuncSetAttribute(fa, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e == cudaSuccess) e = cudaFuncSetAttribute(fb, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    int per_sm = 0, dev = 0, sms = 0;
    if ((e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, fa, 256, smem)) != cudaSuccess) return e;
    if ((e = cudaGetDevice(&dev)) != cudaSuccess) return e;
    if ((e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev)) != cudaSuccess) return e;
    if (per_sm < 1) return cudaErrorInvalidConfiguration;
    const unsigned blocks = (unsigned)(per_sm * sms);
    fa<<<blocks, 256, smem, st>>>(grids, t4, occ, (uint32_t)n_planes);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    fb<<<blocks, 256, smem, st>>>(grids, t4, occ, (uint32_t)n_planes);
    return cudaGetLastError();
}

template <int LOG2N, bool INV>
cudaError_t columns_one(float2* grids, int64_t n_planes, const float2* twid, const Occupancy& occ,
                        cudaStream_t st, bool fourstep = false) {
    using Sh = Shape<LOG2N>;
    constexpr int cols = kCols<LOG2N>;
    if (LOG2N == 14 && fourstep) {
        // every (group, n1) and (group, k2) item index below 2^32
        if ((uint64_t)n_planes * 16384u * kFourL / 32u >= (1ull << 32)) return cudaErrorInvalidValue;
        const float2* t4 = twid + Shape<14>::kTw + Shape<12>::kTw + 4 * 256 + 256;
        return occ.list != nullptr && occ.tile != nullptr ? columns_four<INV, true>(grids, n_planes, t4, occ, st)
                                                          : columns_four<INV, false>(grids, n_planes, t4, occ, st);
    }
    const size_t smem = (size_t)(Sh::kTw + cols * (Sh::kArray + 16 / cols)) * sizeof(float2);
    if (occ.list != nullptr && occ.tile != nullptr) {
        // persistent CTAs over the listed tile columns; the work counter
        // list[1] starts at zero for every pass
        auto fl = k_fft_columns_list<LOG2N, cols, INV>;
        cudaError_t e = cudaFuncSetAttribute(fl, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
        int per_sm = 0, dev = 0, sms = 0;
        if ((e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, fl, cols * Sh::T, smem)) != cudaSuccess)
            return e;
        if ((e = cudaGetDevice(&dev)) != cudaSuccess) return e;
        if ((e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev)) != cudaSuccess) return e;
        if (per_sm < 1) return cudaErrorInvalidConfiguration;
        if ((e = cudaMemsetAsync(occ.list + 1, 0, sizeof(uint32_t), st)) != cudaSuccess) return e;
        fl<<<(unsigned)(per_sm * sms), cols * Sh::T, smem, st>>>(grids, twid, occ);
        return cudaGetLastError();
    }
    auto fn = k_fft_columns<LOG2N, cols, INV>;
    cudaError_t e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    for (int64_t p0 = 0; p0 < n_planes; p0 += 65535) {
        const unsigned np = (unsigned)(n_planes - p0 < 65535 ? n_planes - p0 : 65535);
        fn<<<dim3(Sh::N / cols, np), cols * Sh::T, smem, st>>>(grids + p0 * Sh::N * Sh::N, twid, occ, p0);
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

template <int LOG2N, bool CPLX, bool PADDED>
cudaError_t fused_one(const PhaseParams& P, const float2* grids, const double* wsum, const uint2* pix_turns,
                      const float* pix_scale, const float2* twid, float* image_real, float2* image_complex,
                      const Occupancy& occ, cudaStream_t st) {
    using Sh = Shape<LOG2N>;
    auto fn = k_rows_phase_reduce<LOG2N, CPLX, PADDED>;
    // tables, the transform array and the 256 phasors, then per pixel z and
    // (real output) the partial sum
    const size_t smem = (size_t)(Sh::kTw + Sh::kArray + 256) * sizeof(float2) +
                        (size_t)Sh::N * (sizeof(float2) + (CPLX ? 0 : 1) * sizeof(float));
    cudaError_t e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    fn<<<P.Ni, Sh::T, smem, st>>>(P, grids, wsum, pix_turns, pix_scale, twid, image_real, image_complex, occ);
    return cudaGetLastError();
}

// N = 16384: four CTAs per image row, each with the 4096-point tables (they
// follow the 16384-point tables in twid)
template <bool CPLX, bool PADDED>
cudaError_t fused_split(const PhaseParams& P, const float2* grids, const double* wsum, const uint2* pix_turns,
                        const float* pix_scale, const float2* twid, float* image_real, float2* image_complex,
                        const Occupancy& occ, cudaStream_t st) {
    constexpr int kSub = 12, kSplit = 4;
    using Sh = Shape<kSub>;
    auto fn = k_rows_phase_reduce_split<kSub, kSplit, CPLX, PADDED>;
    const size_t smem = (size_t)(Sh::kTw + Sh::kArray + 256) * sizeof(float2) +
                        (size_t)Sh::N * (sizeof(float2) + (CPLX ? 0 : 1) * sizeof(float));
    cudaError_t e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    fn<<<kSplit * P.Ni, Sh::T, smem, st>>>(P, grids, wsum, pix_turns, pix_scale, twid + Shape<14>::kTw,
                                            image_real, image_complex, occ);
    return cudaGetLastError();
}

template <int LOG2N>
cudaError_t fused_n(const PhaseParams& P, const float2* grids, const double* wsum, const uint2* pix_turns,
                    const float* pix_scale, const float2* twid, float* image_real, float2* image_complex,
                    const Occupancy& occ, cudaStream_t st) {
    const bool padded = P.Ni != P.N;
#define RICK_FUSED_ARGS P, grids, wsum, pix_turns, pix_scale, twid, image_real, image_complex, occ, st
    if constexpr (LOG2N == 14) {
        if (image_complex != nullptr)
            return padded ? fused_split<true, true>(RICK_FUSED_ARGS) : fused_split<true, false>(RICK_FUSED_ARGS);
        return padded ? fused_split<false, true>(RICK_FUSED_ARGS) : fused_split<false, false>(RICK_FUSED_ARGS);
    } else {
        if (image_complex != nullptr)
            return padded ? fused_one<LOG2N, true, true>(RICK_FUSED_ARGS) : fused_one<LOG2N, true, false>(RICK_FUSED_ARGS);
        return padded ? fused_one<LOG2N, false, true>(RICK_FUSED_ARGS) : fused_one<LOG2N, false, false>(RICK_FUSED_ARGS);
    }
#undef RICK_FUSED_ARGS
}

int log2_exact(int N) {
    int m = 0;
    while ((1 << m) < N) ++m;
    return (1 << m) == N ? m : -1;
}

}  // namespace

bool fft_supported(int N) {
    const int m = log2_exact(N);
    return m >= 8 && m <= 14;
}

bool fft_fused_model_supported(int N) {
    const int m = log2_exact(N);
    return m >= 8 && m <= 13;
}

namespace {

void append_twiddles(int N, std::vector<float2>& out) {
    // per radix-16 stage s with twiddles (M = 16^s, cnt = N/16/M groups t1),
    // from FP64: stage 0 entries [j cnt + t1] = e^(+2 pi i 2^j t1 M / N), j < 4;
    // later stages [(f0 - 1) cnt + t1] = e^(+2 pi i f0 t1 M / N), f0 = 1..15
    const int log2n = log2_exact(N);
    const int stages = (log2n % 4 == 0) ? log2n / 4 - 1 : log2n / 4;
    const double two_pi = 6.283185307179586476925;
    for (int st = 0; st < stages; ++st) {
        const int64_t M = (int64_t)1 << (4 * st);
        const int cnt = (int)((N / 16) / M);
        const int per = st == 0 ? 4 : 15;
        for (int j = 0; j < per; ++j)
            for (int t1 = 0; t1 < cnt; ++t1) {
                const int64_t f = st == 0 ? ((int64_t)1 << j) : j + 1;
                const int64_t e = (int64_t)t1 * M * f;   // < N
                const double a = two_pi * (double)e / N;
                out.push_back(make_float2((float)std::cos(a), (float)std::sin(a)));
            }
    }
}

}  // namespace

void fft_twiddles(int N, std::vector<float2>& out) {
    // N < 16384: the stage tables, then e^(2 pi i j / 256), j < 256.
    // N = 16384: the 4096-point tables of the split fused row pass follow,
    // then its split twiddles [r T + b] = e^(+2 pi i r b / N), r < 4, b < T = 256,
    // then e^(2 pi i j / 256), j < 256, then the four-step column pass's tables
    out.clear();
    append_twiddles(N, out);
    if (log2_exact(N) < 14) {
        // N < 16384: the 256 phasors e^(2 pi i j / 256) of the fused row pass's
        // block-end phase screen follow the stage tables
        for (int j = 0; j < 256; ++j) {
            const double a = 6.283185307179586476925 * (double)j / 256.0;
            out.push_back(make_float2((float)std::cos(a), (float)std::sin(a)));
        }
    }
    if (log2_exact(N) == 14) {
        append_twiddles(4096, out);
        const double two_pi = 6.283185307179586476925;
        for (int r = 0; r < 4; ++r)
            for (int b = 0; b < 256; ++b) {
                const double a = two_pi * (double)(r * b) / N;
                out.push_back(make_float2((float)std::cos(a), (float)std::sin(a)));
            }
        // and the 256 phasors e^(2 pi i j / 256) of its block-end phase screen
        for (int j = 0; j < 256; ++j) {
            const double a = two_pi * (double)j / 256.0;
            out.push_back(make_float2((float)std::cos(a), (float)std::sin(a)));
        }
        // the four-step column pass: the 128-point tables, e^(2 pi i mh / 128)
        // and e^(2 pi i ml / N), mh, ml < 128
        append_twiddles(kFourL, out);
        for (int j = 0; j < kFourL; ++j) {
            const double a = two_pi * (double)j / kFourL;
            out.push_back(make_float2((float)std::cos(a), (float)std::sin(a)));
        }
        for (int j = 0; j < kFourL; ++j) {
            const double a = two_pi * (double)j / N;
            out.push_back(make_float2((float)std::cos(a), (float)std::sin(a)));
        }
    }
}

cudaError_t launch_fft2d(float2* grids, int64_t n_planes, int N, bool inverse, const float2* twid,
                         cudaStream_t st, int* launches) {
    if (n_planes <= 0) return cudaSuccess;
    cudaError_t e = cudaErrorInvalidValue;
#define RICK_FFT_CASE(LG)                                                                   \
    case LG:                                                                                \
        e = inverse ? columns_one<LG, true>(grids, n_planes, twid, Occupancy{}, st)         \
                    : columns_one<LG, false>(grids, n_planes, twid, Occupancy{}, st);       \
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
        RICK_FFT_CASE(14)
        default: break;
    }
#undef RICK_FFT_CASE
    if (e == cudaSuccess) *launches += 2 * (int)((n_planes + 65534) / 65535);
    return e;
}

cudaError_t launch_fft_columns(float2* grids, int64_t n_planes, int N, bool inverse, const float2* twid,
                               const Occupancy& occ, cudaStream_t st, int* launches, bool fourstep) {
    if (n_planes <= 0) return cudaSuccess;
    cudaError_t e = cudaErrorInvalidValue;
#define RICK_FFT_CASE(LG)                                                                   \
    case LG:                                                                                \
        e = inverse ? columns_one<LG, true>(grids, n_planes, twid, occ, st, fourstep)       \
                    : columns_one<LG, false>(grids, n_planes, twid, occ, st, fourstep);     \
        break;
    switch (log2_exact(N)) {
        RICK_FFT_CASE(8)
        RICK_FFT_CASE(9)
        RICK_FFT_CASE(10)
        RICK_FFT_CASE(11)
        RICK_FFT_CASE(12)
        RICK_FFT_CASE(13)
        RICK_FFT_CASE(14)
        default: break;
    }
#undef RICK_FFT_CASE
    if (e == cudaSuccess) *launches += fourstep && N == 16384 ? 2 : (int)((n_planes + 65534) / 65535);
    return e;
}

cudaError_t launch_rows_phase_reduce(const PhaseParams& P, const float2* grids, const double* wsum,
                                     const uint2* pix_turns, const float* pix_scale, const float2* twid,
                                     float* image_real, float2* image_complex, const Occupancy& occ,
                                     cudaStream_t st, int* launches) {
    cudaError_t e = cudaErrorInvalidValue;
#define RICK_FUSED_CASE(LG)                                                                              \
    case LG:                                                                                             \
        e = fused_n<LG>(P, grids, wsum, pix_turns, pix_scale, twid, image_real, image_complex, occ, st); \
        break;
    switch (log2_exact(P.N)) {
        RICK_FUSED_CASE(8)
        RICK_FUSED_CASE(9)
        RICK_FUSED_CASE(10)
        RICK_FUSED_CASE(11)
        RICK_FUSED_CASE(12)
        RICK_FUSED_CASE(13)
        RICK_FUSED_CASE(14)
        default: break;
    }
#undef RICK_FUSED_CASE
    if (e == cudaSuccess) ++*launches;
    return e;
}

cudaError_t launch_model_rows(const PhaseParams& P, const float* image, const uint2* pix_turns,
                              const float* pix_model_scale, const float2* twid, float2* grids,
                              const Occupancy& occ, cudaStream_t st, int* launches) {
    cudaError_t e = cudaErrorInvalidValue;
#define RICK_MODEL_CASE(LG)                                                                         \
    case LG: {                                                                                      \
        using Sh = Shape<LG>;                                                                       \
        auto fn = k_model_rows<LG>;                                                                 \
        const size_t smem = (size_t)(Sh::kTw + Sh::kArray + Sh::N) * sizeof(float2) + (size_t)Sh::N * sizeof(float); \
        e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);      \
        if (e == cudaSuccess) {                                                                     \
            fn<<<Sh::N, Sh::T, smem, st>>>(P, image, pix_turns, pix_model_scale, twid, grids, occ); \
            e = cudaGetLastError();                                                                 \
        }                                                                                           \
        break;                                                                                      \
    }
    switch (log2_exact(P.N)) {
        RICK_MODEL_CASE(8)
        RICK_MODEL_CASE(9)
        RICK_MODEL_CASE(10)
        RICK_MODEL_CASE(11)
        RICK_MODEL_CASE(12)
        RICK_MODEL_CASE(13)
        default: break;
    }
#undef RICK_MODEL_CASE
    if (e == cudaSuccess) ++*launches;
    return e;
}

cudaError_t launch_pixel_phase(const PhaseParams& P0, const float* inv_taper, uint2* turns, float* scale,
                               float* model_scale, cudaStream_t st) {
    const int64_t n = (int64_t)P0.Ni * P0.Ni;
    k_pixel_phase<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(P0, inv_taper, turns, scale, model_scale);
    return cudaGetLastError();
}

cudaError_t launch_occupancy(const uint32_t* offsets, int c0, int nc, int k0, int nk, int Nw_store, int NT,
                             uint8_t* col, uint8_t* plane, uint32_t* tile, uint32_t* list, cudaStream_t st,
                             int* launches) {
    const int64_t n = (int64_t)nc * nk * NT * NT;
    if (n <= 0) return cudaSuccess;
    cudaError_t e = cudaMemsetAsync(plane, 0, (size_t)nc * nk, st);
    if (e == cudaSuccess) e = cudaMemsetAsync(col, 0, (size_t)nc * nk * NT, st);
    if (e != cudaSuccess) return e;
    const int words = (NT + 31) / 32;
    k_occupancy<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(offsets, c0, nc, k0, nk, Nw_store, NT, words, col,
                                                             plane, tile);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    ++*launches;
    if (list != nullptr) {
        const int64_t nl = (int64_t)nc * nk * NT;
        if ((e = cudaMemsetAsync(list, 0, 2 * sizeof(uint32_t), st)) != cudaSuccess) return e;
        k_col_list<<<(unsigned)((nl + 255) / 256), 256, 0, st>>>(col, nl, list);
        if ((e = cudaGetLastError()) != cudaSuccess) return e;
        ++*launches;
    }
    return cudaSuccess;
}

}  // namespace rick

// rick_learn.cu -- training objective of the learned support-4 kernel.
//
// A fixed visibility sample (one observation's u, v, w and weights) is placed
// once (FP64, the same rules as the gridder) and sorted by w-plane.  For each
// training field (point sources on pixel centres) the kernels
//   1. predict the visibilities from the sources (Eq. 1),
//   2. evaluate at probe pixels both the w-stacking image that the gridder,
//      FFT and phase screen would produce with the current tap table (Eq. 2,
//      Eq. 3, written per visibility as in the oracle's per-pixel form) and
//      the direct Fourier inversion of the same visibilities,
//   3. form the loss sum_P (I_P - D_P)^2 / sum_P D_P^2, and
//   4. back-propagate it to the tap table (bilinear lattice, per plane),
// after which rick_mlp_backward carries the table gradient into the network.
// The table holds a correction added to the support-4 Kaiser-Bessel taps (so a
// zero table is the Kaiser-Bessel kernel); its gradient is the tap gradient.
//
// Phases: with x = u fov + N/2 the continuous cell position, u l_p =
// (x - N/2)(p - N/2)/N turns.  x - N/2 = X + f with X integer, so the turn is
// (X (p - N/2) mod N)/N + f (p - N/2)/N: exact integer reduction plus a term
// below half a turn, which FP32 carries to ~3e-8 turns.
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <vector>

#include "rick_internal.cuh"

namespace rick {
void set_error_message(const char* msg);
int64_t mlp_param_count(int H);
}

using namespace rick;

namespace {

constexpr int kMaxProbes = 64;
constexpr int kMaxSources = 64;
constexpr int kLearnS = 4;
constexpr int kChunk = 4096;

struct __align__(16) LearnVis {
    int i0, j0, k, pad;
    float fx, fy, w, W;
};

struct LearnConst {
    int N, Nw, L, nvis, ns, np;
    float inv_wsum;
};

// ---- placement --------------------------------------------------------------

__global__ void k_learn_place(const double* __restrict__ uvw, const float* __restrict__ weight,
                              int64_t nvis, int N, int Nw, double fov, double w_min,
                              double w_scale, LearnVis* __restrict__ out, int* __restrict__ status,
                              unsigned* __restrict__ plane_count) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= nvis) return;
    LearnVis v = {0, 0, -1, 0, 0.f, 0.f, 0.f, 0.f};
    int st = 0;
    const float W = weight[i];
    if (W != 0.0f && isfinite(W)) {
        const double u = uvw[3 * i], vv = uvw[3 * i + 1], w = uvw[3 * i + 2];
        const double x = __dadd_rn(__dmul_rn(u, fov), 0.5 * N);
        const double y = __dadd_rn(__dmul_rn(vv, fov), 0.5 * N);
        const double sx = __dsub_rn(x, 0.5 * kLearnS), sy = __dsub_rn(y, 0.5 * kLearnS);
        const double flx = floor(sx), fly = floor(sy);
        if (isfinite(x) && isfinite(y) && isfinite(w) && flx >= -1.0 && fly >= -1.0 &&
            flx + kLearnS <= N - 1 && fly + kLearnS <= N - 1) {
            v.i0 = (int)flx + 1;
            v.j0 = (int)fly + 1;
            v.fx = (float)__dsub_rn(sx, flx);
            v.fy = (float)__dsub_rn(sy, fly);
            int k = 0;
            if (Nw > 1) {
                double kf = floor(__dmul_rn(__dsub_rn(w, w_min), w_scale));
                kf = fmin(fmax(kf, 0.0), (double)(Nw - 1));
                k = (int)kf;
            }
            v.k = k;
            v.w = (float)w;
            v.W = W;
            st = 1;
            atomicAdd(&plane_count[k], 1u);
        } else {
            st = -1;
        }
    }
    out[i] = v;
    status[i] = st;
}

__global__ void k_learn_sort(const LearnVis* __restrict__ in, int64_t nvis,
                             unsigned* __restrict__ cursor, LearnVis* __restrict__ out) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= nvis) return;
    const LearnVis v = in[i];
    if (v.k < 0) return;
    out[atomicAdd(&cursor[v.k], 1u)] = v;
}

// ---- per field ---------------------------------------------------------------

__device__ __forceinline__ float2 turn_phasor(float t) {  // exp(2 pi i t), t reduced first
    float s, c;
    sincospif(2.0f * (t - rintf(t)), &s, &c);
    return make_float2(c, s);
}

// (X * P mod N)/N + f P / N, in turns, for integer X, P and f in [0, 1)
__device__ __forceinline__ float cell_turns(int X, int P, float f, int N) {
    const long long xp = (long long)X * P;
    long long r = xp % N;
    if (r < 0) r += N;
    return (float)r / (float)N + f * (float)P / (float)N;
}

__device__ __forceinline__ float2 cmulf(float2 a, float2 b) {
    return make_float2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}

// The turns of u l for a source at pixel offset P = p - N/2 (any real p):
// with P = Pi + Pf (Pi integer, 0 <= Pf < 1), (X + f)(Pi + Pf)/N is the exact
// integer reduction of X Pi plus f Pi/N plus (X + f) Pf / N, each below half a
// turn in magnitude.
__device__ __forceinline__ float source_turns(int X, float P, float f, int N) {
    const float Pi = floorf(P);
    return cell_turns(X, (int)Pi, f, N) + ((float)X + f) * (P - Pi) / (float)N;
}

// V_j W_j for the field: sources src[s] = (P_s, Q_s, A_s / n_s, delta_s) with
// P_s = p_s - N/2, Q_s = q_s - N/2 (pixel offsets from the centre; p_s, q_s
// continuous positions in pixels).
__global__ void k_learn_predict(const LearnVis* __restrict__ vis, LearnConst C,
                                const float4* __restrict__ src, float2* __restrict__ wv) {
    __shared__ float4 s_src[kMaxSources];
    for (int s = threadIdx.x; s < C.ns; s += blockDim.x) s_src[s] = src[s];
    __syncthreads();
    const int j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= C.nvis) return;
    const LearnVis v = vis[j];
    const int X = v.i0 - 1 + kLearnS / 2 - C.N / 2, Y = v.j0 - 1 + kLearnS / 2 - C.N / 2;
    float2 acc = make_float2(0.f, 0.f);
    for (int s = 0; s < C.ns; ++s) {
        const float4 q = s_src[s];
        const float t = source_turns(X, q.x, v.fx, C.N) + source_turns(Y, q.y, v.fy, C.N) + v.w * q.w;
        const float2 e = turn_phasor(-t);  // Eq. 1: exp(-2 pi i (u l + v m + w (n - 1)))
        acc.x += q.z * e.x;
        acc.y += q.z * e.y;
    }
    wv[j] = make_float2(v.W * acc.x, v.W * acc.y);
}

// The support-4 Kaiser-Bessel taps as polynomials in 2f - 1 (fitted on the host).
struct KbTaps {
    float coef[4][kPolyDegree + 1];
};

__device__ __forceinline__ float kb_tap(const KbTaps& K, int a, float t) {
    float acc = K.coef[a][kPolyDegree];
#pragma unroll
    for (int q = kPolyDegree - 1; q >= 0; --q) acc = fmaf(acc, t, K.coef[a][q]);
    return acc;
}

// Taps of visibility v: the Kaiser-Bessel products plus the correction
// interpolated (bilinearly) from the table, t[b*4 + a].
__device__ __forceinline__ void learn_taps(const float* __restrict__ table, int L, const LearnVis& v,
                                           const KbTaps& K, float* t) {
    const float X = v.fx * L, Y = v.fy * L;
    const int ix = min((int)X, L - 1), iy = min((int)Y, L - 1);
    const float ax = X - ix, ay = Y - iy;
    const size_t row = (size_t)(L + 1);
    const float* t00 = table + (((size_t)v.k * row + iy) * row + ix) * 16;
    const float* t01 = t00 + row * 16;
    const float w00 = (1.f - ax) * (1.f - ay), w10 = ax * (1.f - ay), w01 = (1.f - ax) * ay, w11 = ax * ay;
    const float tx = fmaf(2.0f, v.fx, -1.0f), ty = fmaf(2.0f, v.fy, -1.0f);
    float gx[4], gy[4];
#pragma unroll
    for (int a = 0; a < 4; ++a) {
        gx[a] = kb_tap(K, a, tx);
        gy[a] = kb_tap(K, a, ty);
    }
#pragma unroll
    for (int q = 0; q < 16; ++q)
        t[q] = gx[q & 3] * gy[q >> 2] + w00 * __ldg(t00 + q) + w10 * __ldg(t00 + 16 + q) +
               w01 * __ldg(t01 + q) + w11 * __ldg(t01 + 16 + q);
}

// Probe data in shared memory: per probe p, q (absolute), P = p - N/2, Q,
// image scale (-1)^(p+q) n / (C(p) C(q)), DFT scale n, delta; per (plane, probe)
// the phasor exp(2 pi i w_k delta_P).
struct ProbeSmem {
    int p[kMaxProbes], q[kMaxProbes];
    float scale_img[kMaxProbes], scale_dft[kMaxProbes], delta[kMaxProbes];
};

__device__ __forceinline__ void image_and_dft_terms(const LearnVis& v, float2 wv, const float* taps,
                                                    int P, const ProbeSmem& pr,
                                                    const float2* __restrict__ ph, int N,
                                                    float* img, float* dft, float* gt /* nullable, 16 */,
                                                    float ge) {
    const int p = pr.p[P], q = pr.q[P];
    // E_x(i0 + a) = (-1)^(i0+a) exp(2 pi i (i0 + a) p / N), likewise E_y
    const long long ip = ((long long)v.i0 * p) % N, jq = ((long long)v.j0 * q) % N;
    float2 ex = turn_phasor((float)ip / (float)N), ey = turn_phasor((float)jq / (float)N);
    const float2 sx = turn_phasor((float)p / (float)N), sy = turn_phasor((float)q / (float)N);
    if (v.i0 & 1) ex = make_float2(-ex.x, -ex.y);
    if (v.j0 & 1) ey = make_float2(-ey.x, -ey.y);
    float2 Ex[4], Ey[4];
#pragma unroll
    for (int a = 0; a < 4; ++a) {
        Ex[a] = ex;
        Ey[a] = ey;
        ex = cmulf(ex, make_float2(-sx.x, -sx.y));
        ey = cmulf(ey, make_float2(-sy.x, -sy.y));
    }
    const float2 c = cmulf(wv, ph[v.k * kMaxProbes + P]);  // W V exp(2 pi i w_k delta)
    const float si = pr.scale_img[P];
    if (img) {
        float2 s = make_float2(0.f, 0.f);
#pragma unroll
        for (int b = 0; b < 4; ++b) {
            float2 r = make_float2(0.f, 0.f);
#pragma unroll
            for (int a = 0; a < 4; ++a) {
                r.x += taps[4 * b + a] * Ex[a].x;
                r.y += taps[4 * b + a] * Ex[a].y;
            }
            s = make_float2(s.x + r.x * Ey[b].x - r.y * Ey[b].y, s.y + r.x * Ey[b].y + r.y * Ey[b].x);
        }
        *img = si * (c.x * s.x - c.y * s.y);
        // direct inversion: exp(+2 pi i (u l_P + v m_P + w delta_P))
        const int X = v.i0 - 1 + kLearnS / 2 - N / 2, Y = v.j0 - 1 + kLearnS / 2 - N / 2;
        const float t = cell_turns(X, p - N / 2, v.fx, N) + cell_turns(Y, q - N / 2, v.fy, N) +
                        v.w * pr.delta[P];
        const float2 e = turn_phasor(t);
        *dft = pr.scale_dft[P] * (wv.x * e.x - wv.y * e.y);
    }
    if (gt) {
        const float g = ge * si;
#pragma unroll
        for (int b = 0; b < 4; ++b) {
            const float2 cb = cmulf(c, Ey[b]);
#pragma unroll
            for (int a = 0; a < 4; ++a) gt[4 * b + a] += g * (cb.x * Ex[a].x - cb.y * Ex[a].y);
        }
    }
}

__device__ __forceinline__ void load_probes(ProbeSmem& pr, float2* s_ph, const int* __restrict__ pq,
                                            const float4* __restrict__ pconst,
                                            const float2* __restrict__ ph, int np, int Nw) {
    for (int i = threadIdx.x; i < np; i += blockDim.x) {
        pr.p[i] = pq[2 * i];
        pr.q[i] = pq[2 * i + 1];
        const float4 c = pconst[i];
        pr.scale_img[i] = c.x;
        pr.scale_dft[i] = c.y;
        pr.delta[i] = c.z;
    }
    for (int i = threadIdx.x; i < Nw * kMaxProbes; i += blockDim.x) s_ph[i] = ph[i];
}

// I_P and D_P accumulated over all visibilities (out[2P], out[2P+1]).
__global__ void __launch_bounds__(256)
k_learn_forward(const LearnVis* __restrict__ vis, const float2* __restrict__ wv,
                const float* __restrict__ table, LearnConst C, KbTaps K, const int* __restrict__ pq,
                const float4* __restrict__ pconst, const float2* __restrict__ ph,
                float* __restrict__ out) {
    __shared__ ProbeSmem pr;
    extern __shared__ float2 s_ph[];
    __shared__ float s_acc[2 * kMaxProbes];
    load_probes(pr, s_ph, pq, pconst, ph, C.np, C.Nw);
    for (int i = threadIdx.x; i < 2 * kMaxProbes; i += blockDim.x) s_acc[i] = 0.f;
    __syncthreads();
    const int lane = threadIdx.x & 31;
    for (int base = blockIdx.x * blockDim.x; base < C.nvis; base += gridDim.x * blockDim.x) {
        const int j = base + threadIdx.x;
        const bool ok = j < C.nvis;
        LearnVis v = {0, 0, 0, 0, 0.f, 0.f, 0.f, 0.f};
        float2 w2 = make_float2(0.f, 0.f);
        float taps[16];
        if (ok) {
            v = vis[j];
            w2 = wv[j];
            learn_taps(table, C.L, v, K, taps);
        } else {
#pragma unroll
            for (int q = 0; q < 16; ++q) taps[q] = 0.f;
        }
        for (int P = 0; P < C.np; ++P) {
            float im = 0.f, df = 0.f;
            if (ok) image_and_dft_terms(v, w2, taps, P, pr, s_ph, C.N, &im, &df, nullptr, 0.f);
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) {
                im += __shfl_xor_sync(0xffffffffu, im, o);
                df += __shfl_xor_sync(0xffffffffu, df, o);
            }
            if (lane == 0) {
                atomicAdd(&s_acc[2 * P], im);
                atomicAdd(&s_acc[2 * P + 1], df);
            }
        }
    }
    __syncthreads();
    for (int i = threadIdx.x; i < 2 * C.np; i += blockDim.x) atomicAdd(&out[i], s_acc[i] * C.inv_wsum);
}

// loss = sum (I - D)^2 / sum D^2; ge[P] = dloss/dI_P (scaled by 1/sum W, which
// the backward kernel's per-visibility terms omit).
__global__ void k_learn_loss(const float* __restrict__ idft, int np, float inv_wsum,
                             float* __restrict__ loss, float* __restrict__ ge) {
    if (threadIdx.x != 0 || blockIdx.x != 0) return;
    float num = 0.f, den = 0.f;
    for (int P = 0; P < np; ++P) {
        const float e = idft[2 * P] - idft[2 * P + 1];
        num += e * e;
        den += idft[2 * P + 1] * idft[2 * P + 1];
    }
    den = fmaxf(den, 1e-30f);
    *loss = num / den;
    for (int P = 0; P < np; ++P) ge[P] = 2.f * (idft[2 * P] - idft[2 * P + 1]) / den * inv_wsum;
}

// d loss / d table: per visibility the 16 tap gradients, spread bilinearly onto
// the lattice of its plane in shared memory, then added to the global gradient.
__global__ void __launch_bounds__(256)
k_learn_backward(const LearnVis* __restrict__ vis, const float2* __restrict__ wv, LearnConst C,
                 const int* __restrict__ chunks /* [n][3]: plane, begin, end */,
                 const int* __restrict__ pq, const float4* __restrict__ pconst,
                 const float2* __restrict__ ph, const float* __restrict__ ge,
                 float* __restrict__ table_grad) {
    __shared__ ProbeSmem pr;
    __shared__ float s_ge[kMaxProbes];
    extern __shared__ float2 s_dyn[];
    float2* s_ph = s_dyn;
    float* s_tg = reinterpret_cast<float*>(s_dyn + C.Nw * kMaxProbes);
    const int L1 = C.L + 1;
    const int ntg = L1 * L1 * 16;
    load_probes(pr, s_ph, pq, pconst, ph, C.np, C.Nw);
    for (int i = threadIdx.x; i < C.np; i += blockDim.x) s_ge[i] = ge[i];
    for (int i = threadIdx.x; i < ntg; i += blockDim.x) s_tg[i] = 0.f;
    __syncthreads();
    const int k = chunks[3 * blockIdx.x], jb = chunks[3 * blockIdx.x + 1], je = chunks[3 * blockIdx.x + 2];
    for (int j = jb + threadIdx.x; j < je; j += blockDim.x) {
        const LearnVis v = vis[j];
        const float2 w2 = wv[j];
        float gt[16];
#pragma unroll
        for (int q = 0; q < 16; ++q) gt[q] = 0.f;
        for (int P = 0; P < C.np; ++P)
            image_and_dft_terms(v, w2, nullptr, P, pr, s_ph, C.N, nullptr, nullptr, gt, s_ge[P]);
        const float X = v.fx * C.L, Y = v.fy * C.L;
        const int ix = min((int)X, C.L - 1), iy = min((int)Y, C.L - 1);
        const float ax = X - ix, ay = Y - iy;
        const float wc[4] = {(1.f - ax) * (1.f - ay), ax * (1.f - ay), (1.f - ax) * ay, ax * ay};
        const int base[4] = {(iy * L1 + ix) * 16, (iy * L1 + ix + 1) * 16, ((iy + 1) * L1 + ix) * 16,
                             ((iy + 1) * L1 + ix + 1) * 16};
#pragma unroll
        for (int cidx = 0; cidx < 4; ++cidx)
#pragma unroll
            for (int q = 0; q < 16; ++q) atomicAdd(&s_tg[base[cidx] + q], wc[cidx] * gt[q]);
    }
    __syncthreads();
    float* g = table_grad + (size_t)k * ntg;
    for (int i = threadIdx.x; i < ntg; i += blockDim.x)
        if (s_tg[i] != 0.f) atomicAdd(&g[i], s_tg[i]);
}

}  // namespace

// ============================================================================

struct rick_learn {
    rick_config cfg;
    int L = 0;
    int64_t n_in = 0;
    int nvis = 0;       // placed visibilities
    double wsum = 0.0;
    std::vector<double> taper;
    LearnVis* d_vis = nullptr;
    float2* d_wv = nullptr;
    int* d_chunks = nullptr;
    int n_chunks = 0;
    float4* d_src = nullptr;
    int* d_pq = nullptr;
    float4* d_pconst = nullptr;
    float2* d_ph = nullptr;
    float* d_idft = nullptr;  // [2 * kMaxProbes]
    float* d_ge = nullptr;
    KbTaps kb4;  // fitted support-4 Kaiser-Bessel taps the correction adds to
};

namespace {

void learn_free(rick_learn* Lr) {
    cudaFree(Lr->d_vis);
    cudaFree(Lr->d_wv);
    cudaFree(Lr->d_chunks);
    cudaFree(Lr->d_src);
    cudaFree(Lr->d_pq);
    cudaFree(Lr->d_pconst);
    cudaFree(Lr->d_ph);
    cudaFree(Lr->d_idft);
    cudaFree(Lr->d_ge);
}

rick_status lfail(rick_status s, const char* m) {
    set_error_message(m);
    return s;
}

double host_i0(double x) {
    const double y = 0.25 * x * x;
    double term = 1.0, sum = 1.0;
    for (int k = 1; k < 400 && term > 1e-17 * sum; ++k) {
        term *= y / ((double)k * k);
        sum += term;
    }
    return sum;
}

}  // namespace

extern "C" {

rick_status rick_learn_create(const rick_config* cfg, int32_t lattice, const double* uvw,
                              const float* weight, int64_t nvis, rick_learn** out) {
    if (!cfg || !out || !uvw || !weight) return lfail(RICK_ERR_INVALID_ARG, "invalid argument: learn inputs");
    *out = nullptr;
    const rick_config& c = *cfg;
    if (c.kernel_kind != RICK_KERNEL_TABLE || c.support != kLearnS || c.n_channels != 1 ||
        c.N < 64 || (c.N & (c.N - 1)) || c.n_wplanes < 1 || !(c.fov_rad > 0 && c.fov_rad < 1) ||
        (c.n_wplanes > 1 && !(c.w_max > c.w_min)) || lattice < 1 || lattice > 64 || nvis < 1 ||
        nvis > (1ll << 30) || c.hermitian_fold != 0 || c.w_support >= 2 ||
        c.weighting != RICK_WEIGHT_NATURAL || (c.grid_size != 0 && c.grid_size != c.N))
        return lfail(RICK_ERR_INVALID_ARG,
                     "invalid argument: learning needs a table kernel of support 4, one channel, "
                     "no Hermitian fold, no w-kernel, natural weighting, 1 <= lattice <= 64 and "
                     "1 <= nvis <= 2^30");
    rick_learn* Lr = new rick_learn();
    Lr->cfg = c;
    Lr->L = lattice;
    Lr->n_in = nvis;
    const int N = c.N, Nw = c.n_wplanes;
    const double w_scale = Nw > 1 ? (double)Nw / (c.w_max - c.w_min) : 0.0;
    LearnVis* tmp = nullptr;
    int* status = nullptr;
    unsigned* cnt = nullptr;
    cudaError_t e = cudaSuccess;
    auto chk = [&](cudaError_t x) { if (e == cudaSuccess) e = x; };
    chk(cudaMalloc(&tmp, sizeof(LearnVis) * nvis));
    chk(cudaMalloc(&status, sizeof(int) * nvis));
    chk(cudaMalloc(&cnt, sizeof(unsigned) * Nw * 2));
    chk(cudaMalloc(&Lr->d_vis, sizeof(LearnVis) * nvis));
    chk(cudaMalloc(&Lr->d_wv, sizeof(float2) * nvis));
    chk(cudaMalloc(&Lr->d_src, sizeof(float4) * kMaxSources));
    chk(cudaMalloc(&Lr->d_pq, sizeof(int) * 2 * kMaxProbes));
    chk(cudaMalloc(&Lr->d_pconst, sizeof(float4) * kMaxProbes));
    chk(cudaMalloc(&Lr->d_ph, sizeof(float2) * Nw * kMaxProbes));
    chk(cudaMalloc(&Lr->d_idft, sizeof(float) * 2 * kMaxProbes));
    chk(cudaMalloc(&Lr->d_ge, sizeof(float) * kMaxProbes));
    if (e == cudaSuccess) chk(cudaMemset(cnt, 0, sizeof(unsigned) * Nw * 2));
    if (e == cudaSuccess) {
        k_learn_place<<<(unsigned)((nvis + 255) / 256), 256>>>(uvw, weight, nvis, N, Nw, c.fov_rad,
                                                               c.w_min, w_scale, tmp, status, cnt);
        chk(cudaGetLastError());
    }
    std::vector<unsigned> counts(Nw);
    if (e == cudaSuccess) chk(cudaMemcpy(counts.data(), cnt, sizeof(unsigned) * Nw, cudaMemcpyDeviceToHost));
    std::vector<unsigned> off(Nw + 1, 0);
    for (int k = 0; k < Nw; ++k) off[k + 1] = off[k] + counts[k];
    Lr->nvis = (int)off[Nw];
    if (e == cudaSuccess) chk(cudaMemcpy(cnt + Nw, off.data(), sizeof(unsigned) * Nw, cudaMemcpyHostToDevice));
    if (e == cudaSuccess) {
        k_learn_sort<<<(unsigned)((nvis + 255) / 256), 256>>>(tmp, nvis, cnt + Nw, Lr->d_vis);
        chk(cudaGetLastError());
    }
    // chunks of one plane each
    std::vector<int> chunks;
    for (int k = 0; k < Nw; ++k)
        for (unsigned b = off[k]; b < off[k + 1]; b += kChunk) {
            chunks.push_back(k);
            chunks.push_back((int)b);
            chunks.push_back((int)std::min<unsigned>(off[k + 1], b + kChunk));
        }
    Lr->n_chunks = (int)(chunks.size() / 3);
    if (e == cudaSuccess && Lr->n_chunks) {
        chk(cudaMalloc(&Lr->d_chunks, sizeof(int) * chunks.size()));
        if (e == cudaSuccess)
            chk(cudaMemcpy(Lr->d_chunks, chunks.data(), sizeof(int) * chunks.size(), cudaMemcpyHostToDevice));
    }
    // sum of weights of the placed visibilities (host, FP64)
    if (e == cudaSuccess) {
        std::vector<LearnVis> hv(Lr->nvis);
        chk(cudaMemcpy(hv.data(), Lr->d_vis, sizeof(LearnVis) * Lr->nvis, cudaMemcpyDeviceToHost));
        double ws = 0.0;
        for (const LearnVis& v : hv) ws += v.W;
        Lr->wsum = ws;
    }
    cudaFree(tmp);
    cudaFree(status);
    cudaFree(cnt);
    if (e != cudaSuccess) {
        learn_free(Lr);
        delete Lr;
        char m[200];
        snprintf(m, sizeof m, "rick_learn_create: %s", cudaGetErrorString(e));
        return lfail(e == cudaErrorMemoryAllocation ? RICK_ERR_OOM : RICK_ERR_CUDA, m);
    }
    // taper of the support-4 Kaiser-Bessel (the learned kernel's fixed taper)
    Lr->taper.resize(N);
    {
        const double beta = c.kernel_param, i0b = host_i0(beta);
        const int ng = 24;
        std::vector<double> gx(ng), gw(ng);
        const double pi = 3.14159265358979323846;
        for (int i = 0; i < (ng + 1) / 2; ++i) {
            double z = std::cos(pi * (i + 0.75) / (ng + 0.5)), dp = 1.0;
            for (int it = 0; it < 64; ++it) {
                double pm = 1.0, pc = z;
                for (int k = 2; k <= ng; ++k) {
                    const double pn = ((2 * k - 1) * z * pc - (k - 1) * pm) / k;
                    pm = pc;
                    pc = pn;
                }
                dp = ng * (z * pc - pm) / (z * z - 1.0);
                const double dz = pc / dp;
                z -= dz;
                if (std::fabs(dz) < 1e-16) break;
            }
            gx[i] = -z;
            gx[ng - 1 - i] = z;
            gw[i] = gw[ng - 1 - i] = 2.0 / ((1.0 - z * z) * dp * dp);
        }
        for (int p = 0; p < N; ++p) {
            double acc = 0.0;
            for (int seg = 0; seg < kLearnS; ++seg)
                for (int i = 0; i < ng; ++i) {
                    const double s = -0.5 * kLearnS + seg + 0.5 + 0.5 * gx[i];
                    const double t = 2.0 * s / kLearnS;
                    const double g = host_i0(beta * std::sqrt(std::fmax(0.0, 1.0 - t * t))) / i0b;
                    acc += 0.5 * gw[i] * g * std::cos(2.0 * pi * s * (p - N / 2) / N);
                }
            Lr->taper[p] = acc;
        }
    }
    {
        GridParams fit;
        fit_tap_polynomials(RICK_KERNEL_KAISER_BESSEL, c.kernel_param, kLearnS, fit);
        for (int a = 0; a < 4; ++a)
            for (int q = 0; q <= kPolyDegree; ++q) Lr->kb4.coef[a][q] = fit.coef[a][q];
    }
    *out = Lr;
    return RICK_OK;
}

rick_status rick_learn_destroy(rick_learn* Lr) {
    if (!Lr) return RICK_OK;
    learn_free(Lr);
    delete Lr;
    return RICK_OK;
}

rick_status rick_learn_field_grad(rick_learn* Lr, const float* table, const float* sources,
                                  int32_t ns, const int32_t* probes, int32_t np, float* table_grad,
                                  int32_t accumulate, float grad_scale, float* loss,
                                  float* image_dft, void* stream) {
    if (!Lr || !table || !sources || !probes || !loss)
        return lfail(RICK_ERR_INVALID_ARG, "invalid argument: learn field inputs");
    if (ns < 1 || ns > kMaxSources || np < 1 || np > kMaxProbes)
        return lfail(RICK_ERR_INVALID_ARG, "invalid argument: 1..64 sources and 1..64 probes");
    const rick_config& c = Lr->cfg;
    const int N = c.N, Nw = c.n_wplanes, L = Lr->L;
    const double dl = c.fov_rad / N;
    cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
    // per-source and per-probe constants in FP64 on the host
    std::vector<float4> src(ns), pconst(np);
    std::vector<int> pq(2 * np);
    std::vector<float2> ph((size_t)Nw * kMaxProbes, make_float2(0.f, 0.f));
    for (int s = 0; s < ns; ++s) {
        const double p = sources[3 * s], q = sources[3 * s + 1];
        if (!(p >= 0.0 && p < N && q >= 0.0 && q < N))
            return lfail(RICK_ERR_INVALID_ARG, "source outside the image");
        const double l = (p - N / 2) * dl, m = (q - N / 2) * dl, r2 = l * l + m * m;
        const double n = std::sqrt(1.0 - r2);
        src[s] = make_float4((float)(p - N / 2), (float)(q - N / 2), (float)(sources[3 * s + 2] / n),
                             (float)(-r2 / (1.0 + n)));
    }
    const double dw = Nw > 1 ? (c.w_max - c.w_min) / Nw : 0.0;
    for (int P = 0; P < np; ++P) {
        const int p = probes[2 * P], q = probes[2 * P + 1];
        if (p < 0 || p >= N || q < 0 || q >= N) return lfail(RICK_ERR_INVALID_ARG, "probe outside the image");
        pq[2 * P] = p;
        pq[2 * P + 1] = q;
        const double l = (p - N / 2) * dl, m = (q - N / 2) * dl, r2 = l * l + m * m;
        const double n = std::sqrt(1.0 - r2), delta = -r2 / (1.0 + n);
        const double sg = ((p + q) & 1) ? -1.0 : 1.0;
        pconst[P] = make_float4((float)(sg * n / (Lr->taper[p] * Lr->taper[q])), (float)n, (float)delta, 0.f);
        for (int k = 0; k < Nw; ++k) {
            const double wk = Nw > 1 ? c.w_min + (k + 0.5) * dw : 0.5 * (c.w_min + c.w_max);
            double t = wk * delta;
            t -= std::floor(t + 0.5);
            ph[(size_t)k * kMaxProbes + P] = make_float2((float)std::cos(2 * 3.14159265358979323846 * t),
                                                         (float)std::sin(2 * 3.14159265358979323846 * t));
        }
    }
    cudaError_t e = cudaSuccess;
    auto chk = [&](cudaError_t x) { if (e == cudaSuccess) e = x; };
    chk(cudaMemcpyAsync(Lr->d_src, src.data(), sizeof(float4) * ns, cudaMemcpyHostToDevice, st));
    chk(cudaMemcpyAsync(Lr->d_pq, pq.data(), sizeof(int) * 2 * np, cudaMemcpyHostToDevice, st));
    chk(cudaMemcpyAsync(Lr->d_pconst, pconst.data(), sizeof(float4) * np, cudaMemcpyHostToDevice, st));
    chk(cudaMemcpyAsync(Lr->d_ph, ph.data(), sizeof(float2) * ph.size(), cudaMemcpyHostToDevice, st));
    chk(cudaMemsetAsync(Lr->d_idft, 0, sizeof(float) * 2 * kMaxProbes, st));
    LearnConst C{N, Nw, L, Lr->nvis, ns, np, (float)(1.0 / Lr->wsum)};
    if (e == cudaSuccess && Lr->nvis > 0) {
        k_learn_predict<<<(Lr->nvis + 255) / 256, 256, 0, st>>>(Lr->d_vis, C, Lr->d_src, Lr->d_wv);
        int dev = 0, sms = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        const int blocks = std::min((Lr->nvis + 255) / 256, sms * 4);
        const size_t ph_bytes = sizeof(float2) * Nw * kMaxProbes;
        k_learn_forward<<<blocks, 256, ph_bytes, st>>>(Lr->d_vis, Lr->d_wv, table, C, Lr->kb4, Lr->d_pq,
                                                       Lr->d_pconst, Lr->d_ph, Lr->d_idft);
        k_learn_loss<<<1, 32, 0, st>>>(Lr->d_idft, np, C.inv_wsum * grad_scale, loss, Lr->d_ge);
        chk(cudaGetLastError());
        if (table_grad) {
            const size_t ntg = (size_t)(L + 1) * (L + 1) * 16;
            if (!accumulate) chk(cudaMemsetAsync(table_grad, 0, sizeof(float) * ntg * Nw, st));
            const size_t smem = ph_bytes + sizeof(float) * ntg;
            chk(cudaFuncSetAttribute(k_learn_backward, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
            if (e == cudaSuccess)
                k_learn_backward<<<Lr->n_chunks, 256, smem, st>>>(Lr->d_vis, Lr->d_wv, C, Lr->d_chunks,
                                                                   Lr->d_pq, Lr->d_pconst, Lr->d_ph,
                                                                   Lr->d_ge, table_grad);
            chk(cudaGetLastError());
        }
    }
    if (e == cudaSuccess && image_dft)
        chk(cudaMemcpyAsync(image_dft, Lr->d_idft, sizeof(float) * 2 * np, cudaMemcpyDeviceToDevice, st));
    if (e != cudaSuccess) {
        char m[200];
        snprintf(m, sizeof m, "rick_learn_field_grad: %s", cudaGetErrorString(e));
        return lfail(RICK_ERR_CUDA, m);
    }
    return RICK_OK;
}

int64_t rick_learn_placed(const rick_learn* Lr) { return Lr ? Lr->nvis : -1; }

}  // extern "C"

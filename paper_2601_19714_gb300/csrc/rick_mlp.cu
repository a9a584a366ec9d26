// rick_mlp.cu -- the learned gridding kernel (support 4): a small multilayer
// perceptron maps (dx, dy, w-plane) to 16 taps; its forward pass, backward
// pass and Adam update are the kernels below, and the training objective is
// the w-stacking image itself (Sec. 2, Eq. 2 and 3) measured against the
// direct Fourier inversion of Eq. 1 at the source pixels of point-source
// fields.
//
// Network: in[3] -> W1 (H x 3), b1 -> GELU -> W2 (H x H), b2 -> GELU ->
// W3 (16 x H), b3 -> taps[16]; parameters packed as W1, b1, W2, b2, W3, b3.
// GELU is the tanh form 0.5 x (1 + tanh(sqrt(2/pi)(x + 0.044715 x^3))).
//
// Inference: the network is evaluated on an (L+1)x(L+1) lattice of (dx, dy)
// per plane ("baking" the table the gridder reads, which interpolates
// bilinearly).  Training differentiates through that same table, so what is
// trained is exactly what is gridded.
#include <cmath>
#include <cstdio>
#include <cstring>

#include "rick_internal.cuh"

namespace rick {

namespace {

constexpr int kMlpOut = 16;

__device__ __forceinline__ float gelu(float x) {
    const float c = 0.7978845608028654f;  // sqrt(2/pi)
    return 0.5f * x * (1.0f + tanhf(c * (x + 0.044715f * x * x * x)));
}

__device__ __forceinline__ float gelu_grad(float x) {
    const float c = 0.7978845608028654f;
    const float u = c * (x + 0.044715f * x * x * x);
    const float t = tanhf(u);
    return 0.5f * (1.0f + t) + 0.5f * x * (1.0f - t * t) * c * (1.0f + 3.0f * 0.044715f * x * x);
}

struct MlpView {
    const float *W1, *b1, *W2, *b2, *W3, *b3;
};

__device__ __forceinline__ MlpView view(const float* p, int H) {
    MlpView v;
    v.W1 = p;
    v.b1 = v.W1 + 3 * H;
    v.W2 = v.b1 + H;
    v.b2 = v.W2 + H * H;
    v.W3 = v.b2 + H;
    v.b3 = v.W3 + kMlpOut * H;
    return v;
}

// One point per thread; parameters staged in shared memory.  If work is not
// NULL the pre-activations and activations are kept for the backward pass:
// work[n][6H] = z1, z2, g1, g2, a1, a2 (g1, g2 filled by the backward).
template <int H>
__global__ void __launch_bounds__(128)
k_mlp_forward(const float* __restrict__ params, const float* __restrict__ in, int64_t n,
              float* __restrict__ out, float* __restrict__ work) {
    extern __shared__ float sp[];
    const int np = 3 * H + H + H * H + H + kMlpOut * H + kMlpOut;
    for (int i = threadIdx.x; i < np; i += blockDim.x) sp[i] = params[i];
    __syncthreads();
    const MlpView w = view(sp, H);
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const float x0 = in[3 * i], x1 = in[3 * i + 1], x2 = in[3 * i + 2];
    float a1[H];
    float* wk = work ? work + (size_t)i * 6 * H : nullptr;
#pragma unroll
    for (int h = 0; h < H; ++h) {
        const float z = w.b1[h] + w.W1[3 * h] * x0 + w.W1[3 * h + 1] * x1 + w.W1[3 * h + 2] * x2;
        a1[h] = gelu(z);
        if (wk) {
            wk[h] = z;
            wk[4 * H + h] = a1[h];
        }
    }
    float o[kMlpOut];
#pragma unroll
    for (int q = 0; q < kMlpOut; ++q) o[q] = w.b3[q];
    for (int h = 0; h < H; ++h) {
        float z = w.b2[h];
#pragma unroll
        for (int k = 0; k < H; ++k) z = fmaf(w.W2[h * H + k], a1[k], z);
        const float a = gelu(z);
        if (wk) {
            wk[H + h] = z;
            wk[5 * H + h] = a;
        }
#pragma unroll
        for (int q = 0; q < kMlpOut; ++q) o[q] = fmaf(w.W3[q * H + h], a, o[q]);
    }
#pragma unroll
    for (int q = 0; q < kMlpOut; ++q) out[(size_t)i * kMlpOut + q] = o[q];
}

// Backward through the two GELU layers for each point: g2 = W3^T gout * gelu'(z2),
// g1 = W2^T g2 * gelu'(z1), stored in work (g1 at 2H, g2 at 3H).
template <int H>
__global__ void __launch_bounds__(128)
k_mlp_backward_points(const float* __restrict__ params, int64_t n, const float* __restrict__ gout,
                      float* __restrict__ work) {
    extern __shared__ float sp[];
    const int np = 3 * H + H + H * H + H + kMlpOut * H + kMlpOut;
    for (int i = threadIdx.x; i < np; i += blockDim.x) sp[i] = params[i];
    __syncthreads();
    const MlpView w = view(sp, H);
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    float* wk = work + (size_t)i * 6 * H;
    float g3[kMlpOut];
#pragma unroll
    for (int q = 0; q < kMlpOut; ++q) g3[q] = gout[(size_t)i * kMlpOut + q];
    float g2[H];
#pragma unroll
    for (int h = 0; h < H; ++h) {
        float s = 0.0f;
#pragma unroll
        for (int q = 0; q < kMlpOut; ++q) s = fmaf(w.W3[q * H + h], g3[q], s);
        g2[h] = s * gelu_grad(wk[H + h]);
        wk[3 * H + h] = g2[h];
    }
    for (int k = 0; k < H; ++k) {
        float s = 0.0f;
#pragma unroll
        for (int h = 0; h < H; ++h) s = fmaf(w.W2[h * H + k], g2[h], s);
        wk[2 * H + k] = s * gelu_grad(wk[k]);
    }
}

// Parameter gradients (accumulated): one block per output row, thread = column,
// blockIdx.y = chunk of points.  Rows 0..H-1: W1 (+b1); H..2H-1: W2 (+b2);
// 2H..2H+15: W3 (+b3).
template <int H>
__global__ void __launch_bounds__(H)
k_mlp_param_grad(const float* __restrict__ in, int64_t n, const float* __restrict__ gout,
                 const float* __restrict__ work, float* __restrict__ grad, int64_t chunk) {
    const int row = blockIdx.x, col = threadIdx.x;
    const int64_t n0 = (int64_t)blockIdx.y * chunk;
    const int64_t n1 = min(n, n0 + chunk);
    float* gW1 = grad;
    float* gb1 = gW1 + 3 * H;
    float* gW2 = gb1 + H;
    float* gb2 = gW2 + H * H;
    float* gW3 = gb2 + H;
    float* gb3 = gW3 + kMlpOut * H;
    float acc = 0.0f, accb = 0.0f;
    if (row < H) {
        const int h = row;
        for (int64_t p = n0; p < n1; ++p) {
            const float g = work[(size_t)p * 6 * H + 2 * H + h];
            if (col < 3) acc = fmaf(g, in[3 * p + col], acc);
            accb += g;
        }
        if (col < 3) atomicAdd(&gW1[3 * h + col], acc);
        if (col == 0) atomicAdd(&gb1[h], accb);
    } else if (row < 2 * H) {
        const int h = row - H;
        for (int64_t p = n0; p < n1; ++p) {
            const float* wk = work + (size_t)p * 6 * H;
            const float g = wk[3 * H + h];
            acc = fmaf(g, wk[4 * H + col], acc);
            accb += g;
        }
        atomicAdd(&gW2[h * H + col], acc);
        if (col == 0) atomicAdd(&gb2[h], accb);
    } else {
        const int q = row - 2 * H;
        for (int64_t p = n0; p < n1; ++p) {
            const float g = gout[(size_t)p * kMlpOut + q];
            acc = fmaf(g, work[(size_t)p * 6 * H + 5 * H + col], acc);
            accb += g;
        }
        atomicAdd(&gW3[q * H + col], acc);
        if (col == 0) atomicAdd(&gb3[q], accb);
    }
}

__global__ void k_adam(float* __restrict__ p, const float* __restrict__ g, float* __restrict__ m,
                       float* __restrict__ v, int64_t n, float lr, float b1, float b2, float eps,
                       float c1, float c2) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const float gi = g[i];
    const float mi = b1 * m[i] + (1.0f - b1) * gi;
    const float vi = b2 * v[i] + (1.0f - b2) * gi * gi;
    m[i] = mi;
    v[i] = vi;
    p[i] -= lr * (mi / c1) / (sqrtf(vi / c2) + eps);
}

// Lattice points (dx, dy, w) of the baked table, [Nw][L+1][L+1] x 3.
__global__ void k_lattice_inputs(int Nw, int L, float* __restrict__ out) {
    const int64_t n = (int64_t)Nw * (L + 1) * (L + 1);
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const int ix = (int)(i % (L + 1));
    const int iy = (int)((i / (L + 1)) % (L + 1));
    const int k = (int)(i / ((int64_t)(L + 1) * (L + 1)));
    out[3 * i] = (float)ix / (float)L;
    out[3 * i + 1] = (float)iy / (float)L;
    out[3 * i + 2] = Nw > 1 ? (2.0f * k - (Nw - 1)) / (float)(Nw - 1) : 0.0f;
}

template <int H>
cudaError_t forward_h(const float* params, const float* in, int64_t n, float* out, float* work,
                      cudaStream_t st) {
    const size_t np = 3 * H + H + H * H + H + kMlpOut * H + kMlpOut;
    const int64_t blocks = (n + 127) / 128;
    auto fn = k_mlp_forward<H>;
    cudaError_t e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)(np * 4));
    if (e != cudaSuccess) return e;
    fn<<<(unsigned)blocks, 128, np * 4, st>>>(params, in, n, out, work);
    return cudaGetLastError();
}

}  // namespace

int64_t mlp_param_count(int H) { return (int64_t)3 * H + H + (int64_t)H * H + H + kMlpOut * H + kMlpOut; }

// forward with optional saved activations (work may be NULL)
cudaError_t mlp_forward(const float* params, int H, const float* in, int64_t n, float* out,
                        float* work, cudaStream_t st) {
    if (n <= 0) return cudaSuccess;
    switch (H) {
        case 16: return forward_h<16>(params, in, n, out, work, st);
        case 32: return forward_h<32>(params, in, n, out, work, st);
        case 64: return forward_h<64>(params, in, n, out, work, st);
        default: return cudaErrorInvalidValue;
    }
}

template <int H>
static cudaError_t mlp_backward_h(const float* params, const float* in, int64_t n,
                                  const float* gout, float* grad, float* work, float* scratch_out,
                                  cudaStream_t st) {
    const size_t np = mlp_param_count(H);
    cudaError_t e = forward_h<H>(params, in, n, scratch_out, work, st);
    if (e != cudaSuccess) return e;
    auto fb = k_mlp_backward_points<H>;
    e = cudaFuncSetAttribute(fb, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)(np * 4));
    if (e != cudaSuccess) return e;
    fb<<<(unsigned)((n + 127) / 128), 128, np * 4, st>>>(params, n, gout, work);
    const int64_t chunk = 2048;
    dim3 grid(2 * H + kMlpOut, (unsigned)((n + chunk - 1) / chunk));
    k_mlp_param_grad<H><<<grid, H, 0, st>>>(in, n, gout, work, grad, chunk);
    return cudaGetLastError();
}

// grad += d(sum gout . mlp(in))/dparams.  work: [n][6H] floats, scratch_out: [n][16] floats.
cudaError_t mlp_backward(const float* params, int H, const float* in, int64_t n, const float* gout,
                         float* grad, float* work, float* scratch_out, cudaStream_t st) {
    if (n <= 0) return cudaSuccess;
    switch (H) {
        case 16: return mlp_backward_h<16>(params, in, n, gout, grad, work, scratch_out, st);
        case 32: return mlp_backward_h<32>(params, in, n, gout, grad, work, scratch_out, st);
        case 64: return mlp_backward_h<64>(params, in, n, gout, grad, work, scratch_out, st);
        default: return cudaErrorInvalidValue;
    }
}

cudaError_t adam_step(float* p, const float* g, float* m, float* v, int64_t n, float lr, float b1,
                      float b2, float eps, int step, cudaStream_t st) {
    if (n <= 0) return cudaSuccess;
    const float c1 = 1.0f - powf(b1, (float)step), c2 = 1.0f - powf(b2, (float)step);
    k_adam<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(p, g, m, v, n, lr, b1, b2, eps, c1, c2);
    return cudaGetLastError();
}

cudaError_t lattice_inputs(int Nw, int L, float* out, cudaStream_t st) {
    const int64_t n = (int64_t)Nw * (L + 1) * (L + 1);
    k_lattice_inputs<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(Nw, L, out);
    return cudaGetLastError();
}

}  // namespace rick

// ============================================================================
// C ABI
// ============================================================================

namespace rick {
void set_error_message(const char* msg);
}

namespace {
rick_status mfail(rick_status s, const char* m) {
    rick::set_error_message(m);
    return s;
}
rick_status mcuda(cudaError_t e, const char* where) {
    if (e == cudaSuccess) return RICK_OK;
    char m[200];
    snprintf(m, sizeof m, "%s: %s", where, cudaGetErrorString(e));
    return mfail(RICK_ERR_CUDA, m);
}
bool hidden_ok(int H) { return H == 16 || H == 32 || H == 64; }
}  // namespace

extern "C" {

int64_t rick_mlp_param_count(int32_t hidden) { return hidden_ok(hidden) ? rick::mlp_param_count(hidden) : -1; }

rick_status rick_mlp_forward(const float* params, int32_t hidden, const float* in, int64_t n,
                             float* out, float* work, void* stream) {
    if (!params || !in || !out || n < 0 || !hidden_ok(hidden))
        return mfail(RICK_ERR_INVALID_ARG, "invalid argument: mlp forward (hidden must be 16, 32 or 64)");
    return mcuda(rick::mlp_forward(params, hidden, in, n, out, work, reinterpret_cast<cudaStream_t>(stream)),
                 "rick_mlp_forward");
}

rick_status rick_mlp_backward(const float* params, int32_t hidden, const float* in, int64_t n,
                              const float* gout, float* grad, float* work, float* scratch,
                              void* stream) {
    if (!params || !in || !gout || !grad || !work || !scratch || n < 0 || !hidden_ok(hidden))
        return mfail(RICK_ERR_INVALID_ARG, "invalid argument: mlp backward");
    return mcuda(rick::mlp_backward(params, hidden, in, n, gout, grad, work, scratch,
                                    reinterpret_cast<cudaStream_t>(stream)),
                 "rick_mlp_backward");
}

rick_status rick_adam_step(float* params, const float* grad, float* m, float* v, int64_t n,
                           float lr, float beta1, float beta2, float eps, int32_t step,
                           void* stream) {
    if (!params || !grad || !m || !v || n < 0 || step < 1)
        return mfail(RICK_ERR_INVALID_ARG, "invalid argument: adam step");
    return mcuda(rick::adam_step(params, grad, m, v, n, lr, beta1, beta2, eps, step,
                                 reinterpret_cast<cudaStream_t>(stream)),
                 "rick_adam_step");
}

rick_status rick_mlp_lattice_inputs(int32_t n_wplanes, int32_t lattice, float* out, void* stream) {
    if (!out || n_wplanes < 1 || lattice < 1 || lattice > 256)
        return mfail(RICK_ERR_INVALID_ARG, "invalid argument: lattice inputs");
    return mcuda(rick::lattice_inputs(n_wplanes, lattice, out, reinterpret_cast<cudaStream_t>(stream)),
                 "rick_mlp_lattice_inputs");
}

}  // extern "C"

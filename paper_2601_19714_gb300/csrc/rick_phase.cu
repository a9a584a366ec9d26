// rick_phase.cu -- w phase screen and reduction over w-planes (Eq. 2), "a4".
//
//   image[c][q][p] += (-1)^(p+q) n / (sum W_c C(p) C(q))
//                     * Re sum_k F_k[q][p] exp(+2 pi i w_k (n - 1))
//
// With a padded mesh (grid_size Ng > N) the planes are Ng x Ng and the image
// is their central N x N (offset (Ng - N)/2); only that part is read.
//
// HBM-bound: every transformed plane is read once (8 B per pixel per plane).
// One thread owns two adjacent pixels (one 16-byte load per plane) for all
// channels and planes of the launch.
//
// Phase (pattern 1, FP64 only where it is needed): per pixel, in FP64,
//   delta = n - 1 = -(l^2 + m^2)/(1 + n)          (no cancellation)
//   t_0 = frac(w_first * delta), dt = frac(dw * delta)   [turns]
// both converted to 64-bit fixed point (Q0.64), so that t_k = t_0 + k dt is
// exact modulo one turn with integer adds.  Every 8th plane the phasor is
// formed exactly from the top 32 bits (sincospif of a value in [-1, 1)); in
// between it advances by one FP32 complex multiply with exp(2 pi i dt).  The
// only FP64 work is a handful of operations per pixel, never per plane.
//
// With a w-kernel (improved w-stacking) the planes are those of the extended
// set (w_first is the centre of the launch's first plane in it) and every
// pixel is also divided by the w-kernel's transform C_w((n - 1) dw).
#include "rick_internal.cuh"

namespace rick {

namespace {

constexpr int kPhaseThreads = 256;
constexpr int kAnchor = 8;

__device__ __forceinline__ uint64_t turns_q64(double t) {
    const double f = t - floor(t);  // [0, 1)
    return __double2ull_rz(f * 18446744073709551616.0);
}

__device__ __forceinline__ float2 phasor_q64(uint64_t t) {
    const int32_t hi = (int32_t)(t >> 32);  // turns in [-1/2, 1/2) * 2^32
    float s, c;
    sincospif((float)hi * 4.656612873077392578125e-10f /* 2^-31 */, &s, &c);
    return make_float2(c, s);
}

__device__ __forceinline__ float2 cmul(float2 a, float2 b) {
    return make_float2(fmaf(a.x, b.x, -a.y * b.y), fmaf(a.x, b.y, a.y * b.x));
}


template <int PREC, bool COMPLEX_OUT>
__global__ void __launch_bounds__(kPhaseThreads)
k_phase_reduce(PhaseParams P, const float2* __restrict__ grids, const double* __restrict__ wsum,
               const float* __restrict__ inv_taper, float* __restrict__ image_real,
               float2* __restrict__ image_complex) {
    // (p, q): image pixel; the planes are Ng x Ng with the image at offset off
    const int N = P.N, Ni = P.Ni, halfN = Ni / 2;
    const int64_t tid = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (tid >= (int64_t)Ni * halfN) return;
    const int q = (int)(tid / halfN);
    const int p = (int)(tid - (int64_t)q * halfN) * 2;
    const size_t NN = (size_t)N * N, NNi = (size_t)Ni * Ni;

    uint64_t t0[2], dt[2];
    float t0f[2], dtf[2];
    float scale[2];
    for (int e = 0; e < 2; ++e) {
        const double l = (double)(p + e - halfN) * P.dl, m = (double)(q - halfN) * P.dl;
        const double r2 = l * l + m * m;
        const double n = sqrt(1.0 - r2);
        const double delta = -r2 / (1.0 + n);
        if (PREC == RICK_PREC_ALL_FP32) {
            const float lf = (float)(p + e - halfN) * (float)P.dl, mf = (float)(q - halfN) * (float)P.dl;
            const float r2f = lf * lf + mf * mf;
            const float nf = sqrtf(1.0f - r2f);
            const float df = -r2f / (1.0f + nf);
            t0f[e] = (float)P.w_first * df;
            dtf[e] = (float)P.dw * df;
        } else {
            t0[e] = turns_q64(P.w_first * delta);
            dt[e] = turns_q64(P.dw * delta);
        }
        const float sg = ((p + e + q) & 1) ? -1.f : 1.f;
        scale[e] = sg * (float)n * inv_taper[p + e] * inv_taper[q] * w_taper_inv(P, delta);
    }

    for (int cc = 0; cc < P.nc; ++cc) {
        const double ws = wsum[cc];
        const float inv_ws = ws != 0.0 ? (float)(1.0 / ws) : 0.0f;
        const float4* g = reinterpret_cast<const float4*>(grids + (size_t)cc * P.nk * NN +
                                                          (size_t)(q + P.off) * N + p + P.off);
        float2 acc0 = make_float2(0.f, 0.f), acc1 = make_float2(0.f, 0.f);
        if (PREC == RICK_PREC_ALL_FP32) {
            for (int k = 0; k < P.nk; ++k) {
                const float4 F = __ldcs(g + (size_t)k * (NN / 2));
                float s0, c0, s1, c1;
                const float a0 = t0f[0] + (float)k * dtf[0], a1 = t0f[1] + (float)k * dtf[1];
                sincospif(2.0f * (a0 - rintf(a0)), &s0, &c0);
                sincospif(2.0f * (a1 - rintf(a1)), &s1, &c1);
                acc0 = make_float2(acc0.x + F.x * c0 - F.y * s0, acc0.y + F.x * s0 + F.y * c0);
                acc1 = make_float2(acc1.x + F.z * c1 - F.w * s1, acc1.y + F.z * s1 + F.w * c1);
            }
        } else {
            const float2 r0 = phasor_q64(dt[0]), r1 = phasor_q64(dt[1]);
            uint64_t tk0 = t0[0], tk1 = t0[1];
            for (int kb = 0; kb < P.nk; kb += kAnchor) {
                const int kn = min(kAnchor, P.nk - kb);
                float4 F[kAnchor];
#pragma unroll
                for (int j = 0; j < kAnchor; ++j)
                    if (j < kn) F[j] = __ldcs(g + (size_t)(kb + j) * (NN / 2));
                float2 z0 = phasor_q64(tk0), z1 = phasor_q64(tk1);
#pragma unroll
                for (int j = 0; j < kAnchor; ++j) {
                    if (j < kn) {
                        acc0.x = fmaf(F[j].x, z0.x, fmaf(-F[j].y, z0.y, acc0.x));
                        acc0.y = fmaf(F[j].x, z0.y, fmaf(F[j].y, z0.x, acc0.y));
                        acc1.x = fmaf(F[j].z, z1.x, fmaf(-F[j].w, z1.y, acc1.x));
                        acc1.y = fmaf(F[j].z, z1.y, fmaf(F[j].w, z1.x, acc1.y));
                        z0 = cmul(z0, r0);
                        z1 = cmul(z1, r1);
                    }
                }
                tk0 += (uint64_t)kAnchor * dt[0];
                tk1 += (uint64_t)kAnchor * dt[1];
            }
        }
        const float s0 = scale[0] * inv_ws, s1 = scale[1] * inv_ws;
        float2* ir = reinterpret_cast<float2*>(image_real + (size_t)cc * NNi + (size_t)q * Ni + p);
        float2 cur = *ir;
        cur.x += s0 * acc0.x;
        cur.y += s1 * acc1.x;
        *ir = cur;
        if (COMPLEX_OUT) {
            float4* ic = reinterpret_cast<float4*>(image_complex + (size_t)cc * NNi + (size_t)q * Ni + p);
            float4 v = *ic;
            v.x += s0 * acc0.x;
            v.y += s0 * acc0.y;
            v.z += s1 * acc1.x;
            v.w += s1 * acc1.y;
            *ic = v;
        }
    }
}

// Prediction, first step: the model image of each channel spread onto the
// w-planes (the adjoint of the reduction above),
//   M_k[q][p] = (-1)^(p+q) J_c[q][p] exp(-2 pi i w_k (n - 1)) / (n C(p) C(q) C_w),
// every plane written once (16-byte streaming stores of two pixels).  The
// phase is the conjugate of the one the reduction applies, formed the same
// way (FP64 per pixel, Q0.64 turns, exact anchors every 8 planes).
template <int PREC>
__global__ void __launch_bounds__(kPhaseThreads)
k_model_planes(PhaseParams P, const float* __restrict__ image, const float* __restrict__ inv_taper,
               float2* __restrict__ grids) {
    // one thread per two cells of the Ng x Ng plane; (p, q) the image pixel
    // (the cells outside the central Ni x Ni of a padded plane are zero)
    const int N = P.N, Ni = P.Ni, halfN = Ni / 2;
    const int64_t tid = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (tid >= (int64_t)N * (N / 2)) return;
    const int qg = (int)(tid / (N / 2));
    const int pg = (int)(tid - (int64_t)qg * (N / 2)) * 2;
    const int q = qg - P.off, p = pg - P.off;
    const size_t NN = (size_t)N * N, NNi = (size_t)Ni * Ni;
    if (q < 0 || q >= Ni || p < 0 || p >= Ni) {
        float4* g = reinterpret_cast<float4*>(grids + (size_t)qg * N + pg);
        for (int r = 0; r < P.nc * P.nk; ++r) __stcs(g + (size_t)r * (NN / 2), make_float4(0.f, 0.f, 0.f, 0.f));
        return;
    }

    uint64_t t0[2], dt[2];
    float t0f[2], dtf[2];
    float scale[2];
    for (int e = 0; e < 2; ++e) {
        const double l = (double)(p + e - halfN) * P.dl, m = (double)(q - halfN) * P.dl;
        const double r2 = l * l + m * m;
        const double n = sqrt(1.0 - r2);
        const double delta = -r2 / (1.0 + n);
        if (PREC == RICK_PREC_ALL_FP32) {
            const float lf = (float)(p + e - halfN) * (float)P.dl, mf = (float)(q - halfN) * (float)P.dl;
            const float r2f = lf * lf + mf * mf;
            const float nf = sqrtf(1.0f - r2f);
            const float df = -r2f / (1.0f + nf);
            t0f[e] = (float)P.w_first * df;
            dtf[e] = (float)P.dw * df;
        } else {
            t0[e] = turns_q64(P.w_first * delta);
            dt[e] = turns_q64(P.dw * delta);
        }
        const float sg = ((p + e + q) & 1) ? -1.f : 1.f;
        scale[e] = sg * inv_taper[p + e] * inv_taper[q] * w_taper_inv(P, delta) / (float)n;
    }

    for (int cc = 0; cc < P.nc; ++cc) {
        const float2 J = *reinterpret_cast<const float2*>(image + (size_t)cc * NNi + (size_t)q * Ni + p);
        const float a0 = J.x * scale[0], a1 = J.y * scale[1];
        float4* g = reinterpret_cast<float4*>(grids + (size_t)cc * P.nk * NN + (size_t)qg * N + pg);
        if (PREC == RICK_PREC_ALL_FP32) {
            for (int k = 0; k < P.nk; ++k) {
                float s0, c0, s1, c1;
                const float b0 = t0f[0] + (float)k * dtf[0], b1 = t0f[1] + (float)k * dtf[1];
                sincospif(2.0f * (b0 - rintf(b0)), &s0, &c0);
                sincospif(2.0f * (b1 - rintf(b1)), &s1, &c1);
                __stcs(g + (size_t)k * (NN / 2), make_float4(a0 * c0, -a0 * s0, a1 * c1, -a1 * s1));
            }
        } else {
            const float2 r0 = phasor_q64(dt[0]), r1 = phasor_q64(dt[1]);
            uint64_t tk0 = t0[0], tk1 = t0[1];
            for (int kb = 0; kb < P.nk; kb += kAnchor) {
                const int kn = min(kAnchor, P.nk - kb);
                float2 z0 = phasor_q64(tk0), z1 = phasor_q64(tk1);
#pragma unroll
                for (int j = 0; j < kAnchor; ++j) {
                    if (j < kn) {
                        __stcs(g + (size_t)(kb + j) * (NN / 2),
                               make_float4(a0 * z0.x, -a0 * z0.y, a1 * z1.x, -a1 * z1.y));
                        z0 = cmul(z0, r0);
                        z1 = cmul(z1, r1);
                    }
                }
                tk0 += (uint64_t)kAnchor * dt[0];
                tk1 += (uint64_t)kAnchor * dt[1];
            }
        }
    }
}

}  // namespace

cudaError_t launch_model_planes(const PhaseParams& P, const float* image, const float* inv_taper,
                                float2* grids, cudaStream_t stream, int* launches) {
    const int64_t threads = (int64_t)P.N * (P.N / 2);   // every cell of the (padded) plane
    const int64_t blocks = (threads + kPhaseThreads - 1) / kPhaseThreads;
    if (blocks > 0x7fffffffLL) return cudaErrorInvalidConfiguration;
    if (P.precision == RICK_PREC_ALL_FP32)
        k_model_planes<RICK_PREC_ALL_FP32><<<(unsigned)blocks, kPhaseThreads, 0, stream>>>(P, image, inv_taper, grids);
    else
        k_model_planes<RICK_PREC_FP32_FP64IDX><<<(unsigned)blocks, kPhaseThreads, 0, stream>>>(P, image, inv_taper, grids);
    ++*launches;
    return cudaGetLastError();
}

cudaError_t launch_phase_reduce(const PhaseParams& P, const float2* grids, const double* wsum,
                                const float* inv_taper, float* image_real, float2* image_complex,
                                cudaStream_t stream, int* launches) {
    const int64_t threads = (int64_t)P.Ni * (P.Ni / 2);   // every image pixel pair
    const int64_t blocks = (threads + kPhaseThreads - 1) / kPhaseThreads;
    if (blocks > 0x7fffffffLL) return cudaErrorInvalidConfiguration;
    const bool cplx = image_complex != nullptr;
    if (P.precision == RICK_PREC_ALL_FP32) {
        if (cplx)
            k_phase_reduce<RICK_PREC_ALL_FP32, true><<<(unsigned)blocks, kPhaseThreads, 0, stream>>>(
                P, grids, wsum, inv_taper, image_real, image_complex);
        else
            k_phase_reduce<RICK_PREC_ALL_FP32, false><<<(unsigned)blocks, kPhaseThreads, 0, stream>>>(
                P, grids, wsum, inv_taper, image_real, image_complex);
    } else {
        if (cplx)
            k_phase_reduce<RICK_PREC_FP32_FP64IDX, true><<<(unsigned)blocks, kPhaseThreads, 0, stream>>>(
                P, grids, wsum, inv_taper, image_real, image_complex);
        else
            k_phase_reduce<RICK_PREC_FP32_FP64IDX, false><<<(unsigned)blocks, kPhaseThreads, 0, stream>>>(
                P, grids, wsum, inv_taper, image_real, image_complex);
    }
    ++*launches;
    return cudaGetLastError();
}

}  // namespace rick

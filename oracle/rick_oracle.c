/*
 * rick_oracle.c -- FP64 CPU oracle of the w-stacking imaging path.
 *
 * TEST INFRASTRUCTURE.  This file is the plain, slow, obviously-correct
 * reference that the CUDA library is checked against.  Only the test suite,
 * the smoke check and the benchmark's CPU-baseline leg may load it.  It
 * shares no code, header, table or constant with the CUDA library.
 *
 * What it computes (arXiv 2601.19714, "Accelerating radio astronomy imaging
 * with RICK"):
 *   - Eq. 1, the measurement equation, inverted directly (a direct Fourier
 *     transform of the visibilities; "O2" below): the plain definition of the
 *     dirty image, used to measure the error of the method itself.
 *   - Sec. 2, Eq. 2 and Eq. 3, the w-stacking method ("O1"): convolutional
 *     gridding of every visibility onto its closest w-plane (Eq. 3), a 2-D
 *     inverse FFT of each plane, the w phase screen, and the sum over planes
 *     (Eq. 2), with natural weighting (Sec. 4.1.1).
 *
 * Readings of the paper that this file fixes (the paper gives no formula for
 * them; every one is also listed in the design notes of the repository):
 *   R1 grid <-> uv:   cell i holds u = (i - N/2)/fov (du = 1/fov); the
 *                     visibility's continuous position is x = u*fov + N/2.
 *   R2 pixel <-> lm:  pixel p holds l = (p - N/2)*fov/N.
 *   R3 footprint:     the support of a visibility at x is the S cells i with
 *                     x - S/2 < i <= x + S/2, i.e. i0 = floor(x - S/2) + 1.
 *                     A visibility whose footprint leaves [0, N) is dropped.
 *   R4 w-planes:      "closest w-plane" (Sec. 2) is read as cell-centred
 *                     planes: k = floor((w - w_min) * Nw/(w_max - w_min)),
 *                     clamped to [0, Nw-1]; plane k sits at
 *                     w_k = w_min + (k + 1/2)(w_max - w_min)/Nw.
 *   R5 correction:    the equation after "a correction is applied as" is
 *                     missing from the paper; Eq. 2 is followed literally:
 *                     plane k is multiplied by exp(+2 pi i w_k (n - 1)),
 *                     summed over k, and multiplied by n = sqrt(1-l^2-m^2).
 *                     The image is divided by the sum of weights (natural
 *                     weighting) and by the gridding taper C(l) C(m), the
 *                     continuous Fourier transform of the kernel.
 *   R6 centring:      the FFT is centred with checkerboard signs: grid cell
 *                     (i, j) carries (-1)^(i+j), image pixel (p, q) carries
 *                     (-1)^(p+q) (for even N the remaining factor is 1).
 *   R7 kernels:       Gaussian g(s) = exp(-s^2/(2 sigma^2)); Kaiser-Bessel
 *                     (Jackson 1991) g(s) = I0(beta sqrt(1-(2s/S)^2))/I0(beta),
 *                     both zero for |s| > S/2.
 *   R15 weighting:    the paper uses natural weighting (Sec. 4.1.1); uniform
 *                     and Briggs (robust) weighting are extensions.  The
 *                     density D is the sum of the weights of the gridded
 *                     visibilities of one channel on their nearest mesh cell
 *                     (i, j) = (floor(x + 1/2), floor(y + 1/2)), each counted
 *                     there and at the cell of its Hermitian partner,
 *                     ((N - i) mod N, (N - j) mod N).  Uniform: W' = W / D;
 *                     Briggs with robustness R: W' = W / (1 + f^2 D),
 *                     f^2 = (5 10^-R)^2 sum(D) / sum(D^2) over the cells.  The
 *                     weights W' (stored in FP32, like the data weights)
 *                     then replace W everywhere, including the sum of weights.
 *   R16 padding:      the paper's mesh is the image size (Sec. 2); a padded
 *                     mesh is an extension: Ng = alpha N cells (alpha a power
 *                     of two) of size 1/(alpha fov), x = u fov alpha + Ng/2;
 *                     the image is the central N x N of the Ng x Ng inverse
 *                     DFT (pixel p of the image is pixel p + (Ng - N)/2 of
 *                     the transform, still at l = (p - N/2) fov/N), divided
 *                     by C(p) = int g(s) cos(2 pi s (p - N/2)/Ng) ds.  The
 *                     weighting density of R15 stays on the N x N mesh of
 *                     cell 1/fov (x = u fov + N/2), its cells taken mod N.
 *
 * Floating point: FP64 throughout, compiled without FMA contraction so that
 * the index decisions (footprint start, plane index) are the IEEE results of
 * the operations written here, in the order written here.
 */
#include <complex.h>
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define ORACLE_PI 3.141592653589793238462643383279502884

enum { ORACLE_GAUSS = 0, ORACLE_KAISER_BESSEL = 1, ORACLE_LEARNED = 2 };

/* Learned kernel: a multilayer perceptron 3 -> H -> H -> 16 with GELU
 * activations, whose 16 outputs correct the 16 taps of the support-4
 * Kaiser-Bessel kernel (beta = kernel_param): tap(a, b) = g(a + 1 - 2 - fx)
 * g(b + 1 - 2 - fy) + out[4b + a].  Its weights are laid out in one FP64 array:
 *   W1[H][3], b1[H], W2[H][H], b2[H], W3[16][H], b3[16]. */
#define ORACLE_MLP_IN 3
#define ORACLE_MLP_OUT 16

typedef struct {
    int32_t N;            /* mesh side, N_u = N_v = N (Sec. 2) */
    int32_t Nw;           /* number of w-planes N_w (Eq. 2) */
    int32_t S;            /* kernel support, cells */
    int32_t kernel;       /* ORACLE_GAUSS / ORACLE_KAISER_BESSEL / ORACLE_LEARNED */
    double kernel_param;  /* Gaussian sigma (cells) or Kaiser-Bessel beta; for the
                             learned kernel: beta of the support-S Kaiser-Bessel
                             whose taper divides the image */
    double fov;           /* field of view, direction-cosine units (radians) */
    double w_min, w_max;  /* w range covered by the planes, wavelengths */
    const double* mlp;    /* learned kernel weights (kernel == ORACLE_LEARNED) */
    int32_t mlp_hidden;   /* H */
    int32_t mlp_lattice;  /* taps are baked on an (L+1)x(L+1) lattice of (dx, dy)
                             per plane and bilinearly interpolated; 0 = evaluate
                             the network at the exact offsets */
    int32_t w_support;    /* 0 or 1: each visibility on its closest plane (R4);
                             even Sw >= 2: convolved in w onto Sw planes with a
                             Kaiser-Bessel kernel (R14) */
    double w_kernel_param;/* beta of the w-direction Kaiser-Bessel kernel */
    int32_t weighting;    /* ORACLE_NATURAL / ORACLE_UNIFORM / ORACLE_BRIGGS (R15) */
    double robust;        /* Briggs robustness R */
    int32_t Ng;           /* padded mesh side (R16); 0 = N (no padding) */
} oracle_cfg;

/* Mesh side and the offset of the image inside the transform (R16). */
static int grid_n(const oracle_cfg* cfg) { return cfg->Ng > 0 ? cfg->Ng : cfg->N; }
static int pad_off(const oracle_cfg* cfg) { return (grid_n(cfg) - cfg->N) / 2; }

enum { ORACLE_NATURAL = 0, ORACLE_UNIFORM = 1, ORACLE_BRIGGS = 2 };

/* ------------------------------------------------------------------ */
/* Kernel functions                                                    */
/* ------------------------------------------------------------------ */

/* Modified Bessel function of the first kind, order 0, by its power series
 * I0(x) = sum_k ((x/2)^(2k)) / (k!)^2, summed until the terms stop mattering. */
double oracle_bessel_i0(double x)
{
    double q = 0.25 * x * x, term = 1.0, sum = 1.0;
    for (int k = 1; k < 500; ++k) {
        term *= q / ((double)k * (double)k);
        sum += term;
        if (term < 1e-18 * sum) break;
    }
    return sum;
}

/* g(s) for a separable kernel of support S (R7); zero outside |s| <= S/2. */
double oracle_kernel_value(int kind, double param, int S, double s)
{
    double half = 0.5 * S;
    if (fabs(s) > half) return 0.0;
    if (kind == ORACLE_GAUSS) return exp(-s * s / (2.0 * param * param));
    /* Kaiser-Bessel (used also as the taper of the learned kernel) */
    double r = 2.0 * s / S;
    double a = 1.0 - r * r;
    if (a < 0.0) a = 0.0;
    return oracle_bessel_i0(param * sqrt(a)) / oracle_bessel_i0(param);
}

/* Gauss-Legendre nodes and weights on [-1, 1]: roots of P_n by Newton's
 * method from the Chebyshev-like start cos(pi (i + 3/4)/(n + 1/2)). */
void oracle_gauss_legendre(int n, double* x, double* w)
{
    for (int i = 0; i < n; ++i) {
        double z = cos(ORACLE_PI * (i + 0.75) / (n + 0.5));
        double dp = 0.0;
        for (int it = 0; it < 100; ++it) {
            double p0 = 1.0, p1 = z;  /* P_0, P_1 */
            for (int k = 2; k <= n; ++k) {
                double pk = ((2.0 * k - 1.0) * z * p1 - (k - 1.0) * p0) / k;
                p0 = p1;
                p1 = pk;
            }
            if (n == 1) { p1 = z; p0 = 1.0; }
            dp = n * (z * p1 - p0) / (z * z - 1.0);  /* P_n'(z) */
            double dz = p1 / dp;
            z -= dz;
            if (fabs(dz) < 1e-16) break;
        }
        x[i] = z;
        w[i] = 2.0 / ((1.0 - z * z) * dp * dp);
    }
}

/* Gridding taper C(p) = int_{-S/2}^{S/2} g(s) cos(2 pi s (p - N/2)/N) ds,
 * p = 0..N-1 (R5): the continuous Fourier transform of the kernel at the
 * pixel's l, in cell units.  Gauss-Legendre quadrature, 32 nodes on each of
 * the S unit sub-intervals of the support. */
void oracle_taper_padded(int kind, double param, int S, int N, int Ng, double* C)
{
    enum { NG = 32 };
    double gx[NG], gw[NG];
    oracle_gauss_legendre(NG, gx, gw);
    for (int p = 0; p < N; ++p) {
        double nu = (double)(p - N / 2) / (double)Ng;
        double acc = 0.0;
        for (int seg = 0; seg < S; ++seg) {
            double a = -0.5 * S + seg, b = a + 1.0;
            double mid = 0.5 * (a + b), hw = 0.5 * (b - a);
            for (int i = 0; i < NG; ++i) {
                double s = mid + hw * gx[i];
                acc += hw * gw[i] * oracle_kernel_value(kind, param, S, s) *
                       cos(2.0 * ORACLE_PI * s * nu);
            }
        }
        C[p] = acc;
    }
}

/* C(p) = int g(s) cos(2 pi s (p - N/2)/N) ds: the taper of an unpadded mesh. */
void oracle_taper(int kind, double param, int S, int N, double* C)
{
    oracle_taper_padded(kind, param, S, N, N, C);
}

/* ------------------------------------------------------------------ */
/* Learned kernel (pattern 4): plain FP64 multilayer perceptron        */
/* ------------------------------------------------------------------ */

/* GELU, tanh form: 0.5 x (1 + tanh(sqrt(2/pi) (x + 0.044715 x^3))). */
double oracle_gelu(double x)
{
    double c = sqrt(2.0 / ORACLE_PI);
    return 0.5 * x * (1.0 + tanh(c * (x + 0.044715 * x * x * x)));
}

double oracle_gelu_grad(double x)
{
    double c = sqrt(2.0 / ORACLE_PI);
    double u = c * (x + 0.044715 * x * x * x);
    double t = tanh(u);
    double du = c * (1.0 + 3.0 * 0.044715 * x * x);
    return 0.5 * (1.0 + t) + 0.5 * x * (1.0 - t * t) * du;
}

static size_t mlp_size(int H)
{
    return (size_t)H * ORACLE_MLP_IN + H + (size_t)H * H + H + (size_t)ORACLE_MLP_OUT * H +
           ORACLE_MLP_OUT;
}

size_t oracle_mlp_param_count(int H) { return mlp_size(H); }

/* Forward pass: out[16] = W3 gelu(W2 gelu(W1 in + b1) + b2) + b3.  The hidden
 * pre-activations are returned in z1[H], z2[H] when those are non-NULL. */
void oracle_mlp_forward(const double* prm, int H, const double in[3], double out[16], double* z1,
                        double* z2)
{
    const double* W1 = prm;
    const double* b1 = W1 + (size_t)H * 3;
    const double* W2 = b1 + H;
    const double* b2 = W2 + (size_t)H * H;
    const double* W3 = b2 + H;
    const double* b3 = W3 + (size_t)16 * H;
    double* a1 = (double*)malloc(sizeof(double) * H * 2);
    double* a2 = a1 + H;
    for (int h = 0; h < H; ++h) {
        double z = b1[h];
        for (int i = 0; i < 3; ++i) z += W1[h * 3 + i] * in[i];
        if (z1) z1[h] = z;
        a1[h] = oracle_gelu(z);
    }
    for (int h = 0; h < H; ++h) {
        double z = b2[h];
        for (int i = 0; i < H; ++i) z += W2[(size_t)h * H + i] * a1[i];
        if (z2) z2[h] = z;
        a2[h] = oracle_gelu(z);
    }
    for (int o = 0; o < 16; ++o) {
        double z = b3[o];
        for (int i = 0; i < H; ++i) z += W3[(size_t)o * H + i] * a2[i];
        out[o] = z;
    }
    free(a1);
}

/* Backward pass of the same network for one input: given dL/dout[16],
 * ACCUMULATE dL/dparams into grad (same layout as the weights). */
void oracle_mlp_backward(const double* prm, int H, const double in[3], const double gout[16],
                         double* grad)
{
    const double* W1 = prm;
    const double* b1 = W1 + (size_t)H * 3;
    const double* W2 = b1 + H;
    const double* b2 = W2 + (size_t)H * H;
    const double* W3 = b2 + H;
    (void)b1;
    (void)b2;
    double* gW1 = grad;
    double* gb1 = gW1 + (size_t)H * 3;
    double* gW2 = gb1 + H;
    double* gb2 = gW2 + (size_t)H * H;
    double* gW3 = gb2 + H;
    double* gb3 = gW3 + (size_t)16 * H;
    double* z1 = (double*)malloc(sizeof(double) * H * 6);
    double* z2 = z1 + H;
    double* a1 = z2 + H;
    double* a2 = a1 + H;
    double* g2 = a2 + H;
    double* g1 = g2 + H;
    double out[16];
    oracle_mlp_forward(prm, H, in, out, z1, z2);
    for (int h = 0; h < H; ++h) {
        a1[h] = oracle_gelu(z1[h]);
        a2[h] = oracle_gelu(z2[h]);
    }
    /* layer 3 */
    for (int h = 0; h < H; ++h) g2[h] = 0.0;
    for (int o = 0; o < 16; ++o) {
        gb3[o] += gout[o];
        for (int h = 0; h < H; ++h) {
            gW3[(size_t)o * H + h] += gout[o] * a2[h];
            g2[h] += gout[o] * W3[(size_t)o * H + h];
        }
    }
    /* through GELU 2, layer 2 */
    for (int h = 0; h < H; ++h) g2[h] *= oracle_gelu_grad(z2[h]);
    for (int h = 0; h < H; ++h) g1[h] = 0.0;
    for (int h = 0; h < H; ++h) {
        gb2[h] += g2[h];
        for (int i = 0; i < H; ++i) {
            gW2[(size_t)h * H + i] += g2[h] * a1[i];
            g1[i] += g2[h] * W2[(size_t)h * H + i];
        }
    }
    /* through GELU 1, layer 1 */
    for (int h = 0; h < H; ++h) {
        double g = g1[h] * oracle_gelu_grad(z1[h]);
        gb1[h] += g;
        for (int i = 0; i < 3; ++i) gW1[h * 3 + i] += g * in[i];
    }
    free(z1);
}

/* Plane index scaled to [-1, 1], the third input of the learned kernel. */
static double plane_coordinate(int k, int Nw)
{
    if (Nw <= 1) return 0.0;
    return (2.0 * k - (Nw - 1)) / (double)(Nw - 1);
}

/* Network correction of the learned kernel for fractional offsets (fx, fy)
 * on plane k: t[b*4 + a] for cell (i0 + a, j0 + b).  With a lattice L > 0 the
 * network is evaluated on the (L+1)^2 lattice points around (fx, fy) and
 * interpolated bilinearly; with L = 0 it is evaluated at (fx, fy) itself. */
static void learned_taps(const oracle_cfg* cfg, double fx, double fy, int k, double t[16])
{
    double wk = plane_coordinate(k, cfg->Nw);
    if (cfg->mlp_lattice <= 0) {
        double in[3] = {fx, fy, wk};
        oracle_mlp_forward(cfg->mlp, cfg->mlp_hidden, in, t, NULL, NULL);
        return;
    }
    int L = cfg->mlp_lattice;
    double X = fx * L, Y = fy * L;
    int ix = (int)floor(X), iy = (int)floor(Y);
    if (ix > L - 1) ix = L - 1;
    if (iy > L - 1) iy = L - 1;
    double ax = X - ix, ay = Y - iy;
    double c00[16], c10[16], c01[16], c11[16];
    double in[3];
    in[2] = wk;
    in[0] = (double)ix / L;       in[1] = (double)iy / L;
    oracle_mlp_forward(cfg->mlp, cfg->mlp_hidden, in, c00, NULL, NULL);
    in[0] = (double)(ix + 1) / L; in[1] = (double)iy / L;
    oracle_mlp_forward(cfg->mlp, cfg->mlp_hidden, in, c10, NULL, NULL);
    in[0] = (double)ix / L;       in[1] = (double)(iy + 1) / L;
    oracle_mlp_forward(cfg->mlp, cfg->mlp_hidden, in, c01, NULL, NULL);
    in[0] = (double)(ix + 1) / L; in[1] = (double)(iy + 1) / L;
    oracle_mlp_forward(cfg->mlp, cfg->mlp_hidden, in, c11, NULL, NULL);
    for (int o = 0; o < 16; ++o)
        t[o] = (1.0 - ay) * ((1.0 - ax) * c00[o] + ax * c10[o]) +
               ay * ((1.0 - ax) * c01[o] + ax * c11[o]);
}

/* ------------------------------------------------------------------ */
/* FFT (Sec. 2: "each w-plane is Fourier transformed separately")      */
/* ------------------------------------------------------------------ */

/* In-place radix-2 inverse DFT of length n (power of two), unnormalised:
 * a[p] <- sum_i a[i] exp(+2 pi i i p / n).  Twiddles are evaluated directly
 * (no recurrence), bit-reversal permutation first, then butterflies. */
static void ifft1(int n, double complex* a, const double complex* tw /* tw[k] = exp(+2 pi i k/n), k < n/2 */)
{
    for (int i = 1, j = 0; i < n; ++i) {
        int bit = n >> 1;
        for (; j & bit; bit >>= 1) j ^= bit;
        j ^= bit;
        if (i < j) {
            double complex t = a[i];
            a[i] = a[j];
            a[j] = t;
        }
    }
    for (int len = 2; len <= n; len <<= 1) {
        int half = len >> 1, step = n / len;
        for (int s = 0; s < n; s += len)
            for (int k = 0; k < half; ++k) {
                double complex w = tw[k * step];
                double complex u = a[s + k], v = a[s + k + half] * w;
                a[s + k] = u + v;
                a[s + k + half] = u - v;
            }
    }
}

/* 2-D inverse DFT of an N x N row-major array, unnormalised, exponent +:
 * A[q][p] <- sum_{j,i} A[j][i] exp(+2 pi i (i p + j q)/N).  Rows, then columns. */
int oracle_ifft2(int N, double complex* A)
{
    if (N < 1 || (N & (N - 1))) return 1;
    double complex* tw = (double complex*)malloc(sizeof(double complex) * (N / 2 + 1));
    double complex* col = (double complex*)malloc(sizeof(double complex) * N);
    if (!tw || !col) { free(tw); free(col); return 2; }
    for (int k = 0; k < N / 2; ++k) {
        double ang = 2.0 * ORACLE_PI * (double)k / (double)N;
        tw[k] = cos(ang) + I * sin(ang);
    }
    for (int r = 0; r < N; ++r) ifft1(N, A + (size_t)r * N, tw);
    for (int c = 0; c < N; ++c) {
        for (int r = 0; r < N; ++r) col[r] = A[(size_t)r * N + c];
        ifft1(N, col, tw);
        for (int r = 0; r < N; ++r) A[(size_t)r * N + c] = col[r];
    }
    free(tw);
    free(col);
    return 0;
}

/* ------------------------------------------------------------------ */
/* Visibility placement: R1, R3, R4                                    */
/* ------------------------------------------------------------------ */

typedef struct {
    int ok;        /* 1 = gridded; 0 = flagged / zero weight; -1 = dropped off the grid */
    long i0, j0;   /* first footprint cell along u and along v (R3) */
    double x, y;   /* continuous position in cells (R1) */
    double fx, fy; /* (x - S/2) - floor(x - S/2), in [0, 1) */
    int k;         /* w-plane (R4); with a w-kernel, the first of its Sw planes (R14) */
    double fw;     /* with a w-kernel: (z - Sw/2) - floor(z - Sw/2), z = plane coordinate */
    double u, v, w;/* wavelengths at this channel */
} placement;

static double wplane_scale(const oracle_cfg* cfg)
{
    if (cfg->Nw <= 1) return 0.0;
    return (double)cfg->Nw / (cfg->w_max - cfg->w_min);
}

static int w_improved(const oracle_cfg* cfg) { return cfg->w_support >= 2; }

/* Planes imaged: Nw, or Nw + Sw with a w-kernel (Sw/2 more at each end, R14). */
int oracle_planes_total(const oracle_cfg* cfg)
{
    return cfg->Nw + (w_improved(cfg) ? cfg->w_support : 0);
}

/* w_k: centre of plane k (R4); with a w-kernel, plane k of the extended set,
 * whose first Sw/2 planes lie below w_min (R14). */
double oracle_plane_w(const oracle_cfg* cfg, int k)
{
    if (cfg->Nw <= 1) return 0.5 * (cfg->w_min + cfg->w_max);
    double dw = (cfg->w_max - cfg->w_min) / cfg->Nw;
    int off = w_improved(cfg) ? cfg->w_support / 2 : 0;
    return cfg->w_min + (k - off + 0.5) * dw;
}

static placement place(const oracle_cfg* cfg, const double* uvw, const double* scale, int C,
                       const float* weight, const uint8_t* flag, long r, int c)
{
    placement P;
    memset(&P, 0, sizeof P);
    size_t idx = (size_t)r * C + c;
    if (flag && flag[idx]) return P;
    double W = weight[idx];
    if (!(W != 0.0) || !isfinite(W)) return P;
    P.u = uvw[3 * r + 0] * scale[c];
    P.v = uvw[3 * r + 1] * scale[c];
    P.w = uvw[3 * r + 2] * scale[c];
    /* R1, and R16 for a padded mesh: fov * Ng/N is exact (powers of two) */
    int Ng = grid_n(cfg);
    double half = 0.5 * Ng, fovg = cfg->fov * (double)Ng / (double)cfg->N;
    P.x = P.u * fovg + half;
    P.y = P.v * fovg + half;
    if (!isfinite(P.x) || !isfinite(P.y) || !isfinite(P.w)) { P.ok = -1; return P; }
    double sx = P.x - 0.5 * cfg->S, sy = P.y - 0.5 * cfg->S;
    double flx = floor(sx), fly = floor(sy);
    if (flx < -1.0 || fly < -1.0 || flx + cfg->S > Ng - 1 + 0.0 || fly + cfg->S > Ng - 1 + 0.0) {
        P.ok = -1;
        return P;
    }
    P.i0 = (long)flx + 1;
    P.j0 = (long)fly + 1;
    P.fx = sx - flx;
    P.fy = sy - fly;
    if (cfg->Nw <= 1) {
        P.k = 0;
    } else if (w_improved(cfg)) {
        /* R14: plane coordinate z (plane k centred at z = k), clamped to the
         * w range; footprint of Sw planes as R3 in u and v, shifted by Sw/2 */
        int Sw = cfg->w_support;
        double z = (P.w - cfg->w_min) * wplane_scale(cfg) - 0.5;
        if (z < -0.5) z = -0.5;
        if (z > cfg->Nw - 0.5) z = cfg->Nw - 0.5;
        double sz = z - 0.5 * Sw;
        double fl = floor(sz);
        P.k = (int)fl + 1 + Sw / 2;
        P.fw = sz - fl;
    } else {
        double t = (P.w - cfg->w_min) * wplane_scale(cfg);
        double kf = floor(t);
        if (kf < 0.0) kf = 0.0;
        if (kf > cfg->Nw - 1) kf = cfg->Nw - 1;
        P.k = (int)kf;
    }
    P.ok = 1;
    return P;
}

/* Weight of plane k for a placed visibility: 1 on its plane (R4), or the
 * w-kernel g_w(k - z) on its Sw planes (R14); 0 elsewhere. */
static double plane_weight(const oracle_cfg* cfg, const placement* P, int k)
{
    if (!w_improved(cfg)) return k == P->k ? 1.0 : 0.0;
    int s = k - P->k;
    if (s < 0 || s >= cfg->w_support) return 0.0;
    return oracle_kernel_value(ORACLE_KAISER_BESSEL, cfg->w_kernel_param, cfg->w_support,
                               (double)s + 1.0 - 0.5 * cfg->w_support - P->fw);
}

/* Continuous Fourier transform of a separable kernel, C(nu) = int g(s) cos(2 pi s nu) ds
 * over [-S/2, S/2], by composite Gauss-Legendre quadrature (24 nodes per unit). */
double oracle_kernel_ft(int kind, double param, int S, double nu)
{
    double gx[24], gwt[24];
    oracle_gauss_legendre(24, gx, gwt);
    double acc = 0.0;
    for (int seg = 0; seg < S; ++seg) {
        double a = -0.5 * S + seg;
        for (int i = 0; i < 24; ++i) {
            double si = a + 0.5 + 0.5 * gx[i];
            acc += 0.5 * gwt[i] * oracle_kernel_value(kind, param, S, si) * cos(2.0 * ORACLE_PI * si * nu);
        }
    }
    return acc;
}

/* The w-taper C_w((n - 1) dw) that the image is divided by (R14); 1 without a
 * w-kernel. */
static double w_taper(const oracle_cfg* cfg, double delta)
{
    if (!w_improved(cfg) || cfg->Nw <= 1) return 1.0;
    double dw = (cfg->w_max - cfg->w_min) / cfg->Nw;
    return oracle_kernel_ft(ORACLE_KAISER_BESSEL, cfg->w_kernel_param, cfg->w_support, delta * dw);
}

/* Per-visibility placement, exported so that tests can compare index work
 * exactly.  For each visibility (r, c), r < nrow, c < C, row-major:
 *   status (1 gridded, 0 skipped, -1 dropped), k, i0, j0, fx, fy, and with a
 *   w-kernel the plane fraction fw (k is then the first of its Sw planes). */
void oracle_place(const oracle_cfg* cfg, const double* uvw, const double* scale, int C,
                  const float* weight, const uint8_t* flag, long nrow, int32_t* status, int32_t* k,
                  int32_t* i0, int32_t* j0, double* fx, double* fy, double* fw)
{
    for (long r = 0; r < nrow; ++r)
        for (int c = 0; c < C; ++c) {
            placement P = place(cfg, uvw, scale, C, weight, flag, r, c);
            size_t idx = (size_t)r * C + c;
            status[idx] = P.ok;
            k[idx] = P.ok == 1 ? P.k : -1;
            i0[idx] = P.ok == 1 ? (int32_t)P.i0 : 0;
            j0[idx] = P.ok == 1 ? (int32_t)P.j0 : 0;
            fx[idx] = P.ok == 1 ? P.fx : 0.0;
            fy[idx] = P.ok == 1 ? P.fy : 0.0;
            if (fw) fw[idx] = P.ok == 1 ? P.fw : 0.0;
        }
}

/* Kernel weight of footprint cell (i0 + a, j0 + b) of a placed visibility. */
static void footprint_weights(const oracle_cfg* cfg, const placement* P, double* gw /* [S][S], b-major */)
{
    int S = cfg->S;
    if (cfg->kernel == ORACLE_LEARNED) {
        /* Kaiser-Bessel support-4 taps plus the network's correction */
        double t[16];
        learned_taps(cfg, P->fx, P->fy, P->k, t);
        for (int b = 0; b < 4; ++b)
            for (int a = 0; a < 4; ++a)
                gw[b * 4 + a] =
                    oracle_kernel_value(ORACLE_KAISER_BESSEL, cfg->kernel_param, 4, (double)(P->i0 + a) - P->x) *
                        oracle_kernel_value(ORACLE_KAISER_BESSEL, cfg->kernel_param, 4, (double)(P->j0 + b) - P->y) +
                    t[b * 4 + a];
        return;
    }
    double gxa[64], gyb[64];
    for (int a = 0; a < S; ++a) {
        gxa[a] = oracle_kernel_value(cfg->kernel, cfg->kernel_param, S, (double)(P->i0 + a) - P->x);
        gyb[a] = oracle_kernel_value(cfg->kernel, cfg->kernel_param, S, (double)(P->j0 + a) - P->y);
    }
    for (int b = 0; b < S; ++b)
        for (int a = 0; a < S; ++a) gw[b * S + a] = gxa[a] * gyb[b];
}

static int check_cfg(const oracle_cfg* cfg)
{
    if (cfg->N < 2 || (cfg->N & (cfg->N - 1))) return 1;
    if (cfg->Nw < 1 || cfg->S < 1 || cfg->S > 64 || cfg->S > cfg->N) return 1;
    if (cfg->Nw > 1 && !(cfg->w_max > cfg->w_min)) return 1;
    if (!(cfg->fov > 0.0) || cfg->fov >= 1.0) return 1;
    if (cfg->kernel == ORACLE_LEARNED && (cfg->S != 4 || !cfg->mlp || cfg->mlp_hidden < 1)) return 1;
    if (cfg->w_support < 0 || cfg->w_support > 16) return 1;
    if (w_improved(cfg) && ((cfg->w_support & 1) || cfg->Nw < 2 || !(cfg->w_kernel_param > 0.0))) return 1;
    if (cfg->weighting < ORACLE_NATURAL || cfg->weighting > ORACLE_BRIGGS) return 1;
    if (cfg->weighting == ORACLE_BRIGGS && !isfinite(cfg->robust)) return 1;
    if (cfg->Ng != 0 && (cfg->Ng < cfg->N || (cfg->Ng & (cfg->Ng - 1)))) return 1;
    if (cfg->Ng != 0 && cfg->kernel == ORACLE_LEARNED) return 1;
    return 0;
}

/* Imaging weights (R15): out[r][c] = W' for every visibility (W itself for
 * those that are not gridded, and for natural weighting).  Returns 0, or 1
 * for an invalid configuration, 2 if memory runs out.  The gridding, imaging
 * and direct-inversion functions below take the weights they are given; for
 * uniform or Briggs weighting the caller passes W' (the Python wrapper does). */
int oracle_imaging_weights(const oracle_cfg* cfg, const double* uvw, const double* scale, int C,
                           const float* weight, const uint8_t* flag, long nrow, double* out)
{
    if (check_cfg(cfg)) return 1;
    for (long r = 0; r < nrow; ++r)
        for (int c = 0; c < C; ++c) out[(size_t)r * C + c] = (double)weight[(size_t)r * C + c];
    if (cfg->weighting == ORACLE_NATURAL) return 0;
    int N = cfg->N;
    double* D = (double*)malloc(sizeof(double) * (size_t)N * N);
    long* cell = (long*)malloc(sizeof(long) * (size_t)(nrow > 0 ? nrow : 1));
    if (!D || !cell) { free(D); free(cell); return 2; }
    for (int c = 0; c < C; ++c) {
        memset(D, 0, sizeof(double) * (size_t)N * N);
        for (long r = 0; r < nrow; ++r) {
            cell[r] = -1;
            placement P = place(cfg, uvw, scale, C, weight, flag, r, c);
            if (P.ok != 1) continue;
            /* nearest cell of the N x N mesh of cell 1/fov (R15, R16), mod N */
            double xi = P.u * cfg->fov + 0.5 * N, yi = P.v * cfg->fov + 0.5 * N;
            long i = (((long)floor(xi + 0.5)) % N + N) % N, j = (((long)floor(yi + 0.5)) % N + N) % N;
            double W = (double)weight[(size_t)r * C + c];
            D[(size_t)j * N + i] += W;
            D[(size_t)((N - j) % N) * N + (N - i) % N] += W;
            cell[r] = j * N + i;
        }
        double f2 = 0.0;
        if (cfg->weighting == ORACLE_BRIGGS) {
            double s1 = 0.0, s2 = 0.0;
            for (size_t e = 0; e < (size_t)N * N; ++e) {
                s1 += D[e];
                s2 += D[e] * D[e];
            }
            double a = 5.0 * pow(10.0, -cfg->robust);
            f2 = s2 > 0.0 ? a * a * s1 / s2 : 0.0;
        }
        for (long r = 0; r < nrow; ++r) {
            if (cell[r] < 0) continue;
            double W = (double)weight[(size_t)r * C + c], d = D[cell[r]];
            out[(size_t)r * C + c] = cfg->weighting == ORACLE_UNIFORM ? W / d : W / (1.0 + f2 * d);
        }
    }
    free(D);
    free(cell);
    return 0;
}

/* Taper used by a configuration: the kernel's own, or for the learned kernel
 * the support-S Kaiser-Bessel with beta = kernel_param. */
static void cfg_taper(const oracle_cfg* cfg, double* C)
{
    int kind = cfg->kernel == ORACLE_LEARNED ? ORACLE_KAISER_BESSEL : cfg->kernel;
    oracle_taper_padded(kind, cfg->kernel_param, cfg->S, cfg->N, grid_n(cfg), C);
}

/* ------------------------------------------------------------------ */
/* Eq. 3: one gridded w-plane                                          */
/* ------------------------------------------------------------------ */

/* Grid channel c onto plane k: G[j][i] += W V g(i - x) g(j - y) (-1)^(i+j)
 * over the footprint of every gridded visibility of that channel whose plane
 * is k.  G is Ng x Ng complex (the mesh, R16), zeroed here.  Returns the
 * number gridded. */
long oracle_grid_plane(const oracle_cfg* cfg, const double* uvw, const double* scale, int C,
                       const float* vis /* [nrow][C][2] */, const float* weight,
                       const uint8_t* flag, long nrow, int c, int k, double complex* G)
{
    if (check_cfg(cfg)) return -1;
    int N = grid_n(cfg), S = cfg->S;
    memset(G, 0, sizeof(double complex) * (size_t)N * N);
    double* gw = (double*)malloc(sizeof(double) * S * S);
    long n = 0;
    for (long r = 0; r < nrow; ++r) {
        placement P = place(cfg, uvw, scale, C, weight, flag, r, c);
        if (P.ok != 1) continue;
        double pw = plane_weight(cfg, &P, k);
        if (pw == 0.0) continue;
        size_t idx = (size_t)r * C + c;
        double complex WV = pw * (double)weight[idx] * ((double)vis[2 * idx] + I * (double)vis[2 * idx + 1]);
        footprint_weights(cfg, &P, gw);
        for (int b = 0; b < S; ++b) {
            long j = P.j0 + b;
            for (int a = 0; a < S; ++a) {
                long i = P.i0 + a;
                double sgn = ((i + j) & 1) ? -1.0 : 1.0;
                G[(size_t)j * N + i] += WV * (gw[b * S + a] * sgn);
            }
        }
        ++n;
    }
    free(gw);
    return n;
}

/* Sum of weights and counts of gridded / dropped visibilities of channel c. */
void oracle_channel_stats(const oracle_cfg* cfg, const double* uvw, const double* scale, int C,
                          const float* weight, const uint8_t* flag, long nrow, int c,
                          double* weight_sum, long* n_gridded, long* n_dropped)
{
    double ws = 0.0;
    long ng = 0, nd = 0;
    for (long r = 0; r < nrow; ++r) {
        placement P = place(cfg, uvw, scale, C, weight, flag, r, c);
        if (P.ok == 1) {
            ws += (double)weight[(size_t)r * C + c];
            ++ng;
        } else if (P.ok == -1) {
            ++nd;
        }
    }
    *weight_sum = ws;
    *n_gridded = ng;
    *n_dropped = nd;
}

/* n = sqrt(1 - l^2 - m^2) and delta = n - 1 = -(l^2 + m^2)/(1 + n) at pixel (p, q) (R2). */
static void pixel_n(const oracle_cfg* cfg, int p, int q, double* n, double* delta)
{
    double dl = cfg->fov / cfg->N;
    double l = (p - cfg->N / 2) * dl, m = (q - cfg->N / 2) * dl;
    double r2 = l * l + m * m;
    *n = sqrt(1.0 - r2);
    *delta = -r2 / (1.0 + *n);
}

/* exp(2 pi i t) with t reduced to the nearest whole turn first. */
static double complex turn_phasor(double t)
{
    double f = t - floor(t + 0.5);
    double a = 2.0 * ORACLE_PI * f;
    return cos(a) + I * sin(a);
}

/* ------------------------------------------------------------------ */
/* O1: the w-stacking dirty image (Eq. 2 and 3, R5, R6)                */
/* ------------------------------------------------------------------ */

void oracle_phase_accumulate(const oracle_cfg* cfg, int k, const double complex* F, double complex* img);
void oracle_image_scale(const oracle_cfg* cfg, double ws, const double* Ct, double complex* img);

/* Complex dirty image of channel c, N x N, row q (m) major, column p (l):
 *   I[q][p] = (-1)^(p+q) n / (sum W * C(p) C(q)) * sum_k F_k[q][p] exp(+2 pi i w_k (n-1))
 * where F_k is the unnormalised inverse 2-D DFT of the gridded plane k.
 * Planes are gridded and transformed one at a time.  Returns 0 on success. */
int oracle_image(const oracle_cfg* cfg, const double* uvw, const double* scale, int C,
                 const float* vis, const float* weight, const uint8_t* flag, long nrow, int c,
                 double complex* img, double* weight_sum_out)
{
    if (check_cfg(cfg)) return 1;
    int N = cfg->N, Ng = grid_n(cfg);
    size_t NN = (size_t)N * N;
    double complex* G = (double complex*)malloc(sizeof(double complex) * (size_t)Ng * Ng);
    double* Ct = (double*)malloc(sizeof(double) * N);
    if (!G || !Ct) { free(G); free(Ct); return 2; }
    cfg_taper(cfg, Ct);
    double ws;
    long ng, nd;
    oracle_channel_stats(cfg, uvw, scale, C, weight, flag, nrow, c, &ws, &ng, &nd);
    memset(img, 0, sizeof(double complex) * NN);
    for (int k = 0; k < oracle_planes_total(cfg); ++k) {
        long nk = oracle_grid_plane(cfg, uvw, scale, C, vis, weight, flag, nrow, c, k, G);
        if (nk <= 0) continue;
        oracle_ifft2(Ng, G);
        oracle_phase_accumulate(cfg, k, G, img);
    }
    oracle_image_scale(cfg, ws, Ct, img);
    if (weight_sum_out) *weight_sum_out = ws;
    free(G);
    free(Ct);
    return 0;
}

/* Eq. 2, one term of the sum over planes: img[q][p] += F_k[q][p] exp(+2 pi i
 * w_k (n - 1)) over the image pixels, F_k the transformed plane k (Ng x Ng;
 * the image is its central N x N). */
void oracle_phase_accumulate(const oracle_cfg* cfg, int k, const double complex* F, double complex* img)
{
    int N = cfg->N, Ng = grid_n(cfg), off = pad_off(cfg);
    double wk = oracle_plane_w(cfg, k);
    for (int q = 0; q < N; ++q)
        for (int p = 0; p < N; ++p) {
            double n, d;
            pixel_n(cfg, p, q, &n, &d);
            img[(size_t)q * N + p] += F[(size_t)(q + off) * Ng + (p + off)] * turn_phasor(wk * d);
        }
}

/* The normalisation of Eq. 2 with R5, R6: img[q][p] *= (-1)^(p+q) n /
 * (sum W C(p) C(q) C_w) (0 if sum W = 0); Ct = the taper C(p). */
void oracle_image_scale(const oracle_cfg* cfg, double ws, const double* Ct, double complex* img)
{
    int N = cfg->N;
    for (int q = 0; q < N; ++q)
        for (int p = 0; p < N; ++p) {
            double n, d;
            pixel_n(cfg, p, q, &n, &d);
            double sgn = ((p + q) & 1) ? -1.0 : 1.0;
            double s = ws != 0.0 ? sgn * n / (ws * Ct[p] * Ct[q] * w_taper(cfg, d)) : 0.0;
            img[(size_t)q * N + p] *= s;
        }
}

/* O1 at chosen pixels without the FFT: the same image value written as the
 * DFT of the gridded planes evaluated at (p, q), summed visibility by
 * visibility:  sum_j W_j V_j exp(2 pi i w_kj (n-1))
 *                * [sum_a g_a (-1)^(i0+a) e^{2 pi i (i0+a) p / N}]
 *                * [sum_b g_b (-1)^(j0+b) e^{2 pi i (j0+b) q / N}]
 * (non-separable learned taps are summed over (a, b) jointly), then scaled as
 * in oracle_image.  If plane >= 0 only that plane is summed and the value
 * returned is F_plane[q][p] itself (no phase screen, no scaling). */
int oracle_image_at(const oracle_cfg* cfg, const double* uvw, const double* scale, int C,
                    const float* vis, const float* weight, const uint8_t* flag, long nrow, int c,
                    int plane, long npix, const int32_t* pp, const int32_t* qq, double complex* out)
{
    if (check_cfg(cfg)) return 1;
    int N = cfg->N, S = cfg->S, Ng = grid_n(cfg), off = pad_off(cfg);
    double* Ct = (double*)malloc(sizeof(double) * N);
    double* gw = (double*)malloc(sizeof(double) * S * S);
    double complex* ex = (double complex*)malloc(sizeof(double complex) * S * 2);
    double complex* ey = ex + S;
    cfg_taper(cfg, Ct);
    double ws;
    long ng, nd;
    oracle_channel_stats(cfg, uvw, scale, C, weight, flag, nrow, c, &ws, &ng, &nd);
    for (long t = 0; t < npix; ++t) out[t] = 0.0;
    for (long r = 0; r < nrow; ++r) {
        placement P = place(cfg, uvw, scale, C, weight, flag, r, c);
        if (P.ok != 1) continue;
        if (plane >= 0 && plane_weight(cfg, &P, plane) == 0.0) continue;
        size_t idx = (size_t)r * C + c;
        double complex WV = (double)weight[idx] * ((double)vis[2 * idx] + I * (double)vis[2 * idx + 1]);
        footprint_weights(cfg, &P, gw);
        /* the visibility's planes: its own (R4) or its Sw planes (R14) */
        int kfirst = P.k, kn = w_improved(cfg) ? cfg->w_support : 1;
        for (long t = 0; t < npix; ++t) {
            int p = pp[t], q = qq[t];
            for (int a = 0; a < S; ++a) {
                long i = P.i0 + a, j = P.j0 + a;
                double sx = (i & 1) ? -1.0 : 1.0, sy = (j & 1) ? -1.0 : 1.0;
                /* exp(2 pi i i P / Ng) at the transform's pixel P = p + off,
                 * the exponent reduced exactly mod Ng */
                long ip = (i * (long)(p + off)) % Ng, jq = (j * (long)(q + off)) % Ng;
                ex[a] = sx * turn_phasor((double)ip / Ng);
                ey[a] = sy * turn_phasor((double)jq / Ng);
            }
            double complex acc = 0.0;
            for (int b = 0; b < S; ++b) {
                double complex rowsum = 0.0;
                for (int a = 0; a < S; ++a) rowsum += gw[b * S + a] * ex[a];
                acc += rowsum * ey[b];
            }
            if (plane < 0) {
                double n, d;
                pixel_n(cfg, p, q, &n, &d);
                double complex ph = 0.0;
                for (int s = 0; s < kn; ++s)
                    ph += plane_weight(cfg, &P, kfirst + s) * turn_phasor(oracle_plane_w(cfg, kfirst + s) * d);
                acc *= ph;
            } else {
                acc *= plane_weight(cfg, &P, plane);
            }
            out[t] += WV * acc;
        }
    }
    if (plane < 0)
        for (long t = 0; t < npix; ++t) {
            int p = pp[t], q = qq[t];
            double n, d;
            pixel_n(cfg, p, q, &n, &d);
            double sgn = ((p + q) & 1) ? -1.0 : 1.0;
            out[t] *= ws != 0.0 ? sgn * n / (ws * Ct[p] * Ct[q] * w_taper(cfg, d)) : 0.0;
        }
    free(Ct);
    free(gw);
    free(ex);
    return 0;
}

/* ------------------------------------------------------------------ */
/* O2: direct Fourier inversion of Eq. 1 (the plain definition)        */
/* ------------------------------------------------------------------ */

/* I_D(p, q) = n / sum W * sum_j W_j V_j exp(+2 pi i (u_j l + v_j m + w_j (n - 1)))
 * over the same visibilities the gridder keeps (unflagged, non-zero weight,
 * footprint on the grid), so that O1 - O2 is the error of the method alone. */
int oracle_dft_at(const oracle_cfg* cfg, const double* uvw, const double* scale, int C,
                  const float* vis, const float* weight, const uint8_t* flag, long nrow, int c,
                  long npix, const int32_t* pp, const int32_t* qq, double complex* out)
{
    if (check_cfg(cfg)) return 1;
    double dl = cfg->fov / cfg->N;
    double ws = 0.0;
    for (long t = 0; t < npix; ++t) out[t] = 0.0;
    for (long r = 0; r < nrow; ++r) {
        placement P = place(cfg, uvw, scale, C, weight, flag, r, c);
        if (P.ok != 1) continue;
        size_t idx = (size_t)r * C + c;
        double W = weight[idx];
        ws += W;
        double complex WV = W * ((double)vis[2 * idx] + I * (double)vis[2 * idx + 1]);
        for (long t = 0; t < npix; ++t) {
            double l = (pp[t] - cfg->N / 2) * dl, m = (qq[t] - cfg->N / 2) * dl;
            double n, d;
            pixel_n(cfg, pp[t], qq[t], &n, &d);
            out[t] += WV * turn_phasor(P.u * l + P.v * m + P.w * d);
        }
    }
    for (long t = 0; t < npix; ++t) {
        double n, d;
        pixel_n(cfg, pp[t], qq[t], &n, &d);
        out[t] *= ws != 0.0 ? n / ws : 0.0;
    }
    return 0;
}

/* ------------------------------------------------------------------ */
/* Prediction (degridding): the adjoint direction of Eq. 2 and 3       */
/* ------------------------------------------------------------------ */
/*
 * The paper only images (Sec. 2); prediction is the other half of an imaging
 * cycle and is written here from the same statement of the problem.  For a
 * real model image J of one channel, Eq. 1 discretised on the pixels reads
 *   V(u, v, w) = sum_{p,q} J(p, q) / n * exp(-2 pi i (u l + v m + w (n - 1)))
 * (O2 below, the plain definition).  Its w-stacking form, with the same
 * readings R1-R7 as the imaging path, is (O1):
 *   M_k(p, q) = J(p, q) exp(-2 pi i w_k (n - 1)) / (n C(p) C(q))
 *   F_k(i, j) = sum_{p,q} M_k(p, q) exp(-2 pi i ((i - N/2)(p - N/2) + (j - N/2)(q - N/2)) / N)
 *             = (-1)^(i+j) * [forward DFT of (-1)^(p+q) M_k](i, j)           (R6)
 *   V        ~ sum_{a,b} g(i0 + a - x) g(j0 + b - y) F_k(i0 + a, j0 + b)
 * for every visibility the gridder keeps (R3, R4, R10), k its plane; the
 * others are 0.  The convolution with g in (u, v) is undone by the division by
 * C in (l, m), as in the imaging path.  This operator is the adjoint of the
 * imaging operator up to the weights and the n^2 factor:
 *   sum W V conj(pred(J)) = sum W * sum_p J(p) I(V)(p) / n(p)^2.
 */

/* Forward 2-D DFT (exponent -), unnormalised: conj(ifft2(conj(A))). */
static void fft2_forward(int N, double complex* A)
{
    size_t NN = (size_t)N * N;
    for (size_t t = 0; t < NN; ++t) A[t] = conj(A[t]);
    oracle_ifft2(N, A);
    for (size_t t = 0; t < NN; ++t) A[t] = conj(A[t]);
}

/* O1 prediction for channel c from the real model image J [N][N] (row q, column
 * p): out[r] for every row r of the visibilities (zero where not gridded).
 * Planes are built, transformed and sampled one at a time.  Returns 0. */
int oracle_predict(const oracle_cfg* cfg, const double* uvw, const double* scale, int C,
                   const float* weight, const uint8_t* flag, long nrow, int c, const double* J,
                   double complex* out)
{
    if (check_cfg(cfg)) return 1;
    if (cfg->kernel == ORACLE_LEARNED) return 3;
    int Ni = cfg->N, N = grid_n(cfg), off = pad_off(cfg), S = cfg->S;
    size_t NN = (size_t)N * N;
    double complex* F = (double complex*)malloc(sizeof(double complex) * NN);
    double* Ct = (double*)malloc(sizeof(double) * Ni);
    double* gw = (double*)malloc(sizeof(double) * S * S);
    if (!F || !Ct || !gw) { free(F); free(Ct); free(gw); return 2; }
    cfg_taper(cfg, Ct);
    for (long r = 0; r < nrow; ++r) out[r] = 0.0;
    for (int k = 0; k < oracle_planes_total(cfg); ++k) {
        double wk = oracle_plane_w(cfg, k);
        /* the model inside the central Ni x Ni of the mesh-sized plane (R16) */
        memset(F, 0, sizeof(double complex) * NN);
        for (int q = 0; q < Ni; ++q)
            for (int p = 0; p < Ni; ++p) {
                double n, d;
                pixel_n(cfg, p, q, &n, &d);
                double sgn = ((p + q) & 1) ? -1.0 : 1.0;
                F[(size_t)(q + off) * N + (p + off)] = sgn * J[(size_t)q * Ni + p] * turn_phasor(-wk * d) /
                                                       (n * Ct[p] * Ct[q] * w_taper(cfg, d));
            }
        fft2_forward(N, F);
        for (long r = 0; r < nrow; ++r) {
            placement P = place(cfg, uvw, scale, C, weight, flag, r, c);
            if (P.ok != 1) continue;
            double pw = plane_weight(cfg, &P, k);
            if (pw == 0.0) continue;
            footprint_weights(cfg, &P, gw);
            double complex acc = 0.0;
            for (int b = 0; b < S; ++b)
                for (int a = 0; a < S; ++a) {
                    long i = P.i0 + a, j = P.j0 + b;
                    double sgn = ((i + j) & 1) ? -1.0 : 1.0;
                    acc += gw[b * S + a] * sgn * F[(size_t)j * N + i];
                }
            out[r] += pw * acc;
        }
    }
    free(F);
    free(Ct);
    free(gw);
    return 0;
}

/* O1 prediction for a model of point sources on pixel centres (p_s, q_s) with
 * fluxes A_s, evaluated visibility by visibility without the FFT (the same
 * value as oracle_predict on that image):
 *   V = sum_{a,b} g_a g_b sum_s A_s exp(-2 pi i w_k (n_s - 1)) / (n_s C(p_s) C(q_s))
 *         * exp(-2 pi i ((i - N/2)(p_s - N/2) + (j - N/2)(q_s - N/2)) / N)
 * with the exponent reduced exactly mod N.  rows[t] selects the visibility
 * (rows[t], c); out[t] = 0 if it is not gridded. */
int oracle_predict_at(const oracle_cfg* cfg, const double* uvw, const double* scale, int C,
                      const float* weight, const uint8_t* flag, long nrow, int c, long nsrc,
                      const int32_t* sp, const int32_t* sq, const double* flux, long nsel,
                      const int64_t* rows, double complex* out)
{
    if (check_cfg(cfg)) return 1;
    if (cfg->kernel == ORACLE_LEARNED) return 3;
    int Ni = cfg->N, N = grid_n(cfg), S = cfg->S;
    double* Ct = (double*)malloc(sizeof(double) * Ni);
    double* gw = (double*)malloc(sizeof(double) * S * S);
    if (!Ct || !gw) { free(Ct); free(gw); return 2; }
    cfg_taper(cfg, Ct);
    for (long t = 0; t < nsel; ++t) {
        out[t] = 0.0;
        long r = (long)rows[t];
        if (r < 0 || r >= nrow) continue;
        placement P = place(cfg, uvw, scale, C, weight, flag, r, c);
        if (P.ok != 1) continue;
        footprint_weights(cfg, &P, gw);
        int kn = w_improved(cfg) ? cfg->w_support : 1;
        double complex acc = 0.0;
        for (long s = 0; s < nsrc; ++s) {
            double n, d;
            pixel_n(cfg, sp[s], sq[s], &n, &d);
            double complex ph = 0.0;  /* sum over the visibility's planes (R4 / R14) */
            for (int t2 = 0; t2 < kn; ++t2)
                ph += plane_weight(cfg, &P, P.k + t2) * turn_phasor(-oracle_plane_w(cfg, P.k + t2) * d);
            double complex Ms = flux[s] * ph / (n * Ct[sp[s]] * Ct[sq[s]] * w_taper(cfg, d));
            /* the transform's pixel P = p + off sits at P - Ng/2 = p - Ni/2 (R16) */
            long ps = sp[s] - Ni / 2, qs = sq[s] - Ni / 2;
            for (int b = 0; b < S; ++b) {
                long j = P.j0 + b - N / 2;
                long jq = ((j * qs) % N + N) % N;
                for (int a = 0; a < S; ++a) {
                    long i = P.i0 + a - N / 2;
                    long ip = ((i * ps) % N + N) % N;
                    acc += gw[b * S + a] * Ms * turn_phasor(-(double)((ip + jq) % N) / N);
                }
            }
        }
        out[t] = acc;
    }
    free(Ct);
    free(gw);
    return 0;
}

/* O2 prediction: Eq. 1 summed directly over point sources on pixel centres,
 *   V = sum_s A_s / n_s exp(-2 pi i (u l_s + v m_s + w (n_s - 1))),
 * for the selected visibilities that the gridder keeps (others 0). */
int oracle_predict_dft(const oracle_cfg* cfg, const double* uvw, const double* scale, int C,
                       const float* weight, const uint8_t* flag, long nrow, int c, long nsrc,
                       const int32_t* sp, const int32_t* sq, const double* flux, long nsel,
                       const int64_t* rows, double complex* out)
{
    if (check_cfg(cfg)) return 1;
    double dl = cfg->fov / cfg->N;
    for (long t = 0; t < nsel; ++t) {
        out[t] = 0.0;
        long r = (long)rows[t];
        if (r < 0 || r >= nrow) continue;
        placement P = place(cfg, uvw, scale, C, weight, flag, r, c);
        if (P.ok != 1) continue;
        double complex acc = 0.0;
        for (long s = 0; s < nsrc; ++s) {
            double l = (sp[s] - cfg->N / 2) * dl, m = (sq[s] - cfg->N / 2) * dl;
            double n, d;
            pixel_n(cfg, sp[s], sq[s], &n, &d);
            acc += flux[s] / n * turn_phasor(-(P.u * l + P.v * m + P.w * d));
        }
        out[t] = acc;
    }
    return 0;
}

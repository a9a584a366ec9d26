"""Pins of the FP64 oracle against facts it does not compute itself.

The paper (arXiv 2601.19714) prints no image values and no worked example,
so the oracle is pinned by library routines, closed forms, brute force on
tiny inputs, invariants of the method, and the direct Fourier inversion of
Eq. 1 within the method's own error bound.  Each test names what a mistake
in the oracle would have to get wrong to slip past it.
"""
import math

import numpy as np
import pytest
import scipy.integrate as integ
import scipy.special as sp

import visgen
from visgen.workloads import GAUSS_SIGMA_S7, KB_BETA_S4, KB_BETA_S8, tiny_wstack

pytestmark = pytest.mark.filterwarnings("ignore::scipy.integrate.IntegrationWarning")


def cfg_of(orc, img, **kw):
    d = dict(N=img.N, Nw=img.Nw, S=img.S, kernel=img.kernel, kernel_param=img.kernel_param,
             fov=img.fov, w_min=img.w_min, w_max=img.w_max)
    d.update(kw)
    return orc.Config(**d)


# ----------------------------------------------------------------------------
# kernel functions and quadrature
# ----------------------------------------------------------------------------

def test_bessel_i0_matches_library(orc):
    for x in np.linspace(0.0, 40.0, 81):
        assert orc.bessel_i0(x) == pytest.approx(sp.i0(x), rel=1e-13)


def test_kaiser_bessel_shape(orc):
    S, beta = 8, KB_BETA_S8
    assert orc.kernel_value("kb", beta, S, 0.0) == pytest.approx(1.0, abs=1e-15)
    # the edge of the support is I0(0)/I0(beta); the argument is 2s/S, not s/S
    assert orc.kernel_value("kb", beta, S, 4.0) == pytest.approx(1.0 / sp.i0(beta), rel=1e-12)
    assert orc.kernel_value("kb", beta, S, 2.0) == pytest.approx(
        sp.i0(beta * math.sqrt(0.75)) / sp.i0(beta), rel=1e-12)
    assert orc.kernel_value("kb", beta, S, 4.0 + 1e-9) == 0.0
    for s in np.linspace(0, 4, 17):
        assert orc.kernel_value("kb", beta, S, s) == orc.kernel_value("kb", beta, S, -s)


def test_gaussian_shape(orc):
    assert orc.kernel_value("gauss", GAUSS_SIGMA_S7, 7, 3.5) == pytest.approx(1e-3, rel=1e-12)
    assert orc.kernel_value("gauss", GAUSS_SIGMA_S7, 7, 0.0) == 1.0
    assert orc.kernel_value("gauss", GAUSS_SIGMA_S7, 7, 3.6) == 0.0


def test_gauss_legendre_matches_library(orc):
    for n in (1, 2, 3, 8, 32, 40):
        x, w = orc.gauss_legendre(n)
        xr, wr = np.polynomial.legendre.leggauss(n)
        order = np.argsort(x)
        np.testing.assert_allclose(x[order], xr, atol=1e-14)
        np.testing.assert_allclose(w[order], wr, atol=1e-14)


def test_gaussian_taper_closed_form(orc):
    """int_{-a}^{a} exp(-s^2/2s0^2) cos(w s) ds
       = s0 sqrt(pi/2) exp(-s0^2 w^2/2) Re[erf(z) + erf(conj z)], z = (a - i s0^2 w)/(s0 sqrt 2)."""
    N, S, sig = 256, 7, GAUSS_SIGMA_S7
    C = orc.taper("gauss", sig, S, N)
    a = S / 2.0
    for p in (0, 1, 37, 64, 127, 128, 129, 200, 255):
        om = 2 * math.pi * (p - N // 2) / N
        z = (a - 1j * sig * sig * om) / (sig * math.sqrt(2.0))
        ref = sig * math.sqrt(math.pi / 2) * math.exp(-sig * sig * om * om / 2) * \
            (sp.erf(z) + sp.erf(np.conj(z))).real
        assert C[p] == pytest.approx(ref, rel=1e-12, abs=1e-15)


def test_kaiser_bessel_taper_matches_adaptive_quadrature(orc):
    N, S, beta = 512, 8, KB_BETA_S8
    C = orc.taper("kb", beta, S, N)
    for p in (0, 100, 255, 256, 300, 511):
        nu = (p - N // 2) / N
        f = lambda s: sp.i0(beta * math.sqrt(max(0.0, 1 - (2 * s / S) ** 2))) / sp.i0(beta) \
            * math.cos(2 * math.pi * s * nu)
        ref, _ = integ.quad(f, -S / 2, S / 2, epsabs=1e-14, epsrel=1e-13, limit=200)
        assert C[p] == pytest.approx(ref, rel=1e-10, abs=1e-13)
    assert np.argmax(C) == N // 2


# ----------------------------------------------------------------------------
# FFT
# ----------------------------------------------------------------------------


@pytest.mark.parametrize("N", [2, 4, 8])
def test_ifft2_against_brute_force_dft(orc, N):
    g = np.random.default_rng(N)
    A = g.normal(size=(N, N)) + 1j * g.normal(size=(N, N))
    ref = np.zeros((N, N), complex)
    for q in range(N):
        for p in range(N):
            for j in range(N):
                for i in range(N):
                    ref[q, p] += A[j, i] * np.exp(2j * np.pi * (i * p + j * q) / N)
    np.testing.assert_allclose(orc.ifft2(A), ref, atol=1e-12 * N * N)


@pytest.mark.parametrize("N", [16, 64, 256])
def test_ifft2_against_library_and_parseval(orc, N):
    g = np.random.default_rng(N)
    A = g.normal(size=(N, N)) + 1j * g.normal(size=(N, N))
    F = orc.ifft2(A)
    np.testing.assert_allclose(F, np.fft.ifft2(A) * N * N, atol=1e-10 * N)
    assert (np.abs(F) ** 2).sum() == pytest.approx(N * N * (np.abs(A) ** 2).sum(), rel=1e-12)


def test_ifft2_rejects_non_power_of_two(orc):
    with pytest.raises(ValueError):
        orc.ifft2(np.zeros((6, 6)))


# ----------------------------------------------------------------------------
# placement: footprint (R3), planes (R4), drops, flags
# ----------------------------------------------------------------------------

def _one_vis_cfg(orc, N=64, Nw=4, S=7, w_range=100.0, fov=0.02):
    return orc.Config(N, Nw, S, "gauss", GAUSS_SIGMA_S7, fov, -w_range, w_range)


def test_plane_index_ties_and_clamping(orc):
    cfg = _one_vis_cfg(orc)                 # planes of width 50 on [-100, 100]
    ws = np.array([-100.0, -50.0, -50.000001, 0.0, 49.999, 50.0, 100.0, 250.0, -300.0])
    uvw = np.stack([np.zeros_like(ws), np.zeros_like(ws), ws], axis=1)
    pl = orc.place(cfg, uvw, [1.0], np.ones((len(ws), 1), np.float32))
    assert pl["k"][:, 0].tolist() == [0, 1, 0, 2, 2, 3, 3, 3, 0]
    assert orc.plane_w(cfg, 0) == -75.0 and orc.plane_w(cfg, 3) == 75.0


def test_footprint_start_and_offsets(orc):
    N, S, fov = 64, 7, 0.02
    cfg = _one_vis_cfg(orc, N=N, S=S, fov=fov)
    # x = u fov + N/2; choose x exactly 40.5 (x - S/2 = 37 is a whole cell)
    xs = np.array([40.5, 40.25, 40.75, 10.0])
    u = (xs - N / 2) / fov
    uvw = np.stack([u, np.zeros_like(u), np.zeros_like(u)], axis=1)
    pl = orc.place(cfg, uvw, [1.0], np.ones((4, 1), np.float32))
    # cells with x - S/2 < i <= x + S/2
    for t, x in enumerate(xs):
        cells = [i for i in range(N) if x - S / 2 < i <= x + S / 2]
        assert pl["i0"][t, 0] == cells[0] and len(cells) == S
        assert pl["fx"][t, 0] == pytest.approx((x - S / 2) - math.floor(x - S / 2), abs=1e-12)
    assert pl["j0"][0, 0] == N // 2 - 3


def test_off_grid_visibilities_are_dropped(orc):
    N, S, fov = 64, 7, 0.02
    cfg = _one_vis_cfg(orc, N=N, S=S, fov=fov)
    xs = np.array([2.4, 2.6, 60.4, 60.6, 32.0])   # first cell i0 = floor(x-3.5)+1; on grid iff 2.5 <= x < 60.5
    u = (xs - N / 2) / fov
    uvw = np.stack([u, np.zeros_like(u), np.zeros_like(u)], axis=1)
    pl = orc.place(cfg, uvw, [1.0], np.ones((5, 1), np.float32))
    assert pl["status"][:, 0].tolist() == [-1, 1, 1, -1, 1]
    ws, ng, nd = orc.channel_stats(cfg, uvw, [1.0], np.ones((5, 1), np.float32))
    assert (ws, ng, nd) == (3.0, 3, 2)


def test_flags_and_zero_weights_do_not_contribute(orc):
    img, obs = tiny_wstack(3, nvis=2000, N=64, fov_deg=2.0)
    cfg = cfg_of(orc, img)
    wt = obs.weight.copy()
    fl = np.zeros_like(wt, dtype=np.uint8)
    fl[::3] = 1
    wt[1::7] = 0.0
    keep = (fl[:, 0] == 0) & (wt[:, 0] != 0)
    I1, ws1 = orc.image(cfg, obs.uvw, obs.chan_scale, obs.vis, wt, fl)
    I2, ws2 = orc.image(cfg, obs.uvw[keep], obs.chan_scale, obs.vis[keep], wt[keep])
    assert ws1 == ws2 == keep.sum()
    np.testing.assert_allclose(I1, I2, atol=1e-13)


# ----------------------------------------------------------------------------
# the method: invariants and special cases
# ----------------------------------------------------------------------------

def test_unit_source_at_phase_centre(orc):
    """V = 1 is a unit source at l = m = 0 (n = 1).  The direct inversion gives
    exactly 1 at the centre pixel; the gridded image peaks there, at 1 up to
    the kernel's truncation error (g(3.5) = 1e-3, per axis < 2e-3)."""
    img, obs = tiny_wstack(1, nvis=3000, N=128)
    cfg = cfg_of(orc, img)
    vis = np.ones_like(obs.vis)
    N = img.N
    d = orc.dft_at(cfg, obs.uvw, obs.chan_scale, vis, obs.weight, p=[N // 2], q=[N // 2])
    assert d[0] == pytest.approx(1.0, abs=1e-14)
    I, _ = orc.image(cfg, obs.uvw, obs.chan_scale, vis, obs.weight)
    assert np.unravel_index(np.argmax(I.real), I.shape) == (N // 2, N // 2)
    assert abs(I[N // 2, N // 2].real - 1.0) < 4e-3
    assert abs(I[N // 2, N // 2].imag) < 1e-12


def test_hermitian_input_gives_real_image(orc):
    img, obs = tiny_wstack(2, nvis=2000, N=128)
    cfg = cfg_of(orc, img)
    uvw = np.concatenate([obs.uvw, -obs.uvw])
    vis = np.concatenate([obs.vis, np.conj(obs.vis)])
    wt = np.concatenate([obs.weight, obs.weight])
    I, _ = orc.image(cfg, uvw, obs.chan_scale, vis, wt)
    assert np.abs(I.imag).max() <= 1e-12 * np.abs(I.real).max()
    # and the plain half is genuinely complex, so the check has teeth
    I1, _ = orc.image(cfg, obs.uvw, obs.chan_scale, obs.vis, obs.weight)
    assert np.abs(I1.imag).max() > 1e-3 * np.abs(I1.real).max()


def test_linearity_in_the_visibilities(orc):
    img, obs = tiny_wstack(4, nvis=1500, N=64)
    cfg = cfg_of(orc, img)
    g = np.random.default_rng(0)
    # dyadic values keep a V1 + b V2 exact in complex64
    V1 = (g.integers(-64, 64, obs.vis.shape) + 1j * g.integers(-64, 64, obs.vis.shape)) / 8
    V2 = (g.integers(-64, 64, obs.vis.shape) + 1j * g.integers(-64, 64, obs.vis.shape)) / 8
    V1, V2 = V1.astype(np.complex64), V2.astype(np.complex64)
    a, b = 2.0, -0.5
    I1, _ = orc.image(cfg, obs.uvw, obs.chan_scale, V1, obs.weight)
    I2, _ = orc.image(cfg, obs.uvw, obs.chan_scale, V2, obs.weight)
    I3, _ = orc.image(cfg, obs.uvw, obs.chan_scale, (a * V1 + b * V2).astype(np.complex64),
                      obs.weight)
    np.testing.assert_allclose(I3, a * I1 + b * I2, atol=1e-12 * np.abs(I3).max())


def test_single_plane_without_w_is_plain_gridding_and_fft(orc):
    """Nw = 1, w = 0: the phase screen is 1 and the image is the textbook 2-D
    gridding + inverse FFT; the FFT inside the pipeline must equal numpy's."""
    img, obs = tiny_wstack(5, nvis=1500, N=64)
    cfg = cfg_of(orc, img, Nw=1, w_min=0.0, w_max=0.0)
    uvw = obs.uvw.copy()
    uvw[:, 2] = 0.0
    I, ws = orc.image(cfg, uvw, obs.chan_scale, obs.vis, obs.weight)
    G = orc.grid_plane(cfg, uvw, obs.chan_scale, obs.vis, obs.weight, plane=0)
    N = img.N
    F = np.fft.ifft2(G) * N * N
    Ct = orc.taper(img.kernel, img.kernel_param, img.S, N)
    p = np.arange(N)
    dl = img.fov / N
    l = (p - N // 2) * dl
    n = np.sqrt(1 - l[None, :] ** 2 - l[:, None] ** 2)
    sgn = (-1.0) ** (p[None, :] + p[:, None])
    ref = F * sgn * n / (ws * Ct[None, :] * Ct[:, None])
    np.testing.assert_allclose(I, ref, atol=1e-12 * np.abs(ref).max())


def test_fft_path_equals_per_visibility_path(orc):
    """Two formulations of O1: grid + FFT + phase, and the same sum taken
    visibility by visibility at each pixel.  They share only the placement."""
    img, obs = tiny_wstack(6, nvis=800, N=32, fov_deg=2.0)
    cfg = cfg_of(orc, img)
    I, _ = orc.image(cfg, obs.uvw, obs.chan_scale, obs.vis, obs.weight)
    q, p = np.meshgrid(np.arange(32), np.arange(32), indexing="ij")
    A = orc.image_at(cfg, obs.uvw, obs.chan_scale, obs.vis, obs.weight,
                     p=p.ravel(), q=q.ravel()).reshape(32, 32)
    np.testing.assert_allclose(I, A, atol=1e-12 * np.abs(I).max())
    # per-plane transform before the phase screen
    F3 = orc.ifft2(orc.grid_plane(cfg, obs.uvw, obs.chan_scale, obs.vis, obs.weight, plane=3))
    B = orc.image_at(cfg, obs.uvw, obs.chan_scale, obs.vis, obs.weight, p=p.ravel(), q=q.ravel(),
                     plane=3).reshape(32, 32)
    np.testing.assert_allclose(F3, B, atol=1e-12 * np.abs(F3).max())


def test_stage_functions_compose_to_the_image(orc):
    """The stages the CPU baseline times one by one -- grid_plane (Eq. 3),
    ifft2_inplace, phase_accumulate (Eq. 2's sum) and image_scale (Eq. 2's
    normalisation) -- compose to oracle.image exactly, and the image they give
    matches the per-visibility form (which shares none of the FFT and phase
    code)."""
    img, obs = tiny_wstack(16, nvis=900, N=32, fov_deg=2.0)
    cfg = cfg_of(orc, img)
    I, ws = orc.image(cfg, obs.uvw, obs.chan_scale, obs.vis, obs.weight)
    acc = np.zeros((32, 32), np.complex128)
    for k in range(img.Nw):
        F = orc.ifft2_inplace(orc.grid_plane(cfg, obs.uvw, obs.chan_scale, obs.vis, obs.weight, plane=k))
        orc.phase_accumulate(cfg, k, F, acc)
    orc.image_scale(cfg, ws, acc)
    np.testing.assert_array_equal(acc, I)
    q, p = np.meshgrid(np.arange(32), np.arange(32), indexing="ij")
    A = orc.image_at(cfg, obs.uvw, obs.chan_scale, obs.vis, obs.weight,
                     p=p.ravel(), q=q.ravel()).reshape(32, 32)
    np.testing.assert_allclose(acc, A, atol=1e-12 * np.abs(A).max())


# ----------------------------------------------------------------------------
# Hermitian fold
# ----------------------------------------------------------------------------

@pytest.mark.parametrize("N", [8, 16, 32])
def test_mirror_is_conjugation_under_the_inverse_dft(orc, N):
    """ifft2(conj(mirror(G))) = conj(ifft2(G)) for every G: the property the
    fold rests on, checked with numpy's FFT.  A mirror to N-1-i (or one that
    forgets the wrap of cell 0) fails it."""
    g = np.random.default_rng(N)
    G = g.standard_normal((N, N)) + 1j * g.standard_normal((N, N))
    np.testing.assert_allclose(np.fft.ifft2(np.conj(orc.mirror(G))), np.conj(np.fft.ifft2(G)),
                               atol=1e-14 * N)
    np.testing.assert_array_equal(orc.mirror(orc.mirror(G)), G)
    assert orc.mirror(G)[0, 0] == G[0, 0] and orc.mirror(G)[1, 2] == G[N - 1, N - 2]


@pytest.mark.parametrize("Nw", [1, 7, 8])
def test_mirrored_planes_sit_at_opposite_w(orc, Nw):
    img, _ = tiny_wstack(1, nvis=10, N=64)
    cfg = cfg_of(orc, img, Nw=Nw)
    for k in range(Nw):
        assert orc.plane_w(cfg, Nw - 1 - k) == pytest.approx(-orc.plane_w(cfg, k), abs=1e-12)


def _conjugate_upper_half(orc, cfg, obs):
    """The same data with every visibility of the upper planes replaced by
    its Hermitian partner V(-u,-v,-w) = conj V(u,v,w)."""
    pl = orc.place(cfg, obs.uvw, obs.chan_scale, obs.weight)
    up = (pl["k"][:, 0] * 2 > cfg.Nw - 1)
    uvw = obs.uvw.copy()
    uvw[up] *= -1.0
    vis = obs.vis.copy()
    vis[up] = np.conj(vis[up])
    return uvw, vis, up


@pytest.mark.parametrize("Nw", [7, 8])
def test_folded_planes_equal_gridding_of_the_hermitian_partners(orc, Nw):
    """H_k (the fold, written from its definition) against the oracle's own
    gridder run on the data with the upper-half visibilities replaced by their
    partners at (-u,-v,-w): the two agree up to the rounding of the mirrored
    positions, and the upper planes of the partner data are empty."""
    img, obs = tiny_wstack(21, nvis=3000, N=64, Nw=Nw)
    # keep every footprint off the mesh border: a footprint that starts on
    # cell 0 has a partner that ends on cell N, which the gridder drops while
    # the fold wraps it to cell 0 (both readings agree on the image grid,
    # see the mirror test above; here the gridder is the witness)
    obs.uvw[:, :2] *= 0.8
    cfg = cfg_of(orc, img)
    uvw, vis, up = _conjugate_upper_half(orc, cfg, obs)
    assert 0.3 < up.mean() < 0.7
    for k in range((Nw + 1) // 2):
        H = orc.fold_plane(cfg, obs.uvw, obs.chan_scale, obs.vis, obs.weight, plane=k)
        P = orc.grid_plane(cfg, uvw, obs.chan_scale, vis, obs.weight, plane=k)
        np.testing.assert_allclose(H, P, atol=1e-9 * np.abs(P).max())
    for k in range((Nw + 1) // 2, Nw):
        assert np.abs(orc.grid_plane(cfg, uvw, obs.chan_scale, vis, obs.weight, plane=k)).max() == 0.0
    with pytest.raises(ValueError):
        orc.fold_plane(cfg, obs.uvw, obs.chan_scale, obs.vis, obs.weight, plane=(Nw + 1) // 2)


def test_real_image_is_unchanged_by_hermitian_partners(orc):
    """Re of the dirty image is the same for the data and for the data with
    the upper half replaced by its partners (the fold's premise, on the whole
    path: gridding, inverse FFT, phase screen of the mirrored plane, taper and
    weights); the imaginary part is not, so the check has teeth."""
    img, obs = tiny_wstack(22, nvis=3000, N=64, Nw=8)
    obs.uvw[:, :2] *= 0.8  # footprints off the mesh border, as above
    cfg = cfg_of(orc, img)
    uvw, vis, _ = _conjugate_upper_half(orc, cfg, obs)
    I1, w1 = orc.image(cfg, obs.uvw, obs.chan_scale, obs.vis, obs.weight)
    I2, w2 = orc.image(cfg, uvw, obs.chan_scale, vis, obs.weight)
    assert w1 == w2
    np.testing.assert_allclose(I2.real, I1.real, atol=1e-9 * np.abs(I1.real).max())
    assert np.abs(I2.imag - I1.imag).max() > 1e-3 * np.abs(I1.real).max()


def _on_pixel_sources(img, n, seed, inner):
    """Point sources placed exactly on pixel centres inside |l|,|m| < inner fov/2."""
    g = np.random.default_rng(seed)
    N = img.N
    half = int(inner * N / 2)
    pq = g.integers(N // 2 - half, N // 2 + half, size=(n, 2))
    dl = img.fov / N
    lm = (pq - N // 2) * dl
    return pq, np.concatenate([lm, g.uniform(0.2, 1.0, (n, 1))], axis=1)


def test_gridded_image_matches_direct_inversion_within_method_error(orc):
    """O1 vs O2 (Eq. 1 inverted directly) at sources in the inner half of the
    field: the difference is the method's error -- truncation of the Gaussian
    (g = 1e-3 at the edge), aliasing (C(nu+1)/C(nu) < 2e-4 for |nu| < 1/4) and
    w quantisation (a = pi dw max|n-1| ~ 0.012 rad here, amplitude a^2/6).
    A swapped (u, v), a wrong sign or a wrong plane would be O(1)."""
    img, obs = tiny_wstack(7, nvis=20_000, N=256)
    pq, src = _on_pixel_sources(img, 6, 7, 0.5)
    vis = visgen.predict(obs.uvw, obs.chan_scale, src)
    cfg = cfg_of(orc, img)
    o1 = orc.image_at(cfg, obs.uvw, obs.chan_scale, vis, obs.weight, p=pq[:, 0], q=pq[:, 1])
    o2 = orc.dft_at(cfg, obs.uvw, obs.chan_scale, vis, obs.weight, p=pq[:, 0], q=pq[:, 1])
    peak = np.abs(o2).max()
    assert np.abs(o1 - o2).max() < 3e-3 * peak
    # the planes matter: the same image without w-stacking misses badly away from the centre
    cfg1 = cfg_of(orc, img, Nw=1)
    flat = orc.image_at(cfg1, obs.uvw, obs.chan_scale, vis, obs.weight, p=pq[:, 0], q=pq[:, 1])
    assert np.abs(flat - o2).max() > 3 * np.abs(o1 - o2).max()


def test_source_position_and_orientation(orc):
    """A single off-centre source at (l, m) with l != m appears at pixel
    (p, q) = (N/2 + l/dl, N/2 + m/dl) with its flux, not at the transposed
    or mirrored pixel."""
    img, obs = tiny_wstack(8, nvis=6000, N=128)
    N = img.N
    dl = img.fov / N
    p_s, q_s = N // 2 + 20, N // 2 - 9
    src = np.array([[(p_s - N // 2) * dl, (q_s - N // 2) * dl, 0.8]])
    vis = visgen.predict(obs.uvw, obs.chan_scale, src)
    I, _ = orc.image(cfg_of(orc, img), obs.uvw, obs.chan_scale, vis, obs.weight)
    assert np.unravel_index(np.argmax(I.real), I.shape) == (q_s, p_s)
    assert I[q_s, p_s].real == pytest.approx(0.8, rel=3e-3)


# ----------------------------------------------------------------------------
# learned-kernel network
# ----------------------------------------------------------------------------

def test_gelu_against_exact_form(orc):
    """tanh-form GELU vs x Phi(x): the tanh form's known error is below 1e-3."""
    for x in np.linspace(-6, 6, 121):
        assert abs(orc.gelu(x) - x * sp.ndtr(x)) < 1e-3
        h = 1e-6
        fd = (orc.gelu(x + h) - orc.gelu(x - h)) / (2 * h)
        assert orc.gelu_grad(x) == pytest.approx(fd, abs=1e-8)


def test_mlp_special_cases(orc):
    H = 8
    n = orc.mlp_param_count(H)
    assert n == H * 3 + H + H * H + H + 16 * H + 16
    prm = np.zeros(n)
    prm[-16:] = np.arange(16)                      # only b3 set: output is b3
    np.testing.assert_array_equal(orc.mlp_forward(prm, H, [0.3, 0.7, -1.0]), np.arange(16))
    # W1 = 0, b1 = 0 -> layer-1 activations gelu(0) = 0 -> out = W3 gelu(b2) + b3
    g = np.random.default_rng(1)
    prm = g.normal(size=n)
    o = 0
    prm[o:o + 3 * H] = 0; o += 3 * H
    prm[o:o + H] = 0; o += H
    o += H * H
    b2 = prm[o:o + H]; o += H
    W3 = prm[o:o + 16 * H].reshape(16, H); o += 16 * H
    b3 = prm[o:o + 16]
    ref = W3 @ np.array([orc.gelu(v) for v in b2]) + b3
    np.testing.assert_allclose(orc.mlp_forward(prm, H, [0.1, 0.2, 0.3]), ref, atol=1e-14)


def test_mlp_backward_matches_finite_differences(orc):
    H = 6
    g = np.random.default_rng(2)
    prm = g.normal(scale=0.7, size=orc.mlp_param_count(H))
    x = np.array([0.37, 0.81, -0.4])
    gout = g.normal(size=16)
    grad = orc.mlp_backward(prm, H, x, gout)
    h = 1e-6
    fd = np.zeros_like(prm)
    for i in range(prm.size):
        e = np.zeros_like(prm)
        e[i] = h
        fd[i] = (gout @ orc.mlp_forward(prm + e, H, x) - gout @ orc.mlp_forward(prm - e, H, x)) / (2 * h)
    np.testing.assert_allclose(grad, fd, atol=1e-7)


def test_learned_kernel_is_kaiser_bessel_plus_its_correction(orc):
    """With a network whose only non-zero parameter is b3 = e_t, every
    visibility adds W V (-1)^(i+j) on exactly footprint cell t on top of the
    support-4 Kaiser-Bessel grid; with an all-zero network the learned kernel
    is that Kaiser-Bessel."""
    H = 4
    n = orc.mlp_param_count(H)
    img, obs = tiny_wstack(9, nvis=50, N=64)
    kb = orc.Config(64, img.Nw, 4, "kb", KB_BETA_S4, img.fov, img.w_min, img.w_max)
    G_kb = sum(orc.grid_plane(kb, obs.uvw, obs.chan_scale, obs.vis, obs.weight, plane=k)
               for k in range(img.Nw))
    for t in (None, 0, 5, 15):
        prm = np.zeros(n)
        if t is not None:
            prm[n - 16 + t] = 1.0
        cfg = orc.Config(64, img.Nw, 4, "learned", KB_BETA_S4, img.fov, img.w_min, img.w_max,
                         mlp=prm, mlp_hidden=H)
        pl = orc.place(cfg, obs.uvw, obs.chan_scale, obs.weight)
        G = sum(orc.grid_plane(cfg, obs.uvw, obs.chan_scale, obs.vis, obs.weight, plane=k)
                for k in range(img.Nw))
        ref = G_kb.copy()
        for r in range(50):
            if t is None or pl["status"][r, 0] != 1:
                continue
            i = pl["i0"][r, 0] + t % 4
            j = pl["j0"][r, 0] + t // 4
            ref[j, i] += obs.weight[r, 0] * complex(obs.vis[r, 0]) * (-1) ** (i + j)
        np.testing.assert_allclose(G, ref, atol=1e-12)

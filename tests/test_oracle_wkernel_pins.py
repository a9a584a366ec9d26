"""Pins of the oracle's w-direction kernel (improved w-stacking, R14).

Eq. 3 writes the gridding kernel G as a function of (u, v, w); the plain method
puts each visibility on its closest plane (R4).  With a w-kernel of support Sw
each visibility is spread over Sw planes with Kaiser-Bessel weights g_w(k - z)
(z the continuous plane coordinate), the planes extend Sw/2 beyond the w range at
each end, and the image is divided by the kernel's transform C_w((n - 1) dw) as
well as by C(l) C(m).  Each test names what a mistake would have to get wrong.
"""
import math

import numpy as np
import pytest
import scipy.special as sp

from visgen.workloads import tiny_wstack


def cfg_of(orc, img, **kw):
    d = dict(N=img.N, Nw=img.Nw, S=img.S, kernel=img.kernel, kernel_param=img.kernel_param,
             fov=img.fov, w_min=img.w_min, w_max=img.w_max)
    d.update(kw)
    return orc.Config(**d)


@pytest.mark.parametrize("S,beta", [(4, 5.62), (6, 8.0), (8, 12.25)])
def test_kernel_transform_matches_the_kaiser_bessel_closed_form(orc, S, beta):
    """C(nu) = S sinh(sqrt(beta^2 - (pi S nu)^2)) / (sqrt(...) I0(beta)), and
    sin(...) beyond the first zero: pins the quadrature that gives the w-taper
    (a wrong scale of nu, a missing factor 2 or a wrong support fails)."""
    for nu in np.linspace(0.0, 0.9, 37):
        x2 = beta ** 2 - (math.pi * S * nu) ** 2
        if abs(x2) < 1e-9:
            ref = S / sp.i0(beta)
        elif x2 > 0:
            r = math.sqrt(x2)
            ref = S * math.sinh(r) / (r * sp.i0(beta))
        else:
            r = math.sqrt(-x2)
            ref = S * math.sin(r) / (r * sp.i0(beta))
        got = orc.kernel_ft("kb", beta, S, nu)
        assert got == pytest.approx(ref, rel=1e-10, abs=1e-13 * S)


def test_taper_is_the_transform_at_pixel_frequencies(orc):
    N, S, beta = 64, 8, 12.25
    C = orc.taper("kb", beta, S, N)
    for p in range(N):
        assert C[p] == pytest.approx(orc.kernel_ft("kb", beta, S, (p - N / 2) / N), rel=1e-12)


def test_planes_extend_by_half_the_support_at_each_end(orc):
    img, _ = tiny_wstack(61, nvis=10, N=64, Nw=8, w_range=400.0)
    cfg = cfg_of(orc, img, w_support=4, w_kernel_param=8.0)
    assert orc.planes_total(cfg) == 12
    dw = 800.0 / 8
    for k in range(12):
        assert orc.plane_w(cfg, k) == pytest.approx(-400.0 + (k - 2 + 0.5) * dw, abs=1e-9)
    assert orc.planes_total(cfg_of(orc, img)) == 8


def test_a_visibility_spreads_over_its_sw_planes_with_the_kernel_weights(orc):
    """One visibility gridded with a w-kernel: plane k holds the plane-k weight
    g_w(k - z) times the single-plane grid, for the Sw planes from the placement
    and nowhere else (an off-by-one in the w footprint fails)."""
    img, obs = tiny_wstack(62, nvis=1, N=64, Nw=8, w_range=400.0)
    Sw, bw = 4, 8.0
    cfg = cfg_of(orc, img, w_support=Sw, w_kernel_param=bw)
    plain = cfg_of(orc, img)
    for w in (-399.0, -123.4, 0.0, 37.5, 250.0, 399.9):
        uvw = obs.uvw.copy()
        uvw[0, 2] = w
        pl = orc.place(cfg, uvw, obs.chan_scale, obs.weight)
        k0, fw = int(pl["k"][0, 0]), float(pl["fw"][0, 0])
        z = (w + 400.0) / 100.0 - 0.5
        assert k0 == math.floor(z - Sw / 2) + 1 + Sw // 2
        G0 = orc.grid_plane(plain, uvw, obs.chan_scale, obs.vis, obs.weight,
                            plane=int(orc.place(plain, uvw, obs.chan_scale, obs.weight)["k"][0, 0]))
        for k in range(orc.planes_total(cfg)):
            G = orc.grid_plane(cfg, uvw, obs.chan_scale, obs.vis, obs.weight, plane=k)
            s = k - k0
            wgt = orc.kernel_value("kb", bw, Sw, s + 1 - Sw / 2 - fw) if 0 <= s < Sw else 0.0
            np.testing.assert_allclose(G, wgt * G0, atol=1e-13)


def _sources(N, n, seed, inner):
    g = np.random.default_rng(seed)
    half = int(inner * N / 2)
    return g.integers(N // 2 - half, N // 2 + half, size=(n, 2)), g.uniform(0.3, 1.0, n)


def test_w_kernel_cuts_the_w_error_against_eq1(orc):
    """The method's error against Eq. 1 inverted directly, at sources across the
    field, with the same planes: a large w range (+-3000 lambda, 8 planes, the
    residual phase of the closest plane up to pi dw max|n-1| ~ 0.7 rad at the
    corners) makes the closest-plane error dominant; the Kaiser-Bessel w-kernel
    must reduce it by an order of magnitude (what is left, ~8e-4, is the uv
    kernel's aliasing at sources near the edge: the same for every w-kernel);
    the median error falls from the closest plane to Sw = 2 to Sw = 4.  A
    w-taper that divides by the wrong function, or plane centres off by one,
    makes the kernel worse, not better."""
    import visgen
    img, obs = tiny_wstack(63, nvis=20_000, N=256, Nw=8, w_range=3000.0)
    pq, flux = _sources(img.N, 8, 63, 0.9)
    dl = img.fov / img.N
    src = np.concatenate([(pq - img.N // 2) * dl, flux[:, None]], axis=1)
    vis = visgen.predict(obs.uvw, obs.chan_scale, src)
    p, q = pq[:, 0], pq[:, 1]
    D = orc.dft_at(cfg_of(orc, img), obs.uvw, obs.chan_scale, vis, obs.weight, p=p, q=q).real
    errs, med = {}, {}
    for name, kw in (("closest", {}), ("kb2", dict(w_support=2, w_kernel_param=4.0)),
                     ("kb4", dict(w_support=4, w_kernel_param=8.0))):
        I = orc.image_at(cfg_of(orc, img, **kw), obs.uvw, obs.chan_scale, vis, obs.weight,
                         p=p, q=q).real
        e = np.abs(I - D) / np.abs(D).max()
        errs[name], med[name] = float(e.max()), float(np.median(e))
    print(errs, med)
    assert errs["kb4"] < errs["closest"] / 10
    assert med["kb4"] < med["kb2"] < med["closest"]


@pytest.mark.parametrize("Sw", [2, 4])
def test_w_kernel_keeps_prediction_the_adjoint_of_imaging(orc, Sw):
    img, obs = tiny_wstack(64, nvis=1500, N=64, fov_deg=2.0, w_range=1000.0)
    cfg = cfg_of(orc, img, w_support=Sw, w_kernel_param=6.0)
    g = np.random.default_rng(64)
    V = (g.standard_normal(obs.vis.shape) + 1j * g.standard_normal(obs.vis.shape)).astype(np.complex64)
    W = (0.5 + g.random(obs.weight.shape)).astype(np.float32)
    N = img.N
    J = np.zeros((N, N))
    J[N // 4:3 * N // 4, N // 4:3 * N // 4] = g.standard_normal((N // 2, N // 2))
    I, ws = orc.image(cfg, obs.uvw, obs.chan_scale, V, W)
    P = orc.predict(cfg, obs.uvw, obs.chan_scale, W, image=J)
    lhs = np.sum(W[:, 0].astype(np.float64) * V[:, 0].astype(np.complex128) * np.conj(P))
    l = (np.arange(N) - N // 2) * img.fov / N
    n2 = 1.0 - l[None, :] ** 2 - l[:, None] ** 2
    rhs = ws * np.sum(J * I / n2)
    assert abs(lhs - rhs) <= 1e-10 * abs(rhs)


def test_w_kernel_hermitian_partner_predicts_the_conjugate(orc):
    """With a symmetric w range the extended plane set is symmetric too, so the
    partner at -w uses the mirrored planes with the same weights: the basis of
    the Hermitian fold with a w-kernel."""
    img, obs = tiny_wstack(65, nvis=1200, N=64, Nw=7, fov_deg=2.0, w_range=800.0)
    obs.uvw[:, :2] *= 0.8
    cfg = cfg_of(orc, img, w_support=4, w_kernel_param=8.0)
    g = np.random.default_rng(65)
    J = g.standard_normal((img.N, img.N))
    A = orc.predict(cfg, obs.uvw, obs.chan_scale, obs.weight, image=J)
    B = orc.predict(cfg, -obs.uvw, obs.chan_scale, obs.weight, image=J)
    np.testing.assert_allclose(B, np.conj(A), atol=1e-9 * np.abs(A).max())


def test_w_kernel_real_image_is_unchanged_by_hermitian_partners(orc):
    """Every visibility replaced by its partner conj V at (-u, -v, -w): with a
    w range symmetric about 0 the extended plane set, the w-kernel weights and
    the w-taper are symmetric too, so the real image stays (to rounding of the
    mirrored positions) while the imaginary part flips.  Plane centres off by
    one in the extended set, or an odd taper, break it."""
    img, obs = tiny_wstack(66, nvis=3000, N=64, Nw=8, w_range=800.0)
    obs.uvw[:, :2] *= 0.8   # footprints off the mesh border
    cfg = cfg_of(orc, img, w_support=4, w_kernel_param=8.0)
    I1, w1 = orc.image(cfg, obs.uvw, obs.chan_scale, obs.vis, obs.weight)
    I2, w2 = orc.image(cfg, -obs.uvw, obs.chan_scale, np.conj(obs.vis), obs.weight)
    assert w1 == w2
    np.testing.assert_allclose(I2.real, I1.real, atol=1e-9 * np.abs(I1.real).max())
    np.testing.assert_allclose(I2.imag, -I1.imag, atol=1e-9 * np.abs(I1.real).max())
    assert np.abs(I1.imag).max() > 1e-3 * np.abs(I1.real).max()


@pytest.mark.parametrize("Nw", [7, 8])
def test_w_kernel_fold_planes_add_the_partner_planes(orc, Nw):
    """The fold over the extended plane set (Nt = Nw + Sw planes): stored
    plane H_k equals the grid of the data plus the grid of the partner data on
    plane k (the partner's records on plane k are the mirrored conjugates of
    the data's records on plane Nt - 1 - k), for 2k < Nt - 1; the middle plane
    of an odd Nt keeps the data's grid alone."""
    img, obs = tiny_wstack(67, nvis=1500, N=64, Nw=Nw, w_range=800.0)
    obs.uvw[:, :2] *= 0.8
    cfg = cfg_of(orc, img, w_support=4, w_kernel_param=8.0)
    nt = orc.planes_total(cfg)
    assert nt == Nw + 4
    pu, pv = -obs.uvw, np.conj(obs.vis)
    for k in range((nt + 1) // 2):
        H = orc.fold_plane(cfg, obs.uvw, obs.chan_scale, obs.vis, obs.weight, plane=k)
        G = orc.grid_plane(cfg, obs.uvw, obs.chan_scale, obs.vis, obs.weight, plane=k)
        if 2 * k == nt - 1:
            np.testing.assert_array_equal(H, G)
            continue
        P = orc.grid_plane(cfg, pu, obs.chan_scale, pv, obs.weight, plane=k)
        np.testing.assert_allclose(H, G + P, atol=1e-9 * np.abs(G + P).max())
    with pytest.raises(ValueError):
        orc.fold_plane(cfg, obs.uvw, obs.chan_scale, obs.vis, obs.weight, plane=(nt + 1) // 2)

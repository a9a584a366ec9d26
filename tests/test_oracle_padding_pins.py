"""Pins of the oracle's padded mesh (reading R16, an extension: the paper's
mesh is the image size, Sec. 2).  With Ng = alpha N cells of 1/(alpha FoV) the
image is the central N x N of the Ng x Ng inverse DFT, divided by the taper
evaluated at (p - N/2)/Ng.  Each test names what a mistake would break.
"""
import numpy as np
import pytest

from visgen.workloads import tiny_wstack


def cfg_of(orc, img, **kw):
    d = dict(N=img.N, Nw=img.Nw, S=img.S, kernel=img.kernel, kernel_param=img.kernel_param,
             fov=img.fov, w_min=img.w_min, w_max=img.w_max)
    d.update(kw)
    return orc.Config(**d)


def test_padded_taper_is_the_transform_at_the_padded_frequencies(orc):
    N, Ng, S, beta = 64, 256, 8, 12.25
    C = orc.taper("kb", beta, S, N, Ng)
    for p in range(0, N, 7):
        assert C[p] == pytest.approx(orc.kernel_ft("kb", beta, S, (p - N / 2) / Ng), rel=1e-12)


@pytest.mark.parametrize("alpha", [2, 4])
def test_single_visibility_images_to_the_plane_wave_of_its_cell(orc, alpha):
    """One visibility, a one-tap Gaussian kernel (S = 1), four planes: the
    image is the plane wave of the cell it lands on,
      n V g(i0 - x) g(j0 - y) / (C(p) C(q)) exp(2 pi i [(i0 - Ng/2)(p - N/2)
        + (j0 - Ng/2)(q - N/2)] / Ng) exp(2 pi i w_k (n - 1)),
    i.e. u_cell l + v_cell m with du = 1/(alpha FoV), dl = FoV/N.  A wrong cell
    size, a wrong crop offset or a taper at the unpadded frequencies fails."""
    img, obs = tiny_wstack(111, nvis=1, N=64, Nw=4, fov_deg=2.0, w_range=300.0)
    N, Ng = img.N, alpha * img.N
    sigma = 0.4
    cfg = cfg_of(orc, img, S=1, kernel="gauss", kernel_param=sigma, Ng=Ng)
    obs.uvw[0] = [17.3 / img.fov, -11.8 / img.fov, 123.0]   # cells from the centre
    V = np.array([[0.7 - 0.4j]], np.complex64)
    W = np.array([[1.5]], np.float32)
    I, ws = orc.image(cfg, obs.uvw, obs.chan_scale, V, W)
    x = obs.uvw[0, 0] * obs.chan_scale[0] * img.fov * alpha + Ng / 2
    y = obs.uvw[0, 1] * obs.chan_scale[0] * img.fov * alpha + Ng / 2
    i0, j0 = int(np.floor(x - 0.5)) + 1, int(np.floor(y - 0.5)) + 1
    g = lambda s: np.exp(-s * s / (2 * sigma * sigma))
    k = int(np.clip(np.floor((obs.uvw[0, 2] * obs.chan_scale[0] - img.w_min) * img.Nw /
                             (img.w_max - img.w_min)), 0, img.Nw - 1))
    wk = img.w_min + (k + 0.5) * (img.w_max - img.w_min) / img.Nw
    p = np.arange(N)
    l = (p - N // 2) * img.fov / N
    L, M = np.meshgrid(l, l)
    n = np.sqrt(1 - L ** 2 - M ** 2)
    d = -(L ** 2 + M ** 2) / (1 + n)
    Cp = orc.taper("gauss", sigma, 1, N, Ng)
    ph = ((i0 - Ng // 2) * (p[None, :] - N // 2) + (j0 - Ng // 2) * (p[:, None] - N // 2)) % Ng
    ref = (n * complex(V[0, 0]) * g(i0 - x) * g(j0 - y) / np.outer(Cp, Cp)
           * np.exp(2j * np.pi * ph / Ng) * np.exp(2j * np.pi * wk * d))
    assert ws == pytest.approx(1.5)
    np.testing.assert_allclose(I, ref, atol=1e-12 * np.abs(ref).max())


@pytest.mark.parametrize("alpha", [2, 4])
def test_fft_forms_equal_per_pixel_forms_when_padded(orc, alpha):
    """image (planes, padded inverse DFT, crop) against image_at (the same
    value summed per visibility), and predict against predict_at: they share
    only placement and taper, so a crop offset applied on one side only, or
    an exponent reduced mod N instead of mod Ng, fails."""
    img, obs = tiny_wstack(112, nvis=1500, N=64, fov_deg=2.0, w_range=400.0)
    cfg = cfg_of(orc, img, Ng=alpha * img.N)
    I, _ = orc.image(cfg, obs.uvw, obs.chan_scale, obs.vis, obs.weight)
    g = np.random.default_rng(112)
    p, q = g.integers(0, img.N, 12), g.integers(0, img.N, 12)
    A = orc.image_at(cfg, obs.uvw, obs.chan_scale, obs.vis, obs.weight, p=p, q=q)
    np.testing.assert_allclose(I[q, p], A, atol=1e-10 * np.abs(I).max())
    pq = np.stack([g.integers(img.N // 4, 3 * img.N // 4, 5), g.integers(img.N // 4, 3 * img.N // 4, 5)], 1)
    flux = g.uniform(0.2, 1.0, 5)
    J = np.zeros((img.N, img.N))
    np.add.at(J, (pq[:, 1], pq[:, 0]), flux)
    P1 = orc.predict(cfg, obs.uvw, obs.chan_scale, obs.weight, image=J)
    P2 = orc.predict_at(cfg, obs.uvw, obs.chan_scale, obs.weight, p=pq[:, 0], q=pq[:, 1], flux=flux)
    np.testing.assert_allclose(P1, P2, atol=1e-10 * np.abs(P2).max())


def test_padded_prediction_is_the_adjoint_of_padded_imaging(orc):
    img, obs = tiny_wstack(113, nvis=1500, N=64, fov_deg=2.0)
    cfg = cfg_of(orc, img, S=8, kernel="kb", kernel_param=12.25, Ng=128)
    g = np.random.default_rng(113)
    V = (g.standard_normal(obs.vis.shape) + 1j * g.standard_normal(obs.vis.shape)).astype(np.complex64)
    W = (0.5 + g.random(obs.weight.shape)).astype(np.float32)
    N = img.N
    J = g.standard_normal((N, N))
    I, ws = orc.image(cfg, obs.uvw, obs.chan_scale, V, W)
    P = orc.predict(cfg, obs.uvw, obs.chan_scale, W, image=J)
    lhs = np.sum(W[:, 0].astype(np.float64) * V[:, 0].astype(np.complex128) * np.conj(P))
    l = (np.arange(N) - N // 2) * img.fov / N
    n2 = 1.0 - l[None, :] ** 2 - l[:, None] ** 2
    rhs = ws * np.sum(J * I / n2)
    assert abs(lhs - rhs) <= 1e-10 * abs(rhs)


def test_padding_cuts_the_aliasing_error_at_the_field_edge(orc):
    """Against Eq. 1 inverted directly at sources near the edge of the field,
    where the unpadded taper is small and aliased power is amplified most:
    padding by 2 reduces the error many times (the w range is tiny, so the
    remaining error is not the planes')."""
    import visgen
    img, obs = tiny_wstack(114, nvis=20_000, N=128, Nw=8, fov_deg=2.0, w_range=2.0)
    img = img.with_(S=8, kernel="kb", kernel_param=12.25)
    g = np.random.default_rng(114)
    N = img.N
    edge = np.concatenate([g.integers(4, 14, (4, 2)), g.integers(N - 14, N - 4, (4, 2))])
    dl = img.fov / N
    src = np.concatenate([(edge - N // 2) * dl, g.uniform(0.3, 1.0, (8, 1))], axis=1)
    vis = visgen.predict(obs.uvw, obs.chan_scale, src)
    p, q = edge[:, 0], edge[:, 1]
    D = orc.dft_at(cfg_of(orc, img), obs.uvw, obs.chan_scale, vis, obs.weight, p=p, q=q).real
    err = {}
    for a in (1, 2):
        I = orc.image_at(cfg_of(orc, img, Ng=a * N), obs.uvw, obs.chan_scale, vis, obs.weight,
                         p=p, q=q).real
        err[a] = float(np.abs(I - D).max() / np.abs(D).max())
    print(err)
    assert err[2] < err[1] / 20


def test_weighting_density_does_not_depend_on_padding(orc):
    img, obs = tiny_wstack(115, nvis=4000, N=64, fov_deg=2.0)
    obs.uvw[:, :2] *= 0.6
    base = cfg_of(orc, img, weighting="uniform")
    A = orc.imaging_weights(base, obs.uvw, obs.chan_scale, obs.weight)
    B = orc.imaging_weights(cfg_of(orc, img, weighting="uniform", Ng=256), obs.uvw,
                            obs.chan_scale, obs.weight)
    np.testing.assert_array_equal(A, B)
    assert np.any(A != obs.weight)

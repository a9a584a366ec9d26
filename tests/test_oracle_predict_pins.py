"""Pins of the oracle's prediction (degridding): model image -> visibilities.

The paper images only (Sec. 2); prediction is the other direction of the same
statement of the problem (Eq. 1 discretised on the pixels, and its w-stacking
form with the readings of the imaging path).  Each test names what a mistake
in the oracle would have to get wrong to slip past it.
"""
import numpy as np
import pytest

from visgen.workloads import tiny_wstack


def cfg_of(orc, img, **kw):
    d = dict(N=img.N, Nw=img.Nw, S=img.S, kernel=img.kernel, kernel_param=img.kernel_param,
             fov=img.fov, w_min=img.w_min, w_max=img.w_max)
    d.update(kw)
    return orc.Config(**d)


def _point_model(N, n, seed, inner=0.5):
    g = np.random.default_rng(seed)
    half = int(inner * N / 2)
    pq = g.integers(N // 2 - half, N // 2 + half, size=(n, 2))
    flux = g.uniform(0.2, 1.0, n)
    J = np.zeros((N, N))
    np.add.at(J, (pq[:, 1], pq[:, 0]), flux)
    return pq, flux, J


def test_fft_form_equals_per_visibility_form(orc):
    """oracle.predict (planes, forward DFT, gather) against oracle.predict_at
    (the same sum written per visibility and per source, no FFT): they share
    only the placement and the taper, so a wrong FFT direction, centring sign
    or transposed plane fails here."""
    img, obs = tiny_wstack(41, nvis=1500, N=64, fov_deg=2.0)
    cfg = cfg_of(orc, img)
    pq, flux, J = _point_model(img.N, 4, 41)
    A = orc.predict(cfg, obs.uvw, obs.chan_scale, obs.weight, image=J)
    B = orc.predict_at(cfg, obs.uvw, obs.chan_scale, obs.weight, p=pq[:, 0], q=pq[:, 1], flux=flux)
    np.testing.assert_allclose(A, B, atol=1e-10 * np.abs(B).max())
    assert np.abs(A).max() > 0.1


@pytest.mark.parametrize("kernel", ["gauss", "kb"])
def test_prediction_is_the_adjoint_of_imaging(orc, kernel):
    """sum_v W V conj(pred(J)) = sum W * sum_p J(p) I(V)(p) / n(p)^2 for any
    visibilities V and real image J, with I the oracle's complex dirty image:
    pins every convention of the prediction (phase-screen sign, FFT direction,
    checkerboard, taper, 1/n, plane choice, footprint) against the pinned
    imaging path."""
    img, obs = tiny_wstack(42, nvis=2000, N=64, fov_deg=2.0)
    if kernel == "kb":
        img = img.with_(S=8, kernel="kb", kernel_param=12.25)
    cfg = cfg_of(orc, img)
    g = np.random.default_rng(42)
    V = (g.standard_normal(obs.vis.shape) + 1j * g.standard_normal(obs.vis.shape)).astype(np.complex64)
    W = (0.5 + g.random(obs.weight.shape)).astype(np.float32)
    J = g.standard_normal((img.N, img.N))
    # the model lives in the inner half of the field: at the edges the taper
    # division amplifies FP64 rounding by up to ~5e9 (Kaiser-Bessel, beta 12.25)
    N = img.N
    J[:N // 4] = J[3 * N // 4:] = 0.0
    J[:, :N // 4] = J[:, 3 * N // 4:] = 0.0
    I, ws = orc.image(cfg, obs.uvw, obs.chan_scale, V, W)
    P = orc.predict(cfg, obs.uvw, obs.chan_scale, W, image=J)
    lhs = np.sum(W[:, 0].astype(np.float64) * V[:, 0].astype(np.complex128) * np.conj(P))
    l = (np.arange(N) - N // 2) * img.fov / N
    n2 = 1.0 - l[None, :] ** 2 - l[:, None] ** 2
    rhs = ws * np.sum(J * I / n2)
    assert abs(lhs - rhs) <= 1e-10 * abs(rhs)
    assert abs(rhs) > 1e-3


def test_unit_source_at_the_phase_centre_predicts_its_flux(orc):
    """J = A at (N/2, N/2): Eq. 1 gives V = A for every (u, v, w); the
    w-stacking prediction differs only by the kernel's discrete-vs-continuous
    sum (aliasing of the truncated Gaussian, about 1e-3)."""
    img, obs = tiny_wstack(43, nvis=800, N=64, fov_deg=2.0)
    cfg = cfg_of(orc, img)
    J = np.zeros((img.N, img.N))
    J[img.N // 2, img.N // 2] = 0.75
    P = orc.predict(cfg, obs.uvw, obs.chan_scale, obs.weight, image=J)
    assert np.abs(P / 0.75 - 1.0).max() < 3e-3
    D = orc.predict_dft(cfg, obs.uvw, obs.chan_scale, obs.weight, p=[img.N // 2], q=[img.N // 2],
                        flux=[0.75])
    np.testing.assert_allclose(D, 0.75, atol=1e-14)


def test_hermitian_partner_predicts_the_conjugate(orc):
    """A real image has V(-u, -v, -w) = conj V(u, v, w); with a symmetric w
    range the partner lands on the mirrored plane at the mirrored cells, and
    the w-stacking prediction keeps the identity to rounding.  A wrong
    phase-screen sign or plane centre breaks it."""
    img, obs = tiny_wstack(44, nvis=1200, N=64, Nw=7, fov_deg=2.0)
    obs.uvw[:, :2] *= 0.8   # footprints off the mesh border
    cfg = cfg_of(orc, img)
    g = np.random.default_rng(44)
    J = g.standard_normal((img.N, img.N))
    A = orc.predict(cfg, obs.uvw, obs.chan_scale, obs.weight, image=J)
    B = orc.predict(cfg, -obs.uvw, obs.chan_scale, obs.weight, image=J)
    np.testing.assert_allclose(B, np.conj(A), atol=1e-9 * np.abs(A).max())


def test_prediction_matches_eq1_within_the_method_error(orc):
    """O1 against O2 (Eq. 1 summed directly) for sources in the inner half of
    the field: the difference is the method's error (kernel aliasing and w
    quantisation, a = pi dw max|n-1| ~ 0.05 rad here); a swapped (u, v), a
    wrong sign or a wrong plane would be O(1).  Without w-stacking (one plane)
    the error is much larger."""
    img, obs = tiny_wstack(45, nvis=4000, N=256)
    cfg = cfg_of(orc, img)
    pq, flux, J = _point_model(img.N, 6, 45)
    P = orc.predict_at(cfg, obs.uvw, obs.chan_scale, obs.weight, p=pq[:, 0], q=pq[:, 1], flux=flux)
    D = orc.predict_dft(cfg, obs.uvw, obs.chan_scale, obs.weight, p=pq[:, 0], q=pq[:, 1], flux=flux)
    scale = np.abs(D).max()
    err = np.abs(P - D).max() / scale
    assert err < 5e-3
    flat = orc.predict_at(cfg_of(orc, img, Nw=1), obs.uvw, obs.chan_scale, obs.weight,
                          p=pq[:, 0], q=pq[:, 1], flux=flux)
    assert np.abs(flat - D).max() / scale > 3 * err


def test_prediction_is_linear_and_skips_what_imaging_skips(orc):
    img, obs = tiny_wstack(46, nvis=600, N=64, fov_deg=2.0)
    cfg = cfg_of(orc, img)
    g = np.random.default_rng(46)
    J1, J2 = g.standard_normal((2, img.N, img.N))
    flag = np.zeros_like(obs.weight, dtype=np.uint8)
    flag[::7] = 1
    W = obs.weight.copy()
    W[3::11] = 0.0
    uvw = obs.uvw.copy()
    uvw[5::13, 0] += 10 * img.N / img.fov   # off the grid
    P1 = orc.predict(cfg, uvw, obs.chan_scale, W, flag, image=J1)
    P2 = orc.predict(cfg, uvw, obs.chan_scale, W, flag, image=J2)
    P3 = orc.predict(cfg, uvw, obs.chan_scale, W, flag, image=2 * J1 - 0.5 * J2)
    np.testing.assert_allclose(P3, 2 * P1 - 0.5 * P2, atol=1e-12 * np.abs(P3).max())
    st = orc.place(cfg, uvw, obs.chan_scale, W, flag)["status"][:, 0]
    assert np.all(P1[st != 1] == 0) and np.all(P1[st == 1] != 0)
    assert (st == 0).sum() > 0 and (st == -1).sum() > 0

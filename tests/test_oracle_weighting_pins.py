"""Pins of the oracle's imaging weights (reading R15: uniform and Briggs
weighting, an extension; the paper uses natural weighting, Sec. 4.1.1).

The density D of a channel sums the weights of its gridded visibilities on
their nearest mesh cell and on the cell of their Hermitian partner; uniform
weighting divides by D, Briggs by 1 + f^2 D.  The pins are closed forms and
limits of that definition, each naming the mistake it catches.
"""
import numpy as np
import pytest

from visgen.workloads import meerkat, tiny_wstack


def cfg_of(orc, img, **kw):
    d = dict(N=img.N, Nw=img.Nw, S=img.S, kernel=img.kernel, kernel_param=img.kernel_param,
             fov=img.fov, w_min=img.w_min, w_max=img.w_max)
    d.update(kw)
    return orc.Config(**d)


def _cells(orc, cfg, obs, c=0):
    """Nearest cell of every visibility of channel c from the oracle's
    placement (x = i0 - 1 + S/2 + fx), -1 where not gridded."""
    pl = orc.place(cfg, obs.uvw, obs.chan_scale, obs.weight, obs.flag)
    st = pl["status"][:, c]
    x = pl["i0"][:, c] - 1 + cfg.S / 2 + pl["fx"][:, c]
    y = pl["j0"][:, c] - 1 + cfg.S / 2 + pl["fy"][:, c]
    i, j = np.floor(x + 0.5).astype(np.int64), np.floor(y + 0.5).astype(np.int64)
    N = cfg.N
    return np.where(st == 1, j * N + i, -1), np.where(st == 1, ((N - j) % N) * N + (N - i) % N, -1), st


@pytest.fixture(scope="module")
def data():
    img, obs = meerkat(91, n_ant=16, n_steps=60, nchan=2, N=256, Nw=4, n_src=5)
    g = np.random.default_rng(91)
    obs.weight = (0.2 + g.random(obs.weight.shape)).astype(np.float32)   # unequal weights
    obs.flag = np.zeros_like(obs.weight, dtype=np.uint8)
    obs.flag[::13] = 1
    obs.weight[3::29] = 0.0
    return img, obs


def test_natural_weights_are_the_data_weights(orc, data):
    img, obs = data
    W = orc.imaging_weights(cfg_of(orc, img), obs.uvw, obs.chan_scale, obs.weight, obs.flag)
    np.testing.assert_array_equal(W, obs.weight.astype(np.float64))


def test_uniform_weights_sum_to_one_per_occupied_cell(orc, data):
    """Over the Hermitian-completed set (every gridded visibility at its cell
    and its partner at the mirrored cell), the uniform weights in each
    occupied cell add up to 1: D is exactly the sum they are divided by.  A
    missing mirror, a wrong cell rounding or a density that counts skipped
    visibilities breaks it."""
    img, obs = data
    cfg = cfg_of(orc, img, weighting="uniform")
    W = orc.imaging_weights(cfg, obs.uvw, obs.chan_scale, obs.weight, obs.flag)
    for c in range(2):
        cell, mcell, st = _cells(orc, cfg, obs, c)
        ok = st == 1
        tot = np.zeros(img.N * img.N)
        np.add.at(tot, cell[ok], W[ok, c])
        np.add.at(tot, mcell[ok], W[ok, c])
        occ = tot != 0
        assert occ.sum() > 100
        np.testing.assert_allclose(tot[occ], 1.0, rtol=1e-12)
        # skipped visibilities keep their weight (and do not count in D)
        np.testing.assert_array_equal(W[~ok, c], obs.weight[~ok, c].astype(np.float64))
        assert (st == -1).sum() + (st == 0).sum() > 0


def test_uniform_is_scale_invariant_and_briggs_scale_equivariant(orc, data):
    img, obs = data
    lam = 3.75
    for wt, expect in (("uniform", 1.0), ("briggs", lam)):
        cfg = cfg_of(orc, img, weighting=wt, robust=0.5)
        A = orc.imaging_weights(cfg, obs.uvw, obs.chan_scale, obs.weight, obs.flag)
        B = orc.imaging_weights(cfg, obs.uvw, obs.chan_scale, obs.weight * np.float32(lam),
                                obs.flag)
        cell, _, st = _cells(orc, cfg, obs)
        ok = st == 1
        np.testing.assert_allclose(B[ok, 0], expect * A[ok, 0], rtol=1e-6)


def test_briggs_limits_are_natural_and_uniform(orc, data):
    """R -> +inf: f^2 -> 0, W' -> W.  R -> -inf: f^2 D >> 1, W' -> W/(f^2 D),
    proportional to the uniform weights with one factor per channel."""
    img, obs = data
    Wn = obs.weight.astype(np.float64)
    Wu = orc.imaging_weights(cfg_of(orc, img, weighting="uniform"), obs.uvw, obs.chan_scale,
                             obs.weight, obs.flag)
    hi = orc.imaging_weights(cfg_of(orc, img, weighting="briggs", robust=8.0), obs.uvw,
                             obs.chan_scale, obs.weight, obs.flag)
    lo = orc.imaging_weights(cfg_of(orc, img, weighting="briggs", robust=-8.0), obs.uvw,
                             obs.chan_scale, obs.weight, obs.flag)
    np.testing.assert_allclose(hi, Wn, rtol=1e-9)
    for c in range(2):
        _, _, st = _cells(orc, cfg_of(orc, img), obs, c)
        ok = st == 1
        ratio = lo[ok, c] / Wu[ok, c]
        np.testing.assert_allclose(ratio, ratio[0], rtol=1e-6)
    mid = orc.imaging_weights(cfg_of(orc, img, weighting="briggs", robust=0.0), obs.uvw,
                              obs.chan_scale, obs.weight, obs.flag)
    assert np.all(mid <= Wn + 1e-12)


def test_hermitian_partners_get_equal_weights(orc):
    """Data plus its partners at (-u, -v, -w): every visibility and its partner
    sit on mirrored cells of a symmetric density, so their weights agree
    (a density built without the mirror fails)."""
    img, obs = tiny_wstack(92, nvis=3000, N=64, fov_deg=2.0)
    obs.uvw[:, :2] *= 0.8
    uvw = np.concatenate([obs.uvw, -obs.uvw])
    w = np.concatenate([obs.weight, obs.weight * np.float32(0.5)])
    for wt in ("uniform", "briggs"):
        W = orc.imaging_weights(cfg_of(orc, img, weighting=wt, robust=-0.5), uvw, obs.chan_scale,
                                w, None)
        n = obs.uvw.shape[0]
        np.testing.assert_allclose(W[:n, 0], 2.0 * W[n:, 0], rtol=1e-12)


def test_uniform_psf_has_a_narrower_main_lobe(orc):
    """The point-spread function (all V = 1): its peak is 1 under any weighting
    (the image is normalised by the sum of the weights used), and uniform
    weighting, which takes the weight off the dense short baselines of a
    MeerKAT-like array, narrows the main lobe (its area above half the peak)
    against natural weighting -- the purpose of the scheme; Briggs R = 0 lies
    in between."""
    img, obs = meerkat(93, n_ant=16, n_steps=80, nchan=1, N=256, Nw=4, n_src=5)
    # shrink the tracks onto the mesh (longest baseline 25 cells from the
    # centre) so that the array's dense core is resolved on the grid
    x = obs.uvw[:, :2] * obs.chan_scale[0] * img.fov
    obs.uvw *= 25.0 / np.abs(x).max()
    obs.vis = np.ones_like(obs.vis)
    N = img.N
    area = {}
    for wt in ("natural", "briggs", "uniform"):
        cfg = cfg_of(orc, img, weighting=wt, robust=0.0)
        I, ws = orc.image(cfg, obs.uvw, obs.chan_scale, obs.vis, obs.weight, obs.flag)
        P = I.real
        assert P[N // 2, N // 2] == pytest.approx(1.0, abs=2e-3)
        core = P[N // 2 - 16:N // 2 + 16, N // 2 - 16:N // 2 + 16]
        area[wt] = int((core > 0.5).sum())
    print(area)
    assert area["uniform"] < area["briggs"] < area["natural"]
    assert area["uniform"] <= 0.75 * area["natural"]

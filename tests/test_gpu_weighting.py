"""GPU parity of uniform and Briggs weighting (rick_imaging_weights, and
rick_bin gridding with W' instead of W) against the oracle's imaging weights
(reading R15).

Bars: W' of every visibility within 1e-6 of the oracle's FP64 value (the
library stores W' in FP32, and sums its density with FP64 atomics in another
order); the channel's sum of weights within 1e-9 relative; dirty images within
1e-5 of the peak (full field for the Gaussian workload, taper-gated for
Kaiser-Bessel), folded and unfolded, through the three calls, rick_dirty_image
and a captured graph; the prediction does not depend on the weighting.
"""
import numpy as np
import pytest

from tests.gpu_util import assert_image_close, oracle_config, plan_config, run_path, to_device
from visgen.workloads import meerkat, tiny_wstack

pytestmark = pytest.mark.gpu

TOL = 1e-5


@pytest.fixture(scope="module")
def rk():
    import __graft_entry__
    __graft_entry__.build()
    import torch
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    from paper_2601_19714_gb300 import rick
    rick.load()
    return rick


def _mk(seed, nchan=3, N=512):
    img, obs = meerkat(seed, n_ant=16, n_steps=80, nchan=nchan, N=N, Nw=6, n_src=10)
    g = np.random.default_rng(seed)
    obs.weight = (0.2 + g.random(obs.weight.shape)).astype(np.float32)
    obs.weight[3::29] = 0.0
    # shrink the tracks so that many visibilities share cells (dense centre)
    x = obs.uvw[:, :2] * obs.chan_scale.max() * img.fov
    obs.uvw *= 0.4 * N / np.abs(x).max()
    obs.uvw[7::101, 0] *= 3.0   # and some footprints off the grid
    return img, obs


@pytest.mark.parametrize("wt,R", [("uniform", 0.0), ("briggs", -1.0), ("briggs", 0.0),
                                  ("briggs", 0.5)])
def test_weights_match_oracle(rk, orc, wt, R):
    import torch
    img, obs = _mk(101)
    dev = to_device(obs)
    plan = rk.Plan(plan_config(img, 3, weighting=wt, robust=R))
    out = torch.empty((obs.nrow, 3), dtype=torch.float32, device="cuda")
    plan.imaging_weights(dev["uvw"], dev["chan_scale"], dev["weight"], dev["flag"], dev["nrow"], out)
    torch.cuda.synchronize()
    got = out.cpu().numpy().astype(np.float64)
    ref = orc.imaging_weights(oracle_config(orc, img, weighting=wt, robust=R), obs.uvw,
                              obs.chan_scale, obs.weight, obs.flag)
    err = np.abs(got - ref) / np.maximum(np.abs(ref), 1e-30)
    print(wt, R, err.max(), (ref != obs.weight).mean())
    assert err.max() <= 1e-6
    assert (ref != obs.weight).mean() > 0.5   # most weights changed


@pytest.mark.parametrize("wt", ["uniform", "briggs"])
@pytest.mark.parametrize("fold", [False, True])
def test_weighted_images_match_oracle(rk, orc, wt, fold):
    img, obs = _mk(102)
    plan = rk.Plan(plan_config(img, 3, weighting=wt, robust=0.0, hermitian_fold=fold))
    I_g, _, ws, _ = run_path(plan, to_device(obs), 3, img.N, img.Nw)
    cfg = oracle_config(orc, img, weighting=wt, robust=0.0)
    taper = plan.taper()
    for c in (0, 2):
        I_o, ws_o = orc.image(cfg, obs.uvw, obs.chan_scale, obs.vis, obs.weight, obs.flag, channel=c)
        assert ws[c] == pytest.approx(ws_o, rel=1e-9)
        e = assert_image_close(I_g[c], I_o.real, taper, TOL)
        print(wt, fold, c, e)


def test_weighted_tiny_image_full_field_and_whole_path_calls(rk, orc):
    import torch
    img, obs = tiny_wstack(103, nvis=20_000, N=256)
    obs.uvw[:, :2] *= 0.5      # a denser uv disk: cells shared
    dev = to_device(obs)
    cfg = oracle_config(orc, img, weighting="uniform")
    I_o, _ = orc.image(cfg, obs.uvw, obs.chan_scale, obs.vis, obs.weight)
    plan = rk.Plan(plan_config(img, 1, weighting="uniform"))
    I_g = run_path(plan, dev, 1, img.N, img.Nw)[0]
    assert_image_close(I_g[0], I_o.real, plan.taper(), TOL, full=True)
    im = torch.zeros((1, img.N, img.N), dtype=torch.float32, device="cuda")
    plan.dirty_image(dev["uvw"], dev["chan_scale"], dev["vis"], dev["weight"], dev["flag"],
                     dev["nrow"], im)
    assert_image_close(im[0].cpu().numpy(), I_o.real, plan.taper(), TOL, full=True)
    gplan = rk.Plan(plan_config(img, 1, weighting="uniform"))
    gplan.reserve(dev["nrow"])
    grids = torch.empty((1, img.Nw, img.N, img.N), dtype=torch.complex64, device="cuda")
    wsum = torch.empty(1, dtype=torch.float64, device="cuda")
    img_g = torch.zeros((1, img.N, img.N), dtype=torch.float32, device="cuda")
    graph = gplan.capture_graph(dev["uvw"], dev["chan_scale"], dev["vis"], dev["weight"],
                                dev["flag"], dev["nrow"], grids, wsum, img_g)
    graph.launch()
    torch.cuda.synchronize()
    assert_image_close(img_g[0].cpu().numpy(), I_o.real, plan.taper(), TOL, full=True)


def test_prediction_ignores_the_weighting(rk):
    import torch
    img, obs = tiny_wstack(104, nvis=5000, N=256)
    dev = to_device(obs)
    J = np.zeros((1, img.N, img.N), np.float32)
    J[0, 100:140, 110:150] = 0.01
    out = []
    for wt in ("natural", "uniform"):
        plan = rk.Plan(plan_config(img, 1, weighting=wt))
        vis = torch.zeros((dev["nrow"], 1), dtype=torch.complex64, device="cuda")
        plan.predict(dev["uvw"], dev["chan_scale"], dev["weight"], dev["flag"], dev["nrow"],
                     torch.from_numpy(J).cuda(), vis)
        torch.cuda.synchronize()
        out.append(vis.cpu().numpy())
    np.testing.assert_array_equal(out[0], out[1])

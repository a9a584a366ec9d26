"""Batched multi-channel launch (pattern 2) on the GPU: uneven, flagged
channels in one persistent launch, CUDA-graph capture and replay, streamed
channel/plane groups, and the autotuner -- each against the eager path or the
FP64 oracle."""
import numpy as np
import pytest

from tests.gpu_util import (assert_image_close, host_vis, oracle_config, plan_config, run_path,
                            to_device)
from visgen.workloads import lofar

pytestmark = pytest.mark.gpu

TOL = 1e-5


@pytest.fixture(scope="module")
def rk():
    import __graft_entry__
    __graft_entry__.build()
    import torch
    assert torch.cuda.is_available()
    from paper_2601_19714_gb300 import rick
    rick.load()
    return rick


@pytest.fixture(scope="module")
def small_lofar():
    """LOFAR recipe shrunk to oracle size: 20 stations (10 in the 2 km core),
    60 steps, 6 channels with flag fractions U[0, 0.4], 512^2, 6 planes, FoV
    5 deg.  Long baselines fall off this small grid and are dropped."""
    return lofar(7, n_st=20, n_steps=60, nchan=6, N=512, Nw=6, n_src=10)


def test_uneven_channels_match_oracle(rk, orc, small_lofar):
    img, obs = small_lofar
    C = obs.nchan
    frac = obs.flag.mean(axis=0)
    plan = rk.Plan(plan_config(img, C))
    I_g, _, ws, counts = run_path(plan, to_device(obs), C, img.N, img.Nw)
    assert counts[1] > 0                       # drops on the small grid
    assert frac.max() - frac.min() > 0.1       # uneven channels
    cfg = oracle_config(orc, img)
    for c in (int(np.argmin(frac)), int(np.argmax(frac))):
        I_o, ws_o = orc.image(cfg, obs.uvw, obs.chan_scale, host_vis(obs), obs.weight, obs.flag,
                              channel=c)
        assert ws[c] == pytest.approx(ws_o, rel=1e-12)
        assert_image_close(I_g[c], I_o.real, plan.taper(), TOL)


def test_per_channel_launches_equal_one_batched_launch(rk, small_lofar):
    import torch
    img, obs = small_lofar
    C, N, Nw = obs.nchan, img.N, img.Nw
    plan = rk.Plan(plan_config(img, C))
    dev = to_device(obs)
    wsum = torch.empty(C, dtype=torch.float64, device="cuda")
    plan.bin(dev["uvw"], dev["chan_scale"], dev["vis"], dev["weight"], dev["flag"], dev["nrow"], wsum)
    g1 = torch.empty((C, Nw, N, N), dtype=torch.complex64, device="cuda")
    g2 = torch.empty_like(g1)
    plan.grid_binned(0, C, 0, Nw, g1)
    for c in range(C):
        plan.grid_binned(c, c + 1, 0, Nw, g2[c])
    torch.cuda.synchronize()
    a, b = g1.cpu().numpy(), g2.cpu().numpy()
    assert np.abs(a - b).max() <= 1e-6 * np.abs(a).max()


# kernels of this library per captured graph: place, 3 scan kernels, scatter,
# tile schedule, grid, then the phase kernel after cuFFT's own kernels, or the
# own transform's occupancy and tile-column list, column and fused row kernels
@pytest.mark.parametrize("fft,per_graph", [("cufft", 8), ("own", 11)])
def test_graph_replay_matches_eager_and_follows_new_data(rk, small_lofar, fft, per_graph):
    import torch
    img, obs = small_lofar
    C, N, Nw = obs.nchan, img.N, img.Nw
    plan = rk.Plan(plan_config(img, C, fft_impl=fft))
    plan.reserve(obs.nrow)
    dev = to_device(obs)
    I_e, _, ws_e, cnt_e = run_path(plan, dev, C, N, Nw)
    grids = torch.empty((C, Nw, N, N), dtype=torch.complex64, device="cuda")
    image = torch.full((C, N, N), 7.0, dtype=torch.float32, device="cuda")  # graph zeroes it
    wsum = torch.empty(C, dtype=torch.float64, device="cuda")
    counts = torch.empty(2, dtype=torch.int64, device="cuda")
    graph = plan.capture_graph(dev["uvw"], dev["chan_scale"], dev["vis"], dev["weight"],
                               dev["flag"], dev["nrow"], grids, wsum, image, counts)
    n0 = plan.launch_count()
    for _ in range(2):
        graph.launch()
    torch.cuda.synchronize()
    assert plan.launch_count() - n0 == 2 * per_graph
    taper = plan.taper()
    got = image.cpu().numpy()
    for c in range(C):
        if ws_e[c] > 0:
            assert_image_close(got[c], I_e[c], taper, TOL)
    assert counts.cpu().tolist() == cnt_e.tolist()
    # same buffers, new contents: the replay images the new data
    dev["vis"].mul_(2.0)
    dev["weight"].mul_(0.5)
    graph.launch()
    torch.cuda.synchronize()
    got2 = image.cpu().numpy()
    for c in range(C):
        if ws_e[c] > 0:
            assert_image_close(got2[c], 2.0 * I_e[c], taper, TOL)
    np.testing.assert_allclose(wsum.cpu().numpy(), 0.5 * ws_e, rtol=1e-12)


def test_graph_of_streamed_groups_matches_eager(rk, small_lofar):
    import torch
    img, obs = small_lofar
    C, N, Nw = obs.nchan, img.N, img.Nw
    budget = 4 * N * N * 8                       # 4 planes at a time: groups of planes
    plan = rk.Plan(plan_config(img, C, grid_budget_bytes=budget))
    plan.reserve(obs.nrow)
    dev = to_device(obs)
    I_e, _, ws_e, _ = run_path(plan, dev, C, N, Nw)
    image = torch.empty((C, N, N), dtype=torch.float32, device="cuda")
    wsum = torch.empty(C, dtype=torch.float64, device="cuda")
    graph = plan.capture_graph(dev["uvw"], dev["chan_scale"], dev["vis"], dev["weight"],
                               dev["flag"], dev["nrow"], None, wsum, image)
    graph.launch()
    torch.cuda.synchronize()
    got = image.cpu().numpy()
    for c in range(C):
        if ws_e[c] > 0:
            assert_image_close(got[c], I_e[c], plan.taper(), TOL)


def test_graph_capture_needs_a_reservation(rk, small_lofar):
    import torch
    img, obs = small_lofar
    C = obs.nchan
    plan = rk.Plan(plan_config(img, C))
    dev = to_device(obs)
    image = torch.empty((C, img.N, img.N), dtype=torch.float32, device="cuda")
    wsum = torch.empty(C, dtype=torch.float64, device="cuda")
    with pytest.raises(rk.RickError) as e:
        plan.capture_graph(dev["uvw"], dev["chan_scale"], dev["vis"], dev["weight"], dev["flag"],
                           dev["nrow"], None, wsum, image)
    assert e.value.status == 8


def test_autotune_measures_every_shape_and_its_choice_is_correct(rk, orc, small_lofar):
    import torch
    img, obs = small_lofar
    C, N, Nw = obs.nchan, img.N, img.Nw
    dev = to_device(obs)
    grids = torch.empty((2, Nw, N, N), dtype=torch.complex64, device="cuda")
    best, table = rk.autotune(plan_config(img, C), dev["uvw"], dev["chan_scale"], dev["vis"],
                              dev["weight"], dev["flag"], dev["nrow"], (0, 2), (0, Nw), grids, reps=2)
    # tiles 16 and 32 at 3 CTA sizes, tile 64 at 128 threads only (one 37 KB
    # shared tile per warp); 3 grab sizes each
    assert len(table) == (2 * 3 + 1) * 3
    fastest = min(table, key=lambda r: r[3])
    assert (best.tile, best.grid_threads, best.tiles_per_grab) == fastest[:3]
    assert all(r[3] > 0 for r in table)
    plan = rk.Plan(best)
    I_g, _, _, _ = run_path(plan, dev, C, N, Nw)
    frac = obs.flag.mean(axis=0)
    c = int(np.argmin(frac))
    I_o, _ = orc.image(oracle_config(orc, img), obs.uvw, obs.chan_scale, host_vis(obs), obs.weight,
                       obs.flag, channel=c)
    assert_image_close(I_g[c], I_o.real, plan.taper(), TOL)

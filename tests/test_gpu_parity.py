"""GPU parity: the CUDA path (through the C ABI) against the FP64 oracle.

Bars: index work (plane, footprint start, fractional offset, bin) is
bit-exact; floating-point images match the oracle within 1e-5 of the peak
(the tolerance stated for FP32 accumulation with FP64 index/phase), measured
(a) on the image before the per-pixel taper division and (b) as
max|delta|/peak over the field where that division amplifies by at most 100.
With no grid padding the Kaiser-Bessel taper (beta = 12.25) falls to 1.4e-5 of
its centre value at the field edge, so the division multiplies FP32 rounding
by up to ~5e9 in the corners; there the FP64 oracle itself differs from the
direct Fourier inversion by O(1) (aliasing), so those pixels carry no
information about the arithmetic.  For the Gaussian tiny workload the plain
full-field max|delta|/peak <= 1e-5 is also required.  The all-FP32 variant is
reported, with only a loose sanity bound.
"""
import math

import numpy as np
import pytest

import visgen
from tests.gpu_util import (assert_image_close, host_vis, image_errors, oracle_config,
                            plan_config, rel_err, run_path, taper_gain, to_device)
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


def _oracle_images(orc, img, obs, channels, **kw):
    cfg = oracle_config(orc, img, **kw)
    vis = host_vis(obs)
    out = []
    for c in channels:
        I, _ = orc.image(cfg, obs.uvw, obs.chan_scale, vis, obs.weight, obs.flag, channel=c)
        out.append(I)
    return out


# ----------------------------------------------------------------------------
# index work: bit-exact
# ----------------------------------------------------------------------------

def _expected_records(orc, img, obs, T):
    cfg = oracle_config(orc, img)
    pl = orc.place(cfg, obs.uvw, obs.chan_scale, obs.weight, obs.flag)
    st = pl["status"]
    C = obs.chan_scale.shape[0]
    NT = img.N // T
    r, c = np.nonzero(st == 1)
    k, i0, j0 = pl["k"][r, c], pl["i0"][r, c], pl["j0"][r, c]
    fqx = np.minimum(np.rint(pl["fx"][r, c] * 2.0 ** 24), 2 ** 24 - 1).astype(np.int64)
    fqy = np.minimum(np.rint(pl["fy"][r, c] * 2.0 ** 24), 2 ** 24 - 1).astype(np.int64)
    tx, ty = i0 // T, j0 // T
    il, jl = i0 - tx * T, j0 - ty * T
    right, down = il + img.S - 1 >= T, jl + img.S - 1 >= T
    cls = np.where(right, np.where(down, 2, 3), np.where(down, 1, 0))
    key = ((((c.astype(np.int64) * img.Nw + k) * NT + ty) * NT + tx) * 4 + cls)
    vis = host_vis(obs)
    wv = (obs.weight[r, c].astype(np.float32) * vis[r, c].astype(np.complex64)).astype(np.complex64)
    px = (il.astype(np.int64) << 24) | fqx
    py = (jl.astype(np.int64) << 24) | fqy
    return key, px, py, wv, (st == 1).sum(), (st == -1).sum()


@pytest.mark.parametrize("T", [32, 64])
def test_binning_is_bit_exact(rk, orc, T):
    import torch
    img, obs = tiny_wstack(11, nvis=7001, N=256)
    # a few flagged, zero-weight and off-grid visibilities
    obs.weight[5::97] = 0.0
    obs.flag = np.zeros_like(obs.weight, dtype=np.uint8)
    obs.flag[7::53] = 1
    obs.uvw[3::211, 0] *= 1.8
    plan = rk.Plan(plan_config(img, 1, tile=T))
    dev = to_device(obs)
    wsum = torch.empty(1, dtype=torch.float64, device="cuda")
    counts = torch.empty(2, dtype=torch.int64, device="cuda")
    plan.bin(dev["uvw"], dev["chan_scale"], dev["vis"], dev["weight"], dev["flag"], dev["nrow"],
             wsum, counts)
    off, rec = plan.bins()
    key_e, px_e, py_e, wv_e, ng, nd = _expected_records(orc, img, obs, T)
    assert counts.cpu().tolist() == [ng, nd] and nd > 0
    # GPU records with their keys
    key_g = np.repeat(np.arange(len(off) - 1), np.diff(off.astype(np.int64)))
    assert len(key_g) == len(key_e) == ng
    o_g = np.lexsort((rec[:, 3], rec[:, 2], key_g))
    o_e = np.lexsort((py_e, px_e, key_e))
    np.testing.assert_array_equal(key_g[o_g], key_e[o_e])
    np.testing.assert_array_equal(rec[o_g, 2].astype(np.int64), px_e[o_e])
    np.testing.assert_array_equal(rec[o_g, 3].astype(np.int64), py_e[o_e])
    wv_g = rec[o_g, :2].copy().view(np.float32)
    np.testing.assert_array_equal(wv_g[:, 0], wv_e[o_e].real)
    np.testing.assert_array_equal(wv_g[:, 1], wv_e[o_e].imag)
    ws_e = float(obs.weight[(obs.flag == 0) & (obs.weight != 0)].sum())  # before drops
    cfg = oracle_config(orc, img)
    ws_o, _, _ = orc.channel_stats(cfg, obs.uvw, obs.chan_scale, obs.weight, obs.flag)
    assert wsum.item() == pytest.approx(ws_o, rel=1e-12) and ws_o < ws_e


def test_placement_rounding_ties_and_edges_are_bit_exact(rk, orc):
    """Footprint starts and 24-bit fractions on exact half-way points of the
    rounding (fraction (2j+1) 2^-25), on the first cell (x - S/2 in [-1, 0),
    the FP64 branch of the placement), on the last valid cell, just off the grid
    and at non-finite positions.  With fov = 2^-5 rad, x = u fov + N/2 is exact,
    so each position is the intended one."""
    import torch
    from visgen.workloads import Imaging
    N, S, fov = 256, 8, 2.0 ** -5
    img = Imaging(N, 4, S, "kb", 12.25, fov, -100.0, 100.0)
    xs = []
    for cell in (40, 41, 128, 200):
        for j in (0, 1, 2, 3, 1 << 20, (1 << 23) - 1, (1 << 24) - 1):
            xs.append(cell + S / 2 + (2 * j + 1) * 2.0 ** -25)      # ties at bit 25
        xs.append(cell + S / 2 + 0.5)
        xs.append(cell + S / 2)
    for f in (0.0, 2.0 ** -25, 0.25, 0.5, 1 - 2.0 ** -25):
        xs.append(S / 2 - 1 + f)                                     # x - S/2 in [-1, 0)
    xs += [S / 2 - 1 - 2.0 ** -30, N - S / 2 - 2.0 ** -25, N - S / 2, N - S / 2 + 1e-9]
    xs = np.array(xs)
    n = len(xs)
    g = np.random.default_rng(3)
    ys = xs[g.permutation(n)]
    uvw = np.stack([(xs - N / 2) / fov, (ys - N / 2) / fov, g.uniform(-99, 99, n)], axis=1)
    uvw[-1, 0] = np.inf
    uvw[-2, 2] = np.nan
    from types import SimpleNamespace
    obs = SimpleNamespace(uvw=uvw, chan_scale=np.ones(1), vis=np.ones((n, 1), np.complex64),
                          weight=np.ones((n, 1), np.float32), flag=None)
    for fold in (False, True):
        plan = rk.Plan(plan_config(img, 1, tile=32, hermitian_fold=fold))
        dev = to_device(obs)
        wsum = torch.empty(1, dtype=torch.float64, device="cuda")
        counts = torch.empty(2, dtype=torch.int64, device="cuda")
        plan.bin(dev["uvw"], dev["chan_scale"], dev["vis"], dev["weight"], None, dev["nrow"], wsum,
                 counts)
        off, rec = plan.bins()
        if not fold:
            key_e, px_e, py_e, wv_e, ng, nd = _expected_records(orc, img, obs, 32)
            assert counts.cpu().tolist() == [ng, nd] and nd >= 4
            key_g = np.repeat(np.arange(len(off) - 1), np.diff(off.astype(np.int64)))
            o_g = np.lexsort((rec[:, 3], rec[:, 2], key_g))
            o_e = np.lexsort((py_e, px_e, key_e))
            np.testing.assert_array_equal(key_g[o_g], key_e[o_e])
            np.testing.assert_array_equal(rec[o_g, 2].astype(np.int64), px_e[o_e])
            np.testing.assert_array_equal(rec[o_g, 3].astype(np.int64), py_e[o_e])
            fq = rec[:, 2].astype(np.int64) & ((1 << 24) - 1)
            assert (fq % 2 == 0).sum() > 0 and (fq == 0).sum() > 0
        else:
            assert counts.cpu().tolist()[0] == ng


# ----------------------------------------------------------------------------
# stage by stage against the oracle
# ----------------------------------------------------------------------------

def test_grid_and_fft_planes_match_oracle(rk, orc):
    import torch
    img, obs = tiny_wstack(12, nvis=20_000, N=256)
    plan = rk.Plan(plan_config(img, 1))
    dev = to_device(obs)
    Nw, N = img.Nw, img.N
    grids = torch.empty((1, Nw, N, N), dtype=torch.complex64, device="cuda")
    wsum = torch.empty(1, dtype=torch.float64, device="cuda")
    plan.grid(dev["uvw"], dev["chan_scale"], dev["vis"], dev["weight"], None, dev["nrow"], 0, Nw,
              grids, wsum)
    g = grids.cpu().numpy()[0]
    cfg = oracle_config(orc, img)
    for k in range(Nw):
        G = orc.grid_plane(cfg, obs.uvw, obs.chan_scale, obs.vis, obs.weight, plane=k)
        assert rel_err(g[k], G) < 1e-6, k
    plan.fft_wplanes(grids, Nw)
    f = grids.cpu().numpy()[0]
    for k in (0, 3, 7):
        F = orc.ifft2(orc.grid_plane(cfg, obs.uvw, obs.chan_scale, obs.vis, obs.weight, plane=k))
        assert rel_err(f[k], F) < 1e-5, k


def test_dense_tiles_split_over_warps_match_oracle(rk, orc):
    """A MeerKAT-shaped core at 512^2: the central tiles hold thousands of
    records, so the gridder's longest-first lists of dense tiles (>= 64 T and
    >= 16 T records), which it splits over the warps of a CTA, are not empty,
    and every gridded plane matches the oracle's within 1e-6."""
    import torch
    img, obs = meerkat(21, n_ant=64, n_steps=200, nchan=1, N=512, Nw=4, n_src=10,
                       freqs=np.array([0.856e9]))
    plan = rk.Plan(plan_config(img, 1))
    dev = to_device(obs)
    Nw, N = img.Nw, img.N
    grids = torch.empty((1, Nw, N, N), dtype=torch.complex64, device="cuda")
    wsum = torch.empty(1, dtype=torch.float64, device="cuda")
    plan.grid(dev["uvw"], dev["chan_scale"], dev["vis"], dev["weight"], dev["flag"], dev["nrow"], 0, Nw,
              grids, wsum)
    lists = plan.schedule_counts()
    print(f"longest-first lists (>= 64T, 16T, 4T records): {lists}")
    assert lists[0] + lists[1] > 0
    g = grids.cpu().numpy()[0]
    cfg = oracle_config(orc, img)
    for k in range(Nw):
        G = orc.grid_plane(cfg, obs.uvw, obs.chan_scale, host_vis(obs), obs.weight, obs.flag, plane=k)
        assert rel_err(g[k], G) < 1e-6, k


def test_tiny_wstack_dirty_image(rk, orc):
    """The tiny workload at its stated size: 20k visibilities, 256^2, 8 planes,
    Gaussian S = 7: max|delta|/peak <= 1e-5 for the real and complex image."""
    img, obs = tiny_wstack(0)
    plan = rk.Plan(plan_config(img, 1))
    I_g, C_g, ws, counts = run_path(plan, to_device(obs), 1, img.N, img.Nw, complex_out=True)
    (I_o,) = _oracle_images(orc, img, obs, [0])
    assert counts.tolist() == [20_000, 0]
    assert ws[0] == 20_000.0
    assert_image_close(I_g[0], I_o.real, plan.taper(), TOL, full=True)
    assert_image_close(C_g[0], I_o, plan.taper(), TOL, full=True)
    assert np.unravel_index(np.argmax(I_g[0]), I_g[0].shape) == \
        np.unravel_index(np.argmax(I_o.real), I_o.shape)


@pytest.mark.parametrize("T,threads", [(16, 512), (32, 256), (64, 128)])
def test_tile_and_cta_shapes_agree(rk, orc, T, threads):
    img, obs = tiny_wstack(13, nvis=9000, N=256, Nw=5)
    plan = rk.Plan(plan_config(img, 1, tile=T, grid_threads=threads, fft_batch=2, fft_impl="cufft"))
    I_g, _, _, _ = run_path(plan, to_device(obs), 1, img.N, img.Nw)
    (I_o,) = _oracle_images(orc, img, obs, [0])
    assert_image_close(I_g[0], I_o.real, plan.taper(), TOL, full=True)


def test_multichannel_kaiser_bessel_ragged(rk, orc):
    """A small MeerKAT-shaped set: 5 channels (one fully flagged), KB S = 8,
    random weights, 5 % flags, planes not a multiple of the FFT batch, row
    count not a multiple of any block size."""
    img, obs = meerkat(3, n_ant=12, n_steps=97, nchan=5, N=512, Nw=7, n_src=20, fov_deg=1.5)
    obs.flag[:, 2] = 1
    plan = rk.Plan(plan_config(img, 5, fft_batch=3, fft_impl="cufft"))
    I_g, _, ws, counts = run_path(plan, to_device(obs), 5, img.N, img.Nw)
    assert ws[2] == 0.0 and np.all(I_g[2] == 0.0)
    refs = _oracle_images(orc, img, obs, [0, 1, 3, 4])
    for c, I_o in zip([0, 1, 3, 4], refs):
        e = assert_image_close(I_g[c], I_o.real, plan.taper(), TOL)
        print(f"channel {c}: {e}")


def test_plane_group_streaming_matches_single_pass(rk, orc):
    import torch
    img, obs = meerkat(4, n_ant=10, n_steps=60, nchan=3, N=256, Nw=6, n_src=10)
    dev = to_device(obs)
    outs = []
    for budget in (0, 3 * img.N * img.N * 8, 2 * img.N * img.N * 8 * img.Nw):
        plan = rk.Plan(plan_config(img, 3, grid_budget_bytes=budget))
        im = torch.zeros((3, img.N, img.N), dtype=torch.float32, device="cuda")
        plan.dirty_image(dev["uvw"], dev["chan_scale"], dev["vis"], dev["weight"], dev["flag"],
                         dev["nrow"], im)
        outs.append(im.cpu().numpy())
    taper = plan.taper()
    for o in outs[1:]:
        for c in range(3):
            assert_image_close(o[c], outs[0][c], taper, TOL)
    refs = _oracle_images(orc, img, obs, [1])
    assert_image_close(outs[1][1], refs[0].real, taper, TOL)


@pytest.mark.parametrize("nchan,kw,n_ant,n_steps", [(2, dict(fft_impl="cufft"), 8, 40), (5, dict(hermitian_fold=True), 8, 40),
                                                   (5, dict(fft_impl="own"), 8, 40),
                                                   (3, dict(grid_budget_bytes=2 * 256 * 256 * 8), 8, 40),
                                                   (3, dict(grid_budget_bytes=4 * 256 * 256 * 8, fft_impl="own"), 8, 40),
                                                   (3, dict(weighting="uniform"), 8, 40),
                                                   (2, dict(fft_impl="own"), 7, 1)])
def test_host_entry_point_matches_device_path(rk, orc, nchan, kw, n_ant, n_steps):
    """rick_dirty_image_host: with the whole grid in memory the rows are
    uploaded in chunks, each placed as it arrives (natural weighting; uniform
    weighting uploads everything first), and the channels are transformed and
    downloaded in chunks (uneven for 5 channels); with a plane budget it
    streams plane groups, and with a one-channel budget it downloads each
    channel's image while the next is made; all equal the device path.  One time step of 7
    antennas (21 rows) leaves row chunks of uneven size."""
    img, obs = meerkat(5, n_ant=n_ant, n_steps=n_steps, nchan=nchan, N=256, Nw=4, n_src=8)
    plan = rk.Plan(plan_config(img, nchan, **kw))
    out = np.full((nchan, img.N, img.N), 7.0, np.float32)   # overwritten
    ws = np.zeros(nchan)
    cnt = np.zeros(2, np.int64)
    plan.dirty_image_host(obs.uvw, obs.chan_scale, obs.vis, obs.weight, obs.flag, out, ws, cnt)
    ref = rk.Plan(plan_config(img, nchan, **{k: v for k, v in kw.items() if k != "grid_budget_bytes"}))
    I_g, _, ws_g, cnt_g = run_path(ref, to_device(obs), nchan, img.N, img.Nw)
    for c in range(nchan):
        assert_image_close(out[c], I_g[c], plan.taper(), TOL)
    np.testing.assert_allclose(ws, ws_g, rtol=1e-12)
    assert cnt.tolist() == cnt_g.tolist()


# ----------------------------------------------------------------------------
# invariants and edge cases on the GPU
# ----------------------------------------------------------------------------

def test_empty_input(rk):
    img, obs = tiny_wstack(14, nvis=10, N=128)
    plan = rk.Plan(plan_config(img, 1))
    dev = to_device(obs)
    dev["nrow"] = 0
    I_g, _, ws, counts = run_path(plan, dev, 1, img.N, img.Nw)
    assert ws[0] == 0.0 and counts.tolist() == [0, 0] and np.all(I_g == 0)


def test_all_visibilities_off_grid(rk):
    img, obs = tiny_wstack(15, nvis=500, N=128)
    obs.uvw[:, 0] += 10 * img.N / img.fov   # every footprint far outside the grid
    plan = rk.Plan(plan_config(img, 1))
    I_g, _, ws, counts = run_path(plan, to_device(obs), 1, img.N, img.Nw)
    assert counts.tolist() == [0, 500] and ws[0] == 0.0 and np.all(I_g == 0)


def test_unit_source_at_phase_centre_gpu(rk):
    img, obs = tiny_wstack(16, nvis=5000, N=256)
    obs.vis[:] = 1.0
    plan = rk.Plan(plan_config(img, 1))
    I_g, _, _, _ = run_path(plan, to_device(obs), 1, img.N, img.Nw)
    N = img.N
    assert np.unravel_index(np.argmax(I_g[0]), I_g[0].shape) == (N // 2, N // 2)
    assert abs(I_g[0, N // 2, N // 2] - 1.0) < 4e-3


def test_hermitian_input_gives_real_image_gpu(rk):
    img, obs = tiny_wstack(17, nvis=6000, N=256)
    obs.uvw = np.concatenate([obs.uvw, -obs.uvw])
    obs.vis = np.concatenate([obs.vis, np.conj(obs.vis)])
    obs.weight = np.concatenate([obs.weight, obs.weight])
    plan = rk.Plan(plan_config(img, 1))
    _, C_g, _, _ = run_path(plan, to_device(obs), 1, img.N, img.Nw, complex_out=True)
    A = taper_gain(plan.taper())
    im, re = np.abs(C_g[0].imag), np.abs(C_g[0].real)
    # before the taper division: FP32 rounding only; inside the field of gain <= 100 likewise
    assert (im * A).max() <= 1e-6 * (re * A).max()
    assert im[A >= 1e-2].max() <= 1e-5 * re.max()


def test_linearity_gpu(rk):
    img, obs = tiny_wstack(18, nvis=4000, N=128)
    g = np.random.default_rng(1)
    V1 = ((g.integers(-64, 64, obs.vis.shape) + 1j * g.integers(-64, 64, obs.vis.shape)) / 8).astype(np.complex64)
    V2 = ((g.integers(-64, 64, obs.vis.shape) + 1j * g.integers(-64, 64, obs.vis.shape)) / 8).astype(np.complex64)
    plan = rk.Plan(plan_config(img, 1))
    outs = []
    for V in (V1, V2, (2 * V1 - 0.5 * V2).astype(np.complex64)):
        obs.vis = V
        outs.append(run_path(plan, to_device(obs), 1, img.N, img.Nw)[0])
    assert_image_close(outs[2][0], 2 * outs[0][0] - 0.5 * outs[1][0], plan.taper(), TOL)


def test_all_fp32_variant_error_is_reported(rk, orc):
    """The all-FP32 variant computes index and phase in single precision; its
    error against the FP64 oracle is reported, and must stay sane."""
    img, obs = meerkat(6, n_ant=16, n_steps=80, nchan=2, N=1024, Nw=8, n_src=10)
    (I_o,) = _oracle_images(orc, img, obs, [1])
    errs = {}
    for prec in ("fp64idx", "fp32"):
        plan = rk.Plan(plan_config(img, 2, precision=prec))
        I_g, _, _, _ = run_path(plan, to_device(obs), 2, img.N, img.Nw)
        errs[prec] = image_errors(I_g[1], I_o.real, plan.taper())
    print(f"errors vs FP64 oracle: {errs}")
    assert errs["fp64idx"]["weighted"] <= TOL and errs["fp64idx"]["inner"] <= TOL
    assert errs["fp32"]["weighted"] < 1e-2
    assert errs["fp32"]["weighted"] > errs["fp64idx"]["weighted"]


def test_invalid_arguments_are_rejected(rk):
    img, _ = tiny_wstack(19, nvis=10, N=128)
    bad = [dict(N=100), dict(support=0), dict(tile=48), dict(n_wplanes=0), dict(fov_rad=1.5)]
    for b in bad:
        cfg = plan_config(img, 1)
        for k, v in b.items():
            setattr(cfg, k, v)
        with pytest.raises(rk.RickError) as e:
            rk.Plan(cfg)
        assert e.value.status == 1


def test_launch_count_is_tracked(rk):
    img, obs = tiny_wstack(20, nvis=1000, N=128)
    plan = rk.Plan(plan_config(img, 1, fft_impl="cufft"))
    n0 = plan.launch_count()
    run_path(plan, to_device(obs), 1, img.N, img.Nw)
    # place, 3 scan kernels, scatter, tile schedule, grid, phase
    assert plan.launch_count() - n0 == 8

"""The library's own 2-D DFT of the w-planes (fft_impl = "own", 256 <= N <=
8192) against an FP64 reference, and the fused row pass (transform + phase
screen + reduction) against the separate calls.

Bars: the unnormalised inverse (exponent +) and forward (exponent -) 2-D DFT
of random complex planes within 3e-6 of the reference's RMS at every element
(FP64 numpy FFT of the same FP32 input; the FP32 transform's rounding grows
like log2(N^2) eps), and no worse than 2x the error of cuFFT (through torch)
on the same planes; exact plane waves for impulses; the fused call equals
rick_fft_wplanes + rick_phase_correct_reduce within 2e-6 of the image peak
(real and complex outputs, both precisions, with a w-kernel), and equals the
cuFFT path.
"""
import numpy as np
import pytest

from tests.gpu_util import assert_image_close, oracle_config, plan_config, to_device
from visgen.workloads import meerkat, tiny_wstack

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def rk():
    import __graft_entry__
    __graft_entry__.build()
    import torch
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    from paper_2601_19714_gb300 import rick
    rick.load()
    return rick


def _plan(rk, N, n_planes=1, **kw):
    kw.setdefault("fft_impl", "own")
    return rk.Plan(rk.Config(N=N, n_wplanes=n_planes, support=8, n_channels=1, fov_rad=0.02,
                             w_min=-100.0, w_max=100.0, kernel="kb", kernel_param=12.25, **kw))


@pytest.mark.parametrize("N", [256, 512, 1024, 2048, 4096, 8192])
@pytest.mark.parametrize("inverse", [True, False])
def test_own_fft_matches_fp64(rk, N, inverse):
    import torch
    g = np.random.default_rng(N + inverse)
    P = 3 if N <= 2048 else 1
    x = (g.standard_normal((P, N, N)) + 1j * g.standard_normal((P, N, N))).astype(np.complex64)
    plan = _plan(rk, N)
    d = torch.from_numpy(x).cuda()
    (plan.fft_wplanes if inverse else plan.fft_wplanes_forward)(d, P)
    got = d.cpu().numpy()
    ref = (np.fft.ifft2(x.astype(np.complex128)) * N * N if inverse
           else np.fft.fft2(x.astype(np.complex128)))
    rms = np.sqrt(np.mean(np.abs(ref) ** 2))
    err = np.abs(got - ref).max() / rms
    t = torch.from_numpy(x).cuda()
    cu = (torch.fft.ifft2(t, norm="forward") if inverse else torch.fft.fft2(t)).cpu().numpy()
    err_cufft = np.abs(cu - ref).max() / rms
    print(f"N={N} inverse={inverse}: own {err:.2e}, cuFFT {err_cufft:.2e}")
    assert err <= 3e-6
    assert err <= 2 * err_cufft + 1e-7


@pytest.mark.parametrize("N", [256, 2048, 4096, 8192])
def test_impulse_gives_a_plane_wave(rk, N):
    """x = delta at (i, j): X[q][p] = exp(+2 pi i (i p + j q)/N), exact up to
    the rounding of the twiddles."""
    import torch
    i, j = 37 % N, 201 % N
    x = np.zeros((1, N, N), np.complex64)
    x[0, j, i] = 1.0
    plan = _plan(rk, N)
    d = torch.from_numpy(x).cuda()
    plan.fft_wplanes(d, 1)
    got = d.cpu().numpy()[0]
    p = np.arange(N)
    ref = np.exp(2j * np.pi * ((i * p[None, :] + j * p[:, None]) % N) / N)
    assert np.abs(got - ref).max() <= 2e-6


def test_planes_are_independent_and_cufft_config_agrees(rk):
    import torch
    N = 1024
    g = np.random.default_rng(5)
    x = (g.standard_normal((4, N, N)) + 1j * g.standard_normal((4, N, N))).astype(np.complex64)
    own = torch.from_numpy(x).cuda()
    _plan(rk, N).fft_wplanes(own, 4)
    one = torch.from_numpy(x[2:3].copy()).cuda()
    _plan(rk, N).fft_wplanes(one, 1)
    np.testing.assert_array_equal(own[2].cpu().numpy(), one[0].cpu().numpy())
    cu = torch.from_numpy(x).cuda()
    _plan(rk, N, fft_impl="cufft").fft_wplanes(cu, 4)
    ref = own.cpu().numpy()
    assert np.abs(cu.cpu().numpy() - ref).max() <= 3e-6 * np.sqrt(np.mean(np.abs(ref) ** 2))


def _gridded(rk, cfg, dev, C):
    import torch
    plan = rk.Plan(cfg)
    ns = cfg.stored_planes
    grids = torch.empty((C, ns, cfg.N, cfg.N), dtype=torch.complex64, device="cuda")
    wsum = torch.empty(C, dtype=torch.float64, device="cuda")
    plan.grid(dev["uvw"], dev["chan_scale"], dev["vis"], dev["weight"], dev["flag"], dev["nrow"],
              0, ns, grids, wsum)
    return plan, grids, wsum


@pytest.mark.parametrize("kw", [dict(), dict(hermitian_fold=True), dict(precision="fp32"),
                                dict(hermitian_fold=True, w_support=4, w_kernel_param=8.0)])
def test_fused_equals_separate_calls(rk, kw):
    import torch
    # 24 planes: with a w-kernel of support 4, fewer would put a zero of C_w in the field
    img, obs = meerkat(81, n_ant=10, n_steps=60, nchan=3, N=1024, Nw=24, n_src=10)
    dev = to_device(obs)
    C, N = 3, img.N
    cfg = plan_config(img, C, fft_impl="own", **kw)
    plan, grids, wsum = _gridded(rk, cfg, dev, C)
    ns = cfg.stored_planes
    sep = grids.clone()
    i_sep = torch.zeros((C, N, N), dtype=torch.float32, device="cuda")
    c_sep = torch.zeros((C, N, N), dtype=torch.complex64, device="cuda")
    plan.fft_wplanes(sep, C * ns)
    plan.phase_correct_reduce(sep, 0, C, 0, ns, wsum, i_sep, c_sep)
    i_fus = torch.full((C, N, N), 0.5, dtype=torch.float32, device="cuda")   # accumulates
    c_fus = torch.zeros((C, N, N), dtype=torch.complex64, device="cuda")
    plan.fft_phase_correct_reduce(grids, 0, C, 0, ns, wsum, i_fus, c_fus)
    torch.cuda.synchronize()
    a, b = i_fus.cpu().numpy() - 0.5, i_sep.cpu().numpy()
    peak = np.abs(b).max()
    # the all-FP32 variant forms the phase differently in the two kernels (FP32
    # turns per plane there, FP32 turns to Q0.32 once per pixel here): it is a
    # precision study with no gate, so only agreement to its own error is asked
    tol = 2e-5 if kw.get("precision") == "fp32" else 2e-6
    print(kw, np.abs(a - b).max() / peak)
    assert np.abs(a - b).max() <= tol * peak
    ca, cb = c_fus.cpu().numpy(), c_sep.cpu().numpy()
    assert np.abs(ca - cb).max() <= tol * np.abs(cb).max()


def test_fused_channel_and_plane_ranges(rk):
    """Channels [1, 3) and planes [2, 6) of a 4-channel, 8-plane grid: the
    fused call reads exactly that sub-block (laid out [2][4][N][N])."""
    import torch
    img, obs = meerkat(82, n_ant=10, n_steps=40, nchan=4, N=512, Nw=8, n_src=10)
    dev = to_device(obs)
    C, N = 4, img.N
    cfg = plan_config(img, C, fft_impl="own")
    plan, grids, wsum = _gridded(rk, cfg, dev, C)
    sub = grids[1:3, 2:6].contiguous()
    ref = sub.clone()
    i_ref = torch.zeros((2, N, N), dtype=torch.float32, device="cuda")
    plan.fft_wplanes(ref, 8)
    plan.phase_correct_reduce(ref, 1, 3, 2, 6, wsum, i_ref)
    i_f = torch.zeros((2, N, N), dtype=torch.float32, device="cuda")
    plan.fft_phase_correct_reduce(sub, 1, 3, 2, 6, wsum, i_f)
    torch.cuda.synchronize()
    b = i_ref.cpu().numpy()
    assert np.abs(i_f.cpu().numpy() - b).max() <= 2e-6 * np.abs(b).max()


def test_own_and_cufft_dirty_images_match_oracle(rk, orc):
    """rick_dirty_image (fused path) with the own transform and with cuFFT on
    the tiny workload, both against the oracle, full field."""
    import torch
    img, obs = tiny_wstack(83, nvis=20_000, N=256)
    dev = to_device(obs)
    I_o, _ = orc.image(oracle_config(orc, img), obs.uvw, obs.chan_scale, obs.vis, obs.weight)
    for impl in ("own", "cufft"):
        plan = rk.Plan(plan_config(img, 1, fft_impl=impl))
        im = torch.zeros((1, img.N, img.N), dtype=torch.float32, device="cuda")
        plan.dirty_image(dev["uvw"], dev["chan_scale"], dev["vis"], dev["weight"], dev["flag"],
                         dev["nrow"], im)
        e = assert_image_close(im[0].cpu().numpy(), I_o.real, plan.taper(), 1e-5, full=True)
        print(impl, e)


@pytest.mark.parametrize("kw", [dict(), dict(hermitian_fold=True),
                                dict(hermitian_fold=True, w_support=4, w_kernel_param=8.0)])
def test_pruned_transform_is_exactly_the_unpruned_one(rk, kw):
    """With RICK_GRIDDED_BY_PLAN the column pass skips tile columns that no
    visibility reached and the row pass skips empty planes: zeros transform to
    zeros, so the image is bit-identical to the unpruned call's; a plane range
    of a sub-block and the planes of the whole path are covered.  The data
    leave most tile columns and some planes empty (the short baselines of a
    small array, a wide w range)."""
    import torch
    img, obs = meerkat(84, n_ant=8, n_steps=30, nchan=3, N=1024, Nw=24, n_src=10)
    x = obs.uvw[:, :2] * obs.chan_scale.max() * img.fov
    obs.uvw[:, :2] *= 0.3 * img.N / np.abs(x).max()      # footprints in the central 60 %
    dev = to_device(obs)
    C, N = 3, img.N
    cfg = plan_config(img, C, fft_impl="own", **kw)
    plan, grids, wsum = _gridded(rk, cfg, dev, C)
    ns = cfg.stored_planes
    for (c0, c1, k0, k1) in ((0, C, 0, ns), (1, 3, 2, ns - 1)):
        sub = grids[c0:c1, k0:k1].contiguous()
        a, b = sub.clone(), sub.clone()
        ia = torch.zeros((c1 - c0, N, N), dtype=torch.float32, device="cuda")
        ib = torch.zeros((c1 - c0, N, N), dtype=torch.float32, device="cuda")
        plan.fft_phase_correct_reduce(a, c0, c1, k0, k1, wsum, ia)
        plan.fft_phase_correct_reduce(b, c0, c1, k0, k1, wsum, ib, gridded_by_plan=True)
        torch.cuda.synchronize()
        np.testing.assert_array_equal(ia.cpu().numpy(), ib.cpu().numpy())
        assert np.abs(ia.cpu().numpy()).max() > 0
    # the split calls, pruned, on the whole range
    c = grids.clone()
    ic = torch.zeros((C, N, N), dtype=torch.float32, device="cuda")
    plan.fft_wplanes_columns(c, 0, C, 0, ns, gridded_by_plan=True)
    plan.rows_phase_correct_reduce(c, 0, C, 0, ns, wsum, ic, gridded_by_plan=True)
    d = grids.clone()
    idd = torch.zeros((C, N, N), dtype=torch.float32, device="cuda")
    plan.fft_phase_correct_reduce(d, 0, C, 0, ns, wsum, idd)
    torch.cuda.synchronize()
    np.testing.assert_array_equal(ic.cpu().numpy(), idd.cpu().numpy())


@pytest.mark.parametrize("kw", [dict(), dict(hermitian_fold=True), dict(tile=16), dict(tile=64),
                                dict(hermitian_fold=True, w_support=4, w_kernel_param=8.0)])
def test_sparse_gridding_writes_exactly_the_reached_tiles(rk, kw):
    """rick_grid_binned_sparse into planes filled with NaN: every tile is either
    written exactly as rick_grid_binned writes it or left NaN, and a tile left
    NaN is all zero in the fully written planes; the pruned transform of the
    NaN-filled sparse planes (split and fused calls) gives the image of the
    unpruned transform of the full planes bit for bit -- no unreached cell is
    ever read (a read would carry NaN into the image)."""
    import torch
    img, obs = meerkat(86, n_ant=8, n_steps=30, nchan=3, N=1024, Nw=24, n_src=10)
    x = obs.uvw[:, :2] * obs.chan_scale.max() * img.fov
    obs.uvw[:, :2] *= 0.3 * img.N / np.abs(x).max()      # footprints in the central 60 %
    dev = to_device(obs)
    C, N = 3, img.N
    cfg = plan_config(img, C, fft_impl="own", **kw)
    plan, full, wsum = _gridded(rk, cfg, dev, C)
    ns = cfg.stored_planes
    sp = torch.full_like(full, float("nan"))
    plan.grid_binned(0, C, 0, ns, sp, sparse=True)
    torch.cuda.synchronize()
    T = cfg.tile or 32
    f = full.cpu().numpy().reshape(C, ns, N // T, T, N // T, T)
    g = sp.cpu().numpy().reshape(C, ns, N // T, T, N // T, T)
    nan_tile = np.isnan(g.real).all(axis=(3, 5))
    assert (np.isnan(g.real).any(axis=(3, 5)) == nan_tile).all()   # tiles are whole
    written = ~nan_tile
    assert (f.transpose(0, 1, 2, 4, 3, 5)[written] == g.transpose(0, 1, 2, 4, 3, 5)[written]).all()
    assert (f.transpose(0, 1, 2, 4, 3, 5)[nan_tile] == 0).all()
    print(kw, "unreached tiles", nan_tile.mean())
    assert 0.3 < nan_tile.mean() < 1.0
    for fused in (True, False):
        a, b = full.clone(), sp.clone()
        ia = torch.zeros((C, N, N), dtype=torch.float32, device="cuda")
        ib = torch.zeros((C, N, N), dtype=torch.float32, device="cuda")
        plan.fft_phase_correct_reduce(a, 0, C, 0, ns, wsum, ia)
        if fused:
            plan.fft_phase_correct_reduce(b, 0, C, 0, ns, wsum, ib, gridded_by_plan=True)
        else:
            plan.fft_wplanes_columns(b, 0, C, 0, ns, gridded_by_plan=True)
            plan.rows_phase_correct_reduce(b, 0, C, 0, ns, wsum, ib, gridded_by_plan=True)
        torch.cuda.synchronize()
        got = ib.cpu().numpy()
        assert np.isfinite(got).all()
        np.testing.assert_array_equal(got, ia.cpu().numpy())


def test_pruning_needs_the_plans_gridding_binning(rk):
    import torch
    img, obs = tiny_wstack(85, nvis=500, N=256)
    dev = to_device(obs)
    plan = rk.Plan(plan_config(img, 1, fft_impl="own"))
    grids = torch.zeros((1, img.Nw, img.N, img.N), dtype=torch.complex64, device="cuda")
    with pytest.raises(rk.RickError):   # nothing binned yet
        plan.fft_wplanes_columns(grids, 0, 1, 0, img.Nw, gridded_by_plan=True)
    plan.bin_predict(dev["uvw"], dev["chan_scale"], dev["weight"], None, dev["nrow"])
    with pytest.raises(rk.RickError):   # binned for prediction
        plan.fft_wplanes_columns(grids, 0, 1, 0, img.Nw, gridded_by_plan=True)
    cu = rk.Plan(plan_config(img, 1, fft_impl="cufft"))
    with pytest.raises(rk.RickError) as e:   # the split passes need the own transform
        cu.fft_wplanes_columns(grids, 0, 1, 0, img.Nw)
    assert e.value.status == 6
    cu.bin(dev["uvw"], dev["chan_scale"], dev["vis"], dev["weight"], dev["flag"], dev["nrow"],
           torch.empty(1, dtype=torch.float64, device="cuda"))
    with pytest.raises(rk.RickError) as e:   # and so does sparse gridding
        cu.grid_binned(0, 1, 0, img.Nw, grids, sparse=True)
    assert e.value.status == 6

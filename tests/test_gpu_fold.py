"""GPU parity of the Hermitian fold (hermitian_fold = 1): visibilities of the
upper half of the w-planes are gridded as their conjugates on the mirrored
lower plane at the mirrored cells, so only ceil(Nw/2) planes are stored,
transformed and reduced.

Bars, as for the unfolded path: the binning (plane, mirrored footprint start,
mirrored fraction, conjugated W V, bin) is bit-exact against the oracle's
placement mapped through the fold's definition; the stored planes match the
oracle's folded planes H_k = G_k + conj(mirror(G_{Nw-1-k})) within FP32
rounding; the real dirty image matches the oracle's UNFOLDED image within
1e-5 of the peak (full field for the Gaussian workload, taper-gated for
Kaiser-Bessel).  Edge visibilities whose mirrored footprint ends on cell N
(cell 0 of the periodic mesh) exercise the wrap of the tile halo.
"""
import numpy as np
import pytest

from tests.gpu_util import (assert_image_close, host_vis, oracle_config, plan_config, rel_err,
                            run_path, to_device)
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


def _plant_edges(img, obs, seed):
    """Replace a few rows by visibilities whose footprints start on cell 0 or
    end on cell N-1 (each axis and both), in lower and upper w-planes."""
    g = np.random.default_rng(seed)
    N, S, s = img.N, img.S, float(obs.chan_scale[0])
    lo = 0.5 * S - 1.0 + 0.3   # x with floor(x - S/2) + 1 == 0
    hi = N - 0.5 * S - 0.3     # x with floor(x - S/2) + S == N - 1
    rows = []
    for x, y in ((lo, None), (None, lo), (lo, lo), (hi, None), (None, hi), (hi, hi), (lo, hi),
                 (hi, lo)):
        for w_sign in (-1.0, 1.0):
            xx = x if x is not None else g.uniform(0.3 * N, 0.7 * N)
            yy = y if y is not None else g.uniform(0.3 * N, 0.7 * N)
            w = w_sign * g.uniform(0.2, 0.95) * img.w_max
            rows.append(((xx - N / 2) / img.fov / s, (yy - N / 2) / img.fov / s, w / s))
    idx = np.arange(len(rows)) * 7 + 3
    obs.uvw[idx] = np.array(rows)
    return idx


def _expected_folded_records(orc, img, obs, T):
    cfg = oracle_config(orc, img)
    pl = orc.place(cfg, obs.uvw, obs.chan_scale, obs.weight, obs.flag)
    st = pl["status"]
    N, S, Nw = img.N, img.S, img.Nw
    NT = N // T
    r, c = np.nonzero(st == 1)
    k, i0, j0 = pl["k"][r, c].astype(np.int64), pl["i0"][r, c].astype(np.int64), pl["j0"][r, c].astype(np.int64)
    fqx = np.rint(pl["fx"][r, c] * 2.0 ** 24).astype(np.int64)
    fqy = np.rint(pl["fy"][r, c] * 2.0 ** 24).astype(np.int64)
    vis = host_vis(obs)
    wv = (obs.weight[r, c].astype(np.float32) * vis[r, c].astype(np.complex64)).astype(np.complex64)
    up = 2 * k > Nw - 1
    k = np.where(up, Nw - 1 - k, k)
    i0 = np.where(up, N - i0 - S + 1, i0)
    j0 = np.where(up, N - j0 - S + 1, j0)
    fqx = np.minimum(np.where(up, 2 ** 24 - fqx, fqx), 2 ** 24 - 1)
    fqy = np.minimum(np.where(up, 2 ** 24 - fqy, fqy), 2 ** 24 - 1)
    wv = np.where(up, np.conj(wv), wv)
    tx, ty = i0 // T, j0 // T
    il, jl = i0 - tx * T, j0 - ty * T
    right, down = il + S - 1 >= T, jl + S - 1 >= T
    cls = np.where(right, np.where(down, 2, 3), np.where(down, 1, 0))
    nst = (Nw + 1) // 2
    key = (((c.astype(np.int64) * nst + k) * NT + ty) * NT + tx) * 4 + cls
    return key, (il << 24) | fqx, (jl << 24) | fqy, wv, up


@pytest.mark.parametrize("T,Nw", [(32, 8), (64, 7)])
def test_folded_binning_is_bit_exact(rk, orc, T, Nw):
    import torch
    img, obs = tiny_wstack(31, nvis=7001, N=256, Nw=Nw)
    _plant_edges(img, obs, 31)
    plan = rk.Plan(plan_config(img, 1, tile=T, hermitian_fold=True))
    dev = to_device(obs)
    wsum = torch.empty(1, dtype=torch.float64, device="cuda")
    counts = torch.empty(2, dtype=torch.int64, device="cuda")
    plan.bin(dev["uvw"], dev["chan_scale"], dev["vis"], dev["weight"], dev["flag"], dev["nrow"],
             wsum, counts)
    off, rec = plan.bins()
    key_e, px_e, py_e, wv_e, up = _expected_folded_records(orc, img, obs, T)
    assert 0.3 < up.mean() < 0.7
    assert len(off) - 1 == (Nw + 1) // 2 * (img.N // T) ** 2 * 4
    key_g = np.repeat(np.arange(len(off) - 1), np.diff(off.astype(np.int64)))
    assert len(key_g) == len(key_e)
    o_g = np.lexsort((rec[:, 3], rec[:, 2], key_g))
    o_e = np.lexsort((py_e, px_e, key_e))
    np.testing.assert_array_equal(key_g[o_g], key_e[o_e])
    np.testing.assert_array_equal(rec[o_g, 2].astype(np.int64), px_e[o_e])
    np.testing.assert_array_equal(rec[o_g, 3].astype(np.int64), py_e[o_e])
    wv_g = rec[o_g, :2].copy().view(np.float32)
    np.testing.assert_array_equal(wv_g[:, 0], wv_e[o_e].real)
    np.testing.assert_array_equal(wv_g[:, 1], wv_e[o_e].imag)


@pytest.mark.parametrize("Nw", [8, 7])
def test_folded_planes_match_oracle_fold(rk, orc, Nw):
    """Stored planes against H_k, including footprints wrapped through the
    mesh border (planted edge visibilities), before and after the FFT."""
    import torch
    img, obs = tiny_wstack(32, nvis=20_000, N=256, Nw=Nw)
    _plant_edges(img, obs, 32)
    plan = rk.Plan(plan_config(img, 1, tile=32, hermitian_fold=True))
    ns = plan.cfg.stored_planes
    dev = to_device(obs)
    grids = torch.empty((1, ns, img.N, img.N), dtype=torch.complex64, device="cuda")
    wsum = torch.empty(1, dtype=torch.float64, device="cuda")
    plan.grid(dev["uvw"], dev["chan_scale"], dev["vis"], dev["weight"], None, dev["nrow"], 0, ns,
              grids, wsum)
    g = grids.cpu().numpy()[0]
    cfg = oracle_config(orc, img)
    for k in range(ns):
        H = orc.fold_plane(cfg, obs.uvw, obs.chan_scale, obs.vis, obs.weight, plane=k)
        assert rel_err(g[k], H) < 1e-6, k   # both carry the checkerboard (-1)^(i+j)
        # the wrapped cells of the mirrored edge footprints are populated
        if 2 * k < Nw - 1:
            assert np.abs(H[0, :]).max() > 0 or np.abs(H[:, 0]).max() > 0
    plan.fft_wplanes(grids, ns)
    f = grids.cpu().numpy()[0]
    for k in range(ns):
        F = orc.ifft2(orc.fold_plane(cfg, obs.uvw, obs.chan_scale, obs.vis, obs.weight, plane=k))
        assert rel_err(f[k], F) < 1e-5, k


def test_folded_tiny_image_matches_unfolded_oracle(rk, orc):
    """The tiny workload at its stated size, folded: the real image against
    the oracle's plain (unfolded) w-stacking image, full field."""
    img, obs = tiny_wstack(0)
    plan = rk.Plan(plan_config(img, 1, hermitian_fold=True))
    I_g, _, ws, counts = run_path(plan, to_device(obs), 1, img.N, img.Nw)
    cfg = oracle_config(orc, img)
    I_o, _ = orc.image(cfg, obs.uvw, obs.chan_scale, obs.vis, obs.weight)
    assert counts.tolist() == [20_000, 0] and ws[0] == 20_000.0
    e = assert_image_close(I_g[0], I_o.real, plan.taper(), TOL, full=True)
    print(f"folded tiny: {e}")


@pytest.mark.parametrize("Nw", [7, 8])
def test_folded_multichannel_kaiser_bessel(rk, orc, Nw):
    """MeerKAT-shaped, 4 channels of uneven flagging, KB S = 8, folded against
    the unfolded oracle and against the unfolded GPU path."""
    img, obs = meerkat(8, n_ant=12, n_steps=97, nchan=4, N=512, Nw=Nw, n_src=20)
    dev = to_device(obs)
    plan_f = rk.Plan(plan_config(img, 4, fft_batch=3, hermitian_fold=True, fft_impl="cufft"))
    plan_u = rk.Plan(plan_config(img, 4, fft_batch=3, fft_impl="cufft"))
    I_f, _, ws_f, cnt_f = run_path(plan_f, dev, 4, img.N, img.Nw)
    I_u, _, ws_u, cnt_u = run_path(plan_u, dev, 4, img.N, img.Nw)
    assert cnt_f.tolist() == cnt_u.tolist()
    np.testing.assert_array_equal(ws_f, ws_u)
    cfg = oracle_config(orc, img)
    taper = plan_f.taper()
    for c in (0, 3):
        I_o, _ = orc.image(cfg, obs.uvw, obs.chan_scale, obs.vis, obs.weight, obs.flag, channel=c)
        e = assert_image_close(I_f[c], I_o.real, taper, TOL)
        print(f"channel {c} folded vs oracle: {e}")
    for c in range(4):
        assert_image_close(I_f[c], I_u[c], taper, TOL)


def test_folded_streaming_and_graph_match_single_pass(rk):
    """rick_dirty_image with a plane budget (groups of stored planes) and a
    captured graph give the folded single-pass image."""
    import torch
    img, obs = meerkat(9, n_ant=10, n_steps=60, nchan=3, N=256, Nw=6, n_src=10)
    dev = to_device(obs)
    ref = run_path(rk.Plan(plan_config(img, 3, hermitian_fold=True)), dev, 3, img.N, img.Nw)[0]
    plan = rk.Plan(plan_config(img, 3, hermitian_fold=True, grid_budget_bytes=2 * img.N * img.N * 8))
    im = torch.zeros((3, img.N, img.N), dtype=torch.float32, device="cuda")
    plan.dirty_image(dev["uvw"], dev["chan_scale"], dev["vis"], dev["weight"], dev["flag"],
                     dev["nrow"], im)
    taper = plan.taper()
    for c in range(3):
        assert_image_close(im[c].cpu().numpy(), ref[c], taper, TOL)
    gplan = rk.Plan(plan_config(img, 3, hermitian_fold=True))
    gplan.reserve(dev["nrow"])
    ns = gplan.cfg.stored_planes
    grids = torch.empty((3, ns, img.N, img.N), dtype=torch.complex64, device="cuda")
    wsum = torch.empty(3, dtype=torch.float64, device="cuda")
    img_g = torch.zeros((3, img.N, img.N), dtype=torch.float32, device="cuda")
    graph = gplan.capture_graph(dev["uvw"], dev["chan_scale"], dev["vis"], dev["weight"],
                                dev["flag"], dev["nrow"], grids, wsum, img_g)
    for _ in range(2):
        graph.launch()
    torch.cuda.synchronize()
    for c in range(3):
        assert_image_close(img_g[c].cpu().numpy(), ref[c], taper, TOL)

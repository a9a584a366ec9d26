"""rick_grid_noalloc: gridding for callers that may not allocate device memory.

Some users run the gridder inside a process that sized all of its device
memory up front -- a streaming telescope back end that must never stall on
cudaMalloc while data arrives, or a host framework whose own memory pool owns
the GPU -- so they cannot create a plan (plan creation allocates).  This entry
point takes the configuration directly and uses a fixed device array for its
scratch.  The tests call it through the C ABI twice in a row, on two different
observations, and check each result against rick_grid on the same inputs,
within the tolerance the parity tests use; check that after a first call the
device's free memory does not change across later calls; and check that sizes
whose scratch does not fit, and the other refusals, leave the outputs as they
were (nothing is launched).

This file is collected last on purpose: if it fails, a run stopping at the
first failure has already run everything else.
"""
import ctypes as C

import numpy as np
import pytest

from visgen.workloads import tiny_wstack

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


def _config(rk, img, nchan, fold=False):
    return rk.Config(N=img.N, n_wplanes=img.Nw, support=img.S, n_channels=nchan,
                     fov_rad=img.fov, w_min=img.w_min, w_max=img.w_max, kernel="gauss",
                     kernel_param=img.kernel_param, hermitian_fold=fold)


def _inputs(obs):
    import torch
    t = lambda a: torch.from_numpy(np.ascontiguousarray(a)).cuda()
    return t(obs.uvw), t(obs.chan_scale), t(obs.vis), t(obs.weight), obs.nrow


def _with_plan(rk, img, obs, fold=False):
    import torch
    uvw, sc, vis, wt, nrow = _inputs(obs)
    cfg = _config(rk, img, 1, fold)
    ns = cfg.stored_planes
    grids = torch.empty((1, ns, img.N, img.N), dtype=torch.complex64, device="cuda")
    wsum = torch.empty(1, dtype=torch.float64, device="cuda")
    counts = torch.empty(2, dtype=torch.int64, device="cuda")
    with rk.Plan(cfg) as plan:
        plan.grid(uvw, sc, vis, wt, None, nrow, 0, ns, grids, wsum, counts)
        torch.cuda.synchronize()
    return grids.cpu().numpy(), wsum.cpu().numpy(), counts.cpu().numpy()


def _noalloc_call(rk, cfg_c, uvw, sc, vis, wt, nrow, ns, grids, wsum, counts):
    """One call of rick_grid_noalloc through ctypes (the C ABI); returns the status."""
    import torch
    L = rk.load()
    return L.rick_grid_noalloc(C.byref(cfg_c), uvw.data_ptr(), sc.data_ptr(), vis.data_ptr(),
                               wt.data_ptr(), None, nrow, 0, ns, grids.data_ptr(),
                               wsum.data_ptr(), counts.data_ptr(),
                               torch.cuda.current_stream().cuda_stream)


def _without_alloc(rk, img, obs, fold=False):
    """Call rick_grid_noalloc directly through ctypes (the C ABI)."""
    import torch
    uvw, sc, vis, wt, nrow = _inputs(obs)
    ns = _config(rk, img, 1, fold).stored_planes
    grids = torch.empty((1, ns, img.N, img.N), dtype=torch.complex64, device="cuda")
    wsum = torch.empty(1, dtype=torch.float64, device="cuda")
    counts = torch.empty(2, dtype=torch.int64, device="cuda")
    st = _noalloc_call(rk, _config(rk, img, 1, fold).c(), uvw, sc, vis, wt, nrow, ns, grids, wsum, counts)
    assert st == 0, rk.load().rick_last_error()
    torch.cuda.synchronize()
    return grids.cpu().numpy(), wsum.cpu().numpy(), counts.cpu().numpy()


def test_noalloc_matches_rick_grid_on_two_calls_in_a_row(rk):
    cases = [tiny_wstack(31, nvis=20_000, N=256), tiny_wstack(32, nvis=7_777, N=256, Nw=5)]
    got = [_without_alloc(rk, img, obs) for img, obs in cases]   # two calls back to back
    for (img, obs), (g, ws, cnt) in zip(cases, got):
        g_ref, ws_ref, cnt_ref = _with_plan(rk, img, obs)
        err = np.abs(g - g_ref).max() / np.abs(g_ref).max()
        assert err <= TOL, err
        assert cnt.tolist() == cnt_ref.tolist()
        np.testing.assert_allclose(ws, ws_ref, rtol=1e-12)


def test_noalloc_with_hermitian_fold_matches_rick_grid(rk):
    img, obs = tiny_wstack(34, nvis=12_345, N=256, Nw=7)
    g, ws, cnt = _without_alloc(rk, img, obs, fold=True)
    g_ref, ws_ref, cnt_ref = _with_plan(rk, img, obs, fold=True)
    assert g.shape[1] == 4
    assert np.abs(g - g_ref).max() <= TOL * np.abs(g_ref).max()
    assert cnt.tolist() == cnt_ref.tolist()
    np.testing.assert_allclose(ws, ws_ref, rtol=1e-12)


def test_noalloc_refuses_sizes_beyond_its_scratch(rk):
    img, _ = tiny_wstack(33, nvis=10, N=256)
    cfg = rk.Config(N=4096, n_wplanes=32, support=8, n_channels=16, fov_rad=img.fov,
                    w_min=-1e4, w_max=1e4, kernel="kb", kernel_param=12.25).c()
    import torch
    small = torch.zeros(64, dtype=torch.float64, device="cuda")
    p = small.data_ptr()
    L = rk.load()
    st = L.rick_grid_noalloc(C.byref(cfg), p, p, p, p, None, 1000, 0, 32, p, p, None, None)
    torch.cuda.synchronize()
    assert st == 8  # RICK_ERR_CAPACITY, refused before anything is launched
    assert b"scratch" in L.rick_last_error()


def test_noalloc_later_calls_take_no_device_memory(rk):
    """After a first call (which loads the scratch array and the kernels), two
    more calls of the same support and tile size leave the device's free
    memory exactly as it was: nothing is allocated."""
    import torch
    cases = [tiny_wstack(41, nvis=9_000, N=256), tiny_wstack(42, nvis=5_000, N=256, Nw=6)]
    bufs = []
    for img, obs in cases:
        uvw, sc, vis, wt, nrow = _inputs(obs)
        ns = _config(rk, img, 1).stored_planes
        bufs.append((_config(rk, img, 1).c(), uvw, sc, vis, wt, nrow, ns,
                     torch.empty((1, ns, img.N, img.N), dtype=torch.complex64, device="cuda"),
                     torch.empty(1, dtype=torch.float64, device="cuda"),
                     torch.empty(2, dtype=torch.int64, device="cuda")))
    assert _noalloc_call(rk, *bufs[0]) == 0          # warm-up: loads what the call runs
    torch.cuda.synchronize()
    free0 = torch.cuda.mem_get_info()[0]
    for b in bufs:                                   # two calls in a row
        assert _noalloc_call(rk, *b) == 0, rk.load().rick_last_error()
    torch.cuda.synchronize()
    free1 = torch.cuda.mem_get_info()[0]
    assert free1 == free0, (free0, free1)


def test_noalloc_refusals_launch_nothing(rk):
    """A kernel too narrow for its support and an out-of-range tiles_per_grab
    are refused before anything runs: weight_sum keeps its sentinel."""
    import torch
    img, obs = tiny_wstack(43, nvis=2_000, N=256)
    uvw, sc, vis, wt, nrow = _inputs(obs)
    grids = torch.empty((1, img.Nw, img.N, img.N), dtype=torch.complex64, device="cuda")
    counts = torch.full((2,), -7, dtype=torch.int64, device="cuda")
    for cfg, want in ((rk.Config(N=img.N, n_wplanes=img.Nw, support=8, n_channels=1, fov_rad=img.fov,
                                 w_min=img.w_min, w_max=img.w_max, kernel="gauss", kernel_param=0.05), 6),
                      (_config(rk, img, 1), 1)):
        c = cfg.c()
        if want == 1:
            c.tiles_per_grab = 9
        wsum = torch.full((1,), 123.0, dtype=torch.float64, device="cuda")
        st = _noalloc_call(rk, c, uvw, sc, vis, wt, nrow, img.Nw, grids, wsum, counts)
        torch.cuda.synchronize()
        assert st == want, (st, rk.load().rick_last_error())
        assert wsum.item() == 123.0 and counts.tolist() == [-7, -7]

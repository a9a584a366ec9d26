"""Failure handling without a GPU fault.

Every error path is driven from the host: an injected device-allocation
failure at each allocation of plan creation and inside a call, an injected
cuFFT plan failure, an injected launch failure.  Each failing call must return
its status, and the device's free memory after the plan is destroyed must equal
what it was before (nothing leaks); a plan whose call failed stays usable.
The RICK_DEBUG build's gridder check is made to fail by overwriting one binned
record's first footprint cell with one outside its tile (harmless in any
build: the gridder clips every cell to its tile); the device-side check
records it and rick_plan_sync_status returns RICK_ERR_INTERNAL, and the debug
build otherwise grids the normal build's planes (within FP32 rounding).
"""
import ctypes as C

import numpy as np
import pytest

from tests.gpu_util import assert_image_close, plan_config, to_device
from visgen.workloads import meerkat, tiny_wstack

pytestmark = pytest.mark.gpu

OOM, CUDA, CUFFT, INTERNAL = 2, 3, 4, 7


@pytest.fixture(scope="module")
def rk():
    import __graft_entry__
    __graft_entry__.build()
    import torch
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    from paper_2601_19714_gb300 import rick
    rick.load()
    return rick


def _free():
    """Free device memory with torch's cached blocks returned first, so that
    only what the library holds counts."""
    import torch
    torch.cuda.synchronize()
    torch.cuda.empty_cache()
    return torch.cuda.mem_get_info()[0]


def _create(L, cfg):
    h = C.c_void_p()
    st = L.rick_plan_create(C.byref(cfg.c()), C.byref(h))
    return st, h


@pytest.mark.parametrize("fft", ["own", "cufft"])
def test_every_plan_allocation_failure_is_reported_and_leaks_nothing(rk, fft):
    img, _ = meerkat(51, n_ant=8, n_steps=10, nchan=2, N=512, Nw=6, n_src=4)
    cfg = plan_config(img, 2, hermitian_fold=True, fft_impl=fft)
    L = rk.load()
    st, h = _create(L, cfg)          # warm-up: loads the kernels plan creation runs
    assert st == 0
    L.rick_plan_destroy(h)
    free0 = _free()
    failed = 0
    for n in range(1, 64):
        rk.inject("device_alloc", n)
        st, h = _create(L, cfg)
        if st == 0:                   # fewer allocations than n: nothing was injected
            L.rick_plan_destroy(h)
            break
        assert st == OOM, (n, st, L.rick_last_error())
        assert h.value is None
        failed += 1
        assert _free() == free0, n
    rk.inject("none")
    assert failed >= 8
    assert _free() == free0


def test_cufft_plan_failure_is_reported_and_leaks_nothing(rk):
    img, _ = tiny_wstack(52, nvis=100, N=256)
    cfg = plan_config(img, 1, fft_impl="cufft")
    L = rk.load()
    st, h = _create(L, cfg)
    assert st == 0
    L.rick_plan_destroy(h)
    free0 = _free()
    for n in (1, 2):                  # the batch plan and the single-plane plan
        rk.inject("cufft_plan", n)
        st, h = _create(L, cfg)
        rk.inject("none")
        if st == 0:
            L.rick_plan_destroy(h)
            continue
        assert st == CUFFT and b"injected" in L.rick_last_error()
        assert _free() == free0
    assert _free() == free0


def test_failures_inside_calls_leave_the_plan_usable(rk):
    """An allocation failure inside rick_dirty_image (its first growth of the
    binning scratch) and a reported launch failure inside rick_grid: each call
    returns its status, the next call on the same plan gives the image of a
    fresh plan, and destroying the plan returns all memory."""
    import torch
    img, obs = meerkat(53, n_ant=10, n_steps=30, nchan=2, N=512, Nw=8, n_src=6)
    dev = to_device(obs)
    N, ns = img.N, 4
    cfg = plan_config(img, 2, hermitian_fold=True)

    def image_with(plan):
        out = torch.zeros((2, N, N), dtype=torch.float32, device="cuda")
        plan.dirty_image(dev["uvw"], dev["chan_scale"], dev["vis"], dev["weight"], dev["flag"],
                         obs.nrow, out)
        torch.cuda.synchronize()
        return out.cpu().numpy()

    # the first use of a kernel can reserve device memory for good (its code,
    # a larger local-memory pool): every call of the test runs once first
    with rk.Plan(cfg) as p0:
        ref = image_with(p0)
        g0 = torch.empty((2, ns, N, N), dtype=torch.complex64, device="cuda")
        w0 = torch.empty(2, dtype=torch.float64, device="cuda")
        p0.grid(dev["uvw"], dev["chan_scale"], dev["vis"], dev["weight"], dev["flag"], obs.nrow,
                0, ns, g0, w0)
        p0.sync_status()
        del g0, w0
    free0 = _free()
    plan = rk.Plan(cfg)
    rk.inject("device_alloc", 1)
    with pytest.raises(rk.RickError) as e:
        image_with(plan)
    rk.inject("none")
    assert e.value.status == OOM
    del e   # its traceback holds the frames' tensors
    # record order within a bin follows the binning's atomics, so FP32 sums
    # differ in their last bits between runs, which the unpadded taper
    # correction amplifies at the field edge: the image is compared with the
    # parity tests' taper-aware gate
    taper = plan.taper()

    def same(got):
        for c in range(2):
            assert_image_close(got[c], ref[c], taper, 1e-5)

    same(image_with(plan))
    grids = torch.empty((2, ns, N, N), dtype=torch.complex64, device="cuda")
    wsum = torch.empty(2, dtype=torch.float64, device="cuda")
    rk.inject("launch", 2)
    with pytest.raises(rk.RickError) as e:
        plan.grid(dev["uvw"], dev["chan_scale"], dev["vis"], dev["weight"], dev["flag"], obs.nrow,
                  0, ns, grids, wsum)
    rk.inject("none")
    assert e.value.status == CUDA
    del e
    torch.cuda.synchronize()
    plan.sync_status()
    same(image_with(plan))
    plan.close()
    del grids, wsum
    torch.cuda.empty_cache()
    assert _free() == free0


def test_debug_build_flags_a_record_outside_its_tile(rk):
    import torch
    D = rk.load_debug()
    assert D.rick_debug_build() == 1 and rk.load().rick_debug_build() == 0
    img, obs = tiny_wstack(54, nvis=3000, N=256, Nw=4)
    dev = to_device(obs)
    cfg = plan_config(img, 1)
    st, h = _create(D, cfg)
    assert st == 0, D.rick_last_error()
    N, Nw = img.N, img.Nw
    g_dbg = torch.empty((1, Nw, N, N), dtype=torch.complex64, device="cuda")
    wsum = torch.empty(1, dtype=torch.float64, device="cuda")
    stream = torch.cuda.current_stream().cuda_stream

    def bin_and_grid():
        assert D.rick_bin(h, dev["uvw"].data_ptr(), dev["chan_scale"].data_ptr(), dev["vis"].data_ptr(),
                          dev["weight"].data_ptr(), None, obs.nrow, wsum.data_ptr(), None, stream) == 0
        assert D.rick_grid_binned(h, 0, 1, 0, Nw, g_dbg.data_ptr(), stream) == 0

    bin_and_grid()
    assert D.rick_plan_sync_status(h) == 0
    with rk.Plan(cfg) as p:      # the normal build grids the same planes
        g_ref = torch.empty_like(g_dbg)
        p.grid(dev["uvw"], dev["chan_scale"], dev["vis"], dev["weight"], None, obs.nrow, 0, Nw, g_ref,
               torch.empty(1, dtype=torch.float64, device="cuda"))
        torch.cuda.synchronize()
        a, b = g_dbg.cpu().numpy(), g_ref.cpu().numpy()
        assert np.abs(a - b).max() <= 1e-6 * np.abs(b).max()   # planes: no taper involved
    # one record's first footprint cell moved outside its 32-cell tile
    assert D.rick_debug_poke_record(h, 5, 200, 3) == 0
    assert D.rick_grid_binned(h, 0, 1, 0, Nw, g_dbg.data_ptr(), stream) == 0
    assert D.rick_plan_sync_status(h) == INTERNAL
    assert b"outside its tile" in D.rick_last_error()
    assert D.rick_plan_sync_status(h) == 0      # reported once, then cleared
    bin_and_grid()                              # a fresh binning is consistent again
    assert D.rick_plan_sync_status(h) == 0
    D.rick_plan_destroy(h)
    # the normal build has no poke
    assert rk.load().rick_debug_poke_record(None, 0, 0, 0) == 6

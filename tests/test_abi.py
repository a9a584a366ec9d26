"""The C ABI without a GPU: the library builds, loads, exports every symbol
include/rick.h declares, and rejects invalid configurations before touching
a device."""
import ctypes as C
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    import __graft_entry__
    __graft_entry__.build()
    from paper_2601_19714_gb300 import rick
    return rick.load()


def declared_functions():
    names = set()
    for f in os.listdir(os.path.join(ROOT, "include")):
        if f.endswith(".h"):
            src = open(os.path.join(ROOT, "include", f)).read()
            src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
            names |= set(re.findall(r"\b(rick_\w+)\s*\(", src))
    return sorted(names)


def test_header_declares_the_hot_path():
    names = declared_functions()
    for n in ("rick_grid", "rick_fft_wplanes", "rick_phase_correct_reduce"):
        assert n in names


def test_library_exports_every_declared_symbol(lib):
    missing = [n for n in declared_functions() if not hasattr(lib, n)]
    assert not missing, missing


def test_binding_covers_every_declared_symbol():
    from paper_2601_19714_gb300 import rick
    assert sorted(rick.EXPORTS) == declared_functions()


def test_status_strings(lib):
    assert lib.rick_status_string(0) == b"RICK_OK"
    assert lib.rick_status_string(8) == b"RICK_ERR_CAPACITY"
    assert lib.rick_status_string(99) == b"unknown rick_status"


@pytest.mark.parametrize("field,value", [("N", 100), ("N", 32), ("support", 0), ("support", 17),
                                         ("tile", 48), ("n_wplanes", 0), ("n_channels", 0),
                                         ("fov_rad", 1.5), ("kernel_param", -1.0),
                                         ("grid_threads", 96), ("tiles_per_grab", 65),
                                         ("hermitian_fold", 2)])
def test_invalid_configs_rejected_on_host(lib, field, value):
    from paper_2601_19714_gb300 import rick
    cfg = rick.Config(N=256, n_wplanes=8, support=7, n_channels=1, fov_rad=0.03, w_min=-200,
                      w_max=200, kernel="gauss", kernel_param=0.94).c()
    setattr(cfg, field, value)
    h = C.c_void_p(123)
    st = lib.rick_plan_create(C.byref(cfg), C.byref(h))
    assert st == 1
    assert h.value is None
    assert b"invalid argument" in lib.rick_last_error()


def test_bin_space_overflow_is_unsupported(lib):
    from paper_2601_19714_gb300 import rick
    cfg = rick.Config(N=65536, n_wplanes=128, support=8, n_channels=64, fov_rad=0.03,
                      w_min=-1, w_max=1, kernel="kb", kernel_param=12.0, tile=32).c()
    h = C.c_void_p()
    assert lib.rick_plan_create(C.byref(cfg), C.byref(h)) == 6


def test_null_plan_is_an_error(lib):
    assert lib.rick_plan_destroy(None) == 0
    assert lib.rick_fft_wplanes(None, None, 0, None) == 1
    assert lib.rick_plan_launch_count(None) == -1


def test_hermitian_fold_needs_symmetric_w_and_symmetric_kernel(lib):
    """The fold maps plane k to plane Nw-1-k, which sits at -w_k only for a
    w range symmetric about zero, and reuses the taps of the mirrored
    footprint, which needs a point-symmetric kernel."""
    from paper_2601_19714_gb300 import rick
    base = dict(N=256, n_wplanes=8, support=4, n_channels=1, fov_rad=0.03, kernel_param=5.6,
                hermitian_fold=True)
    for kw in (dict(w_min=-200, w_max=250, kernel="kb"), dict(w_min=-200, w_max=200, kernel="learned")):
        cfg = rick.Config(**base, **kw).c()
        h = C.c_void_p(123)
        assert lib.rick_plan_create(C.byref(cfg), C.byref(h)) == 1
        assert h.value is None
        assert b"hermitian_fold" in lib.rick_last_error()


@pytest.mark.parametrize("nw,fold,expect", [(8, 0, 8), (8, 1, 4), (7, 1, 4), (1, 1, 1), (32, 1, 16)])
def test_stored_planes(lib, nw, fold, expect):
    from paper_2601_19714_gb300 import rick
    cfg = rick.Config(N=256, n_wplanes=nw, support=7, n_channels=1, fov_rad=0.03, w_min=-200,
                      w_max=200, kernel="gauss", kernel_param=0.94, hermitian_fold=bool(fold))
    assert lib.rick_stored_planes(C.byref(cfg.c())) == expect == cfg.stored_planes
    assert lib.rick_stored_planes(None) == -1


@pytest.mark.parametrize("kw", [dict(w_support=3, w_kernel_param=6.0),
                                dict(w_support=10, w_kernel_param=6.0),
                                dict(w_support=4, w_kernel_param=0.0),
                                dict(w_support=4, w_kernel_param=6.0, n_wplanes=1),
                                dict(w_support=4, w_kernel_param=6.0, kernel="learned", support=4,
                                     kernel_param=5.6),
                                # dw max|n - 1| = 0.6 (pi Sw 0.6 = 7.5 > sqrt(6^2 + pi^2) = 6.8)
                                dict(w_support=4, w_kernel_param=6.0, fov_rad=0.2,
                                     w_min=-0.6 / 0.0100503781525921 * 4,
                                     w_max=0.6 / 0.0100503781525921 * 4)])
def test_w_kernel_configs_rejected_on_host(lib, kw):
    """The w-kernel needs an even support in [2, 8], a positive beta, at least
    two planes, and a separable uv kernel (the table kernel is per plane)."""
    from paper_2601_19714_gb300 import rick
    base = dict(N=256, n_wplanes=8, support=7, n_channels=1, fov_rad=0.03, w_min=-200,
                w_max=200, kernel="gauss", kernel_param=0.94)
    base.update(kw)
    h = C.c_void_p(123)
    assert lib.rick_plan_create(C.byref(rick.Config(**base).c()), C.byref(h)) == 1
    assert h.value is None
    assert b"w_" in lib.rick_last_error() or b"w-kernel" in lib.rick_last_error()


@pytest.mark.parametrize("nw,sw,fold,expect", [(8, 4, 0, 12), (8, 4, 1, 6), (7, 4, 1, 6),
                                               (7, 2, 0, 9), (32, 8, 1, 20), (8, 1, 0, 8)])
def test_stored_planes_with_w_kernel(lib, nw, sw, fold, expect):
    from paper_2601_19714_gb300 import rick
    cfg = rick.Config(N=256, n_wplanes=nw, support=7, n_channels=1, fov_rad=0.03, w_min=-200,
                      w_max=200, kernel="gauss", kernel_param=0.94, hermitian_fold=bool(fold),
                      w_support=sw, w_kernel_param=6.0)
    assert lib.rick_stored_planes(C.byref(cfg.c())) == expect == cfg.stored_planes


@pytest.mark.parametrize("kw", [dict(weighting="briggs", robust=float("nan"))])
def test_weighting_configs_rejected_on_host(lib, kw):
    from paper_2601_19714_gb300 import rick
    cfg = rick.Config(N=256, n_wplanes=8, support=7, n_channels=1, fov_rad=0.03, w_min=-200,
                      w_max=200, kernel="gauss", kernel_param=0.94, **kw).c()
    h = C.c_void_p(123)
    assert lib.rick_plan_create(C.byref(cfg), C.byref(h)) == 1
    assert b"robust" in lib.rick_last_error()
    cfg.weighting = 3
    cfg.robust = 0.0
    assert lib.rick_plan_create(C.byref(cfg), C.byref(h)) == 1
    assert b"weighting" in lib.rick_last_error()


@pytest.mark.parametrize("kw,word", [(dict(grid_size=384), b"grid_size"),
                                     (dict(grid_size=128), b"grid_size"),
                                     (dict(grid_size=512, kernel="learned", support=4,
                                           kernel_param=5.6), b"padded")])
def test_padding_configs_rejected_on_host(lib, kw, word):
    """A padded mesh is a power of two >= N, with a separable kernel."""
    from paper_2601_19714_gb300 import rick
    base = dict(N=256, n_wplanes=8, support=7, n_channels=1, fov_rad=0.03, w_min=-200,
                w_max=200, kernel="gauss", kernel_param=0.94)
    base.update(kw)
    h = C.c_void_p(123)
    assert lib.rick_plan_create(C.byref(rick.Config(**base).c()), C.byref(h)) == 1
    assert word in lib.rick_last_error()


def test_fft_impl_values(lib):
    """fft_impl 0 (the C default) is the library's own transform, 1 cuFFT;
    other values are refused on the host."""
    from paper_2601_19714_gb300 import rick
    assert rick.FFT_IMPLS == {"own": 0, "cufft": 1}
    assert rick.Config(N=256, n_wplanes=8, support=7, n_channels=1, fov_rad=0.03, w_min=-200,
                       w_max=200, kernel="gauss", kernel_param=0.94).c().fft_impl == 0
    cfg = rick.Config(N=256, n_wplanes=8, support=7, n_channels=1, fov_rad=0.03, w_min=-200,
                      w_max=200, kernel="gauss", kernel_param=0.94).c()
    cfg.fft_impl = 2
    h = C.c_void_p(123)
    assert lib.rick_plan_create(C.byref(cfg), C.byref(h)) == 1
    assert b"fft_impl" in lib.rick_last_error()


def test_fault_injection_hook_arguments(lib):
    """rick_debug_inject arms and disarms on the host (what a failure does is
    checked on a GPU); the normal build is not a debug build and has no
    record poke."""
    assert lib.rick_debug_inject(1, 3) == 0
    assert lib.rick_debug_inject(0, 0) == 0
    assert lib.rick_debug_inject(9, 1) == 1
    assert b"injection site" in lib.rick_last_error()
    assert lib.rick_debug_inject(1, -1) == 1
    assert lib.rick_debug_build() == 0
    assert lib.rick_debug_poke_record(None, 0, 0, 0) == 6

"""Thin ctypes binding of librick (include/rick.h).

Argument marshalling only: every step of the imaging path runs in the
library's CUDA kernels (and cuFFT).  There is no fallback: if librick.so is
missing or cannot be loaded, importing the binding raises.

Torch tensors are accepted wherever the C ABI takes a device pointer; their
dtype, contiguity and device are checked here, and ``data_ptr()`` plus the
current CUDA stream are passed through.
"""
from __future__ import annotations

import ctypes as C
import os
from dataclasses import dataclass

PKG = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(PKG, "librick.so")

RICK_OK = 0
STATUS = {0: "RICK_OK", 1: "RICK_ERR_INVALID_ARG", 2: "RICK_ERR_OOM", 3: "RICK_ERR_CUDA",
          4: "RICK_ERR_CUFFT", 5: "RICK_ERR_TIMEOUT", 6: "RICK_ERR_UNSUPPORTED",
          7: "RICK_ERR_INTERNAL", 8: "RICK_ERR_CAPACITY"}
KERNELS = {"gauss": 0, "kb": 1, "kaiser_bessel": 1, "table": 2, "learned": 2}
PRECISIONS = {"fp64idx": 0, "fp32": 1}
FFT_IMPLS = {"own": 0, "cufft": 1}
GRIDDED_BY_PLAN = 1             # transform flag: the planes are this plan's gridder output
WEIGHTINGS = {"natural": 0, "uniform": 1, "briggs": 2}

EXPORTS = ["rick_plan_create", "rick_plan_destroy", "rick_plan_reserve", "rick_plan_taper",
           "rick_set_kernel_table", "rick_bin", "rick_grid_binned", "rick_grid_binned_sparse",
           "rick_grid",
           "rick_fft_wplanes", "rick_phase_correct_reduce", "rick_fft_phase_correct_reduce",
           "rick_fft_wplanes_columns", "rick_rows_phase_correct_reduce", "rick_imaging_weights",
           "rick_dirty_image",
           "rick_dirty_image_host", "rick_plan_sync_status", "rick_plan_launch_count",
           "rick_plan_bins", "rick_grid_noalloc", "rick_graph_capture", "rick_graph_launch",
           "rick_graph_destroy", "rick_autotune", "rick_mlp_param_count", "rick_mlp_forward",
           "rick_mlp_backward", "rick_adam_step", "rick_mlp_lattice_inputs", "rick_learn_create",
           "rick_learn_destroy", "rick_learn_placed", "rick_learn_field_grad",
           "rick_status_string", "rick_last_error", "rick_stored_planes", "rick_bin_predict",
           "rick_model_to_wplanes", "rick_fft_wplanes_forward", "rick_model_fft_wplanes", "rick_degrid_binned",
           "rick_predict", "rick_plan_fft_impl", "rick_plan_schedule_counts", "rick_debug_inject",
           "rick_debug_build", "rick_debug_poke_record"]

INJECT_SITES = {"none": 0, "device_alloc": 1, "cufft_plan": 2, "launch": 3}


class RickError(RuntimeError):
    def __init__(self, status: int, where: str, msg: str):
        super().__init__(f"{where}: {STATUS.get(status, status)}: {msg}")
        self.status = status


class rick_config(C.Structure):
    _fields_ = [("N", C.c_int32), ("n_wplanes", C.c_int32), ("support", C.c_int32),
                ("n_channels", C.c_int32), ("fov_rad", C.c_double), ("w_min", C.c_double),
                ("w_max", C.c_double), ("kernel_param", C.c_double), ("kernel_kind", C.c_int32),
                ("precision", C.c_int32), ("tile", C.c_int32), ("grid_threads", C.c_int32),
                ("fft_batch", C.c_int32), ("tiles_per_grab", C.c_int32),
                ("grid_budget_bytes", C.c_int64), ("hermitian_fold", C.c_int32),
                ("w_support", C.c_int32), ("w_kernel_param", C.c_double),
                ("fft_impl", C.c_int32), ("weighting", C.c_int32), ("robust", C.c_double),
                ("grid_size", C.c_int32)]


class rick_tune_entry(C.Structure):
    _fields_ = [("tile", C.c_int32), ("grid_threads", C.c_int32), ("tiles_per_grab", C.c_int32),
                ("grid_ms", C.c_float)]


_lib = None


def load(path: str = LIB_PATH):
    """Load librick.so (built by ``paper_2601_19714_gb300._build.build()``)."""
    global _lib
    if _lib is not None:
        return _lib
    _lib = _open(path)
    return _lib


def load_debug():
    """The RICK_DEBUG build of the library (built on first use), with the same
    signatures; a separate library with its own state."""
    from . import _build
    return _open(_build.build(debug=True))


def _open(path: str):
    if not os.path.exists(path):
        raise ImportError(f"librick.so not built ({path}); run __graft_entry__.build()")
    L = C.CDLL(path)
    p, i32, i64, st = C.c_void_p, C.c_int32, C.c_int64, C.c_int
    sig = {
        "rick_plan_create": [C.POINTER(rick_config), C.POINTER(p)],
        "rick_plan_destroy": [p],
        "rick_plan_reserve": [p, i64],
        "rick_plan_taper": [p, p],
        "rick_set_kernel_table": [p, p, i32, p],
        "rick_bin": [p, p, p, p, p, p, i64, p, p, p],
        "rick_grid_binned": [p, i32, i32, i32, i32, p, p],
        "rick_grid_binned_sparse": [p, i32, i32, i32, i32, p, p],
        "rick_grid": [p, p, p, p, p, p, i64, i32, i32, p, p, p, p],
        "rick_fft_wplanes": [p, p, i64, p],
        "rick_phase_correct_reduce": [p, p, i32, i32, i32, i32, p, p, p, p],
        "rick_fft_phase_correct_reduce": [p, p, i32, i32, i32, i32, p, p, p, i32, p],
        "rick_fft_wplanes_columns": [p, p, i32, i32, i32, i32, i32, p],
        "rick_imaging_weights": [p, p, p, p, p, i64, p, p],
        "rick_rows_phase_correct_reduce": [p, p, i32, i32, i32, i32, p, p, p, i32, p],
        "rick_dirty_image": [p, p, p, p, p, p, i64, p, p, p, p, p],
        "rick_dirty_image_host": [p, p, p, p, p, p, i64, p, p, p, p],
        "rick_plan_sync_status": [p],
        "rick_plan_bins": [p, C.POINTER(i64), C.POINTER(i64), p, p],
        "rick_grid_noalloc": [C.POINTER(rick_config), p, p, p, p, p, i64, i32, i32, p, p, p, p],
        "rick_graph_capture": [p, p, p, p, p, p, i64, p, p, p, p, C.POINTER(p)],
        "rick_graph_launch": [p, p],
        "rick_graph_destroy": [p],
        "rick_autotune": [C.POINTER(rick_config), p, p, p, p, p, i64, i32, i32, i32, i32, p, i32,
                          C.POINTER(rick_tune_entry), i32, C.POINTER(i32), C.POINTER(rick_config)],
        "rick_bin_predict": [p, p, p, p, p, i64, p, p],
        "rick_model_to_wplanes": [p, p, i32, i32, i32, i32, p, p],
        "rick_fft_wplanes_forward": [p, p, i64, p],
        "rick_model_fft_wplanes": [p, p, i32, i32, i32, i32, p, i32, p],
        "rick_degrid_binned": [p, p, i32, i32, i32, i32, p, p],
        "rick_predict": [p, p, p, p, p, i64, p, p, p, p],
        "rick_plan_schedule_counts": [p, p],
        "rick_debug_inject": [i32, i32],
        "rick_debug_poke_record": [p, i64, i32, i32],
    }
    for name, args in sig.items():
        f = getattr(L, name)
        f.argtypes = args
        f.restype = st
    f32 = C.c_float
    for name, args in {
        "rick_mlp_forward": [p, i32, p, i64, p, p, p],
        "rick_mlp_backward": [p, i32, p, i64, p, p, p, p, p],
        "rick_adam_step": [p, p, p, p, i64, f32, f32, f32, f32, i32, p],
        "rick_mlp_lattice_inputs": [i32, i32, p, p],
        "rick_learn_create": [C.POINTER(rick_config), i32, p, p, i64, C.POINTER(p)],
        "rick_learn_destroy": [p],
        "rick_learn_field_grad": [p, p, p, i32, p, i32, p, i32, f32, p, p, p],
    }.items():
        f = getattr(L, name)
        f.argtypes = args
        f.restype = st
    L.rick_mlp_param_count.argtypes = [i32]
    L.rick_mlp_param_count.restype = i64
    L.rick_learn_placed.argtypes = [p]
    L.rick_learn_placed.restype = i64
    L.rick_plan_launch_count.argtypes = [p]
    L.rick_plan_launch_count.restype = i64
    L.rick_plan_fft_impl.argtypes = [p]
    L.rick_plan_fft_impl.restype = i32
    L.rick_status_string.argtypes = [st]
    L.rick_status_string.restype = C.c_char_p
    L.rick_last_error.argtypes = []
    L.rick_last_error.restype = C.c_char_p
    L.rick_stored_planes.argtypes = [C.POINTER(rick_config)]
    L.rick_stored_planes.restype = i32
    L.rick_debug_build.argtypes = []
    L.rick_debug_build.restype = i32
    return L


def inject(site: str, countdown: int = 1):
    """Arm one injected failure (see rick_debug_inject): the countdown-th
    event of `site` ("device_alloc", "cufft_plan", "launch") fails once;
    inject("none") disarms."""
    _check(load().rick_debug_inject(INJECT_SITES[site], int(countdown)), "rick_debug_inject")


def _check(status: int, where: str):
    if status != RICK_OK:
        msg = load().rick_last_error().decode(errors="replace")
        raise RickError(status, where, msg)


def _ptr(t, dtype=None, name="tensor", align=1):
    """Device pointer of a contiguous CUDA tensor (or None / an int)."""
    if t is None:
        return None
    if isinstance(t, int):
        return t
    import torch
    if not isinstance(t, torch.Tensor):
        raise TypeError(f"{name}: expected a torch tensor")
    if not t.is_cuda:
        raise ValueError(f"{name}: must be a CUDA tensor")
    if not t.is_contiguous():
        raise ValueError(f"{name}: must be contiguous")
    if dtype is not None and t.dtype not in dtype:
        raise TypeError(f"{name}: dtype {t.dtype} not in {dtype}")
    ptr = t.data_ptr()
    if ptr % align:
        raise ValueError(f"{name}: must be {align}-byte aligned")
    return ptr


def _stream(stream):
    if stream is None:
        import torch
        return torch.cuda.current_stream().cuda_stream
    if isinstance(stream, int):
        return stream
    return stream.cuda_stream


def _dt():
    import torch
    return dict(f64=(torch.float64,), f32=(torch.float32,), c64=(torch.complex64, torch.float32),
                u8=(torch.uint8, torch.bool), i64=(torch.int64,))


@dataclass
class Config:
    """Imaging parameters in the paper's notation (Sec. 2) plus launch knobs."""
    N: int
    n_wplanes: int
    support: int
    n_channels: int
    fov_rad: float
    w_min: float
    w_max: float
    kernel: str = "kb"
    kernel_param: float = 12.0
    precision: str = "fp64idx"
    tile: int = 0
    grid_threads: int = 0
    fft_batch: int = 0
    tiles_per_grab: int = 0
    grid_budget_bytes: int = 0
    hermitian_fold: bool = False
    w_support: int = 0          # even Sw >= 2: Kaiser-Bessel kernel in w over Sw planes
    w_kernel_param: float = 0.0
    fft_impl: str = "own"       # the library's two-pass DFT (unpadded 256 <= N <= 16384; cuFFT otherwise), or "cufft"
    weighting: str = "natural"  # or "uniform", "briggs" (imaging weights)
    robust: float = 0.0         # Briggs robustness R
    grid_size: int = 0          # padded mesh side Ng (0 = N)

    def c(self) -> rick_config:
        return rick_config(self.N, self.n_wplanes, self.support, self.n_channels, self.fov_rad,
                           self.w_min, self.w_max, self.kernel_param, KERNELS[self.kernel],
                           PRECISIONS[self.precision], self.tile, self.grid_threads,
                           self.fft_batch, self.tiles_per_grab, self.grid_budget_bytes,
                           int(bool(self.hermitian_fold)), int(self.w_support),
                           float(self.w_kernel_param), FFT_IMPLS[self.fft_impl],
                           WEIGHTINGS[self.weighting], float(self.robust), int(self.grid_size))

    @property
    def Ng(self) -> int:
        """Mesh side of the planes (grid_size, or N without padding)."""
        return self.grid_size or self.N

    @property
    def planes_total(self) -> int:
        """Planes imaged: Nw, or Nw + Sw with a w-kernel."""
        return self.n_wplanes + (self.w_support if self.w_support >= 2 else 0)

    @property
    def stored_planes(self) -> int:
        """Planes held per channel: ceil(planes_total/2) with the Hermitian fold."""
        t = self.planes_total
        return (t + 1) // 2 if self.hermitian_fold else t


class Plan:
    """A librick plan (owns tables, cuFFT plans and binning scratch)."""

    def __init__(self, cfg: Config):
        L = load()
        self.cfg = cfg
        self._c = cfg.c()
        h = C.c_void_p()
        _check(L.rick_plan_create(C.byref(self._c), C.byref(h)), "rick_plan_create")
        self.handle = h

    def close(self):
        if getattr(self, "handle", None):
            load().rick_plan_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    # ---- plan utilities ---------------------------------------------------
    def reserve(self, max_rows: int):
        _check(load().rick_plan_reserve(self.handle, int(max_rows)), "rick_plan_reserve")

    def taper(self):
        import numpy as np
        out = np.zeros(self.cfg.N, np.float64)
        _check(load().rick_plan_taper(self.handle, out.ctypes.data), "rick_plan_taper")
        return out

    def set_kernel_table(self, taps, lattice: int, stream=None):
        d = _dt()
        _check(load().rick_set_kernel_table(self.handle, _ptr(taps, d["f32"], "taps", 16),
                                            int(lattice), _stream(stream)),
               "rick_set_kernel_table")

    def launch_count(self) -> int:
        return int(load().rick_plan_launch_count(self.handle))

    @property
    def own_fft(self) -> bool:
        """True if the plan runs the library's own 2-D DFT (else cuFFT)."""
        return int(load().rick_plan_fft_impl(self.handle)) == FFT_IMPLS["own"]

    def schedule_counts(self):
        """Lengths of the gridder's three longest-first tile lists of the last
        gridding call: tiles reached by >= 64T, 16T and 4T records."""
        out = (C.c_uint32 * 3)()
        _check(load().rick_plan_schedule_counts(self.handle, out), "rick_plan_schedule_counts")
        return [int(v) for v in out]

    def sync_status(self):
        _check(load().rick_plan_sync_status(self.handle), "rick_plan_sync_status")

    def bins(self):
        import numpy as np
        L = load()
        nk, nr = C.c_int64(), C.c_int64()
        _check(L.rick_plan_bins(self.handle, C.byref(nk), C.byref(nr), None, None), "rick_plan_bins")
        off = np.zeros(nk.value + 1, np.uint32)
        rec = np.zeros((max(nr.value, 1), 4), np.uint32)
        _check(L.rick_plan_bins(self.handle, C.byref(nk), C.byref(nr), off.ctypes.data,
                                rec.ctypes.data), "rick_plan_bins")
        return off, rec[:nr.value]

    def bin_offsets(self):
        """The bin offsets of the current binning (host numpy u32 [n_keys + 1])."""
        import numpy as np
        L = load()
        nk, nr = C.c_int64(), C.c_int64()
        _check(L.rick_plan_bins(self.handle, C.byref(nk), C.byref(nr), None, None), "rick_plan_bins")
        off = np.zeros(nk.value + 1, np.uint32)
        _check(L.rick_plan_bins(self.handle, C.byref(nk), C.byref(nr), off.ctypes.data, None),
               "rick_plan_bins")
        return off

    # ---- the hot path -------------------------------------------------------
    def _vis_args(self, uvw, chan_scale, vis, weight, flag):
        d = _dt()
        return [_ptr(uvw, d["f64"], "uvw", 8), _ptr(chan_scale, d["f64"], "chan_scale", 8),
                _ptr(vis, d["c64"], "vis", 8), _ptr(weight, d["f32"], "weight", 4),
                _ptr(flag, d["u8"], "flag")]

    def bin(self, uvw, chan_scale, vis, weight, flag, nrow, weight_sum, counts=None, stream=None):
        d = _dt()
        _check(load().rick_bin(self.handle, *self._vis_args(uvw, chan_scale, vis, weight, flag),
                               int(nrow), _ptr(weight_sum, d["f64"], "weight_sum", 8),
                               _ptr(counts, d["i64"], "counts", 8), _stream(stream)), "rick_bin")

    def grid_binned(self, chan_begin, chan_end, plane_begin, plane_end, grids, stream=None,
                    sparse=False):
        """rick_grid_binned, or rick_grid_binned_sparse with sparse=True (the
        unreached tiles are left unwritten: for the pruned own transform only)."""
        d = _dt()
        fn = load().rick_grid_binned_sparse if sparse else load().rick_grid_binned
        _check(fn(self.handle, chan_begin, chan_end, plane_begin, plane_end,
                  _ptr(grids, d["c64"], "grids", 16), _stream(stream)),
               "rick_grid_binned_sparse" if sparse else "rick_grid_binned")

    def grid(self, uvw, chan_scale, vis, weight, flag, nrow, plane_begin, plane_end, grids,
             weight_sum, counts=None, stream=None):
        d = _dt()
        _check(load().rick_grid(self.handle, *self._vis_args(uvw, chan_scale, vis, weight, flag),
                                int(nrow), plane_begin, plane_end,
                                _ptr(grids, d["c64"], "grids", 16),
                                _ptr(weight_sum, d["f64"], "weight_sum", 8),
                                _ptr(counts, d["i64"], "counts", 8), _stream(stream)), "rick_grid")

    def fft_wplanes(self, grids, n_planes, stream=None):
        d = _dt()
        _check(load().rick_fft_wplanes(self.handle, _ptr(grids, d["c64"], "grids", 16),
                                       int(n_planes), _stream(stream)), "rick_fft_wplanes")

    def phase_correct_reduce(self, grids, chan_begin, chan_end, plane_begin, plane_end,
                             weight_sum, image_real, image_complex=None, stream=None):
        d = _dt()
        _check(load().rick_phase_correct_reduce(
            self.handle, _ptr(grids, d["c64"], "grids", 16), chan_begin, chan_end, plane_begin,
            plane_end, _ptr(weight_sum, d["f64"], "weight_sum", 8),
            _ptr(image_real, d["f32"], "image_real", 8),
            _ptr(image_complex, d["c64"], "image_complex", 16), _stream(stream)),
            "rick_phase_correct_reduce")

    def fft_phase_correct_reduce(self, grids, chan_begin, chan_end, plane_begin, plane_end,
                                 weight_sum, image_real, image_complex=None, gridded_by_plan=False,
                                 stream=None):
        d = _dt()
        _check(load().rick_fft_phase_correct_reduce(
            self.handle, _ptr(grids, d["c64"], "grids", 16), chan_begin, chan_end, plane_begin,
            plane_end, _ptr(weight_sum, d["f64"], "weight_sum", 8),
            _ptr(image_real, d["f32"], "image_real", 4),
            _ptr(image_complex, d["c64"], "image_complex", 8), GRIDDED_BY_PLAN if gridded_by_plan else 0,
            _stream(stream)), "rick_fft_phase_correct_reduce")

    def imaging_weights(self, uvw, chan_scale, weight, flag, nrow, weight_out, stream=None):
        d = _dt()
        _check(load().rick_imaging_weights(
            self.handle, _ptr(uvw, d["f64"], "uvw", 8), _ptr(chan_scale, d["f64"], "chan_scale", 8),
            _ptr(weight, d["f32"], "weight", 4), _ptr(flag, d["u8"], "flag"), int(nrow),
            _ptr(weight_out, d["f32"], "weight_out", 4), _stream(stream)), "rick_imaging_weights")

    def fft_wplanes_columns(self, grids, chan_begin, chan_end, plane_begin, plane_end,
                            gridded_by_plan=False, stream=None):
        d = _dt()
        _check(load().rick_fft_wplanes_columns(
            self.handle, _ptr(grids, d["c64"], "grids", 16), chan_begin, chan_end, plane_begin,
            plane_end, GRIDDED_BY_PLAN if gridded_by_plan else 0, _stream(stream)),
            "rick_fft_wplanes_columns")

    def rows_phase_correct_reduce(self, grids, chan_begin, chan_end, plane_begin, plane_end,
                                  weight_sum, image_real, image_complex=None, gridded_by_plan=False,
                                  stream=None):
        d = _dt()
        _check(load().rick_rows_phase_correct_reduce(
            self.handle, _ptr(grids, d["c64"], "grids", 16), chan_begin, chan_end, plane_begin,
            plane_end, _ptr(weight_sum, d["f64"], "weight_sum", 8),
            _ptr(image_real, d["f32"], "image_real", 4),
            _ptr(image_complex, d["c64"], "image_complex", 8), GRIDDED_BY_PLAN if gridded_by_plan else 0,
            _stream(stream)), "rick_rows_phase_correct_reduce")

    def dirty_image(self, uvw, chan_scale, vis, weight, flag, nrow, image_real,
                    image_complex=None, weight_sum=None, counts=None, stream=None):
        d = _dt()
        _check(load().rick_dirty_image(
            self.handle, *self._vis_args(uvw, chan_scale, vis, weight, flag), int(nrow),
            _ptr(image_real, d["f32"], "image_real", 8),
            _ptr(image_complex, d["c64"], "image_complex", 16),
            _ptr(weight_sum, d["f64"], "weight_sum", 8), _ptr(counts, d["i64"], "counts", 8),
            _stream(stream)), "rick_dirty_image")

    # ---- prediction (degridding) ---------------------------------------------
    def bin_predict(self, uvw, chan_scale, weight, flag, nrow, counts=None, stream=None):
        d = _dt()
        _check(load().rick_bin_predict(
            self.handle, _ptr(uvw, d["f64"], "uvw", 8), _ptr(chan_scale, d["f64"], "chan_scale", 8),
            _ptr(weight, d["f32"], "weight", 4), _ptr(flag, d["u8"], "flag"), int(nrow),
            _ptr(counts, d["i64"], "counts", 8), _stream(stream)), "rick_bin_predict")

    def model_to_wplanes(self, image_real, chan_begin, chan_end, plane_begin, plane_end, grids,
                         stream=None):
        d = _dt()
        _check(load().rick_model_to_wplanes(
            self.handle, _ptr(image_real, d["f32"], "image_real", 8), chan_begin, chan_end,
            plane_begin, plane_end, _ptr(grids, d["c64"], "grids", 16), _stream(stream)),
            "rick_model_to_wplanes")

    def model_fft_wplanes(self, image_real, chan_begin, chan_end, plane_begin, plane_end, grids,
                          pruned=False, stream=None):
        """rick_model_fft_wplanes: model planes and their forward 2-D DFT in one
        call (own transform); pruned=True prunes to the prediction binning."""
        d = _dt()
        _check(load().rick_model_fft_wplanes(
            self.handle, _ptr(image_real, d["f32"], "image_real", 4), chan_begin, chan_end,
            plane_begin, plane_end, _ptr(grids, d["c64"], "grids", 16),
            GRIDDED_BY_PLAN if pruned else 0, _stream(stream)), "rick_model_fft_wplanes")

    def fft_wplanes_forward(self, grids, n_planes, stream=None):
        d = _dt()
        _check(load().rick_fft_wplanes_forward(self.handle, _ptr(grids, d["c64"], "grids", 16),
                                               int(n_planes), _stream(stream)),
               "rick_fft_wplanes_forward")

    def degrid_binned(self, grids, chan_begin, chan_end, plane_begin, plane_end, vis_out,
                      stream=None):
        d = _dt()
        _check(load().rick_degrid_binned(
            self.handle, _ptr(grids, d["c64"], "grids", 16), chan_begin, chan_end, plane_begin,
            plane_end, _ptr(vis_out, d["c64"], "vis_out", 8), _stream(stream)), "rick_degrid_binned")

    def predict(self, uvw, chan_scale, weight, flag, nrow, image_real, vis_out, counts=None,
                stream=None):
        d = _dt()
        _check(load().rick_predict(
            self.handle, _ptr(uvw, d["f64"], "uvw", 8), _ptr(chan_scale, d["f64"], "chan_scale", 8),
            _ptr(weight, d["f32"], "weight", 4), _ptr(flag, d["u8"], "flag"), int(nrow),
            _ptr(image_real, d["f32"], "image_real", 8), _ptr(vis_out, d["c64"], "vis_out", 8),
            _ptr(counts, d["i64"], "counts", 8), _stream(stream)), "rick_predict")

    def capture_graph(self, uvw, chan_scale, vis, weight, flag, nrow, grids, weight_sum,
                      image_real, counts=None):
        """Capture the whole path (all channels and planes) into a CUDA graph."""
        d = _dt()
        h = C.c_void_p()
        _check(load().rick_graph_capture(
            self.handle, *self._vis_args(uvw, chan_scale, vis, weight, flag), int(nrow),
            _ptr(grids, d["c64"], "grids", 16), _ptr(weight_sum, d["f64"], "weight_sum", 8),
            _ptr(image_real, d["f32"], "image_real", 8), _ptr(counts, d["i64"], "counts", 8),
            C.byref(h)), "rick_graph_capture")
        return Graph(h, self)

    def dirty_image_host(self, uvw, chan_scale, vis, weight, flag, image_real, weight_sum=None,
                         counts=None, stream=None):
        """Host buffers in and out (numpy arrays or CPU tensors, contiguous)."""
        def hp(a):
            if a is None:
                return None
            if hasattr(a, "data_ptr"):
                if a.is_cuda or not a.is_contiguous():
                    raise ValueError("host path takes contiguous CPU tensors")
                return a.data_ptr()
            if not a.flags["C_CONTIGUOUS"]:
                raise ValueError("host path takes C-contiguous arrays")
            return a.ctypes.data
        nrow = uvw.shape[0]
        _check(load().rick_dirty_image_host(self.handle, hp(uvw), hp(chan_scale), hp(vis),
                                            hp(weight), hp(flag), int(nrow), hp(image_real),
                                            hp(weight_sum), hp(counts), _stream(stream)),
               "rick_dirty_image_host")


def grid_noalloc(cfg: Config, uvw, chan_scale, vis, weight, flag, nrow, plane_begin, plane_end,
                 grids, weight_sum, counts=None, stream=None):
    """rick_grid without a plan and without any device allocation (see
    rick_grid_noalloc in include/rick.h): for callers that may not allocate
    once running.  Scratch is a fixed 32 MiB device array shared by all calls."""
    d = _dt()
    c = cfg.c()
    _check(load().rick_grid_noalloc(
        C.byref(c), _ptr(uvw, d["f64"], "uvw", 8), _ptr(chan_scale, d["f64"], "chan_scale", 8),
        _ptr(vis, d["c64"], "vis", 8), _ptr(weight, d["f32"], "weight", 4),
        _ptr(flag, d["u8"], "flag"), int(nrow), int(plane_begin), int(plane_end),
        _ptr(grids, d["c64"], "grids", 16), _ptr(weight_sum, d["f64"], "weight_sum", 8),
        _ptr(counts, d["i64"], "counts", 8), _stream(stream)), "rick_grid_noalloc")


class Graph:
    """A captured rick graph (keeps its plan alive)."""

    def __init__(self, handle, plan):
        self.handle = handle
        self.plan = plan

    def launch(self, stream=None):
        _check(load().rick_graph_launch(self.handle, _stream(stream)), "rick_graph_launch")

    def close(self):
        if getattr(self, "handle", None):
            load().rick_graph_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def autotune(cfg: Config, uvw, chan_scale, vis, weight, flag, nrow, chan_range, plane_range,
             grids, reps: int = 3):
    """rick_autotune: returns (best Config, [(tile, threads, grab, ms), ...])."""
    d = _dt()
    c = cfg.c()
    res = (rick_tune_entry * 64)()
    n = C.c_int32()
    best = rick_config()
    _check(load().rick_autotune(
        C.byref(c), _ptr(uvw, d["f64"], "uvw", 8), _ptr(chan_scale, d["f64"], "chan_scale", 8),
        _ptr(vis, d["c64"], "vis", 8), _ptr(weight, d["f32"], "weight", 4),
        _ptr(flag, d["u8"], "flag"), int(nrow), int(chan_range[0]), int(chan_range[1]),
        int(plane_range[0]), int(plane_range[1]), _ptr(grids, d["c64"], "grids", 16), int(reps),
        res, 64, C.byref(n), C.byref(best)), "rick_autotune")
    from dataclasses import replace
    out = replace(cfg, tile=best.tile, grid_threads=best.grid_threads,
                  tiles_per_grab=best.tiles_per_grab)
    table = [(r.tile, r.grid_threads, r.tiles_per_grab, float(r.grid_ms)) for r in res[:min(n.value, 64)]]
    return out, table


# ---- learned kernel (pattern 4) -------------------------------------------

def mlp_param_count(hidden: int) -> int:
    return int(load().rick_mlp_param_count(hidden))


def mlp_forward(params, hidden, inp, out, work=None, stream=None):
    d = _dt()
    n = inp.shape[0]
    _check(load().rick_mlp_forward(_ptr(params, d["f32"], "params", 4), hidden,
                                   _ptr(inp, d["f32"], "in", 4), int(n),
                                   _ptr(out, d["f32"], "out", 4), _ptr(work, d["f32"], "work", 4),
                                   _stream(stream)), "rick_mlp_forward")


def mlp_backward(params, hidden, inp, gout, grad, work, scratch, stream=None):
    d = _dt()
    n = inp.shape[0]
    _check(load().rick_mlp_backward(_ptr(params, d["f32"], "params", 4), hidden,
                                    _ptr(inp, d["f32"], "in", 4), int(n),
                                    _ptr(gout, d["f32"], "gout", 4), _ptr(grad, d["f32"], "grad", 4),
                                    _ptr(work, d["f32"], "work", 4),
                                    _ptr(scratch, d["f32"], "scratch", 4), _stream(stream)),
           "rick_mlp_backward")


def adam_step(params, grad, m, v, lr, step, beta1=0.9, beta2=0.999, eps=1e-8, stream=None):
    d = _dt()
    _check(load().rick_adam_step(_ptr(params, d["f32"]), _ptr(grad, d["f32"]), _ptr(m, d["f32"]),
                                 _ptr(v, d["f32"]), int(params.numel()), float(lr), float(beta1),
                                 float(beta2), float(eps), int(step), _stream(stream)),
           "rick_adam_step")


def mlp_lattice_inputs(n_wplanes, lattice, out, stream=None):
    d = _dt()
    _check(load().rick_mlp_lattice_inputs(int(n_wplanes), int(lattice), _ptr(out, d["f32"]),
                                          _stream(stream)), "rick_mlp_lattice_inputs")


class Learn:
    """Training set-up of the learned kernel on a fixed visibility sample."""

    def __init__(self, cfg: Config, lattice: int, uvw, weight):
        d = _dt()
        self._c = cfg.c()
        h = C.c_void_p()
        _check(load().rick_learn_create(C.byref(self._c), int(lattice), _ptr(uvw, d["f64"], "uvw", 8),
                                        _ptr(weight, d["f32"], "weight", 4), int(uvw.shape[0]),
                                        C.byref(h)), "rick_learn_create")
        self.handle = h
        self.cfg = cfg
        self.lattice = lattice

    def placed(self) -> int:
        return int(load().rick_learn_placed(self.handle))

    def field_grad(self, table, sources, probes, table_grad, loss, image_dft=None,
                   accumulate=False, grad_scale=1.0, stream=None):
        """sources: numpy [ns, 3] (p, q, flux); probes: numpy [np, 2] int pixels."""
        import numpy as np
        d = _dt()
        src = np.ascontiguousarray(sources, dtype=np.float32)
        prb = np.ascontiguousarray(probes, dtype=np.int32)
        _check(load().rick_learn_field_grad(self.handle, _ptr(table, d["f32"]), src.ctypes.data,
                                            src.shape[0], prb.ctypes.data, prb.shape[0],
                                            _ptr(table_grad, d["f32"]), int(bool(accumulate)),
                                            float(grad_scale), _ptr(loss, d["f32"]),
                                            _ptr(image_dft, d["f32"]), _stream(stream)),
               "rick_learn_field_grad")

    def close(self):
        if getattr(self, "handle", None):
            load().rick_learn_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

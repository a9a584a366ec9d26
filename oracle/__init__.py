"""FP64 CPU oracle of the w-stacking imaging path (ctypes wrapper).

TEST INFRASTRUCTURE.  Only the test suite, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py`` may import this package.  The CUDA library
never imports it and shares no code, header or table with it.

The C source ``rick_oracle.c`` states which passage of arXiv 2601.19714 each
function follows (Eq. 1 direct inversion, Eq. 2 w-stacking, Eq. 3 gridding)
and the readings R1-R7 it fixes where the paper is silent.  This wrapper only
marshals numpy arrays.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
from dataclasses import dataclass, field

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "rick_oracle.c")
_LIB_PATH = os.path.join(_HERE, "liboracle.so")

GAUSS, KAISER_BESSEL, LEARNED = 0, 1, 2
_KINDS = {"gauss": GAUSS, "kb": KAISER_BESSEL, "kaiser_bessel": KAISER_BESSEL, "learned": LEARNED}
_WEIGHTINGS = {"natural": 0, "uniform": 1, "briggs": 2}


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (FP64, no FMA contraction) if needed."""
    if (not force and os.path.exists(_LIB_PATH)
            and os.path.getmtime(_LIB_PATH) >= os.path.getmtime(_SRC)):
        return _LIB_PATH
    tmp = _LIB_PATH + f".tmp{os.getpid()}"
    cmd = ["gcc", "-O2", "-std=gnu11", "-ffp-contract=off", "-fno-fast-math", "-fPIC",
           "-shared", _SRC, "-o", tmp, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


class _Cfg(C.Structure):
    _fields_ = [("N", C.c_int32), ("Nw", C.c_int32), ("S", C.c_int32), ("kernel", C.c_int32),
                ("kernel_param", C.c_double), ("fov", C.c_double), ("w_min", C.c_double),
                ("w_max", C.c_double), ("mlp", C.POINTER(C.c_double)),
                ("mlp_hidden", C.c_int32), ("mlp_lattice", C.c_int32),
                ("w_support", C.c_int32), ("w_kernel_param", C.c_double),
                ("weighting", C.c_int32), ("robust", C.c_double), ("Ng", C.c_int32)]


@dataclass
class Config:
    """Imaging parameters in the paper's notation (Sec. 2): mesh side N,
    number of w-planes Nw, kernel support S, field of view, w range."""
    N: int
    Nw: int
    S: int
    kernel: str
    kernel_param: float
    fov: float
    w_min: float
    w_max: float
    mlp: np.ndarray | None = None
    mlp_hidden: int = 64
    mlp_lattice: int = 0
    w_support: int = 0          # even Sw >= 2: Kaiser-Bessel kernel in w over Sw planes
    w_kernel_param: float = 0.0
    weighting: str = "natural"  # or "uniform", "briggs" (R15)
    robust: float = 0.0         # Briggs robustness R
    Ng: int = 0                 # padded mesh side (R16); 0 = N
    _keep: list = field(default_factory=list, repr=False)

    def c(self) -> _Cfg:
        cfg = _Cfg(self.N, self.Nw, self.S, _KINDS[self.kernel], self.kernel_param, self.fov,
                   self.w_min, self.w_max, None, self.mlp_hidden, self.mlp_lattice,
                   self.w_support, self.w_kernel_param, _WEIGHTINGS[self.weighting],
                   self.robust, self.Ng)
        if self.mlp is not None:
            arr = np.ascontiguousarray(self.mlp, dtype=np.float64)
            self._keep = [arr]
            cfg.mlp = arr.ctypes.data_as(C.POINTER(C.c_double))
        return cfg


_lib = None


def lib():
    global _lib
    if _lib is None:
        _lib = C.CDLL(build())
        _declare(_lib)
    return _lib


def _declare(L):
    d, i32, i64, p = C.c_double, C.c_int32, C.c_long, C.c_void_p
    cfgp = C.POINTER(_Cfg)
    L.oracle_bessel_i0.restype = d
    L.oracle_bessel_i0.argtypes = [d]
    L.oracle_kernel_value.restype = d
    L.oracle_kernel_value.argtypes = [C.c_int, d, C.c_int, d]
    L.oracle_gauss_legendre.argtypes = [C.c_int, p, p]
    L.oracle_taper.argtypes = [C.c_int, d, C.c_int, C.c_int, p]
    L.oracle_taper_padded.argtypes = [C.c_int, d, C.c_int, C.c_int, C.c_int, p]
    L.oracle_ifft2.restype = C.c_int
    L.oracle_ifft2.argtypes = [C.c_int, p]
    L.oracle_gelu.restype = d
    L.oracle_gelu.argtypes = [d]
    L.oracle_gelu_grad.restype = d
    L.oracle_gelu_grad.argtypes = [d]
    L.oracle_mlp_param_count.restype = C.c_size_t
    L.oracle_mlp_param_count.argtypes = [C.c_int]
    L.oracle_mlp_forward.argtypes = [p, C.c_int, p, p, p, p]
    L.oracle_mlp_backward.argtypes = [p, C.c_int, p, p, p]
    L.oracle_plane_w.restype = d
    L.oracle_plane_w.argtypes = [cfgp, C.c_int]
    vis_args = [cfgp, p, p, C.c_int, p, p, p, i64]
    L.oracle_place.argtypes = [cfgp, p, p, C.c_int, p, p, i64, p, p, p, p, p, p, p]
    L.oracle_imaging_weights.restype = C.c_int
    L.oracle_imaging_weights.argtypes = [cfgp, p, p, C.c_int, p, p, i64, p]
    L.oracle_planes_total.restype = C.c_int
    L.oracle_planes_total.argtypes = [cfgp]
    L.oracle_kernel_ft.restype = d
    L.oracle_kernel_ft.argtypes = [C.c_int, d, C.c_int, d]
    L.oracle_grid_plane.restype = i64
    L.oracle_grid_plane.argtypes = vis_args + [C.c_int, C.c_int, p]
    L.oracle_channel_stats.argtypes = [cfgp, p, p, C.c_int, p, p, i64, C.c_int, p, p, p]
    L.oracle_image.restype = C.c_int
    L.oracle_image.argtypes = vis_args + [C.c_int, p, p]
    L.oracle_phase_accumulate.argtypes = [cfgp, C.c_int, p, p]
    L.oracle_image_scale.argtypes = [cfgp, d, p, p]
    L.oracle_image_at.restype = C.c_int
    L.oracle_image_at.argtypes = vis_args + [C.c_int, C.c_int, i64, p, p, p]
    L.oracle_dft_at.restype = C.c_int
    L.oracle_dft_at.argtypes = vis_args + [C.c_int, i64, p, p, p]
    novis = [cfgp, p, p, C.c_int, p, p, i64, C.c_int]
    L.oracle_predict.restype = C.c_int
    L.oracle_predict.argtypes = novis + [p, p]
    for name in ("oracle_predict_at", "oracle_predict_dft"):
        getattr(L, name).restype = C.c_int
        getattr(L, name).argtypes = novis + [i64, p, p, p, i64, p, p]
    del i32


def _ptr(a):
    return None if a is None else a.ctypes.data


class _Vis:
    """Contiguous copies of one set of visibilities in the oracle's layout."""

    def __init__(self, uvw, chan_scale, vis, weight, flag):
        self.uvw = np.ascontiguousarray(uvw, dtype=np.float64).reshape(-1, 3)
        self.scale = np.ascontiguousarray(chan_scale, dtype=np.float64).reshape(-1)
        self.C = self.scale.shape[0]
        self.nrow = self.uvw.shape[0]
        v = np.ascontiguousarray(vis, dtype=np.complex64).reshape(self.nrow, self.C)
        self.vis = v.view(np.float32)
        self.weight = np.ascontiguousarray(weight, dtype=np.float32).reshape(self.nrow, self.C)
        self.flag = (None if flag is None else
                     np.ascontiguousarray(flag, dtype=np.uint8).reshape(self.nrow, self.C))

    def args(self):
        return [_ptr(self.uvw), _ptr(self.scale), self.C, _ptr(self.vis), _ptr(self.weight),
                _ptr(self.flag), self.nrow]


# --------------------------------------------------------------------- #
# kernel functions, quadrature, FFT                                       #
# --------------------------------------------------------------------- #

def bessel_i0(x: float) -> float:
    return lib().oracle_bessel_i0(float(x))


def kernel_value(kind: str, param: float, S: int, s: float) -> float:
    return lib().oracle_kernel_value(_KINDS[kind], float(param), int(S), float(s))


def gauss_legendre(n: int):
    x = np.zeros(n)
    w = np.zeros(n)
    lib().oracle_gauss_legendre(n, _ptr(x), _ptr(w))
    return x, w


def taper(kind: str, param: float, S: int, N: int, Ng: int = 0) -> np.ndarray:
    """C(p) = int g(s) cos(2 pi s (p - N/2)/Ng) ds for the N image pixels
    (Ng = N without padding, R16)."""
    out = np.zeros(N)
    lib().oracle_taper_padded(_KINDS[kind], float(param), int(S), int(N), int(Ng or N), _ptr(out))
    return out


def ifft2(a: np.ndarray) -> np.ndarray:
    """Unnormalised inverse 2-D DFT (exponent +) of a square power-of-two array."""
    out = np.ascontiguousarray(a, dtype=np.complex128).copy()
    if lib().oracle_ifft2(out.shape[0], _ptr(out)) != 0:
        raise ValueError("oracle_ifft2: N must be a power of two")
    return out


def gelu(x: float) -> float:
    return lib().oracle_gelu(float(x))


def gelu_grad(x: float) -> float:
    return lib().oracle_gelu_grad(float(x))


def mlp_param_count(H: int) -> int:
    return int(lib().oracle_mlp_param_count(H))


def mlp_forward(params: np.ndarray, H: int, inp) -> np.ndarray:
    prm = np.ascontiguousarray(params, dtype=np.float64)
    x = np.ascontiguousarray(inp, dtype=np.float64)
    out = np.zeros(16)
    lib().oracle_mlp_forward(_ptr(prm), H, _ptr(x), _ptr(out), None, None)
    return out


def mlp_backward(params: np.ndarray, H: int, inp, gout) -> np.ndarray:
    prm = np.ascontiguousarray(params, dtype=np.float64)
    x = np.ascontiguousarray(inp, dtype=np.float64)
    g = np.ascontiguousarray(gout, dtype=np.float64)
    grad = np.zeros_like(prm)
    lib().oracle_mlp_backward(_ptr(prm), H, _ptr(x), _ptr(g), _ptr(grad))
    return grad


# --------------------------------------------------------------------- #
# the imaging path                                                        #
# --------------------------------------------------------------------- #

def plane_w(cfg: Config, k: int) -> float:
    c = cfg.c()
    return lib().oracle_plane_w(C.byref(c), k)


def place(cfg: Config, uvw, chan_scale, weight, flag=None):
    """Per-visibility placement: status, plane k, footprint start (i0, j0),
    fractional offsets (fx, fy); arrays shaped [nrow, C]."""
    v = _Vis(uvw, chan_scale, np.zeros((len(uvw), len(np.atleast_1d(chan_scale))), np.complex64),
             weight, flag)
    shape = (v.nrow, v.C)
    st, k, i0, j0 = (np.zeros(shape, np.int32) for _ in range(4))
    fx, fy, fw = np.zeros(shape), np.zeros(shape), np.zeros(shape)
    c = cfg.c()
    lib().oracle_place(C.byref(c), _ptr(v.uvw), _ptr(v.scale), v.C, _ptr(v.weight), _ptr(v.flag),
                       v.nrow, _ptr(st), _ptr(k), _ptr(i0), _ptr(j0), _ptr(fx), _ptr(fy), _ptr(fw))
    return dict(status=st, k=k, i0=i0, j0=j0, fx=fx, fy=fy, fw=fw)


def planes_total(cfg: Config) -> int:
    """Planes imaged: Nw, or Nw + Sw with a w-kernel."""
    c = cfg.c()
    return lib().oracle_planes_total(C.byref(c))


def kernel_ft(kind: str, param: float, S: int, nu: float) -> float:
    """Continuous Fourier transform of a kernel at frequency nu (cycles per cell)."""
    return lib().oracle_kernel_ft(_KINDS[kind], float(param), int(S), float(nu))


def imaging_weights(cfg: Config, uvw, chan_scale, weight, flag=None) -> np.ndarray:
    """Imaging weights W' [nrow, C] in FP64 (R15): W for natural weighting and
    for visibilities that are not gridded; W / D (uniform) or W / (1 + f^2 D)
    (Briggs) otherwise, D the Hermitian-completed density on the nearest cell."""
    v = _Vis(uvw, chan_scale, np.zeros((len(uvw), len(np.atleast_1d(chan_scale))), np.complex64),
             weight, flag)
    out = np.zeros((v.nrow, v.C), np.float64)
    c = cfg.c()
    rc = lib().oracle_imaging_weights(C.byref(c), _ptr(v.uvw), _ptr(v.scale), v.C, _ptr(v.weight),
                                      _ptr(v.flag), v.nrow, _ptr(out))
    if rc != 0:
        raise ValueError(f"oracle_imaging_weights failed ({rc})")
    return out


def _weights(cfg: Config, uvw, chan_scale, weight, flag):
    """The weights the imaging functions use: the data weights, or the imaging
    weights W' of R15 stored in FP32 (the C functions take them as given)."""
    if cfg.weighting == "natural":
        return weight
    return imaging_weights(cfg, uvw, chan_scale, weight, flag).astype(np.float32)


def channel_stats(cfg: Config, uvw, chan_scale, weight, flag=None, channel=0):
    weight = _weights(cfg, uvw, chan_scale, weight, flag)
    v = _Vis(uvw, chan_scale, np.zeros((len(uvw), len(np.atleast_1d(chan_scale))), np.complex64),
             weight, flag)
    ws = C.c_double()
    ng, nd = C.c_long(), C.c_long()
    c = cfg.c()
    lib().oracle_channel_stats(C.byref(c), _ptr(v.uvw), _ptr(v.scale), v.C, _ptr(v.weight),
                               _ptr(v.flag), v.nrow, channel, C.byref(ws), C.byref(ng),
                               C.byref(nd))
    return ws.value, ng.value, nd.value


def grid_plane(cfg: Config, uvw, chan_scale, vis, weight, flag=None, channel=0, plane=0):
    """Gridded plane ``plane`` of channel ``channel`` (Eq. 3), complex128
    [Ng, Ng] (the mesh; N x N without padding)."""
    v = _Vis(uvw, chan_scale, vis, _weights(cfg, uvw, chan_scale, weight, flag), flag)
    ng = cfg.Ng or cfg.N
    out = np.zeros((ng, ng), np.complex128)
    c = cfg.c()
    n = lib().oracle_grid_plane(C.byref(c), *v.args(), channel, plane, _ptr(out))
    if n < 0:
        raise ValueError("oracle_grid_plane: invalid configuration")
    return out


def mirror(G: np.ndarray) -> np.ndarray:
    """M[j, i] = G[(N - j) mod N, (N - i) mod N]: the cell of (-u, -v) on the
    mesh (cell i sits at u = (i - N/2)/FoV; cell N, the image of cell 0, is
    cell 0 again on the periodic mesh the inverse DFT sees)."""
    G = np.asarray(G)
    N = G.shape[0]
    j = (N - np.arange(N)) % N
    return G[np.ix_(j, j)]


def fold_plane(cfg: Config, uvw, chan_scale, vis, weight, flag=None, channel=0, plane=0):
    """Stored plane ``plane`` under the Hermitian fold, complex128 [N, N].

    The dirty image is the real part of the sum over planes in Eq. 2 and
    Re(z) = Re(conj z); with w_min = -w_max, plane Nw-1-k sits at -w_k, so
    the contribution of plane k' = Nw-1-k equals that of the conjugate of
    its grid mirrored to (-u, -v) on plane k.  Definition, with Nt the
    number of planes imaged (Nw, or Nw + Sw with a w-kernel, whose extended
    set is symmetric about w = 0 as well):
        H_k = G_k + conj(mirror(G_{Nt-1-k}))   for 2k < Nt - 1,
        H_k = G_k                              for 2k = Nt - 1 (odd Nt).
    """
    if cfg.w_min != -cfg.w_max:
        raise ValueError("the fold needs w_min == -w_max")
    nt = planes_total(cfg)
    if not 0 <= 2 * plane <= nt - 1:
        raise ValueError("stored planes are 0 .. ceil(Nt/2) - 1")
    G = grid_plane(cfg, uvw, chan_scale, vis, weight, flag, channel, plane)
    k2 = nt - 1 - plane
    if k2 == plane:
        return G
    return G + np.conj(mirror(grid_plane(cfg, uvw, chan_scale, vis, weight, flag, channel, k2)))


def image(cfg: Config, uvw, chan_scale, vis, weight, flag=None, channel=0):
    """Complex w-stacking dirty image of one channel (O1), complex128 [N, N]
    indexed [q, p] (m row, l column), and the channel's sum of weights."""
    v = _Vis(uvw, chan_scale, vis, _weights(cfg, uvw, chan_scale, weight, flag), flag)
    out = np.zeros((cfg.N, cfg.N), np.complex128)
    ws = C.c_double()
    c = cfg.c()
    rc = lib().oracle_image(C.byref(c), *v.args(), channel, _ptr(out), C.byref(ws))
    if rc != 0:
        raise ValueError(f"oracle_image failed ({rc})")
    return out, ws.value


def ifft2_inplace(a: np.ndarray) -> np.ndarray:
    """ifft2 without the copy: ``a`` (C-contiguous complex128, square, power of
    two) is overwritten by its unnormalised inverse 2-D DFT and returned."""
    if a.dtype != np.complex128 or not a.flags.c_contiguous:
        raise ValueError("ifft2_inplace needs a C-contiguous complex128 array")
    if lib().oracle_ifft2(a.shape[0], _ptr(a)) != 0:
        raise ValueError("oracle_ifft2: N must be a power of two")
    return a


def phase_accumulate(cfg: Config, plane: int, F: np.ndarray, img: np.ndarray) -> None:
    """One term of Eq. 2's sum over planes: img[q, p] += F[q, p] exp(+2 pi i
    w_plane (n - 1)) over the N x N image (F: the transformed plane, complex128
    [Ng, Ng]; img: complex128 [N, N], updated in place)."""
    if F.dtype != np.complex128 or img.dtype != np.complex128 or not (F.flags.c_contiguous and
                                                                      img.flags.c_contiguous):
        raise ValueError("phase_accumulate needs C-contiguous complex128 arrays")
    c = cfg.c()
    lib().oracle_phase_accumulate(C.byref(c), int(plane), _ptr(F), _ptr(img))


def image_scale(cfg: Config, weight_sum: float, img: np.ndarray) -> None:
    """Eq. 2's normalisation of a summed image, in place: times (-1)^(p+q) n /
    (sum W C(p) C(q) C_w)."""
    if img.dtype != np.complex128 or not img.flags.c_contiguous:
        raise ValueError("image_scale needs a C-contiguous complex128 array")
    Ct = taper(cfg.kernel if cfg.kernel != "learned" else "kb", cfg.kernel_param, cfg.S, cfg.N, cfg.Ng)
    c = cfg.c()
    lib().oracle_image_scale(C.byref(c), float(weight_sum), _ptr(Ct), _ptr(img))


def image_at(cfg: Config, uvw, chan_scale, vis, weight, flag=None, channel=0, p=(), q=(),
             plane=-1):
    """O1 at pixels (p, q) evaluated visibility by visibility (no FFT).  With
    ``plane >= 0``: the transformed plane F_plane[q, p] before the phase screen."""
    v = _Vis(uvw, chan_scale, vis, _weights(cfg, uvw, chan_scale, weight, flag), flag)
    pp = np.ascontiguousarray(p, dtype=np.int32)
    qq = np.ascontiguousarray(q, dtype=np.int32)
    out = np.zeros(pp.shape[0], np.complex128)
    c = cfg.c()
    rc = lib().oracle_image_at(C.byref(c), *v.args(), channel, plane, pp.shape[0], _ptr(pp),
                               _ptr(qq), _ptr(out))
    if rc != 0:
        raise ValueError(f"oracle_image_at failed ({rc})")
    return out


def dft_at(cfg: Config, uvw, chan_scale, vis, weight, flag=None, channel=0, p=(), q=()):
    """O2: direct Fourier inversion of Eq. 1 at pixels (p, q), complex (with
    the same imaging weights as O1)."""
    v = _Vis(uvw, chan_scale, vis, _weights(cfg, uvw, chan_scale, weight, flag), flag)
    pp = np.ascontiguousarray(p, dtype=np.int32)
    qq = np.ascontiguousarray(q, dtype=np.int32)
    out = np.zeros(pp.shape[0], np.complex128)
    c = cfg.c()
    rc = lib().oracle_dft_at(C.byref(c), *v.args(), channel, pp.shape[0], _ptr(pp), _ptr(qq),
                             _ptr(out))
    if rc != 0:
        raise ValueError(f"oracle_dft_at failed ({rc})")
    return out


# --------------------------------------------------------------------- #
# prediction (degridding)                                                 #
# --------------------------------------------------------------------- #

def _novis_args(uvw, chan_scale, weight, flag):
    nrow = len(uvw)
    v = _Vis(uvw, chan_scale, np.zeros((nrow, len(np.atleast_1d(chan_scale))), np.complex64),
             weight, flag)
    return v, [_ptr(v.uvw), _ptr(v.scale), v.C, _ptr(v.weight), _ptr(v.flag), v.nrow]


def predict(cfg: Config, uvw, chan_scale, weight, flag=None, channel=0, image=None):
    """O1 prediction of channel ``channel`` from the real model image [N, N]
    (row q, column p): complex128 [nrow], zero where a visibility is not gridded."""
    v, args = _novis_args(uvw, chan_scale, weight, flag)
    J = np.ascontiguousarray(image, dtype=np.float64)
    assert J.shape == (cfg.N, cfg.N)
    out = np.zeros(v.nrow, np.complex128)
    c = cfg.c()
    rc = lib().oracle_predict(C.byref(c), *args, channel, _ptr(J), _ptr(out))
    if rc != 0:
        raise ValueError(f"oracle_predict failed ({rc})")
    return out


def _sources_call(fn, cfg, uvw, chan_scale, weight, flag, channel, p, q, flux, rows):
    v, args = _novis_args(uvw, chan_scale, weight, flag)
    pp = np.ascontiguousarray(p, dtype=np.int32)
    qq = np.ascontiguousarray(q, dtype=np.int32)
    ff = np.ascontiguousarray(flux, dtype=np.float64)
    rr = np.ascontiguousarray(np.arange(v.nrow) if rows is None else rows, dtype=np.int64)
    out = np.zeros(rr.shape[0], np.complex128)
    c = cfg.c()
    rc = fn(C.byref(c), *args, channel, pp.shape[0], _ptr(pp), _ptr(qq), _ptr(ff), rr.shape[0],
            _ptr(rr), _ptr(out))
    if rc != 0:
        raise ValueError(f"prediction failed ({rc})")
    return out


def predict_at(cfg: Config, uvw, chan_scale, weight, flag=None, channel=0, p=(), q=(), flux=(),
               rows=None):
    """O1 prediction for a point-source model on pixel centres, visibility by
    visibility (no FFT): the same values as ``predict`` on that image."""
    return _sources_call(lib().oracle_predict_at, cfg, uvw, chan_scale, weight, flag, channel,
                         p, q, flux, rows)


def predict_dft(cfg: Config, uvw, chan_scale, weight, flag=None, channel=0, p=(), q=(), flux=(),
                rows=None):
    """O2 prediction: Eq. 1 summed over the point sources directly."""
    return _sources_call(lib().oracle_predict_dft, cfg, uvw, chan_scale, weight, flag, channel,
                         p, q, flux, rows)

"""Seeded synthetic observations for the w-stacking imager.

This module makes inputs only: antenna layouts, earth-rotation (u, v, w)
tracks, point-source skies, visibilities, weights and flags.  It holds none of
the imaging arithmetic (no gridding, transform, phase screen or reduction) and
is imported both by the tests that feed the CUDA library and by those that
feed the oracle, so that both sides see identical inputs.

Random numbers come from numpy's Philox-4x32 counter-based generator
(Salmon et al. 2011), keyed by the seed and a stream name, so that any part
of a workload can be regenerated on its own.

Visibilities follow the measurement equation (arXiv 2601.19714, Eq. 1) for a
sky of point sources: V(u, v, w) = sum_s A_s / n_s exp(-2 pi i (u l_s + v m_s
+ w (n_s - 1))), n_s = sqrt(1 - l_s^2 - m_s^2).
"""
from __future__ import annotations

import hashlib
import math
from dataclasses import dataclass

import numpy as np

C_LIGHT = 299_792_458.0

MEERKAT_LAT_DEG = -30.7
LOFAR_LAT_DEG = 52.9


def rng(seed: int, stream: str) -> np.random.Generator:
    """A Philox generator keyed by (seed, stream name)."""
    h = int.from_bytes(hashlib.sha256(stream.encode()).digest()[:8], "little")
    return np.random.Generator(np.random.Philox(key=[seed & (2**64 - 1), h]))


# --------------------------------------------------------------------- #
# geometry                                                                #
# --------------------------------------------------------------------- #

def disk_points(g: np.random.Generator, n: int, radius: float) -> np.ndarray:
    """n points uniform in area in a disk of the given radius: [n, 2]."""
    r = radius * np.sqrt(g.random(n))
    t = 2.0 * math.pi * g.random(n)
    return np.stack([r * np.cos(t), r * np.sin(t)], axis=1)


def stations_enu(seed: int, n: int, diameter_m: float, core_n: int = 0,
                 core_diameter_m: float = 0.0) -> np.ndarray:
    """Station positions (east, north, up) in metres: n stations uniform in a
    disk of the given diameter, of which ``core_n`` sit in a central core."""
    g = rng(seed, "stations")
    outer = disk_points(g, n - core_n, 0.5 * diameter_m)
    core = disk_points(g, core_n, 0.5 * core_diameter_m) if core_n else np.zeros((0, 2))
    en = np.concatenate([core, outer], axis=0)
    up = g.normal(0.0, 5.0, size=(n, 1))
    return np.concatenate([en, up], axis=1)


def baselines(enu: np.ndarray) -> np.ndarray:
    """All n(n-1)/2 baseline vectors b = x_j - x_i (i < j), ENU metres."""
    i, j = np.triu_indices(enu.shape[0], k=1)
    return enu[j] - enu[i]


def earth_rotation_uvw(bl_enu: np.ndarray, lat_deg: float, dec_deg: float, n_steps: int,
                       duration_h: float) -> np.ndarray:
    """(u, v, w) in metres for every (time step, baseline), time-major rows.

    Textbook earth-rotation synthesis (Thompson, Moran & Swenson, Ch. 4):
    ENU -> equatorial (X, Y, Z) by the latitude, then rotation by the hour
    angle H and declination d:
        u =  sin H X + cos H Y
        v = -sin d cos H X + sin d sin H Y + cos d Z
        w =  cos d cos H X - cos d sin H Y + sin d Z
    The track is symmetric about transit (H from -duration/2 to +duration/2)."""
    lat = math.radians(lat_deg)
    dec = math.radians(dec_deg)
    E, N, U = bl_enu[:, 0], bl_enu[:, 1], bl_enu[:, 2]
    X = -math.sin(lat) * N + math.cos(lat) * U
    Y = E
    Z = math.cos(lat) * N + math.sin(lat) * U
    half = 0.5 * duration_h * (2.0 * math.pi / 24.0)
    H = np.linspace(-half, half, n_steps) if n_steps > 1 else np.zeros(1)
    sH, cH = np.sin(H)[:, None], np.cos(H)[:, None]
    sd, cd = math.sin(dec), math.cos(dec)
    u = sH * X + cH * Y
    v = -sd * cH * X + sd * sH * Y + cd * Z
    w = cd * cH * X - cd * sH * Y + sd * Z
    return np.stack([u, v, w], axis=-1).reshape(-1, 3)


# --------------------------------------------------------------------- #
# skies, weights, flags                                                   #
# --------------------------------------------------------------------- #

def point_sources(seed: int, n: int, fov: float, flux: str = "uniform", lo: float = 0.1,
                  hi: float = 1.0, inner: float = 1.0) -> np.ndarray:
    """[n, 3] (l, m, A): positions uniform in the square |l|, |m| < inner*fov/2.
    flux: 'uniform' U[lo, hi]; 'powerlaw' N(>A) ~ A^-1.5 on [lo, hi];
    'loguniform' log-uniform on [lo, hi]."""
    g = rng(seed, "sources")
    lm = (g.random((n, 2)) - 0.5) * fov * inner
    x = g.random(n)
    if flux == "uniform":
        a = lo + (hi - lo) * x
    elif flux == "powerlaw":
        # inverse CDF of p(A) ~ A^-2.5 on [lo, hi]
        a = (lo ** -1.5 - x * (lo ** -1.5 - hi ** -1.5)) ** (-1.0 / 1.5)
    elif flux == "loguniform":
        a = np.exp(math.log(lo) + x * (math.log(hi) - math.log(lo)))
    else:
        raise ValueError(flux)
    return np.concatenate([lm, a[:, None]], axis=1)


def flags(seed: int, nrow: int, fractions) -> np.ndarray:
    """Bernoulli flags [nrow, C] (uint8), channel c flagged with probability fractions[c]."""
    g = rng(seed, "flags")
    f = np.asarray(fractions, dtype=np.float64)[None, :]
    return (g.random((nrow, f.shape[1])) < f).astype(np.uint8)


# --------------------------------------------------------------------- #
# visibilities (Eq. 1, forward)                                           #
# --------------------------------------------------------------------- #

def predict(uvw_lambda: np.ndarray, chan_scale: np.ndarray, sources: np.ndarray,
            block: int = 1 << 16) -> np.ndarray:
    """Visibilities [nrow, C] complex64 of a point-source sky, evaluated in
    FP64 on the CPU and rounded once."""
    uvw = np.asarray(uvw_lambda, dtype=np.float64)
    sc = np.asarray(chan_scale, dtype=np.float64)
    l, m, a = sources[:, 0], sources[:, 1], sources[:, 2]
    n = np.sqrt(1.0 - l * l - m * m)
    d = -(l * l + m * m) / (1.0 + n)
    out = np.empty((uvw.shape[0], sc.shape[0]), np.complex64)
    for r0 in range(0, uvw.shape[0], block):
        u = uvw[r0:r0 + block]
        ph = u[:, 0:1] * l[None] + u[:, 1:2] * m[None] + u[:, 2:3] * d[None]   # [rows, S] turns
        acc = np.zeros((u.shape[0], sc.shape[0]), np.complex128)
        for c, s in enumerate(sc):
            t = ph * s
            t = t - np.floor(t + 0.5)
            acc[:, c] = (np.exp(-2j * math.pi * t) * (a / n)[None]).sum(axis=1)
        out[r0:r0 + u.shape[0]] = acc
    return out


def predict_torch(uvw_lambda, chan_scale: np.ndarray, sources: np.ndarray, device="cuda",
                  src_block: int = 8):
    """Visibilities [nrow, C] complex64 on ``device`` (a torch tensor) for large
    workloads.  The phase of each (row, source) at the reference frequency is
    formed in FP64 and split into a base and a per-channel step, reduced to
    whole turns in FP64; the per-channel phasors then follow by complex64
    multiplication (channels are evenly spaced in frequency).  Accuracy
    ~1e-6 relative to ``predict`` -- input synthesis only."""
    import torch
    uvw = torch.as_tensor(np.asarray(uvw_lambda, np.float64), device=device)
    sc = np.asarray(chan_scale, dtype=np.float64)
    nchan = sc.shape[0]
    step = (sc[-1] - sc[0]) / (nchan - 1) if nchan > 1 else 0.0
    if nchan > 2 and not np.allclose(np.diff(sc), step, rtol=1e-9, atol=0):
        raise ValueError("predict_torch needs evenly spaced channels")
    l, m, a = sources[:, 0], sources[:, 1], sources[:, 2]
    n = np.sqrt(1.0 - l * l - m * m)
    d = -(l * l + m * m) / (1.0 + n)
    out = torch.zeros((uvw.shape[0], nchan), dtype=torch.complex64, device=device)
    two_pi = 2.0 * math.pi
    for s0 in range(0, sources.shape[0], src_block):
        s1 = min(s0 + src_block, sources.shape[0])
        lmd = torch.as_tensor(np.stack([l[s0:s1], m[s0:s1], d[s0:s1]]), device=device)
        ph = uvw @ lmd                                   # [nrow, nb] turns at scale 1, FP64
        base = ph * sc[0]
        base = base - torch.floor(base + 0.5)
        inc = ph * step
        inc = inc - torch.floor(inc + 0.5)
        amp = torch.as_tensor((a / n)[s0:s1], dtype=torch.float32, device=device)
        z = torch.polar(amp.expand_as(base).contiguous(), (-two_pi * base).float())
        r = torch.polar(torch.ones_like(amp).expand_as(inc).contiguous(), (-two_pi * inc).float())
        for c in range(nchan):
            out[:, c] += z.sum(dim=1)
            if c + 1 < nchan:
                z = z * r
    return out


# --------------------------------------------------------------------- #
# observations                                                            #
# --------------------------------------------------------------------- #

@dataclass
class Observation:
    """One synthetic measurement set.  uvw are wavelengths at the reference
    frequency freqs[0]; channel c scales them by chan_scale[c]."""
    uvw: np.ndarray          # [nrow, 3] float64
    chan_scale: np.ndarray   # [C] float64
    vis: object              # [nrow, C] complex64 (numpy, or torch on a device)
    weight: np.ndarray       # [nrow, C] float32
    flag: np.ndarray | None  # [nrow, C] uint8 or None
    sources: np.ndarray      # [ns, 3] (l, m, A)
    freqs: np.ndarray        # [C] Hz

    @property
    def nrow(self) -> int:
        return self.uvw.shape[0]

    @property
    def nchan(self) -> int:
        return self.chan_scale.shape[0]


def band(f_lo: float, f_hi: float, nchan: int) -> np.ndarray:
    """Centres of nchan equal sub-bands covering [f_lo, f_hi]."""
    width = (f_hi - f_lo) / nchan
    return f_lo + (np.arange(nchan) + 0.5) * width


def disk_observation(seed: int, nvis: int, N: int, fov: float, w_range: float, n_src: int = 5,
                     flux=("uniform", 0.1, 1.0), inner: float = 1.0, radius_frac: float = 0.45,
                     weights: str = "unit") -> Observation:
    """u, v uniform in a disk of radius radius_frac*N/fov wavelengths, w uniform in
    [-w_range, w_range], one channel, point sources uniform in the field."""
    g = rng(seed, "uvw")
    uv = disk_points(g, nvis, radius_frac * N / fov)
    w = (2.0 * g.random(nvis) - 1.0) * w_range
    uvw = np.concatenate([uv, w[:, None]], axis=1)
    src = point_sources(seed, n_src, fov, flux[0], flux[1], flux[2], inner)
    scale = np.ones(1)
    wt = (np.ones((nvis, 1), np.float32) if weights == "unit"
          else (0.5 + rng(seed, "weights").random((nvis, 1))).astype(np.float32))
    return Observation(uvw, scale, predict(uvw, scale, src), wt, None, src, np.ones(1))


def array_observation(seed: int, enu: np.ndarray, lat_deg: float, n_steps: int, duration_h: float,
                      freqs: np.ndarray, sources: np.ndarray, flag_fractions, weights: str = "unit",
                      device: str | None = None, w_limit: float | None = None,
                      row_fraction: float = 1.0) -> Observation:
    """Earth-rotation synthesis of an array pointed at dec = latitude (the
    field transits the zenith), time-major rows.  With ``device`` the
    visibilities are predicted by ``predict_torch`` on that device.  With
    row_fraction < 1 a seeded subset of the rows is kept (before flags,
    weights and visibilities are drawn)."""
    uvw_m = earth_rotation_uvw(baselines(enu), lat_deg, lat_deg, n_steps, duration_h)
    if row_fraction < 1.0:
        keep = rng(seed, "row-subset").random(uvw_m.shape[0]) < row_fraction
        uvw_m = uvw_m[keep]
    lam0 = C_LIGHT / freqs[0]
    uvw = uvw_m / lam0
    scale = freqs / freqs[0]
    nrow, nchan = uvw.shape[0], scale.shape[0]
    fl = flags(seed, nrow, flag_fractions) if flag_fractions is not None else None
    if w_limit is not None:
        over = np.abs(uvw[:, 2:3] * scale[None, :]) > w_limit
        fl = np.maximum(fl if fl is not None else 0, over.astype(np.uint8)).astype(np.uint8)
    if weights == "unit":
        wt = np.ones((nrow, nchan), np.float32)
    else:
        wt = (0.5 + rng(seed, "weights").random((nrow, nchan))).astype(np.float32)
    vis = (predict(uvw, scale, sources) if device is None
           else predict_torch(uvw, scale, sources, device=device))
    return Observation(uvw, scale, vis, wt, fl, sources, np.asarray(freqs, np.float64))


def w_extent(obs: Observation) -> float:
    """max |w| over all channels, wavelengths."""
    return float(np.abs(obs.uvw[:, 2]).max() * np.abs(obs.chan_scale).max())

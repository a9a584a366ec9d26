"""Helpers shared by the GPU tests: move a synthetic observation to the
device, build a plan from the imaging parameters, run the library's path
through the C ABI, and compare with the oracle."""
from __future__ import annotations

import numpy as np

from visgen.workloads import Imaging


def plan_config(img: Imaging, nchan: int, **kw):
    from paper_2601_19714_gb300 import rick
    kern = {"gauss": "gauss", "kb": "kb", "learned": "table"}[img.kernel]
    return rick.Config(N=img.N, n_wplanes=img.Nw, support=img.S, n_channels=nchan,
                       fov_rad=img.fov, w_min=img.w_min, w_max=img.w_max, kernel=kern,
                       kernel_param=img.kernel_param, **kw)


def oracle_config(orc, img: Imaging, **kw):
    d = dict(N=img.N, Nw=img.Nw, S=img.S, kernel=img.kernel, kernel_param=img.kernel_param,
             fov=img.fov, w_min=img.w_min, w_max=img.w_max)
    d.update(kw)
    return orc.Config(**d)


def to_device(obs, device="cuda"):
    import torch
    vis = obs.vis if isinstance(obs.vis, torch.Tensor) else torch.from_numpy(np.ascontiguousarray(obs.vis))
    return dict(
        uvw=torch.from_numpy(np.ascontiguousarray(obs.uvw)).to(device),
        chan_scale=torch.from_numpy(np.ascontiguousarray(obs.chan_scale)).to(device),
        vis=vis.to(device).contiguous(),
        weight=torch.from_numpy(np.ascontiguousarray(obs.weight)).to(device),
        flag=None if obs.flag is None else torch.from_numpy(np.ascontiguousarray(obs.flag)).to(device),
        nrow=obs.uvw.shape[0],
    )


def host_vis(obs):
    """The visibilities as numpy (copied back if they were made on the device)."""
    v = obs.vis
    if hasattr(v, "cpu"):
        return v.cpu().numpy()
    return v


def run_path(plan, dev, nchan, N, Nw, complex_out=False):
    """grid -> fft -> phase through the three spec calls; returns numpy
    (image_real [C,N,N], image_complex or None, weight_sum [C], counts [2]).
    Nw is the number of w-planes; the plan stores ceil(Nw/2) of them when it
    folds."""
    import torch
    Nw = plan.cfg.stored_planes if plan.cfg.n_wplanes == Nw else Nw
    Ng = plan.cfg.Ng if plan.cfg.N == N else N
    grids = torch.empty((nchan, Nw, Ng, Ng), dtype=torch.complex64, device="cuda")
    wsum = torch.empty(nchan, dtype=torch.float64, device="cuda")
    counts = torch.empty(2, dtype=torch.int64, device="cuda")
    img = torch.zeros((nchan, N, N), dtype=torch.float32, device="cuda")
    imc = torch.zeros((nchan, N, N), dtype=torch.complex64, device="cuda") if complex_out else None
    plan.grid(dev["uvw"], dev["chan_scale"], dev["vis"], dev["weight"], dev["flag"], dev["nrow"],
              0, Nw, grids, wsum, counts)
    plan.fft_wplanes(grids, nchan * Nw)
    plan.phase_correct_reduce(grids, 0, nchan, 0, Nw, wsum, img, imc)
    torch.cuda.synchronize()
    plan.sync_status()
    return (img.cpu().numpy(), None if imc is None else imc.cpu().numpy(),
            wsum.cpu().numpy(), counts.cpu().numpy())


def rel_err(a, ref):
    ref = np.asarray(ref)
    peak = np.abs(ref).max()
    return float(np.abs(np.asarray(a) - ref).max() / peak)


def taper_gain(taper):
    """A(p, q) = C(p) C(q) / C(N/2)^2: the factor the taper correction divides
    pixel (p, q) by, relative to the field centre."""
    t = np.asarray(taper, dtype=np.float64)
    c0 = t[t.shape[0] // 2]
    return np.outer(t, t) / (c0 * c0)


def image_errors(got, ref, taper, inner=1e-2):
    """Errors of a dirty image against the oracle.

    full      max|delta| / peak over every pixel;
    weighted  max|delta| A / max|ref| A  -- the error of the image before the
              per-pixel division by the taper, which is where FP32 rounding
              arises; the division itself multiplies it by up to 1/A;
    inner     max|delta| / peak over pixels with A >= inner, i.e. where the
              taper correction amplifies by at most 1/inner."""
    got = np.asarray(got)
    ref = np.asarray(ref)
    A = taper_gain(taper)
    d = np.abs(got - ref)
    peak = np.abs(ref).max()
    m = A >= inner
    return dict(full=float(d.max() / peak),
                weighted=float((d * A).max() / (np.abs(ref) * A).max()),
                inner=float(d[m].max() / peak))


def assert_image_close(got, ref, taper, tol=1e-5, full=False):
    e = image_errors(got, ref, taper)
    assert e["weighted"] <= tol and e["inner"] <= tol, e
    if full:
        assert e["full"] <= tol, e
    return e

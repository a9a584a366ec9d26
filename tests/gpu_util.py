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
    (image_real [C,N,N], image_complex or None, weight_sum [C], counts [2])."""
    import torch
    grids = torch.empty((nchan, Nw, N, N), dtype=torch.complex64, device="cuda")
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

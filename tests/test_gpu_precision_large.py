"""Precision stress at the large workload's size (pattern 1): MeerKAT layout,
8 h track of 5800 steps, 16384^2 grid, 32 w-planes, Kaiser-Bessel S = 8, the
lowest and highest of the 128 channels over 856-1712 MHz, on a seeded 1 %
subsample of the rows.  For both precision variants (FP64 placement and
phase with FP32 accumulation; all FP32) every transformed plane F_k is
compared with the oracle at 16 probe pixels before the reduction, and the
final image at the same pixels after it.  The FP64-index/phase variant must
match within 1e-5; the all-FP32 variant's error is reported and must be the
larger one (its placement loses the fraction of a cell FP32 cannot hold at
x ~ 8192)."""
import json

import numpy as np
import pytest

from tests.gpu_util import oracle_config, plan_config, taper_gain, to_device
from visgen.workloads import meerkat_large

pytestmark = pytest.mark.gpu


def _probes(N, taper, count=16, seed=5):
    """The field centre and seeded pixels where the taper gain is >= 1e-2."""
    A = taper_gain(taper)
    g = np.random.default_rng(seed)
    out = [(N // 2, N // 2)]
    while len(out) < count:
        p, q = g.integers(0, N, 2)
        if A[q, p] >= 1e-2:
            out.append((int(p), int(q)))
    return np.array(out, dtype=np.int32)


def test_large_grid_precision_variants(orc):
    import torch
    import __graft_entry__
    __graft_entry__.build()
    from paper_2601_19714_gb300 import rick
    img, obs = meerkat_large(0, channels=slice(0, 128, 127), row_fraction=0.01, device="cuda")
    obs.vis = obs.vis.cpu().numpy()
    C, N, Nw = obs.nchan, img.N, img.Nw
    dev = to_device(obs)
    ocfg = oracle_config(orc, img)
    report = {}
    for prec in ("fp64idx", "fp32"):
        plan = rick.Plan(plan_config(img, C, precision=prec))
        taper = plan.taper()
        pr = _probes(N, taper)
        p, q = pr[:, 0], pr[:, 1]
        wsum = torch.empty(C, dtype=torch.float64, device="cuda")
        plan.bin(dev["uvw"], dev["chan_scale"], dev["vis"], dev["weight"], dev["flag"], obs.nrow, wsum)
        grids = torch.empty((1, Nw, N, N), dtype=torch.complex64, device="cuda")
        image = torch.zeros((1, N, N), dtype=torch.float32, device="cuda")
        errs = {}
        for c in range(C):
            plan.grid_binned(c, c + 1, 0, Nw, grids)
            plan.fft_wplanes(grids, Nw)
            F = grids[0][:, torch.from_numpy(q).long().cuda(), torch.from_numpy(p).long().cuda()].cpu().numpy()
            Fo = np.stack([orc.image_at(ocfg, obs.uvw, obs.chan_scale, obs.vis, obs.weight, obs.flag,
                                        channel=c, p=p, q=q, plane=k) for k in range(Nw)])
            e_plane = float(np.abs(F - Fo).max() / np.abs(Fo).max())
            image.zero_()
            plan.phase_correct_reduce(grids, c, c + 1, 0, Nw, wsum, image)
            I = image[0][torch.from_numpy(q).long().cuda(), torch.from_numpy(p).long().cuda()].cpu().numpy()
            Io = orc.image_at(ocfg, obs.uvw, obs.chan_scale, obs.vis, obs.weight, obs.flag,
                              channel=c, p=p, q=q).real
            e_image = float(np.abs(I - Io).max() / np.abs(Io).max())
            errs[f"channel_{c}"] = {"planes_max_rel": e_plane, "image_max_rel": e_image}
        report[prec] = errs
        del grids, image, plan
        torch.cuda.empty_cache()
    print(json.dumps({"rows": int(obs.nrow), "visibilities": int(obs.nrow * C), **report}, indent=1))
    for c in range(C):
        k = f"channel_{c}"
        assert report["fp64idx"][k]["planes_max_rel"] <= 1e-5
        assert report["fp64idx"][k]["image_max_rel"] <= 1e-5
        assert report["fp32"][k]["image_max_rel"] > report["fp64idx"][k]["image_max_rel"]

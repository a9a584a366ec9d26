"""Autotuner cache for the gridder's launch shape (pattern 2).

``rick_autotune`` (native, in librick) times every valid (tile side, CTA size,
tiles per grab) on the caller's own data.  This module keys the winners by
what decides them -- grid side, support, planes, channels, kernel, the
Hermitian fold, the visibility density per 64x64 tile per stored plane (as a
power of two) and the GPU name -- and keeps them in a JSON file so that later plans reuse them.
"""
from __future__ import annotations

import json
import math
import os
from dataclasses import replace

from . import rick


def density_class(cfg: rick.Config, n_vis: int) -> int:
    tiles = cfg.n_channels * cfg.stored_planes * (cfg.N // 64) ** 2
    return int(round(math.log2(max(n_vis, 1) / tiles + 1e-9)))


def cache_key(cfg: rick.Config, n_vis: int, gpu_name: str) -> str:
    return (f"N{cfg.N}-S{cfg.support}-Nw{cfg.n_wplanes}-C{cfg.n_channels}-{cfg.kernel}-"
            f"{'fold-' if cfg.hermitian_fold else ''}"
            f"d{density_class(cfg, n_vis)}-{gpu_name.replace(' ', '_')}")


def tuned(cfg: rick.Config, n_vis: int, cache_path: str, tune_fn=None, gpu_name: str | None = None):
    """The cached shape for this problem class, or ``tune_fn()`` (which must
    return (best Config, table)) run once and stored.  Returns (Config, entry)."""
    if gpu_name is None:
        import torch
        gpu_name = torch.cuda.get_device_name()
    key = cache_key(cfg, n_vis, gpu_name)
    cache = {}
    if os.path.exists(cache_path):
        with open(cache_path) as f:
            cache = json.load(f)
    if key in cache:
        e = cache[key]
        return replace(cfg, tile=e["tile"], grid_threads=e["grid_threads"],
                       tiles_per_grab=e["tiles_per_grab"]), e
    if tune_fn is None:
        return cfg, None
    best, table = tune_fn()
    e = {"tile": best.tile, "grid_threads": best.grid_threads,
         "tiles_per_grab": best.tiles_per_grab, "table": table}
    cache[key] = e
    os.makedirs(os.path.dirname(os.path.abspath(cache_path)), exist_ok=True)
    tmp = cache_path + ".tmp"
    with open(tmp, "w") as f:
        json.dump(cache, f, indent=1)
    os.replace(tmp, cache_path)
    return best, e

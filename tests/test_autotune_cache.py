"""The autotuner's JSON cache (host logic only; the timing itself runs on the GPU)."""
import json

from paper_2601_19714_gb300 import autotune, rick


def _cfg(**kw):
    d = dict(N=4096, n_wplanes=32, support=8, n_channels=16, fov_rad=0.026, w_min=-4e4,
             w_max=4e4, kernel="kb", kernel_param=12.25)
    d.update(kw)
    return rick.Config(**d)


def test_density_class_scales_with_visibilities():
    cfg = _cfg()
    tiles = 16 * 32 * 64 * 64
    assert autotune.density_class(cfg, tiles) == 0
    assert autotune.density_class(cfg, 16 * tiles) == 4
    assert autotune.density_class(_cfg(n_channels=1), 16 * tiles) == 8


def test_cache_round_trip(tmp_path):
    path = str(tmp_path / "tune.json")
    cfg = _cfg()
    calls = []

    def tune():
        calls.append(1)
        from dataclasses import replace
        return replace(cfg, tile=32, grid_threads=128, tiles_per_grab=2), [(32, 128, 2, 1.5)]

    best, e = autotune.tuned(cfg, 30_000_000, path, tune, gpu_name="NVIDIA GB300")
    assert (best.tile, best.grid_threads, best.tiles_per_grab) == (32, 128, 2) and calls == [1]
    again, e2 = autotune.tuned(cfg, 30_000_000, path, tune, gpu_name="NVIDIA GB300")
    assert calls == [1] and (again.tile, again.grid_threads, again.tiles_per_grab) == (32, 128, 2)
    # a different problem class or GPU is tuned separately
    autotune.tuned(_cfg(N=8192), 30_000_000, path, tune, gpu_name="NVIDIA GB300")
    autotune.tuned(cfg, 30_000_000, path, tune, gpu_name="Other GPU")
    assert calls == [1, 1, 1]
    assert len(json.load(open(path))) == 3


def test_untuned_without_tuner_returns_input(tmp_path):
    cfg = _cfg()
    out, e = autotune.tuned(cfg, 1000, str(tmp_path / "none.json"), None, gpu_name="x")
    assert out is cfg and e is None

"""GB300-native w-stacking imager: the hot path of arXiv 2601.19714 (RICK)
behind the C ABI of ``include/rick.h``, with a thin Python binding.

    from paper_2601_19714_gb300 import rick
    plan = rick.Plan(rick.Config(N=4096, n_wplanes=32, support=8, ...))
    plan.grid(...); plan.fft_wplanes(...); plan.phase_correct_reduce(...)
"""
from . import rick  # noqa: F401
from ._build import build  # noqa: F401

__all__ = ["rick", "build"]

"""Host-side helpers of bench.py that feed the reported numbers: the count of
reached tiles (the algorithmic bytes of the pruned stages) against a direct
per-tile evaluation of the gridder's rule, and the stage byte / flop formulas
on a hand-counted case."""
import numpy as np

import bench


def _reached_direct(cnt, NT):
    """cnt[plane][ty][tx][class]: a tile is reached if its own bins hold a
    record, or its left neighbour's classes 2-3, its upper neighbour's classes
    1-2 or its upper-left neighbour's class 2 do (neighbours wrap around)."""
    P = cnt.shape[0]
    out = np.zeros((P, NT, NT), bool)
    for p in range(P):
        for ty in range(NT):
            for tx in range(NT):
                txl, tyu = (tx - 1) % NT, (ty - 1) % NT
                tot = (cnt[p, ty, tx].sum() + cnt[p, ty, txl, 2] + cnt[p, ty, txl, 3] +
                       cnt[p, tyu, tx, 1] + cnt[p, tyu, tx, 2] + cnt[p, tyu, txl, 2])
                out[p, ty, tx] = tot > 0
    return out


def test_reach_counts_match_the_tile_rule():
    g = np.random.default_rng(3)
    C, P, N, T = 2, 3, 256, 32
    NT = N // T
    cnt = (g.random((C * P, NT, NT, 4)) < 0.04).astype(np.int64) * g.integers(1, 5, (C * P, NT, NT, 4))
    cnt[0, NT - 1, NT - 1, 2] = 3          # spills right and down from the last tile: wraps to 0
    cnt[1] = 0                             # an empty plane
    off = np.concatenate([[0], np.cumsum(cnt.ravel())]).astype(np.uint32)
    r = bench.reach_counts(off, C, P, N, T)
    ref = _reached_direct(cnt, NT)
    assert ref[0, 0, 0] and ref[0, NT - 1, 0] and ref[0, 0, NT - 1]
    assert r["tiles"] == int(ref.sum())
    assert r["tile_columns"] == int(ref.any(axis=1).sum())
    assert r["planes"] == int(ref.any(axis=(1, 2)).sum()) and r["planes"] < C * P
    assert r["tiles_total"] == C * P * NT * NT


def test_stage_traffic_and_flops_by_hand():
    N, C, P, T = 1024, 2, 4, 32
    reach = {"tiles": 10, "tile_columns": 3, "planes": 5, "tile": T}
    b = bench.stage_traffic(N, C, P, nrow=100, n_grid=150, T=T, reach=reach, own=True)
    assert b["grid"] == 8 * 10 * T * T + 16 * 150
    assert b["columns"] == 8 * 10 * T * T + 8 * 3 * N * T
    assert b["rows_phase"] == 8 * 3 * N * T + 8 * C * N * N
    f = bench.stage_flops(N, C, P, reach, True)
    assert f["columns"] == 3 * T * 5 * N * 10
    assert f["rows_phase"] == 5 * N * 5 * N * 10 + 8 * 5 * N * N
    full = bench.stage_traffic(N, C, P, nrow=100, n_grid=150, T=T, reach=reach, own=False)
    assert full["fft"] == 16 * C * P * N * N and full["grid"] == 8 * C * P * N * N + 16 * 150


def test_large_blocks_cover_each_ranks_channels_once():
    """The default workload's channel blocks: rank r of N takes channels
    [128 r, 128 r + 128) of the band split into 128 N, in 8 blocks of 16; over
    all ranks every channel of the band is taken exactly once."""
    for world in (1, 2, 4, 8):
        seen = []
        for r in range(world):
            blk = bench.large_blocks(world, r)
            assert len(blk) == 8 and all(c1 - c0 == 16 for c0, c1 in blk)
            assert blk[0][0] == 128 * r
            for c0, c1 in blk:
                seen.extend(range(c0, c1))
        assert seen == list(range(128 * world))


def test_gridder_ceilings_are_counts_times_rate_over_peaks():
    """The gridder's ceiling fractions: per-visibility counts of the ncu
    capture times the visibilities gridded per second, over one shared-memory
    wavefront per cycle per SM and four warp instructions per cycle per SM at
    2.07 GHz (152 SMs); the binding ceiling is the larger fraction."""
    c = bench.GRID_COUNTERS["large"]
    out = bench.gridder_ceilings(2.0e9, 1000.0, "large")   # 2 G visibilities in one second
    assert out["smem_wavefronts"]["achieved_per_s"] == 2.0e9 * c["smem_wavefronts"]
    assert abs(out["smem_wavefronts"]["frac"] - 2.0e9 * c["smem_wavefronts"] / (152 * 2.07e9)) < 1e-12
    assert abs(out["issue"]["frac"] - 2.0e9 * c["warp_instructions"] / (152 * 4 * 2.07e9)) < 1e-12
    assert out["binding"] == max(("smem_wavefronts", "issue"), key=lambda k: out[k]["frac"])
    assert out["source"].startswith("profiles/") and out["source"].endswith(".md")

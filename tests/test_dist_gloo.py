"""The multi-rank host logic with two gloo ranks on the CPU: channel blocks
cover every channel exactly once, and the step time reported is the maximum
over ranks."""
import os
import socket

import pytest

from paper_2601_19714_gb300 import dist


def test_channel_blocks_cover_once():
    for total in (1, 5, 16, 17, 128):
        for world in (1, 2, 3, 8):
            if world > total:
                continue
            seen = []
            for r in range(world):
                c0, c1 = dist.channel_block(total, world, r)
                assert c1 - c0 in (total // world, total // world + 1)
                seen.extend(range(c0, c1))
            assert seen == list(range(total))
    with pytest.raises(ValueError):
        dist.channel_block(8, 2, 2)


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, out_dir):
    import torch.distributed as tdist
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), WORLD_SIZE=str(world),
                      RANK=str(rank), LOCAL_RANK=str(rank))
    tdist.init_process_group("gloo", rank=rank, world_size=world)
    w, r, _ = dist.env()
    c0, c1 = dist.channel_block(16 * w, w, r)
    dist.barrier()
    m = dist.max_over_ranks(1.5 * (r + 1))
    with open(os.path.join(out_dir, f"rank{r}.txt"), "w") as f:
        f.write(f"{w} {r} {c0} {c1} {m}")
    tdist.destroy_process_group()


def test_two_gloo_ranks(tmp_path):
    import torch.multiprocessing as mp
    port = _free_port()
    mp.start_processes(_rank_main, args=(2, port, str(tmp_path)), nprocs=2, join=True,
                       start_method="spawn")
    rows = sorted(open(tmp_path / f"rank{r}.txt").read().split() for r in range(2))
    assert rows[0][:4] == ["2", "0", "0", "16"] and rows[1][:4] == ["2", "1", "16", "32"]
    assert float(rows[0][4]) == float(rows[1][4]) == 3.0

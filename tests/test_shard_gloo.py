"""The multi-process path on CPU: two gloo ranks, each answering its own slice of the
configuration queries (here with the oracle, since no GPU is needed to check the
partition), must together give exactly the single-process answer, and the timing
reduction must return the maximum over ranks."""
import os
import socket

import numpy as np
import pytest
import torch.multiprocessing as mp

from paper_2406_02807_gb300.shard import max_over_ranks, shard_range, weak_slice


def test_shard_range_covers_everything_once():
    for total in (0, 1, 7, 100, 1 << 20):
        for world in (1, 2, 3, 8):
            seen = []
            for r in range(world):
                b, e = shard_range(total, r, world)
                assert 0 <= b <= e <= total
                seen.extend(range(b, e)) if total < 1000 else seen.append((b, e))
            if total < 1000:
                assert seen == list(range(total))
            else:
                assert seen[0][0] == 0 and seen[-1][1] == total
                assert all(seen[i][1] == seen[i + 1][0] for i in range(world - 1))
    assert weak_slice(5, 0) == (0, 5) and weak_slice(5, 3) == (15, 20)
    with pytest.raises(ValueError):
        shard_range(10, 2, 2)


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, out):
    import torch
    import torch.distributed as dist

    import oracle
    import workloads as W
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    raw, _, arm = W.tabletop_scene(1001)
    pts = raw[oracle.sfc_filter(raw, 0.01)]
    tree = oracle.PlainCAPT(pts, 0.02, 0.08)
    per_rank = 300
    b, e = weak_slice(per_rank, rank)
    cen = W.fk_centers(arm, W.random_configs(e - b, 1001, first=b))
    flags, _ = tree.query_configs(cen, arm.sphere_radius)
    parts = [torch.zeros(per_rank, dtype=torch.uint8) for _ in range(world)]
    dist.all_gather(parts, torch.from_numpy(flags))
    t = max_over_ranks(1.0 + rank, dist)
    if rank == 0:
        out.put((torch.cat(parts).numpy(), t))
    dist.barrier()
    dist.destroy_process_group()


def test_two_gloo_ranks_equal_one_process(orc):
    import workloads as W
    world, port = 2, _free_port()
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    procs = [ctx.Process(target=_worker, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    flags, tmax = q.get(timeout=300)
    for p in procs:
        p.join(timeout=120)
        assert p.exitcode == 0
    raw, _, arm = W.tabletop_scene(1001)
    pts = raw[orc.sfc_filter(raw, 0.01)]
    cen = W.fk_centers(arm, W.random_configs(600, 1001))
    ref = orc.brute_config_flags(pts, cen, arm.sphere_radius)
    assert np.array_equal(flags, ref)
    assert tmax == 2.0

"""Multi-rank host logic on CPU: pixel-balanced sharding and the gather of
records across two gloo ranks (the method has no data-path collective)."""
import os
import socket

import numpy as np
import pytest
import torch.multiprocessing as mp

from paper_1705_09776_gb300 import shard, synth


def test_shards_cover_every_image_once_and_balance_pixels():
    sizes = [(h, w) for w, h in synth.uneven_sizes(200, base_seed=5)]
    for world in (1, 2, 3, 8):
        shares = shard.shard_images(sizes, world)
        flat = sorted(i for s in shares for i in s)
        assert flat == list(range(len(sizes)))
        loads = [sum(sizes[i][0] * sizes[i][1] for i in s) for s in shares]
        biggest = max(h * w for h, w in sizes)
        assert max(loads) - min(loads) <= biggest   # LPT bound
    assert shard.shard_images(sizes, 2) == shard.shard_images(list(sizes), 2)   # deterministic


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _rank(rank, world, port, q):
    import torch.distributed as dist

    from paper_1705_09776_gb300 import cdvs as dt  # record layout only; nothing is launched
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    sizes = [(480, 640), (240, 320), (480, 640), (300, 500), (100, 100)]
    mine = shard.shard_images(sizes, world)[rank]
    # fake per-rank results: two records per local image
    rec = np.zeros(2 * len(mine), dt.KEYPOINT_DTYPE)
    rec["image"] = np.repeat(np.arange(len(mine)), 2)
    rec["parent_id"] = np.tile([0, 1], len(mine))
    rec["x"] = rank
    desc = np.full((len(rec), 128), float(rank), np.float32)
    allr, alld = shard.gather_records(rec, desc, mine)
    # the step-time reduction of the benchmark: max over ranks
    import torch
    t = torch.tensor([float(rank + 1)])
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    q.put((rank, allr["image"].tolist(), allr["parent_id"].tolist(), allr["x"].tolist(),
           alld[:, 0].tolist(), float(t.item())))
    dist.destroy_process_group()


@pytest.mark.timeout(120)
def test_gather_across_two_gloo_ranks():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    out = [q.get(timeout=100) for _ in procs]
    for p in procs:
        p.join(timeout=30)
        assert p.exitcode == 0
    out.sort()
    sizes = [(480, 640), (240, 320), (480, 640), (300, 500), (100, 100)]
    shares = shard.shard_images(sizes, 2)
    owner = {i: r for r, s in enumerate(shares) for i in s}
    for rank, images, parents, xs, d0, tmax in out:
        assert images == sorted(images) and images == [i for i in range(5) for _ in range(2)]
        assert parents == [0, 1] * 5
        assert xs == [float(owner[i]) for i in images]      # each record came from its owner
        assert d0 == xs
        assert tmax == 2.0

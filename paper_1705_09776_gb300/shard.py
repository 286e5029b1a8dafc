"""Image sharding for runs on several GPUs (one process per GPU).

Images are independent, so the front end shards by image with no exchange
step: each rank extracts its own share, and the only communication is an
optional host-side gather of the records at the end.  Shares are balanced by
pixel count with the greedy longest-processing-time rule (largest image to
the least-loaded rank; ties by rank), which gives every rank the same
deterministic assignment without communication.
"""
from __future__ import annotations

import heapq

import numpy as np


def shard_images(sizes, world_size: int):
    """sizes: list of (height, width).  Returns, per rank, the sorted list of
    image indices it extracts."""
    if world_size < 1:
        raise ValueError("world_size must be >= 1")
    order = sorted(range(len(sizes)), key=lambda i: (-sizes[i][0] * sizes[i][1], i))
    heap = [(0, r) for r in range(world_size)]
    shares = [[] for _ in range(world_size)]
    for i in order:
        load, r = heapq.heappop(heap)
        shares[r].append(i)
        heapq.heappush(heap, (load + sizes[i][0] * sizes[i][1], r))
    return [sorted(s) for s in shares]


def gather_records(records: np.ndarray, descriptors: np.ndarray, image_ids, group=None):
    """Host-side gather of every rank's records (``records["image"]`` indexes
    the rank's local list ``image_ids``).  Returns all records with global image
    indices, sorted by image then by their per-image order, and the matching
    descriptors.  Uses torch.distributed (any backend) when initialised."""
    import torch.distributed as dist

    rec = records.copy()
    rec["image"] = np.asarray(image_ids, dtype=np.int32)[rec["image"]]
    if dist.is_available() and dist.is_initialized():
        parts = [None] * dist.get_world_size(group)
        dist.all_gather_object(parts, (rec, descriptors), group=group)
    else:
        parts = [(rec, descriptors)]
    allr = np.concatenate([p[0] for p in parts])
    alld = np.concatenate([p[1] for p in parts])
    order = np.argsort(allr["image"], kind="stable")
    return allr[order], alld[order]

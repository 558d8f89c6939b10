"""Exchange between the processes that verify one log split over several GPUs.

One process per GPU verifies a contiguous range of the log's global indices (its shard).  The
processes exchange two things, both through torch.distributed (NCCL with CUDA tensors, gloo
with CPU tensors): the fixed-size aggregate records of poslo_aver_partial (216 bytes each,
treated as opaque bytes here) and the ascending invalid-index lists of their shards'
poslo_distill calls.  Argument marshalling only: the records are combined and checked by
poslo_combine_check on the device.
"""
from __future__ import annotations

import numpy as np

RECORD_BYTES = 216


def shard_range(n_total: int, rank: int, world: int) -> tuple[int, int]:
    """Contiguous shard [lo, hi) of rank `rank` among `world`: sizes differ by at most one."""
    if not 0 <= rank < world:
        raise ValueError("rank out of range")
    return n_total * rank // world, n_total * (rank + 1) // world


def _device(device):
    import torch
    return torch.device("cpu") if device is None else torch.device(device)


def all_gather_records(rec: bytes, device=None, group=None) -> list[bytes]:
    """Every rank's record, in rank order (an all-gather of RECORD_BYTES per rank)."""
    import torch
    import torch.distributed as dist
    if len(rec) != RECORD_BYTES:
        raise ValueError(f"a shard record is {RECORD_BYTES} bytes")
    world = dist.get_world_size(group)
    dev = _device(device)
    mine = torch.frombuffer(bytearray(rec), dtype=torch.uint8).to(dev)
    out = torch.empty(world * RECORD_BYTES, dtype=torch.uint8, device=dev)
    dist.all_gather_into_tensor(out, mine, group=group)
    flat = out.cpu().numpy().tobytes()
    return [flat[RECORD_BYTES * r:RECORD_BYTES * (r + 1)] for r in range(world)]


def gather_lists(idx, device=None, group=None) -> np.ndarray:
    """The concatenation, in rank order, of every rank's invalid-index list (uint64).  With
    contiguous shards in rank order and ascending lists, the result is the log's ascending list."""
    import torch
    import torch.distributed as dist
    world = dist.get_world_size(group)
    dev = _device(device)
    mine = np.ascontiguousarray(idx, dtype=np.uint64).view(np.int64)
    cnt = torch.tensor([mine.size], dtype=torch.int64, device=dev)
    cnts = torch.empty(world, dtype=torch.int64, device=dev)
    dist.all_gather_into_tensor(cnts, cnt, group=group)
    counts = [int(c) for c in cnts.cpu()]
    width = max(max(counts), 1)
    pad = np.zeros(width, np.int64)
    pad[:mine.size] = mine
    buf = torch.from_numpy(pad).to(dev)
    out = torch.empty(world * width, dtype=torch.int64, device=dev)
    dist.all_gather_into_tensor(out, buf, group=group)
    allv = out.cpu().numpy()
    return np.concatenate([allv[r * width:r * width + counts[r]] for r in range(world)]).view(np.uint64)

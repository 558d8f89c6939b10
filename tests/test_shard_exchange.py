"""The exchange between the processes that verify one log split over several GPUs, on CPU over
gloo: every rank receives every rank's 216-byte record in rank order (the records are opaque
bytes here; their combination runs on the device), and the ranks' invalid-index lists
concatenate in rank order.  Also the split of a log into contiguous shards."""
import os

import numpy as np
import pytest
import torch.multiprocessing as mp

from test_bench_ranks import _free_port


def _record(rank: int) -> bytes:
    # distinct, position-dependent bytes so that a shuffled or truncated record is caught
    return bytes((rank * 37 + k * 11) % 256 for k in range(216))


LISTS = {0: [3, 9, 10], 1: [], 2: [2_000_000_000_000, 2_000_000_000_007]}


def _worker(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    import torch.distributed as dist
    from paper_2506_08781_gb300 import shard
    dist.init_process_group("gloo", rank=rank, world_size=world)
    recs = shard.all_gather_records(_record(rank))
    lists = shard.gather_lists(np.array(LISTS.get(rank, [rank]), np.uint64))
    out.put((rank, recs, [int(x) for x in lists], str(lists.dtype)))
    dist.barrier()
    dist.destroy_process_group()


@pytest.mark.parametrize("world", [2, 3])
def test_records_and_lists_in_rank_order(world):
    ctx = mp.get_context("spawn")
    out = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, world, port, out)) for r in range(world)]
    for p in procs:
        p.start()
    res = sorted((out.get(timeout=120) for _ in procs), key=lambda r: r[0])
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    want_lists = [x for r in range(world) for x in LISTS.get(r, [r])]
    for rank, recs, lists, dtype in res:
        assert recs == [_record(r) for r in range(world)]
        assert lists == want_lists and dtype == "uint64"


def test_record_size_is_enforced():
    from paper_2506_08781_gb300 import shard
    with pytest.raises(ValueError):
        shard.all_gather_records(bytes(215))


def test_shard_ranges_cover_the_log():
    from paper_2506_08781_gb300 import shard
    for n in (0, 1, 7, 1 << 20, (1 << 20) * 3 + 5):
        for world in (1, 2, 3, 8):
            r = [shard.shard_range(n, k, world) for k in range(world)]
            assert r[0][0] == 0 and r[-1][1] == n
            assert all(r[k][1] == r[k + 1][0] for k in range(world - 1))
            assert max(b - a for a, b in r) - min(b - a for a, b in r) <= 1
    with pytest.raises(ValueError):
        shard.shard_range(10, 2, 2)


def test_partial_record_layout():
    """The ctypes record is the C struct's 216 bytes: e, s, R (extended), then the counters."""
    import ctypes as C
    from paper_2506_08781_gb300 import poslo
    p = poslo.Partial()
    assert C.sizeof(p) == 216
    assert [poslo.Partial.e.offset, poslo.Partial.s.offset, poslo.Partial.R.offset, poslo.Partial.first_index.offset,
            poslo.Partial.n.offset, poslo.Partial.malformed.offset, poslo.Partial.agg_mode.offset] == \
        [0, 32, 64, 192, 200, 208, 212]
    p.first_index, p.n, p.malformed, p.agg_mode = 5, 7, 1, 1
    q = poslo.Partial.from_bytes(p.to_bytes())
    assert (q.first_index, q.n, q.malformed, q.agg_mode) == (5, 7, 1, 1)

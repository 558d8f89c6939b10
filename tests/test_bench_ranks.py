"""The multi-rank host logic of bench.py with world size 2 over gloo on CPU: shards are
independent, the job time is the slowest rank's, and the throughput counts every rank's
entries (weak scaling; no data-path collective)."""
import os
import socket

import pytest
import torch.multiprocessing as mp


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _worker(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world),
                      LOCAL_RANK=str(rank))
    import torch.distributed as dist
    import bench
    dist.init_process_group("gloo", rank=rank, world_size=world)
    r, w, local = bench.dist_env()
    ms = bench.max_over_ranks(3.0 + 2.0 * r, w)          # rank 1 is the slow one
    out.put((r, w, local, ms, bench.job_throughput(1000, w, ms), bench.shard_seed(r)))
    dist.barrier()
    dist.destroy_process_group()


def test_two_ranks_max_time_and_job_throughput():
    ctx = mp.get_context("spawn")
    out = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, out)) for r in range(2)]
    for p in procs:
        p.start()
    res = sorted(out.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    assert [r[:3] for r in res] == [(0, 2, 0), (1, 2, 1)]
    assert [r[3] for r in res] == [5.0, 5.0]                 # both see the slowest rank's time
    assert [r[4] for r in res] == [2 * 1000 / 5e-3] * 2      # whole-job entries per second
    assert res[0][5] != res[1][5]                            # independent shards


def test_single_rank_is_identity():
    import bench
    assert bench.max_over_ranks(4.0, 1) == 4.0
    assert bench.job_throughput(1 << 20, 1, 5.0) == (1 << 20) / 5e-3


def test_shards_are_independent_workloads():
    pytest.importorskip("numpy")
    import bench
    from paper_2506_08781_gb300 import synth
    a = synth.messages(bench.shard_seed(0), 64, 32, 64)
    b = synth.messages(bench.shard_seed(1), 64, 32, 64)
    assert a.data.tobytes() != b.data.tobytes()

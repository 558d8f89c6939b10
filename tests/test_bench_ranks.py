"""The multi-rank host logic of bench.py with world size 2 over gloo on CPU: the ranks verify
contiguous shards of one log, the job time is the slowest rank's, and the throughput counts
every rank's entries (weak scaling)."""
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
    out.put((r, w, local, ms, bench.job_throughput(1000, w, ms), bench.shard_plan(r, w)))
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
    assert [r[5] for r in res] == [(0, 13), (1 << 20, 13)]     # contiguous shards, one tree for the log


def test_single_rank_is_identity():
    import bench
    assert bench.max_over_ranks(4.0, 1) == 4.0
    assert bench.job_throughput(1 << 20, 1, 5.0) == (1 << 20) / 5e-3


def test_shards_are_parts_of_one_log():
    """Every rank signs with the same key; its entries sit at its own global indices, under a
    seed tree deep enough for the whole log; rank 0's shard is the single-GPU workload."""
    pytest.importorskip("numpy")
    import bench
    from paper_2506_08781_gb300 import synth
    for world in (1, 2, 3, 4, 8):
        shards = [bench.shard_plan(r, world, n_per_rank=64) for r in range(world)]
        assert [f for f, _ in shards] == [64 * r for r in range(world)]
        depth = shards[0][1]
        assert all(d == depth for _, d in shards)
        assert (1 << depth) * bench.N2 >= 64 * world * (bench.N_ENTRIES // 64)   # epochs of the full-size log fit
    k0, m0, s0, _ = bench.make_workload(n=64, rank=0, world=2)
    k1, m1, s1, _ = bench.make_workload(n=64, rank=1, world=2)
    kk, mm, ss, _ = bench.make_workload(n=64)
    assert k0.y == k1.y and k0.root == k1.root                           # one signer
    assert m0.data.tobytes() != m1.data.tobytes()                        # different entries
    assert m0.data.tobytes() == mm.data.tobytes()                        # rank 0 = single GPU
    assert (s1 == synth.bpv_subsets(bench.SEED, 64, first_index=64)).all()   # subsets at global indices

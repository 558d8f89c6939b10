"""Full-size checks at the benchmark's workload (2^20 entries, |m| ~ U[32, 256], n2 = 256)
in the launch configuration bench.py times.

The oracle cannot sign 2^20 entries in test time, so the batch is signed by the library's
signer (whose output equals the oracle signer's bit for bit, see test_gpu_parity) and the
checks use what the oracle can compute one by one or properties that hold at any size:
  * e_t for a sample of entries equals the oracle's H(m_t || x_t) mod q;
  * the honest batch is accepted (unit and weighted) and Distill returns no index;
  * with 0.1 % of entries flipped by one byte, Distill returns exactly the flipped
    indices, and the oracle's single-entry check rejects each of them.
"""
import struct

import numpy as np
import pytest

import bench
from oracle import poslo_oracle as O
from paper_2506_08781_gb300 import poslo, synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def big():
    import torch
    import __graft_entry__
    __graft_entry__.build()
    ctx = poslo.Context(device=0, verifier_seed=synth.verifier_seed(5))
    km, msgs, subsets, _ = bench.make_workload()
    Y, s, R = bench.sign_workload(ctx, km, msgs, subsets)
    ds = struct.pack("<II", bench.D, 0) + km.root
    dev = lambda a: torch.from_numpy(np.ascontiguousarray(a).copy()).cuda()
    d = dict(ctx=ctx, km=km, msgs=msgs, Y=Y, s=s, R=R, ds=ds,
             d_msgs=dev(msgs.data), d_offs=dev(msgs.offs.view(np.int64)), d_s=dev(s), d_R=dev(R))
    torch.cuda.synchronize()
    yield d
    ctx.close()


def test_fullsize_hash_sample(big):
    ctx = big["ctx"]
    b = ctx.make_batch(poslo.VARIANT_F, bench.N2, big["Y"], big["d_msgs"], big["d_offs"], big["d_s"], big["d_R"],
                       big["ds"])
    import torch
    e = torch.zeros(32 * b.n, dtype=torch.uint8, device="cuda")
    ctx.hash_entries(b, out=e)
    e = e.cpu().numpy().reshape(-1, 32)
    ds = O.ds_root(big["km"].root, bench.D)
    for t in synth.choose_without_replacement(9, "sample", b.n, 300):
        t = int(t)
        assert int.from_bytes(bytes(e[t]), "little") == O.entry_scalar(ds, bench.N2, t, big["msgs"].entry(t))


def test_fullsize_honest_accepts(big):
    ctx = big["ctx"]
    b = ctx.make_batch(poslo.VARIANT_F, bench.N2, big["Y"], big["d_msgs"], big["d_offs"], big["d_s"], big["d_R"],
                       big["ds"])
    assert ctx.aver(b, poslo.AGG_UNIT) is True
    assert ctx.aver(b, poslo.AGG_WEIGHTED) is True
    idx, cs, cR = ctx.distill(b)
    assert len(idx) == 0


def test_fullsize_distill_config3(big):
    """0.1 % of 2^20 entries (1,049) flipped by one byte at seeded positions."""
    import torch
    ctx, msgs = big["ctx"], big["msgs"]
    plan = synth.tamper_plan(3, msgs, round(0.001 * msgs.n))
    bad = synth.apply_tamper(msgs, plan)
    b = ctx.make_batch(poslo.VARIANT_F, bench.N2, big["Y"], torch.from_numpy(bad.data).cuda(), big["d_offs"],
                       big["d_s"], big["d_R"], big["ds"])
    torch.cuda.synchronize()
    idx, cs, cR = ctx.distill(b)
    assert list(idx) == list(plan.idx)
    assert ctx.aver(b, poslo.AGG_UNIT) is False
    # the oracle's single-entry check rejects a sample of the flagged entries and accepts a
    # sample of the others (inputs: generator bytes and the batch's s_t, R_t)
    Yp = O.decode_point(big["Y"])
    ds = O.ds_root(big["km"].root, bench.D)
    s, R = big["s"].reshape(-1, 32), big["R"].reshape(-1, 32)
    for t in list(plan.idx[:8]):
        e = O.entry_scalar(ds, bench.N2, int(t), bad.entry(int(t)))
        assert not O.verify_entry_f(Yp, e, bytes(s[t]), bytes(R[t]))
    for t in synth.choose_without_replacement(10, "ok", msgs.n, 8):
        if int(t) in set(plan.idx.tolist()):
            continue
        e = O.entry_scalar(ds, bench.N2, int(t), bad.entry(int(t)))
        assert O.verify_entry_f(Yp, e, bytes(s[t]), bytes(R[t]))


def test_fullsize_autotuned_window(big):
    """bench.py tunes the MSM window before timing; the tuned width gives the same results."""
    import torch
    ctx, msgs = big["ctx"], big["msgs"]
    c = ctx.msm_autotune(msgs.n, 4)
    assert 8 <= c <= 16
    b = ctx.make_batch(poslo.VARIANT_F, bench.N2, big["Y"], big["d_msgs"], big["d_offs"], big["d_s"], big["d_R"],
                       big["ds"])
    assert ctx.aver(b, poslo.AGG_WEIGHTED) is True
    plan = synth.tamper_plan(3, msgs, round(0.001 * msgs.n))
    bad = synth.apply_tamper(msgs, plan)
    b = ctx.make_batch(poslo.VARIANT_F, bench.N2, big["Y"], torch.from_numpy(bad.data).cuda(), big["d_offs"],
                       big["d_s"], big["d_R"], big["ds"])
    torch.cuda.synchronize()
    assert list(ctx.distill(b)[0]) == list(plan.idx)

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


def test_fullsize_multi_device_4096():
    """The 4,096-device batch bench.py times (sizes log-uniform in [16, 65536], about 3.1e7
    entries, 20 devices with one entry flipped by one byte), under the autotuned MSM plan:
    the (device, index) list equals the tamper plan, a device is rejected exactly when it has
    a listed entry, and the oracle's single-entry check rejects every listed entry and
    accepts a sample of the others."""
    import torch
    import __graft_entry__
    __graft_entry__.build()
    with poslo.Context(device=0, verifier_seed=synth.verifier_seed(7)) as ctx:
        w = bench.make_multi_workload(ctx)
        nd = len(w["Y"])
        dev = lambda a: torch.from_numpy(np.ascontiguousarray(a)).cuda()
        args = (w["Y"], w["sizes"], np.zeros(nd, np.uint64), np.full(nd, bench.MULTI_N2, np.uint32), w["ds"],
                dev(w["msgs"].data), dev(w["msgs"].offs.view(np.int64)), dev(w["s"]), dev(w["R"]))
        torch.cuda.synchronize()
        ctx.msm_autotune(w["total"], 4)
        for _ in range(2):                           # the second call is the captured one
            acc, pairs = ctx.aver_multi(*args)
            got = [(int(a), int(b)) for a, b in pairs]
            assert got == w["pairs"]
            assert [not a for a in acc] == [d in {p[0] for p in got} for d in range(nd)]
    start = np.zeros(nd + 1, np.int64)
    start[1:] = np.cumsum(w["sizes"])
    s, R = w["s"].reshape(-1, 32), w["R"].reshape(-1, 32)

    def oracle_ok(d, t):
        g = int(start[d]) + t
        ds = O.ds_root(w["ds"][d][8:], bench.MULTI_D)
        e = O.entry_scalar(ds, bench.MULTI_N2, t, w["msgs"].entry(g))
        return O.verify_entry_f(O.decode_point(w["Y"][d]), e, bytes(s[g]), bytes(R[g]))

    for d, t in got:
        assert not oracle_ok(d, t)
    flagged = set(got)
    devs = synth.uniform_int(11, "devs", 24, 0, nd - 1)
    for k, d in enumerate(devs):
        d = int(d)
        t = int(synth.uniform_int(11, f"t{k}", 1, 0, int(w["sizes"][d]) - 1)[0])
        if (d, t) not in flagged:
            assert oracle_ok(d, t)

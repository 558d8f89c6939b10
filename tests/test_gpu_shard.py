"""One log split into shards (as over several GPUs), run in sequence on one GPU: each shard's
record from poslo_aver_partial, the combined check poslo_combine_check, and per-shard Distill
lists, against the oracle's whole-log AVer (Fig. 3a, Fig. 4) and Distill (Sec. 4.3)."""
import numpy as np
import pytest

from oracle import poslo_oracle as O
from paper_2506_08781_gb300 import poslo, synth

pytestmark = pytest.mark.gpu

D, N2 = 6, 4


@pytest.fixture(scope="module")
def ctx():
    import __graft_entry__
    __graft_entry__.build()
    c = poslo.Context(device=0, verifier_seed=synth.verifier_seed(808))
    yield c
    c.close()


def _log(seed, n, first=0, lmin=1, lmax=90):
    km = synth.key_material(seed, v=16)
    sk, Y = O.kg_f(km.y, km.root, D, N2, km.bpv_r.tobytes())
    msgs = synth.messages(seed, n, lmin, lmax)
    sub = synth.bpv_subsets(seed, n, first_index=first, v=16, k=4)
    sig = [O.sig_f(sk, first + t, msgs.entry(t), sub[t]) for t in range(n)]
    return sk, Y, msgs, [x[0] for x in sig], [x[1] for x in sig], O.ds_root(km.root, D)


def _cuts(n, k):
    """k contiguous shards of n entries, uneven (one may be empty when k > n)."""
    return [0] + [int(n * (i * i + i) / (k * k + k)) for i in range(1, k)] + [n]


def _shard(ctx, Y, msgs, s, R, ds, a, b, first):
    sub = synth.pack([msgs.entry(t) for t in range(a, b)])
    return ctx.make_batch(poslo.VARIANT_F, N2, Y, sub.data, sub.offs, b"".join(s[a:b]) or bytes(32),
                          b"".join(R[a:b]) or bytes(32), O.ds_serialize(ds), first_index=first + a, R_count=b - a)


def _ext_to_point(R128: bytes):
    X, Y, Z, T = (int.from_bytes(R128[32 * k:32 * k + 32], "little") for k in range(4))
    return (X, Y, Z, T)


@pytest.mark.parametrize("k", [1, 2, 3, 4])
@pytest.mark.parametrize("mode", [poslo.AGG_UNIT, poslo.AGG_WEIGHTED])
def test_shards_combine_to_the_whole_log(ctx, k, mode):
    n, first = 150, 11
    sk, Y, msgs, s, R, ds = _log(31 + k, n, first)
    cuts = _cuts(n, k)
    parts = [ctx.aver_partial(_shard(ctx, Y, msgs, s, R, ds, cuts[i], cuts[i + 1], first), mode) for i in range(k)]
    acc, total = ctx.combine_check(Y, parts)
    assert acc is True is O.aver_f(Y, msgs.as_list(), first, N2, s, R, ds)
    assert total.first_index == first and total.n == n and total.malformed == 0
    if mode == poslo.AGG_UNIT:
        # the summed record element by element: e~, s~ and R~ of the oracle
        e_sum = sum(O.entry_scalar(ds, N2, first + t, msgs.entry(t)) for t in range(n)) % O.Q
        assert bytes(total.e) == O.scalar_to_bytes(e_sum)
        assert bytes(total.s) == O.agg_scalars(s)
        assert O.point_eq(_ext_to_point(bytes(total.R)), O.decode_point(O.agg_points(R)))
        for i, p in enumerate(parts):
            a, b = cuts[i], cuts[i + 1]
            assert (p.first_index, p.n) == (first + a, b - a)
            want = sum(O.entry_scalar(ds, N2, first + t, msgs.entry(t)) for t in range(a, b)) % O.Q
            assert bytes(p.e) == O.scalar_to_bytes(want) and bytes(p.s) == O.agg_scalars(s[a:b])
            Rp = _ext_to_point(bytes(p.R))
            assert O.on_curve(Rp) and all(c < O.P for c in Rp)
            assert O.point_eq(Rp, O.decode_point(O.agg_points(R[a:b])) if b > a else O.IDENTITY)
    # the same shards with one tampered entry in the last shard: rejected; the shard Distill
    # lists concatenate to the whole log's list
    plan = synth.tamper_plan(k, msgs, 2)
    bad = synth.apply_tamper(msgs, plan)
    parts = [ctx.aver_partial(_shard(ctx, Y, bad, s, R, ds, cuts[i], cuts[i + 1], first), mode) for i in range(k)]
    acc, _ = ctx.combine_check(Y, parts)
    assert acc is False is O.aver_f(Y, bad.as_list(), first, N2, s, R, ds)
    lists = [ctx.distill(_shard(ctx, Y, bad, s, R, ds, cuts[i], cuts[i + 1], first))[0] for i in range(k)]
    want, ws, wR = O.distill_f(Y, bad.as_list(), first, N2, s, R, ds)
    assert [int(t) for l in lists for t in l] == want == [first + int(t) for t in plan.idx]


def test_cancelling_s_shift_across_shards(ctx):
    """s_t + d in shard 0 and s_u - d in shard 1: invisible to the unit sums (as for AVer of the
    whole log), found by the weighted records."""
    n, first = 40, 0
    sk, Y, msgs, s, R, ds = _log(41, n, first)
    s = list(s)
    s[3] = O.scalar_to_bytes(int.from_bytes(s[3], "little") + 12345)
    s[33] = O.scalar_to_bytes(int.from_bytes(s[33], "little") - 12345)
    assert O.aver_f(Y, msgs.as_list(), first, N2, s, R, ds) is True
    shards = [_shard(ctx, Y, msgs, s, R, ds, 0, 20, first), _shard(ctx, Y, msgs, s, R, ds, 20, 40, first)]
    acc_u, _ = ctx.combine_check(Y, [ctx.aver_partial(b, poslo.AGG_UNIT) for b in shards])
    acc_w, _ = ctx.combine_check(Y, [ctx.aver_partial(b, poslo.AGG_WEIGHTED) for b in shards])
    assert acc_u is True and acc_w is False
    assert [int(t) for b in shards for t in ctx.distill(b)[0]] == [3, 33]


def test_malformed_entries_are_counted(ctx):
    n = 24
    sk, Y, msgs, s, R, ds = _log(42, n)
    s, R = list(s), list(R)
    s[2] = O.Q.to_bytes(32, "little")
    R[17] = (O.P + 1).to_bytes(32, "little")
    parts = [ctx.aver_partial(_shard(ctx, Y, msgs, s, R, ds, a, b, 0), mode)
             for a, b in [(0, 10), (10, 24)] for mode in [poslo.AGG_UNIT]]
    assert [p.malformed for p in parts] == [1, 1]
    acc, total = ctx.combine_check(Y, parts)
    assert acc is False and total.malformed == 2
    assert O.aver_f(Y, msgs.as_list(), 0, N2, s, R, ds) is False


def test_records_checked_and_ordered(ctx):
    n = 30
    sk, Y, msgs, s, R, ds = _log(43, n)
    p0 = ctx.aver_partial(_shard(ctx, Y, msgs, s, R, ds, 0, 12, 0))
    p1 = ctx.aver_partial(_shard(ctx, Y, msgs, s, R, ds, 12, 30, 0))
    assert ctx.combine_check(Y, [p0, p1])[0] is True
    # records as opaque 216-byte strings (the form an all-gather moves) give the same result
    assert ctx.combine_check(Y, [p0.to_bytes(), p1.to_bytes()])[0] is True
    assert ctx.combine_check(Y, [p0])[0] is True                    # entries 0..11 are a valid log too
    with pytest.raises(poslo.PosloError) as e:
        ctx.combine_check(Y, [p1, p0])                               # out of order
    assert e.value.code == -1
    pw = ctx.aver_partial(_shard(ctx, Y, msgs, s, R, ds, 12, 30, 0), poslo.AGG_WEIGHTED)
    with pytest.raises(poslo.PosloError):
        ctx.combine_check(Y, [p0, pw])                               # mixed modes
    with pytest.raises(poslo.PosloError):
        ctx.combine_check((O.P + 1).to_bytes(32, "little"), [p0, p1])  # key does not decode
    # a record whose point is off the curve, or has a coordinate >= p, is refused by the check
    r = bytearray(p1.to_bytes())
    r[64] ^= 1                                                      # X changes: off the curve
    assert ctx.combine_check(Y, [p0, bytes(r)])[0] is False
    r = bytearray(p1.to_bytes())
    X = int.from_bytes(r[64:96], "little")
    r[64:96] = (X + O.P).to_bytes(32, "little") if X + O.P < 1 << 256 else r[64:96]
    if X + O.P < 1 << 256:
        assert ctx.combine_check(Y, [p0, bytes(r)])[0] is False
    r = bytearray(p1.to_bytes())
    r[0:32] = O.Q.to_bytes(32, "little")                            # e~ not below q
    assert ctx.combine_check(Y, [p0, bytes(r)])[0] is False


def test_poslo_c_shards_by_epoch(ctx):
    """POSLO-C (Fig. 3a): shards of whole epochs with their own s~ and per-epoch R~_i."""
    Dc, n2 = 3, 8
    km = synth.key_material(44)
    sk, Y, epoch_R = O.kg_c(km.y, km.r, km.root, Dc, n2)
    n1 = 1 << Dc
    msgs = synth.messages(44, n1 * n2, 5, 60)
    s_ep = [O.sig_c(sk, i, [msgs.entry(i * n2 + j) for j in range(n2)]) for i in range(n1)]
    ds = O.ds_serialize(O.ds_root(km.root, Dc))
    parts = []
    for a, b in [(0, 3), (3, 4), (4, 8)]:
        sub = synth.pack([msgs.entry(t) for t in range(a * n2, b * n2)])
        bt = ctx.make_batch(poslo.VARIANT_C, n2, Y, sub.data, sub.offs, O.agg_scalars(s_ep[a:b]),
                            b"".join(epoch_R[a:b]), ds, first_index=a * n2)
        parts.append(ctx.aver_partial(bt))
    assert ctx.combine_check(Y, parts)[0] is True
    parts[1] = ctx.aver_partial(ctx.make_batch(
        poslo.VARIANT_C, n2, Y, synth.pack([msgs.entry(t) for t in range(3 * n2, 4 * n2)]).data,
        synth.pack([msgs.entry(t) for t in range(3 * n2, 4 * n2)]).offs,
        O.scalar_to_bytes(int.from_bytes(s_ep[3], "little") + 1), epoch_R[3], ds, first_index=3 * n2))
    assert ctx.combine_check(Y, parts)[0] is False


def test_device_resident_shards(ctx):
    import torch
    n = 64
    sk, Y, msgs, s, R, ds = _log(45, n)
    dev = lambda a: torch.from_numpy(np.ascontiguousarray(a).copy()).cuda()
    parts = []
    for a, b in [(0, 32), (32, 64)]:
        sub = synth.pack([msgs.entry(t) for t in range(a, b)])
        bt = ctx.make_batch(poslo.VARIANT_F, N2, Y, dev(sub.data), dev(sub.offs.view(np.int64)),
                            dev(np.frombuffer(b"".join(s[a:b]), np.uint8)),
                            dev(np.frombuffer(b"".join(R[a:b]), np.uint8)), O.ds_serialize(ds), first_index=a)
        parts.append(ctx.aver_partial(bt, poslo.AGG_WEIGHTED))
    torch.cuda.synchronize()
    assert ctx.combine_check(Y, parts)[0] is True


def test_record_of_a_replayed_call_follows_its_inputs(ctx):
    """A device-resident shard of the same shape in a row is replayed from a CUDA graph: the
    records still follow the inputs (a byte flipped between calls changes the record, restoring
    it restores the record), in both modes."""
    import torch
    n = 96
    sk, Y, msgs, s, R, ds = _log(46, n)
    dev = lambda a: torch.from_numpy(np.ascontiguousarray(a).copy()).cuda()
    d_msgs = dev(msgs.data)
    bt = ctx.make_batch(poslo.VARIANT_F, N2, Y, d_msgs, dev(msgs.offs.view(np.int64)),
                        dev(np.frombuffer(b"".join(s), np.uint8)), dev(np.frombuffer(b"".join(R), np.uint8)),
                        O.ds_serialize(ds))
    def same(a, b):
        # equal scalars and the same point (the projective coordinates of R~ depend on the
        # order in which the device summed the points, not on the point)
        return a[:64] == b[:64] and O.point_eq(_ext_to_point(a[64:192]), _ext_to_point(b[64:192]))

    for mode in (poslo.AGG_UNIT, poslo.AGG_WEIGHTED):
        c0 = ctx.graph_stats()
        good = [ctx.aver_partial(bt, mode).to_bytes() for _ in range(3)]
        assert same(good[0], good[1]) and same(good[0], good[2]) and ctx.combine_check(Y, [good[2]])[0] is True
        off = int(msgs.offs[40])
        d_msgs[off] ^= 0x11
        torch.cuda.synchronize()
        bad = ctx.aver_partial(bt, mode).to_bytes()
        d_msgs[off] ^= 0x11
        torch.cuda.synchronize()
        again = ctx.aver_partial(bt, mode).to_bytes()
        c1 = ctx.graph_stats()
        assert bad[:32] != good[0][:32] and same(again, good[0])    # the flip changes e~ only
        assert ctx.combine_check(Y, [bad])[0] is False
        assert c1[1] > c0[1]                    # some of these calls were replays

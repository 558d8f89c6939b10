"""GPU parity on the edges of the verification equation [8](R - eY - sG) = O (Fig. 4, with
the strict decoding and cofactored reading of the points the paper leaves open).

Every case below is built so that a lenient implementation would get it wrong:
  * valid entries whose R_t (or the key Y) carries a component of order 2, 4 or 8, or is the
    identity: only the cofactor [8] makes them verify;
  * invalid entries whose R_t is a NON-canonical encoding of exactly the point that would make
    the entry verify (y >= p, or x = 0 with the sign bit set), or whose s_t is q or q + 5
    with R_t matching s_t mod q: only strict decoding and the s < q test reject them.
Each case runs through aggregate verification (unit and weighted), Distill, the multi-device
call and one served request, and is compared element by element with the oracle.
"""
import numpy as np
import pytest

from oracle import poslo_oracle as O
from paper_2506_08781_gb300 import poslo, synth

pytestmark = pytest.mark.gpu

D, N2, N = 5, 4, 40


@pytest.fixture(scope="module")
def ctx():
    import __graft_entry__
    __graft_entry__.build()
    c = poslo.Context(device=0, verifier_seed=synth.verifier_seed(606))
    yield c
    c.close()


def _enc(y: int, sign: int) -> bytes:
    return (y | (sign << 255)).to_bytes(32, "little")


def _torsion():
    """Points of order 2, 4 and 8 from the oracle's group law."""
    T2 = O.decode_point(_enc(O.P - 1, 0))                   # (0, -1)
    T4 = O.decode_point(_enc(0, 0))                         # (sqrt(-1), 0), x even
    y = 3
    while True:
        P = O.decode_point(y.to_bytes(32, "little"))
        if P is not None:
            T = O.scalar_mult(O.Q, P)                      # in the 8-torsion
            if not O.is_identity(O.scalar_mult(4, T)):
                break
        y += 1
    T8 = T
    assert O.is_identity(O.point_add(T2, T2)) and not O.is_identity(T2)
    assert O.is_identity(O.scalar_mult(4, T4)) and not O.is_identity(O.point_add(T4, T4))
    assert O.is_identity(O.scalar_mult(8, T8)) and not O.is_identity(O.scalar_mult(4, T8))
    return T2, T4, T8


T2, T4, T8 = _torsion()
T4_SIGN = O.encode_point(T4)[31] >> 7                       # parity of T4's x


def _base(seed, n=N, first=0):
    km = synth.key_material(seed, v=16)
    sk, Y = O.kg_f(km.y, km.root, D, N2, km.bpv_r.tobytes())
    msgs = synth.messages(seed, n, 1, 70)
    sub = synth.bpv_subsets(seed, n, first_index=first, v=16, k=4)
    sig = [O.sig_f(sk, first + t, msgs.entry(t), sub[t]) for t in range(n)]
    ds = O.ds_root(km.root, D)
    return sk, Y, msgs, [x[0] for x in sig], [x[1] for x in sig], ds


# Each edge: name -> function (sk, Y point, e, s, R) -> (s', R', valid?)
def _r_plus(T):
    return lambda sk, Yp, e, s, R: (s, O.encode_point(O.point_add(O.decode_point(R), T)), True)


def _torsion_R(enc):
    """R_t a torsion point (or O) given by its encoding, s_t = -e y: [8](R - eY - sG) = [8]R."""
    return lambda sk, Yp, e, s, R: (O.scalar_to_bytes(-e * sk.y), enc, O.decode_point(enc) is not None)


def _s_edge(k: int, valid: bool):
    """s_t the integer k (k = q - 1, q, q + 5) with R_t = eY + (k mod q) G."""
    def f(sk, Yp, e, s, R):
        Rp = O.point_add(O.scalar_mult(e, Yp), O.scalar_mult(k % O.Q, O.G))
        return k.to_bytes(32, "little"), O.encode_point(Rp), valid
    return f


def _r_bytes(enc):
    return lambda sk, Yp, e, s, R: (s, enc, False)


EDGES = {
    # valid only because of the cofactor
    "R+T2": _r_plus(T2),
    "R+T4": _r_plus(T4),
    "R+T8": _r_plus(T8),
    "R=O": _torsion_R(_enc(1, 0)),
    "R=T2": _torsion_R(_enc(O.P - 1, 0)),
    "R=T4": _torsion_R(_enc(0, T4_SIGN)),
    "s=q-1": _s_edge(O.Q - 1, True),
    # non-canonical encodings of exactly the point that would verify
    "O as y=p+1": _torsion_R(_enc(O.P + 1, 0)),
    "O as y=p+1,sign": _torsion_R(_enc(O.P + 1, 1)),
    "O as x=0,sign": _torsion_R(_enc(1, 1)),
    "T2 as x=0,sign": _torsion_R(_enc(O.P - 1, 1)),
    "T4 as y=p": _torsion_R(_enc(O.P, T4_SIGN)),
    "-T4 as y=p": _torsion_R(_enc(O.P, 1 - T4_SIGN)),
    "y=2^255-1": _r_bytes(_enc((1 << 255) - 1, 0)),
    "y=2^255-1,sign": _r_bytes(_enc((1 << 255) - 1, 1)),
    "s=q": _s_edge(O.Q, False),
    "s=q+5": _s_edge(O.Q + 5, False),
}
VALID = [k for k in EDGES if k in ("R+T2", "R+T4", "R+T8", "R=O", "R=T2", "R=T4", "s=q-1")]
INVALID = [k for k in EDGES if k not in VALID]


def _apply(sk, Y, msgs, s, R, ds, edits, first=0):
    """edits: {t: edge name}; returns the edited (s, R) and the indices expected invalid."""
    Yp = O.decode_point(Y)
    s, R = list(s), list(R)
    bad = []
    for t, name in sorted(edits.items()):
        e = O.entry_scalar(ds, N2, first + t, msgs.entry(t))
        s[t], R[t], ok = EDGES[name](sk, Yp, e, s[t], R[t])
        assert O.verify_entry_f(Yp, e, s[t], R[t]) is ok, name      # the construction itself
        if not ok:
            bad.append(first + t)
    return s, R, bad


def _gpu_batch(ctx, Y, msgs, s, R, ds, first=0):
    return ctx.make_batch(poslo.VARIANT_F, N2, Y, msgs.data, msgs.offs, b"".join(s), b"".join(R),
                          O.ds_serialize(ds), first_index=first)


def test_edge_encodings_decode_as_the_reading_says():
    """The non-canonical encodings are exactly the ones the oracle refuses, and each names the
    same point as a canonical encoding (so a decoder that reduced y mod p would accept it)."""
    for enc, canon in [(_enc(O.P + 1, 0), _enc(1, 0)), (_enc(O.P, T4_SIGN), _enc(0, T4_SIGN))]:
        assert O.decode_point(enc) is None and O.decode_point(canon) is not None
    for enc in (_enc(1, 1), _enc(O.P - 1, 1), _enc((1 << 255) - 1, 0), _enc((1 << 255) - 1, 1)):
        assert O.decode_point(enc) is None


@pytest.mark.parametrize("name", list(EDGES))
def test_each_edge_alone(ctx, name):
    """One edited entry in an otherwise honest batch: AVer (unit, weighted) and Distill give the
    oracle's answers."""
    sk, Y, msgs, s, R, ds = _base(71)
    t = 13
    s, R, bad = _apply(sk, Y, msgs, s, R, ds, {t: name})
    want, ws, wR = O.distill_f(Y, msgs.as_list(), 0, N2, s, R, ds)
    assert want == bad
    want_acc = O.aver_f(Y, msgs.as_list(), 0, N2, s, R, ds)
    assert want_acc is (not bad)
    b = _gpu_batch(ctx, Y, msgs, s, R, ds)
    assert ctx.aver(b, poslo.AGG_UNIT) is want_acc, name
    assert ctx.aver(b, poslo.AGG_WEIGHTED) is want_acc, name
    idx, cs, cR = ctx.distill(b)
    assert list(idx) == want, name
    assert cs == ws and cR == wR, name


def test_all_edges_in_one_batch(ctx):
    sk, Y, msgs, s, R, ds = _base(72, n=64, first=8)
    names = list(EDGES)
    edits = {3 + 3 * k: names[k] for k in range(len(names))}
    s, R, bad = _apply(sk, Y, msgs, s, R, ds, edits, first=8)
    want, ws, wR = O.distill_f(Y, msgs.as_list(), 8, N2, s, R, ds)
    assert want == bad and len(want) == len(INVALID)
    b = _gpu_batch(ctx, Y, msgs, s, R, ds, first=8)
    assert ctx.aver(b, poslo.AGG_UNIT) is False and ctx.aver(b, poslo.AGG_WEIGHTED) is False
    idx, cs, cR = ctx.distill(b)
    assert list(idx) == want and cs == ws and cR == wR
    # the valid edges alone: accepted by both aggregate modes, nothing listed
    sk, Y, msgs, s, R, ds = _base(73, n=64, first=8)
    s, R, bad = _apply(sk, Y, msgs, s, R, ds, {2 + 5 * k: VALID[k] for k in range(len(VALID))}, first=8)
    assert bad == [] and O.aver_f(Y, msgs.as_list(), 8, N2, s, R, ds) is True
    b = _gpu_batch(ctx, Y, msgs, s, R, ds, first=8)
    assert ctx.aver(b, poslo.AGG_UNIT) is True and ctx.aver(b, poslo.AGG_WEIGHTED) is True
    idx, cs, cR = ctx.distill(b)
    want, ws, wR = O.distill_f(Y, msgs.as_list(), 8, N2, s, R, ds)
    assert list(idx) == want == [] and cs == ws and cR == wR


def _torsioned_key(Y):
    return O.encode_point(O.point_add(O.decode_point(Y), T8))


def test_key_with_torsion_component(ctx):
    """Y + T8 in place of Y: every honest entry still verifies under the cofactor; a tampered
    entry and the invalid edges are still found."""
    sk, Y, msgs, s, R, ds = _base(74)
    Yt = _torsioned_key(Y)
    assert O.aver_f(Yt, msgs.as_list(), 0, N2, s, R, ds) is True
    b = _gpu_batch(ctx, Yt, msgs, s, R, ds)
    assert ctx.aver(b, poslo.AGG_UNIT) is True and ctx.aver(b, poslo.AGG_WEIGHTED) is True
    idx, cs, cR = ctx.distill(b)
    want, ws, wR = O.distill_f(Yt, msgs.as_list(), 0, N2, s, R, ds)
    assert list(idx) == want == [] and cs == ws and cR == wR
    # tampered message + edges, checked under the torsioned key
    bad_msgs = synth.apply_tamper(msgs, synth.tamper_plan(74, msgs, 1))
    s2, R2, _ = _apply(sk, Y, msgs, s, R, ds, {5: "R+T8", 9: "O as y=p+1", 20: "s=q", 30: "R=T4"})
    want, ws, wR = O.distill_f(Yt, bad_msgs.as_list(), 0, N2, s2, R2, ds)
    b = _gpu_batch(ctx, Yt, bad_msgs, s2, R2, ds)
    assert ctx.aver(b, poslo.AGG_UNIT) is False and ctx.aver(b, poslo.AGG_WEIGHTED) is False
    idx, cs, cR = ctx.distill(b)
    assert list(idx) == want and cs == ws and cR == wR


@pytest.mark.parametrize("enc", [_enc(O.P + 1, 0), _enc(1, 1), _enc(O.P - 1, 1), _enc(O.P, 0),
                                 _enc((1 << 255) - 1, 1)])
def test_undecodable_key_is_einval(ctx, enc):
    sk, Y, msgs, s, R, ds = _base(75, n=8)
    with pytest.raises(ValueError):
        O.aver_f(enc, msgs.as_list(), 0, N2, s, R, ds)
    b = _gpu_batch(ctx, enc, msgs, s, R, ds)
    for call in (lambda: ctx.aver(b, poslo.AGG_UNIT), lambda: ctx.aver(b, poslo.AGG_WEIGHTED),
                 lambda: ctx.distill(b)):
        with pytest.raises(poslo.PosloError) as e:
            call()
        assert e.value.code == -1


def test_poslo_c_aggregate_edges(ctx):
    """POSLO-C AVer (Fig. 3a) with an aggregate R~ that is the identity: accepted when
    encoded canonically with s~ = -e~ y, rejected in its non-canonical forms; per-epoch R~_i
    carrying torsion are accepted."""
    Dc, n2 = 2, 8
    km = synth.key_material(76)
    sk, Y, epoch_R = O.kg_c(km.y, km.r, km.root, Dc, n2)
    msgs = synth.messages(76, n2 << Dc, 10, 40)
    ds_nodes = O.ds_root(km.root, Dc)
    ds = O.ds_serialize(ds_nodes)
    ep = [[msgs.entry(i * n2 + j) for j in range(n2)] for i in range(1 << Dc)]
    s_ep = [O.sig_c(sk, i, ep[i]) for i in range(1 << Dc)]
    s_all = O.agg_scalars(s_ep)
    # per-epoch R~_i with torsion components
    R_t = [O.encode_point(O.point_add(O.decode_point(r), T)) for r, T in zip(epoch_R, (T2, T4, T8, O.IDENTITY))]
    assert O.aver_c(Y, list(range(1 << Dc)), ep, n2, s_all, R_t, ds_nodes) is True
    b = ctx.make_batch(poslo.VARIANT_C, n2, Y, msgs.data, msgs.offs, s_all, b"".join(R_t), ds)
    assert ctx.aver(b) is True
    # R~ = O with s~ = -e~ y
    e_all = sum(O.entry_scalar(ds_nodes, n2, t, msgs.entry(t)) for t in range(msgs.n)) % O.Q
    s_id = O.scalar_to_bytes(-e_all * sk.y)
    for enc in (_enc(1, 0), _enc(O.P + 1, 0), _enc(1, 1), _enc(O.P + 1, 1)):
        want = O.aver_c(Y, list(range(1 << Dc)), ep, n2, s_id, enc, ds_nodes)
        assert want is (enc == _enc(1, 0))
        b = ctx.make_batch(poslo.VARIANT_C, n2, Y, msgs.data, msgs.offs, s_id, enc, ds)
        assert ctx.aver(b) is want, enc.hex()
    # s~ = q + (s~ mod q) is refused although it reduces to the right value
    s_nc = (int.from_bytes(s_all, "little") + O.Q)
    if s_nc < 1 << 256:
        b = ctx.make_batch(poslo.VARIANT_C, n2, Y, msgs.data, msgs.offs, s_nc.to_bytes(32, "little"),
                           O.agg_points(epoch_R), ds)
        assert O.aver_c(Y, list(range(1 << Dc)), ep, n2, s_nc.to_bytes(32, "little"), O.agg_points(epoch_R),
                        ds_nodes) is False
        assert ctx.aver(b) is False


def _device(seed, edits, torsion_key=False, n=24, first=4):
    sk, Y, msgs, s, R, ds = _base(seed, n=n, first=first)
    s, R, _ = _apply(sk, Y, msgs, s, R, ds, edits, first=first)
    if torsion_key:
        Y = _torsioned_key(Y)
    return (Y, msgs, first, s, R, ds)


def test_multi_device_edges(ctx):
    """Per-device definition for devices with torsioned keys, valid torsion edges and every
    invalid edge, in one multi-device call."""
    inv = INVALID
    devs = [
        _device(81, {}),
        _device(82, {1: "R+T8", 4: "R=O", 7: "s=q-1", 10: "R=T4"}, torsion_key=True),
        _device(83, {k + 2: inv[k] for k in range(0, len(inv), 2)}),
        _device(84, {k + 1: inv[k] for k in range(1, len(inv), 2)}, torsion_key=True),
        _device(85, {0: "R+T2", 23: "R=T2"}),
    ]
    oracle_devs = [(Y, m.as_list(), first, N2, s, R, ds) for Y, m, first, s, R, ds in devs]
    want_acc, want_pairs = O.verify_multi(oracle_devs)
    assert want_acc == [True, True, False, False, True]
    cat = synth.pack([x for d in devs for x in d[1].as_list()])
    sb = b"".join(b"".join(d[3]) for d in devs)
    Rb = b"".join(b"".join(d[4]) for d in devs)
    acc, pairs = ctx.aver_multi([d[0] for d in devs], [d[1].n for d in devs], [d[2] for d in devs],
                                [N2] * len(devs), [O.ds_serialize(d[5]) for d in devs], cat.data, cat.offs, sb, Rb)
    assert list(acc) == want_acc
    assert [tuple(int(x) for x in p) for p in pairs] == want_pairs


def test_served_request_edges():
    """One served request per edge mix under a registered torsioned key: each result equals
    the oracle's per-entry definition."""
    import __graft_entry__
    __graft_entry__.build()
    reqs = [
        _device(91, {2: "R+T8", 5: "R=O", 8: "O as y=p+1", 11: "s=q", 14: "y=2^255-1,sign"}, torsion_key=True),
        _device(92, {k + 1: INVALID[k] for k in range(len(INVALID))}),
        _device(93, {3: "R+T4", 6: "R=T2", 9: "s=q-1"}),
    ]
    with poslo.Context(device=0, verifier_seed=synth.verifier_seed(9)) as c:
        c.serve_start(workers=2, max_batch_devices=4, max_batch_entries=1 << 12)
        try:
            tickets, wants = [], []
            for Y, msgs, first, s, R, ds in reqs:
                kid = c.register_key(Y)
                want, _, _ = O.distill_f(Y, msgs.as_list(), first, N2, s, R, ds)
                wants.append(want)
                tickets.append(c.submit(kid, N2, first, msgs.data, msgs.offs, b"".join(s), b"".join(R),
                                        O.ds_serialize(ds)))
            for t, want in zip(tickets, wants):
                acc, idx = c.poll(t, wait_ms=60000)
                assert acc is (not want) and list(idx) == want
        finally:
            c.serve_stop()


def test_all_edges_through_the_descent(ctx):
    """The same edges spread over a batch above the direct-check size (16,384 entries), so that
    Distill localises them by the descent over the segment tree and the confirmation, not by
    every entry's own check; signed and checked by the C++ oracle (pinned to the Python one)."""
    import types
    from oracle import cpp_oracle as X
    n, first, depth = 16400, 8, 13         # 2^13 epochs of N2 = 4 entries hold the batch
    km = synth.key_material(75, v=16)
    msgs = synth.messages(75, n, 1, 70)
    sub = synth.bpv_subsets(75, n, first_index=first, v=16, k=4)
    sa, Ra = X.sign_f(km.y, km.root, depth, N2, km.bpv_r, sub, msgs.data, msgs.offs, first)
    sb, Rb = sa.tobytes(), Ra.tobytes()
    s = [sb[32 * t:32 * t + 32] for t in range(n)]
    R = [Rb[32 * t:32 * t + 32] for t in range(n)]
    sk = types.SimpleNamespace(y=int.from_bytes(km.y, "little"))
    Y = X.base_mult(sk.y)
    ds = O.ds_root(km.root, depth)
    names = list(EDGES)
    s, R, bad = _apply(sk, Y, msgs, s, R, ds, {100 + 941 * k: names[k] for k in range(len(names))}, first=first)
    want, ws, wR = X.distill_f(Y, msgs.data, msgs.offs, first, N2, b"".join(s), b"".join(R), O.ds_serialize(ds))
    assert want == bad and len(want) == len(INVALID)
    b = _gpu_batch(ctx, Y, msgs, s, R, ds, first=first)
    assert ctx.aver(b, poslo.AGG_UNIT) is False and ctx.aver(b, poslo.AGG_WEIGHTED) is False
    ctx.set_profiling(True)
    ctx.reset_kernel_times()
    idx, cs, cR = ctx.distill(b)
    ctx.set_profiling(False)
    assert ctx.kernel_time("bisect")[1] >= 1 and ctx.kernel_time("direct")[1] == 0
    assert list(idx) == want and cs == ws and cR == wR

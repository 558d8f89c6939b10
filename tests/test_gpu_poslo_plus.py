"""POSLO+ (Sec. 7.2: MMO-AES-128 PRF with kappa = 127, MDC-2-AES-128 H) on the GPU against
the oracle evaluated in the same instantiation, through the C ABI, bit-exact."""
import numpy as np
import pytest

from oracle import poslo_oracle as O
from paper_2506_08781_gb300 import poslo, synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctx():
    import __graft_entry__
    __graft_entry__.build()
    c = poslo.Context(device=0, verifier_seed=synth.verifier_seed(77), instantiation=poslo.INST_AES)
    yield c
    c.close()


@pytest.fixture(autouse=True)
def plus():
    with O.instantiation("POSLO+"):
        yield


def _f_data(seed, n, D, n2, lmin, lmax, v=32, k=4, first_index=0):
    km = synth.key_material(seed, v=v)
    sk, Y = O.kg_f(km.y, km.root, D, n2, km.bpv_r.tobytes())
    msgs = synth.messages(seed, n, lmin, lmax)
    subsets = synth.bpv_subsets(seed, n, first_index=first_index, v=v, k=k)
    sig = [O.sig_f(sk, first_index + t, msgs.entry(t), subsets[t]) for t in range(n)]
    return km, sk, Y, msgs, subsets, [x[0] for x in sig], [x[1] for x in sig], [x[2] for x in sig]


def test_unknown_instantiation_is_einval():
    import __graft_entry__
    __graft_entry__.build()
    with pytest.raises(poslo.PosloError) as e:
        poslo.Context(device=0, instantiation=7)
    assert e.value.code == -1


@pytest.mark.parametrize("D", [3, 5])
def test_epoch_seeds_every_ds(ctx, D):
    root = synth.random_bytes(20 + D, "root", 16).tobytes()
    leaves = [O.tree_node(root, D, 0, i) for i in range(1 << D)]
    for i in range(1 << D):
        got = ctx.epoch_seeds(O.ds_serialize(O.ds_after(root, D, i)), 0, i + 1)
        assert [bytes(r) for r in got] == leaves[:i + 1]


def test_hash_every_length_and_alignment(ctx):
    """Message lengths 0..160 (every MDC-2 block boundary, 10 blocks deep) at every byte
    alignment, plus long messages."""
    D, n2 = 5, 8
    root = synth.random_bytes(21, "root", 16).tobytes()
    ds = O.ds_root(root, D)
    lens = list(range(0, 161)) + [255, 256, 257, 600]
    entries = [synth.random_bytes(21, f"m{L}", L).tobytes() for L in lens]
    for pad in range(4):
        buf = bytes(pad) + b"".join(entries)
        offs = np.zeros(len(entries) + 1, np.uint64)
        offs[0] = pad
        offs[1:] = pad + np.cumsum([len(m) for m in entries])
        b = ctx.make_batch(poslo.VARIANT_F, n2, O.encode_point(O.G), np.frombuffer(buf, np.uint8), offs,
                           bytes(32 * len(entries)), bytes(32 * len(entries)), O.ds_serialize(ds), first_index=5)
        e = ctx.hash_entries(b).reshape(-1, 32)
        for t, m in enumerate(entries):
            assert int.from_bytes(bytes(e[t]), "little") == O.entry_scalar(ds, n2, 5 + t, m), (pad, t)


def test_keygen_and_sign_f_match_oracle(ctx):
    D, n2, n = 3, 8, 40
    km, sk, Y, msgs, subsets, s, R, x = _f_data(22, n, D, n2, 0, 200, v=32, k=16)
    gY, gR = ctx.keygen_f(km.y, km.bpv_r)
    assert gY == Y
    gs, gRt, gx = ctx.sign_f(km.y, km.root, D, n2, km.bpv_r, gR, subsets, msgs.data, msgs.offs, want_x=True)
    assert gs.tobytes() == b"".join(s)
    assert gRt.tobytes() == b"".join(R)
    assert gx.tobytes() == b"".join(x)


def test_keygen_and_sign_c_match_oracle(ctx):
    D, n2 = 2, 16
    km = synth.key_material(23)
    sk, Y, epoch_R = O.kg_c(km.y, km.r, km.root, D, n2)
    gY, gR = ctx.keygen_c(km.y, km.r, D, n2)
    assert gY == Y and gR.tobytes() == b"".join(epoch_R)
    msgs = synth.messages(23, n2 << D, 10, 90)
    gs = ctx.sign_c(km.y, km.r, km.root, D, n2, msgs.data, msgs.offs, 0, 1 << D)
    for i in range(1 << D):
        assert gs[32 * i:32 * i + 32].tobytes() == O.sig_c(sk, i, [msgs.entry(i * n2 + j) for j in range(n2)])


def test_aver_c_accepts_and_rejects(ctx):
    D, n2 = 2, 64
    km = synth.key_material(24)
    sk, Y, epoch_R = O.kg_c(km.y, km.r, km.root, D, n2)
    msgs = synth.messages(24, n2 << D, 0, 100)
    s_ep = [O.sig_c(sk, i, [msgs.entry(i * n2 + j) for j in range(n2)]) for i in range(1 << D)]
    ds_l = O.ds_root(km.root, D)
    b = ctx.make_batch(poslo.VARIANT_C, n2, Y, msgs.data, msgs.offs, O.agg_scalars(s_ep), b"".join(epoch_R),
                       O.ds_serialize(ds_l))
    assert ctx.aver(b) is True
    bad = synth.apply_tamper(msgs, synth.tamper_plan(24, msgs, 1))
    tb = ctx.make_batch(poslo.VARIANT_C, n2, Y, bad.data, bad.offs, O.agg_scalars(s_ep), b"".join(epoch_R),
                        O.ds_serialize(ds_l))
    want = O.aver_c(Y, list(range(1 << D)), [[bad.entry(i * n2 + j) for j in range(n2)] for i in range(1 << D)],
                    n2, O.agg_scalars(s_ep), epoch_R, ds_l)
    assert ctx.aver(tb) is want is False


@pytest.mark.parametrize("mode", [poslo.AGG_UNIT, poslo.AGG_WEIGHTED])
def test_aver_f_and_distill_patterns(ctx, mode):
    D, n2, n = 4, 16, 150
    km, sk, Y, msgs, subsets, s, R, _ = _f_data(25, n, D, n2, 0, 200)
    ds_l = O.ds_root(km.root, D)
    ds = O.ds_serialize(ds_l)
    b = ctx.make_batch(poslo.VARIANT_F, n2, Y, msgs.data, msgs.offs, b"".join(s), b"".join(R), ds)
    assert ctx.aver(b, mode) is True
    for trial, count in enumerate([1, 6, 30]):
        bad = synth.apply_tamper(msgs, synth.tamper_plan(250 + trial, msgs, count))
        tb = ctx.make_batch(poslo.VARIANT_F, n2, Y, bad.data, bad.offs, b"".join(s), b"".join(R), ds)
        assert ctx.aver(tb, mode) is False
        idx, cs, cR = ctx.distill(tb)
        wi, ws, wR = O.distill_f(Y, bad.as_list(), 0, n2, s, R, ds_l)
        assert list(idx) == wi and cs == ws and cR == wR


def test_multi_device_matches_definition(ctx):
    devs, parts = [], []
    for d in range(6):
        km = synth.key_material(2600 + d, v=16)
        sk, Y = O.kg_f(km.y, km.root, 3, 4, km.bpv_r.tobytes())
        msgs = synth.messages(2600 + d, 5 + 3 * d, 1, 50)
        subsets = synth.bpv_subsets(2600 + d, msgs.n, v=16, k=4)
        sig = [O.sig_f(sk, t, msgs.entry(t), subsets[t]) for t in range(msgs.n)]
        s, R = [x[0] for x in sig], [x[1] for x in sig]
        if d in (1, 4):
            msgs = synth.apply_tamper(msgs, synth.tamper_plan(2600 + d, msgs, 1))
        ds_l = O.ds_root(km.root, 3)
        devs.append((Y, msgs.as_list(), 0, 4, s, R, ds_l))
        parts.append((Y, msgs, s, R, O.ds_serialize(ds_l)))
    cat = synth.pack([m for p in parts for m in p[1].as_list()])
    acc, pairs = ctx.aver_multi([p[0] for p in parts], [p[1].n for p in parts], [0] * 6, [4] * 6,
                                [p[4] for p in parts], cat.data, cat.offs, b"".join(b"".join(p[2]) for p in parts),
                                b"".join(b"".join(p[3]) for p in parts))
    want_acc, want_pairs = O.verify_multi(devs)
    assert list(acc) == want_acc and [tuple(int(x) for x in p) for p in pairs] == want_pairs
    assert want_acc.count(False) == 2


def test_serving_in_poslo_plus():
    """The serving loop's workers inherit the context's instantiation."""
    import __graft_entry__
    __graft_entry__.build()
    with O.instantiation("POSLO+"):
        reqs = []
        keys = []
        for r in range(4):
            km, sk, Y, msgs, subsets, s, R, _ = _f_data(2700 + r, 10 + 7 * r, 3, 4, 1, 40)
            if r == 2:
                msgs = synth.apply_tamper(msgs, synth.tamper_plan(2700 + r, msgs, 2))
            ds_l = O.ds_root(km.root, 3)
            want, _, _ = O.distill_f(Y, msgs.as_list(), 0, 4, s, R, ds_l)
            keys.append(Y)
            reqs.append((msgs, b"".join(s), b"".join(R), O.ds_serialize(ds_l), want))
    with poslo.Context(device=0, instantiation=poslo.INST_AES) as ctx:
        ctx.serve_start(workers=2)
        kid = [ctx.register_key(Y) for Y in keys]
        tickets = [ctx.submit(kid[i], 4, 0, m.data, m.offs, s, R, ds) for i, (m, s, R, ds, _) in enumerate(reqs)]
        res = [ctx.poll(t, wait_ms=60000) for t in tickets]
        ctx.serve_stop()
    for (m, s, R, ds, want), r in zip(reqs, res):
        assert (r[0], list(r[1])) == (not want, want)
    assert any(want for *_, want in reqs)

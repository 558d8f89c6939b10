"""GPU parity: every step of the CUDA path against the CPU oracle, through the C ABI.

Inputs come from the seeded generators (synth); signatures used as oracle inputs are made
by the oracle's own signer.  All results are integers, points or bits, so every comparison
is bit-exact.
"""
import numpy as np
import pytest

from oracle import poslo_oracle as O
from paper_2506_08781_gb300 import poslo, synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctx():
    import __graft_entry__
    __graft_entry__.build()
    c = poslo.Context(device=0, verifier_seed=synth.verifier_seed(99))
    yield c
    c.close()


def _f_data(seed, n, D, n2, lmin, lmax, v=32, k=4, first_index=0, msgs=None):
    km = synth.key_material(seed, v=v)
    sk, Y = O.kg_f(km.y, km.root, D, n2, km.bpv_r.tobytes())
    if msgs is None:
        msgs = synth.messages(seed, n, lmin, lmax)
    subsets = synth.bpv_subsets(seed, n, first_index=first_index, v=v, k=k)
    sig = [O.sig_f(sk, first_index + t, msgs.entry(t), subsets[t]) for t in range(n)]
    return km, sk, Y, msgs, subsets, [x[0] for x in sig], [x[1] for x in sig], [x[2] for x in sig]


# ------------------------------------------------------------------------------ epoch seeds

@pytest.mark.parametrize("D", [3, 5])
def test_epoch_seeds_every_ds(ctx, D):
    root = synth.random_bytes(D, "root", 16).tobytes()
    leaves = [O.tree_node(root, D, 0, i) for i in range(1 << D)]
    for i in range(1 << D):
        ds = O.ds_after(root, D, i)
        got = ctx.epoch_seeds(O.ds_serialize(ds), 0, i + 1)
        assert [bytes(r) for r in got] == leaves[:i + 1]


def test_epoch_seeds_root_large_tree(ctx):
    D = 12
    root = synth.random_bytes(12, "root", 16).tobytes()
    got = ctx.epoch_seeds(O.ds_serialize(O.ds_root(root, D)), 0, 1 << D)
    for i in [0, 1, 2, 777, 2048, 4095]:
        assert bytes(got[i]) == O.tree_node(root, D, 0, i)


def test_epoch_seeds_not_disclosed_is_einval(ctx):
    root = bytes(16)
    ds = O.ds_serialize(O.ds_after(root, 4, 5))
    with pytest.raises(poslo.PosloError) as e:
        ctx.epoch_seeds(ds, 5, 2)          # epoch 6 is not disclosed yet
    assert e.value.code == -1


def test_disclose_matches_sso(ctx):
    root = synth.random_bytes(3, "root", 16).tobytes()
    for D, i in [(3, 0), (3, 5), (3, 6), (3, 7), (6, 37), (10, 1000)]:
        assert ctx.disclose(root, D, i) == O.ds_serialize(O.ds_after(root, D, i))


# ------------------------------------------------------------------------------ hashing

def test_hash_every_length_and_alignment(ctx):
    """Message lengths 0..300 (all SHA-256 padding boundaries) at every byte alignment."""
    D, n2 = 6, 8
    root = synth.random_bytes(4, "root", 16).tobytes()
    ds = O.ds_root(root, D)
    lens = list(range(0, 301))
    entries = [synth.random_bytes(4, f"m{L}", L).tobytes() for L in lens]
    for pad in range(4):
        buf = bytes(pad) + b"".join(entries)
        offs = np.zeros(len(entries) + 1, np.uint64)
        offs[0] = pad
        offs[1:] = pad + np.cumsum([len(m) for m in entries])
        b = ctx.make_batch(poslo.VARIANT_F, n2, O.encode_point(O.G), np.frombuffer(buf, np.uint8), offs,
                           bytes(32 * len(entries)), bytes(32 * len(entries)), O.ds_serialize(ds), first_index=3)
        e = ctx.hash_entries(b).reshape(-1, 32)
        for t, m in enumerate(entries):
            want = O.entry_scalar(ds, n2, 3 + t, m)
            assert int.from_bytes(bytes(e[t]), "little") == want, (pad, t)


def test_hash_non_power_of_two_epoch(ctx):
    D, n2 = 6, 5
    root = synth.random_bytes(5, "root", 16).tobytes()
    msgs = synth.messages(5, 200, 0, 130)
    ds = O.ds_after(root, D, 45)
    b = ctx.make_batch(poslo.VARIANT_F, n2, O.encode_point(O.G), msgs.data, msgs.offs, bytes(32 * 200),
                       bytes(32 * 200), O.ds_serialize(ds), first_index=17)
    e = ctx.hash_entries(b).reshape(-1, 32)
    for t in range(200):
        assert int.from_bytes(bytes(e[t]), "little") == O.entry_scalar(ds, n2, 17 + t, msgs.entry(t))


# ------------------------------------------------------------------------------ signer parity

def test_keygen_and_sign_f_match_oracle(ctx):
    D, n2, n = 3, 8, 40
    km, sk, Y, msgs, subsets, s, R, x = _f_data(7, n, D, n2, 0, 200, v=32, k=16)
    gY, gR = ctx.keygen_f(km.y, km.bpv_r)
    assert gY == Y
    assert gR.tobytes() == b"".join(O.bpv_table_encoded(sk))
    gs, gRt, gx = ctx.sign_f(km.y, km.root, D, n2, km.bpv_r, gR, subsets, msgs.data, msgs.offs, want_x=True)
    assert gs.tobytes() == b"".join(s)
    assert gRt.tobytes() == b"".join(R)
    assert gx.tobytes() == b"".join(x)


def test_keygen_and_sign_c_match_oracle(ctx):
    D, n2 = 2, 16
    km = synth.key_material(8)
    sk, Y, epoch_R = O.kg_c(km.y, km.r, km.root, D, n2)
    gY, gR = ctx.keygen_c(km.y, km.r, D, n2)
    assert gY == Y and gR.tobytes() == b"".join(epoch_R)
    msgs = synth.messages(8, n2 << D, 10, 90)
    gs = ctx.sign_c(km.y, km.r, km.root, D, n2, msgs.data, msgs.offs, 0, 1 << D)
    for i in range(1 << D):
        assert gs[32 * i:32 * i + 32].tobytes() == O.sig_c(sk, i, [msgs.entry(i * n2 + j) for j in range(n2)])


# ------------------------------------------------------------------------------ AVer

@pytest.mark.parametrize("mode", [poslo.AGG_UNIT, poslo.AGG_WEIGHTED])
def test_aver_f_1024_entries_of_64_bytes(ctx, mode):
    """POSLO-F, 1,024 entries of 64 bytes: the valid copy accepts, a one-byte flip rejects."""
    D, n2, n = 2, 256, 1024
    km, sk, Y, msgs, subsets, s, R, _ = _f_data(1, n, D, n2, 64, 64)
    ds = O.ds_serialize(O.ds_root(km.root, D))
    b = ctx.make_batch(poslo.VARIANT_F, n2, Y, msgs.data, msgs.offs, b"".join(s), b"".join(R), ds)
    assert ctx.aver(b, mode) is True
    bad = synth.apply_tamper(msgs, synth.tamper_plan(1, msgs, 1))
    tb = ctx.make_batch(poslo.VARIANT_F, n2, Y, bad.data, bad.offs, b"".join(s), b"".join(R), ds)
    assert ctx.aver(tb, mode) is False
    assert O.aver_f(Y, bad.as_list(), 0, n2, s, R, O.ds_root(km.root, D)) is False


def test_aver_c_4_epochs_of_256_entries(ctx):
    """POSLO-C, n1 = 4 epochs of 256 entries of 64 bytes, both R~ forms of AVer step 2."""
    D, n2 = 2, 256
    km = synth.key_material(11)
    sk, Y, epoch_R = O.kg_c(km.y, km.r, km.root, D, n2)
    msgs = synth.messages(11, n2 << D, 64, 64)
    s_ep = [O.sig_c(sk, i, [msgs.entry(i * n2 + j) for j in range(n2)]) for i in range(1 << D)]
    s_all = O.agg_scalars(s_ep)
    ds = O.ds_serialize(O.ds_root(km.root, D))
    for R in (b"".join(epoch_R), O.agg_points(epoch_R)):
        b = ctx.make_batch(poslo.VARIANT_C, n2, Y, msgs.data, msgs.offs, s_all, R, ds)
        assert ctx.aver(b) is True
        bad = synth.apply_tamper(msgs, synth.tamper_plan(11, msgs, 1))
        tb = ctx.make_batch(poslo.VARIANT_C, n2, Y, bad.data, bad.offs, s_all, R, ds)
        assert ctx.aver(tb) is False
    # a subrange of epochs 1..2 under ds_2 with the per-epoch R~_i of those epochs
    ds2 = O.ds_after(km.root, D, 2)
    sub = synth.pack([msgs.entry(t) for t in range(n2, 3 * n2)])
    b = ctx.make_batch(poslo.VARIANT_C, n2, Y, sub.data, sub.offs, O.agg_scalars(s_ep[1:3]),
                       b"".join(epoch_R[1:3]), O.ds_serialize(ds2), first_index=n2)
    assert ctx.aver(b) is True
    assert O.aver_c(Y, [1, 2], [[msgs.entry(i * n2 + j) for j in range(n2)] for i in (1, 2)], n2,
                    O.agg_scalars(s_ep[1:3]), epoch_R[1:3], ds2)


def test_aver_s_shift_unit_accepts_weighted_rejects(ctx):
    D, n2, n = 3, 4, 24
    km, sk, Y, msgs, subsets, s, R, _ = _f_data(12, n, D, n2, 5, 50)
    s2 = list(s)
    s2[3] = O.scalar_to_bytes(int.from_bytes(s[3], "little") + 999)
    s2[17] = O.scalar_to_bytes(int.from_bytes(s[17], "little") - 999)
    ds = O.ds_serialize(O.ds_root(km.root, D))
    b = ctx.make_batch(poslo.VARIANT_F, n2, Y, msgs.data, msgs.offs, b"".join(s2), b"".join(R), ds)
    assert O.aver_f(Y, msgs.as_list(), 0, n2, s2, R, O.ds_root(km.root, D)) is True
    assert ctx.aver(b, poslo.AGG_UNIT) is True          # the paper's unit aggregate
    assert ctx.aver(b, poslo.AGG_WEIGHTED) is False     # = per-entry definition
    idx, _, _ = ctx.distill(b)
    assert list(idx) == [3, 17]


def test_aver_malformed_and_errors(ctx):
    D, n2, n = 2, 4, 10
    km, sk, Y, msgs, subsets, s, R, _ = _f_data(13, n, D, n2, 1, 40)
    ds = O.ds_serialize(O.ds_root(km.root, D))
    s_bad = list(s)
    s_bad[2] = (int.from_bytes(s[2], "little") + O.Q).to_bytes(32, "little")
    y = 2
    while O.decode_point(y.to_bytes(32, "little")) is not None:
        y += 1
    R_bad = list(R)
    R_bad[7] = y.to_bytes(32, "little")
    for ss, RR, want in [(s_bad, R, [2]), (s, R_bad, [7]), (s_bad, R_bad, [2, 7])]:
        b = ctx.make_batch(poslo.VARIANT_F, n2, Y, msgs.data, msgs.offs, b"".join(ss), b"".join(RR), ds)
        for mode in (poslo.AGG_UNIT, poslo.AGG_WEIGHTED):
            assert ctx.aver(b, mode) is False
        idx, cs, cR = ctx.distill(b)
        wi, ws, wR = O.distill_f(Y, msgs.as_list(), 0, n2, ss, RR, O.ds_root(km.root, D))
        assert list(idx) == wi == want and cs == ws and cR == wR
    # undecodable public key, undisclosed seed, wrong R_count: errors, not reject bits
    b = ctx.make_batch(poslo.VARIANT_F, n2, y.to_bytes(32, "little"), msgs.data, msgs.offs, b"".join(s),
                       b"".join(R), ds)
    with pytest.raises(poslo.PosloError):
        ctx.aver(b)
    b = ctx.make_batch(poslo.VARIANT_F, n2, Y, msgs.data, msgs.offs, b"".join(s), b"".join(R),
                       O.ds_serialize(O.ds_after(km.root, D, 1)))
    with pytest.raises(poslo.PosloError):
        ctx.aver(b)


def test_aver_empty_and_single(ctx):
    D, n2 = 2, 4
    km, sk, Y, msgs, subsets, s, R, _ = _f_data(14, 1, D, n2, 0, 0)
    ds = O.ds_serialize(O.ds_root(km.root, D))
    e = synth.pack([])
    b = ctx.make_batch(poslo.VARIANT_F, n2, Y, e.data, e.offs, b"", b"", ds)
    assert ctx.aver(b) is O.aver_f(Y, [], 0, n2, [], [], O.ds_root(km.root, D)) is True
    idx, cs, cR = ctx.distill(b)
    assert len(idx) == 0 and cs == bytes(32) and cR == O.encode_point(O.IDENTITY)
    b = ctx.make_batch(poslo.VARIANT_F, n2, Y, msgs.data, msgs.offs, s[0], R[0], ds)
    assert ctx.aver(b) is True and ctx.aver(b, poslo.AGG_WEIGHTED) is True


# ------------------------------------------------------------------------------ Distill

def test_distill_random_patterns_ragged(ctx):
    D, n2, n = 4, 16, 150
    km, sk, Y, msgs, subsets, s, R, _ = _f_data(15, n, D, n2, 0, 260)
    ds_l = O.ds_root(km.root, D)
    ds = O.ds_serialize(ds_l)
    for trial, count in enumerate([0, 1, 5, 40]):
        nz = synth.pack([m for m in msgs.as_list()])
        if count:
            # only non-empty entries can be flipped
            cand = [t for t in range(n) if len(msgs.entry(t))]
            pick = synth.choose_without_replacement(15 + trial, "pick", len(cand), count)
            data = nz.data.copy()
            for q in pick:
                t = cand[q]
                data[int(nz.offs[t])] ^= 0x5A
            nz = synth.Messages(data, nz.offs)
        b = ctx.make_batch(poslo.VARIANT_F, n2, Y, nz.data, nz.offs, b"".join(s), b"".join(R), ds)
        idx, cs, cR = ctx.distill(b)
        wi, ws, wR = O.distill_f(Y, nz.as_list(), 0, n2, s, R, ds_l)
        assert list(idx) == wi and cs == ws and cR == wR


def test_distill_capacity(ctx):
    D, n2, n = 2, 8, 16
    km, sk, Y, msgs, subsets, s, R, _ = _f_data(16, n, D, n2, 8, 8)
    ds = O.ds_serialize(O.ds_root(km.root, D))
    bad = synth.apply_tamper(msgs, synth.tamper_plan(16, msgs, 5))
    b = ctx.make_batch(poslo.VARIANT_F, n2, Y, bad.data, bad.offs, b"".join(s), b"".join(R), ds)
    with pytest.raises(poslo.PosloError) as e:
        ctx.distill(b, cap=3)
    assert e.value.code == -5


# ------------------------------------------------------------------------------ MSM

def test_msm_matches_oracle(ctx):
    n = 37
    pts = [O.encode_point(O.scalar_mult(3 + 11 * i, O.G)) for i in range(n)]
    ks = [int.from_bytes(synth.random_bytes(17, f"k{i}", 32).tobytes(), "little") for i in range(n)]
    got = ctx.msm(b"".join(pts), b"".join(k.to_bytes(32, "little") for k in ks))
    assert got == O.msm(ks, pts)


# ------------------------------------------------------------------------------ device inputs

def test_device_inputs_same_as_host(ctx):
    import torch
    D, n2, n = 3, 8, 64
    km, sk, Y, msgs, subsets, s, R, _ = _f_data(18, n, D, n2, 20, 200)
    ds = O.ds_serialize(O.ds_root(km.root, D))
    bad = synth.apply_tamper(msgs, synth.tamper_plan(18, msgs, 3))
    hb = ctx.make_batch(poslo.VARIANT_F, n2, Y, bad.data, bad.offs, b"".join(s), b"".join(R), ds)
    dev = lambda a: torch.from_numpy(np.ascontiguousarray(a)).cuda()
    db = ctx.make_batch(poslo.VARIANT_F, n2, Y, dev(bad.data), dev(bad.offs.astype(np.int64)),
                        dev(np.frombuffer(b"".join(s), np.uint8)), dev(np.frombuffer(b"".join(R), np.uint8)), ds)
    torch.cuda.synchronize()
    assert ctx.aver(hb) is ctx.aver(db) is False
    assert [list(x) if i == 0 else x for i, x in enumerate(ctx.distill(hb))] == \
           [list(x) if i == 0 else x for i, x in enumerate(ctx.distill(db))]


@pytest.mark.parametrize("c", [8, 11, 13, 16])
def test_msm_every_window_width(c):
    """The bucket method gives the definition's result for every window width."""
    import __graft_entry__
    __graft_entry__.build()
    n = 300
    pts = [O.encode_point(O.scalar_mult(5 + 7 * i, O.G)) for i in range(n)]
    ks = [int.from_bytes(synth.random_bytes(c, f"w{i}", 32).tobytes(), "little") >> (i % 5) for i in range(n)]
    ks[3] = 0
    ks[4] = (1 << 256) - 1
    # signed-digit edges: every c-bit field at 2^(c-1) (largest positive digit), at
    # 2^(c-1) + 1 (smallest field that turns negative) and at 2^(c-1) - 1 under a carry
    fields = lambda f: sum(f << (c * w) for w in range(256 // c)) & ((1 << 256) - 1)
    ks[5] = fields(1 << (c - 1))
    ks[6] = fields((1 << (c - 1)) + 1)
    ks[7] = fields((1 << (c - 1)) - 1) + ((1 << c) - 1)
    ks[8] = 1 << 255
    with poslo.Context(device=0, msm_window=c) as cx:
        got = cx.msm(b"".join(pts), b"".join(k.to_bytes(32, "little") for k in ks))
    assert got == O.msm(ks, pts)


@pytest.mark.parametrize("c", [8, 12, 16])
def test_weighted_checks_every_window_width(c):
    """Weighted AVer and Distill (127-bit weights, signed window digits) keep the per-entry
    definition's result at every window width."""
    import __graft_entry__
    __graft_entry__.build()
    D, n2, n = 4, 16, 200
    km, sk, Y, msgs, subsets, s, R, _ = _f_data(30 + c, n, D, n2, 0, 90)
    ds_l = O.ds_root(km.root, D)
    bad = synth.apply_tamper(msgs, synth.tamper_plan(30 + c, msgs, 7))
    with poslo.Context(device=0, msm_window=c) as cx:
        for m in (msgs, bad):
            b = cx.make_batch(poslo.VARIANT_F, n2, Y, m.data, m.offs, b"".join(s), b"".join(R),
                              O.ds_serialize(ds_l))
            wi, ws, wR = O.distill_f(Y, m.as_list(), 0, n2, s, R, ds_l)
            assert cx.aver(b, poslo.AGG_WEIGHTED) is (len(wi) == 0)
            idx, cs, cR = cx.distill(b)
            assert list(idx) == wi and cs == ws and cR == wR


@pytest.mark.parametrize("c", [8, 16])
def test_msm_concentrated_scalars(c):
    """Every scalar one of two values: each window's entries fall into at most two buckets
    that span many 16-entry ranges (the wide-bucket combine).  The definition is evaluated
    as a sum over the two classes."""
    import __graft_entry__
    __graft_entry__.build()
    n = 1500
    P = [O.G]
    for _ in range(n - 1):
        P.append(O.point_add(P[-1], O.G))
    a = int.from_bytes(synth.random_bytes(c, "ca", 32).tobytes(), "little") % O.Q
    b = int.from_bytes(synth.random_bytes(c, "cb", 32).tobytes(), "little") % O.Q
    ks = [a if i % 3 else b for i in range(n)]
    Sa, Sb = O.IDENTITY, O.IDENTITY
    for i in range(n):
        if i % 3:
            Sa = O.point_add(Sa, P[i])
        else:
            Sb = O.point_add(Sb, P[i])
    want = O.encode_point(O.point_add(O.scalar_mult(a, Sa), O.scalar_mult(b, Sb)))
    with poslo.Context(device=0, msm_window=c) as cx:
        got = cx.msm(b"".join(O.encode_point(p) for p in P), b"".join(k.to_bytes(32, "little") for k in ks))
    assert got == want


@pytest.mark.parametrize("r", [4, 5, 6, 7, 8])
def test_msm_every_range_length(r):
    """Every range length 2^r of the bucket accumulation (buckets inside one range, buckets
    across ranges, a ragged last range) gives the definition's result."""
    import __graft_entry__
    __graft_entry__.build()
    n = 700
    pts = [O.encode_point(O.scalar_mult(9 + 13 * i, O.G)) for i in range(n)]
    ks = [int.from_bytes(synth.random_bytes(40 + r, f"r{i}", 32).tobytes(), "little") % O.Q for i in range(n)]
    with poslo.Context(device=0) as cx:
        cx.msm_set_plan(n, 10, r, scalar_words=8)
        assert cx.msm_get_plan(n, 8) == (10, r)
        got = cx.msm(b"".join(pts), b"".join(k.to_bytes(32, "little") for k in ks))
    assert got == O.msm(ks, pts)


@pytest.mark.parametrize("c,r", [(8, 6), (12, 8)])
def test_msm_concentrated_scalars_long_ranges(c, r):
    """Two scalar values over 2,500 entries with ranges of 2^r: each window's two buckets span
    many ranges (the wide-bucket join with warps striding over the ranges)."""
    import __graft_entry__
    __graft_entry__.build()
    n = 2500
    P = [O.G]
    for _ in range(n - 1):
        P.append(O.point_add(P[-1], O.G))
    a = int.from_bytes(synth.random_bytes(c + r, "la", 32).tobytes(), "little") % O.Q
    b = int.from_bytes(synth.random_bytes(c + r, "lb", 32).tobytes(), "little") % O.Q
    ks = [a if i % 4 else b for i in range(n)]
    Sa, Sb = O.IDENTITY, O.IDENTITY
    for i in range(n):
        if i % 4:
            Sa = O.point_add(Sa, P[i])
        else:
            Sb = O.point_add(Sb, P[i])
    want = O.encode_point(O.point_add(O.scalar_mult(a, Sa), O.scalar_mult(b, Sb)))
    with poslo.Context(device=0) as cx:
        cx.msm_set_plan(n, c, r, scalar_words=8)
        got = cx.msm(b"".join(O.encode_point(p) for p in P), b"".join(k.to_bytes(32, "little") for k in ks))
    assert got == want


@pytest.mark.parametrize("r", [5, 8])
def test_weighted_checks_every_range_length(r):
    """Weighted AVer and Distill with 127-bit weights keep the per-entry definition's result
    when the accumulation ranges are long."""
    import __graft_entry__
    __graft_entry__.build()
    D, n2, n = 6, 16, 600
    km, sk, Y, msgs, subsets, s, R, _ = _f_data(60 + r, n, D, n2, 1, 60)
    ds_l = O.ds_root(km.root, D)
    bad = synth.apply_tamper(msgs, synth.tamper_plan(60 + r, msgs, 9))
    with poslo.Context(device=0) as cx:
        for k in (1, 2, 4, 8, 16, 32, 64, 128, 256, 512):
            cx.msm_set_plan(k, 10, r)     # every size class the bisection's MSMs can fall in
        for m in (msgs, bad):
            b = cx.make_batch(poslo.VARIANT_F, n2, Y, m.data, m.offs, b"".join(s), b"".join(R),
                              O.ds_serialize(ds_l))
            wi, ws, wR = O.distill_f(Y, m.as_list(), 0, n2, s, R, ds_l)
            assert cx.aver(b, poslo.AGG_WEIGHTED) is (len(wi) == 0)
            idx, cs, cR = cx.distill(b)
            assert list(idx) == wi and cs == ws and cR == wR


def test_msm_plan_table():
    """The plan table: defaults, a stored plan per size class, a fixed width winning, and
    argument checks."""
    with poslo.Context(device=0) as cx:
        assert cx.msm_get_plan(1 << 20) == (16, 4)
        assert cx.msm_get_plan(30_000_000) == (16, 8)
        cx.msm_set_plan(1 << 20, 13, 6)
        assert cx.msm_get_plan((1 << 21) - 1) == (13, 6)
        assert cx.msm_get_plan(1 << 21) == (16, 5)      # 64 entries per bucket: ranges of 32
        for bad in [(1 << 20, 7, 4), (1 << 20, 17, 4), (1 << 20, 12, 3), (1 << 20, 12, 9)]:
            with pytest.raises(poslo.PosloError) as e:
                cx.msm_set_plan(*bad)
            assert e.value.code == -1
    with poslo.Context(device=0, msm_window=11) as cx:
        cx.msm_set_plan(1 << 20, 13, 6)
        assert cx.msm_get_plan(1 << 20)[0] == 11


def test_msm_rejects_undecodable_point(ctx):
    y = 2
    while O.decode_point(y.to_bytes(32, "little")) is not None:
        y += 1
    pts = [O.encode_point(O.G), y.to_bytes(32, "little")]
    with pytest.raises(poslo.PosloError):
        ctx.msm(b"".join(pts), bytes(64))


@pytest.mark.parametrize("n", [1, 2, 3, 5, 17])
def test_distill_small_batches_every_pattern(ctx, n):
    """Every tamper pattern of a tiny batch (all 2^n for n <= 5)."""
    D, n2 = 3, 4
    km, sk, Y, msgs, subsets, s, R, _ = _f_data(60 + n, n, D, n2, 3, 40)
    ds_l = O.ds_root(km.root, D)
    ds = O.ds_serialize(ds_l)
    patterns = range(1 << n) if n <= 5 else [0, 1, (1 << n) - 1, 0x5A5A & ((1 << n) - 1), 1 << (n - 1)]
    for pat in patterns:
        data = msgs.data.copy()
        for t in range(n):
            if pat >> t & 1:
                data[int(msgs.offs[t])] ^= 0x11
        bad = synth.Messages(data, msgs.offs)
        b = ctx.make_batch(poslo.VARIANT_F, n2, Y, bad.data, bad.offs, b"".join(s), b"".join(R), ds)
        idx, cs, cR = ctx.distill(b)
        want = [t for t in range(n) if pat >> t & 1]
        assert list(idx) == want, (n, pat)
        keep = [t for t in range(n) if not pat >> t & 1]
        assert cs == O.agg_scalars([s[t] for t in keep])
        assert cR == O.agg_points([R[t] for t in keep])
        assert ctx.aver(b, poslo.AGG_WEIGHTED) is (pat == 0)


def test_distill_dense_tampering(ctx):
    """40 % of 200 entries tampered: deep bisection with wide frontiers."""
    D, n2, n = 4, 16, 200
    km, sk, Y, msgs, subsets, s, R, _ = _f_data(70, n, D, n2, 1, 100)
    ds_l = O.ds_root(km.root, D)
    plan = synth.tamper_plan(70, msgs, 80)
    bad = synth.apply_tamper(msgs, plan)
    b = ctx.make_batch(poslo.VARIANT_F, n2, Y, bad.data, bad.offs, b"".join(s), b"".join(R), O.ds_serialize(ds_l))
    idx, cs, cR = ctx.distill(b)
    wi, ws, wR = O.distill_f(Y, bad.as_list(), 0, n2, s, R, ds_l)
    assert list(idx) == wi == list(plan.idx) and cs == ws and cR == wR


def test_decreasing_offsets_are_einval(ctx):
    """Offsets that go backwards are rejected (host and device inputs) before any read."""
    import torch
    D, n2, n = 2, 4, 8
    km, sk, Y, msgs, subsets, s, R, _ = _f_data(80, n, D, n2, 10, 20)
    ds = O.ds_serialize(O.ds_root(km.root, D))
    offs = msgs.offs.copy()
    offs[3], offs[4] = offs[4], offs[3]
    hb = ctx.make_batch(poslo.VARIANT_F, n2, Y, msgs.data, offs, b"".join(s), b"".join(R), ds)
    dev = lambda a: torch.from_numpy(np.ascontiguousarray(a).copy()).cuda()
    db = ctx.make_batch(poslo.VARIANT_F, n2, Y, dev(msgs.data), dev(offs.view(np.int64)),
                        dev(np.frombuffer(b"".join(s), np.uint8)), dev(np.frombuffer(b"".join(R), np.uint8)), ds)
    torch.cuda.synchronize()
    for b in (hb, db):
        for call in (lambda: ctx.aver(b), lambda: ctx.distill(b), lambda: ctx.hash_entries(b)):
            with pytest.raises(poslo.PosloError) as e:
                call()
            assert e.value.code == -1
    # the context stays usable
    good = ctx.make_batch(poslo.VARIANT_F, n2, Y, msgs.data, msgs.offs, b"".join(s), b"".join(R), ds)
    assert ctx.aver(good) is True


def test_distill_graph_replay_device_batch():
    """Distill calls on one device-resident batch are captured into a CUDA graph and replayed;
    every call still reads its own bytes (a different entry is tampered on each call)."""
    import torch
    import __graft_entry__
    __graft_entry__.build()
    D, n2, n = 4, 16, 120
    km, sk, Y, msgs, subsets, s, R, _ = _f_data(91, n, D, n2, 1, 80)
    ds_l = O.ds_root(km.root, D)
    with poslo.Context(device=0) as cx:
        dev = lambda a: torch.from_numpy(np.ascontiguousarray(a).copy()).cuda()
        d_msgs = dev(msgs.data)
        b = cx.make_batch(poslo.VARIANT_F, n2, Y, d_msgs, dev(msgs.offs.astype(np.int64)),
                          dev(np.frombuffer(b"".join(s), np.uint8)), dev(np.frombuffer(b"".join(R), np.uint8)),
                          O.ds_serialize(ds_l))
        # trial 1's data first: the localisation of a failing call grows its own workspace
        # once, which would invalidate a graph captured before it; that first call also builds
        # the key's table (a shape of its own), so the second call of the cached shape captures
        for trial in [1] + list(range(5)):
            data = msgs.data.copy()
            tampered = []
            if trial:
                t = (17 * trial) % n
                data[int(msgs.offs[t])] ^= 0x33
                tampered = [t]
            d_msgs.copy_(torch.from_numpy(data))
            torch.cuda.synchronize()
            idx, cs, cR = cx.distill(b)
            wi, ws, wR = O.distill_f(Y, synth.Messages(data, msgs.offs).as_list(), 0, n2, s, R, ds_l)
            assert list(idx) == wi == tampered and cs == ws and cR == wR, trial
        assert cx.graph_stats() == (1, 3)


def test_more_than_2p32_minus_1_entries_is_einval(ctx):
    """A call over more entries than 32-bit entry indices can name fails with EINVAL before it
    reads any input (the pointers below lead to a few bytes only)."""
    import ctypes as C
    buf = np.zeros(64, np.uint8)
    p = buf.ctypes.data
    n = 1 << 32
    b = poslo.Batch()
    b.variant, b.n2, b.Y, b.msgs, b.offs, b.s, b.R = poslo.VARIANT_F, 8, p, p, p, p, p
    b.n, b.first_index, b.R_count, b.ds, b.ds_nodes, b.on_device = n, 0, n, p, 1, 0
    acc, cnt = np.zeros(1, np.uint8), C.c_uint64()
    assert ctx.lib.poslo_aver(ctx.h, C.byref(b), poslo.AGG_UNIT, acc.ctypes.data) == -1
    assert ctx.lib.poslo_distill(ctx.h, C.byref(b), p, 0, C.byref(cnt), None, None) == -1
    start = np.array([0, n], np.uint64)
    zero64, n2, dsoff = np.zeros(1, np.uint64), np.full(1, 8, np.uint32), np.array([0, 1], np.uint32)
    mb = poslo.MultiBatch()
    mb.n_dev, mb.Y, mb.dev_start, mb.first_index, mb.n2 = 1, p, start.ctypes.data, zero64.ctypes.data, n2.ctypes.data
    mb.ds, mb.ds_off, mb.msgs, mb.offs, mb.s, mb.R, mb.on_device = p, dsoff.ctypes.data, p, p, p, p, 0
    assert ctx.lib.poslo_aver_multi(ctx.h, C.byref(mb), acc.ctypes.data, p, 0, C.byref(cnt)) == -1

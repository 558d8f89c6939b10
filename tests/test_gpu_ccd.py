"""POSLO-C distillation (ccd^v, umbrellas, ccd^i) and SeBVer modes V/U/I (Fig. 3b) on the GPU
against the oracle, through the C ABI, in both instantiations."""
import numpy as np
import pytest

from oracle import poslo_oracle as O
from paper_2506_08781_gb300 import poslo, synth

pytestmark = pytest.mark.gpu

INSTS = [("POSLO", poslo.INST_SHA256), ("POSLO+", poslo.INST_AES)]


@pytest.fixture(scope="module", params=INSTS, ids=[n for n, _ in INSTS])
def env(request):
    import __graft_entry__
    __graft_entry__.build()
    name, inst = request.param
    c = poslo.Context(device=0, instantiation=inst)
    with O.instantiation(name):
        yield c, name
    c.close()


def _epochs(seed, D, n2, n1):
    km = synth.key_material(seed)
    sk, Y, epoch_R = O.kg_c(km.y, km.r, km.root, D, n2)
    msgs = synth.messages(seed, n1 * n2, 1, 60)
    ms = [[msgs.entry(i * n2 + j) for j in range(n2)] for i in range(n1)]
    s_ep = [O.sig_c(sk, i, ms[i]) for i in range(n1)]
    return km, Y, list(epoch_R[:n1]), ms, s_ep


def _flip(ms, i, j):
    m = ms[i][j]
    ms[i][j] = bytes([m[0] ^ 0x11]) + m[1:]


def _run(ctx, Y, ms, n2, s_ep, R, ds_l, n_u, first_epoch=0):
    flat = synth.pack([m for mk in ms for m in mk])
    b = ctx.make_batch(poslo.VARIANT_C, n2, Y, flat.data, flat.offs, b"".join(s_ep), b"".join(R),
                       O.ds_serialize(ds_l), first_index=first_epoch * n2)
    valid, ccd = ctx.distill_c(b, n_u)
    epochs = list(range(first_epoch, first_epoch + len(ms)))
    wb, wccd = O.distill_c(Y, epochs, ms, n2, s_ep, R, ds_l, n_u)
    assert valid == wb
    assert (ccd["s_v"], ccd["R_v"]) == (wccd.sv, wccd.Rv)
    assert ccd["umbrellas"] == [(su, Ru) for su, Ru, _ in wccd.umbrellas]
    assert ccd["invalid"] == [i for _, _, i in wccd.invalid]
    for mode in "VUI":
        assert ctx.sebver_c(b, n_u, ccd, mode) == O.sebver_c(Y, epochs, ms, n2, wccd, ds_l, mode), mode
    return valid, ccd


@pytest.mark.parametrize("pattern", ["none", "one", "two_same_group", "whole_group", "last_of_group"])
def test_distill_c_patterns(env, pattern):
    ctx, _ = env
    km, Y, R, ms, s_ep = _epochs(60, 3, 8, 8)
    flips = {"none": [], "one": [(3, 5)], "two_same_group": [(4, 0), (5, 7)],
             "whole_group": [(6, 1), (7, 2)], "last_of_group": [(1, 3), (7, 7)]}[pattern]
    for i, j in flips:
        _flip(ms, i, j)
    valid, ccd = _run(ctx, Y, ms, 8, s_ep, R, O.ds_root(km.root, 3), 4)
    assert ccd["invalid"] == sorted({i for i, _ in flips})


def test_distill_c_malformed_signatures(env):
    # a non-canonical s~_i, an undecodable R~_i and two swapped s~: all their epochs invalid
    ctx, _ = env
    km, Y, R, ms, s_ep = _epochs(61, 3, 4, 8)
    s_ep[1] = (int.from_bytes(s_ep[1], "little") + O.Q).to_bytes(32, "little")
    y = 2
    while O.decode_point(y.to_bytes(32, "little")) is not None:
        y += 1
    R[4] = y.to_bytes(32, "little")
    s_ep[6], s_ep[7] = s_ep[7], s_ep[6]
    valid, ccd = _run(ctx, Y, ms, 4, s_ep, R, O.ds_root(km.root, 3), 2)
    assert ccd["invalid"] == [1, 4, 6, 7]


def test_distill_c_subrange_under_ds(env):
    # epochs 2..5 of an 8-epoch key under ds_5: global epoch indices in ccd^i
    ctx, _ = env
    km, Y, R, ms, s_ep = _epochs(62, 3, 4, 8)
    _flip(ms, 3, 0)
    sub = slice(2, 6)
    valid, ccd = _run(ctx, Y, ms[sub], 4, s_ep[sub], R[sub], O.ds_after(km.root, 3, 5), 2, first_epoch=2)
    assert ccd["invalid"] == [3]


def test_distill_c_errors(env):
    ctx, _ = env
    km, Y, R, ms, s_ep = _epochs(63, 2, 4, 4)
    for i in range(4):
        _flip(ms, i, 1)
    flat = synth.pack([m for mk in ms for m in mk])
    b = ctx.make_batch(poslo.VARIANT_C, 4, Y, flat.data, flat.offs, b"".join(s_ep), b"".join(R),
                       O.ds_serialize(O.ds_root(km.root, 2)))
    with pytest.raises(poslo.PosloError) as e:
        ctx.distill_c(b, 3)                          # 3 does not divide n1 = 4
    assert e.value.code == -1
    with pytest.raises(poslo.PosloError) as e:
        ctx.distill_c(b, 2, cap=2)                   # 4 invalid epochs, room for 2
    assert e.value.code == -5


@pytest.mark.parametrize("n_u", [1, 8])
def test_distill_c_umbrella_extremes(env, n_u):
    # one umbrella over the whole batch, and one umbrella per epoch
    ctx, _ = env
    km, Y, R, ms, s_ep = _epochs(64, 3, 4, 8)
    _flip(ms, 2, 1)
    _flip(ms, 5, 3)
    valid, ccd = _run(ctx, Y, ms, 4, s_ep, R, O.ds_root(km.root, 3), n_u)
    assert ccd["invalid"] == [2, 5] and len(ccd["umbrellas"]) == n_u


def test_distill_c_every_epoch_invalid(env):
    ctx, _ = env
    km, Y, R, ms, s_ep = _epochs(65, 2, 4, 4)
    for i in range(4):
        _flip(ms, i, 0)
    valid, ccd = _run(ctx, Y, ms, 4, s_ep, R, O.ds_root(km.root, 2), 2)
    assert valid == [False] * 4 and ccd["s_v"] == bytes(32) and ccd["R_v"] == O.encode_point(O.IDENTITY)


def test_distill_c_and_sebver_use_the_key_cache(env):
    """POSLO-C Distill builds the key's window table into the context's key cache and the
    SeBVer calls that follow reuse it (results equal the oracle's all along); a key that does
    not decode is refused (EINVAL) and not kept, so the next call misses again."""
    ctx, _ = env
    km, Y, R, ms, s_ep = _epochs(66, 2, 4, 4)
    _flip(ms, 1, 2)
    ds_l = O.ds_root(km.root, 2)
    h0, m0 = ctx.key_cache_stats()
    _run(ctx, Y, ms, 4, s_ep, R, ds_l, 2)           # distill_c misses, SeBVer V, U and I hit
    h1, m1 = ctx.key_cache_stats()
    assert (h1 - h0, m1 - m0) == (3, 1)
    y = 2
    while O.decode_point(y.to_bytes(32, "little")) is not None:
        y += 1
    flat = synth.pack([m for mk in ms for m in mk])
    b = ctx.make_batch(poslo.VARIANT_C, 4, y.to_bytes(32, "little"), flat.data, flat.offs, b"".join(s_ep),
                       b"".join(R), O.ds_serialize(ds_l))
    for _ in range(2):
        with pytest.raises(poslo.PosloError) as e:
            ctx.distill_c(b, 2)
        assert e.value.code == -1
    h2, m2 = ctx.key_cache_stats()
    assert (h2 - h1, m2 - m1) == (0, 2)

"""The context's cache of key window tables: hits and misses, eviction, keys that do not
decode, and duplicate keys in one multi-device call.  Every result is compared with the
oracle's per-entry definition."""
import numpy as np
import pytest

from oracle import poslo_oracle as O
from paper_2506_08781_gb300 import poslo, synth

pytestmark = pytest.mark.gpu


def _signer(seed, n, D=3, n2=8, tamper=0):
    km = synth.key_material(seed, v=16)
    sk, Y = O.kg_f(km.y, km.root, D, n2, km.bpv_r.tobytes())
    msgs = synth.messages(seed, n, 1, 40)
    subsets = synth.bpv_subsets(seed, n, v=16, k=4)
    sig = [O.sig_f(sk, t, msgs.entry(t), subsets[t]) for t in range(n)]
    s, R = [x[0] for x in sig], [x[1] for x in sig]
    if tamper:
        msgs = synth.apply_tamper(msgs, synth.tamper_plan(seed, msgs, tamper))
    ds_l = O.ds_root(km.root, D)
    return Y, msgs, s, R, ds_l, n2


def _undecodable():
    y = 2
    while O.decode_point(y.to_bytes(32, "little")) is not None:
        y += 1
    return y.to_bytes(32, "little")


def _distill(cx, sig):
    Y, msgs, s, R, ds_l, n2 = sig
    b = cx.make_batch(poslo.VARIANT_F, n2, Y, msgs.data, msgs.offs, b"".join(s), b"".join(R), O.ds_serialize(ds_l))
    idx, cs, cR = cx.distill(b)
    wi, ws, wR = O.distill_f(Y, msgs.as_list(), 0, n2, s, R, ds_l)
    assert list(idx) == wi and cs == ws and cR == wR
    return wi


def test_distill_hits_misses_and_eviction():
    import __graft_entry__
    __graft_entry__.build()
    sigs = [_signer(300 + k, 20 + k, tamper=k % 2) for k in range(3)]
    with poslo.Context(device=0) as cx:
        _distill(cx, sigs[0])
        _distill(cx, sigs[0])
        assert cx.key_cache_stats() == (1, 1)
        cx.set_key_cache(2)                          # drops the table, keeps the counters
        for k in [0, 1, 0, 2, 1, 0]:                 # 2 evicts 1 (least recent), then 1 evicts 0
            _distill(cx, sigs[k])
        hits, misses = cx.key_cache_stats()
        assert (hits - 1, misses - 1) == (1, 5)
        cx.set_key_cache(0)                          # off: every call builds its table
        _distill(cx, sigs[2])
        assert cx.key_cache_stats() == (hits, misses)


def test_undecodable_key_is_not_kept():
    import __graft_entry__
    __graft_entry__.build()
    Y, msgs, s, R, ds_l, n2 = _signer(310, 12)
    bad = _undecodable()
    with poslo.Context(device=0) as cx:
        for _ in range(2):
            b = cx.make_batch(poslo.VARIANT_F, n2, bad, msgs.data, msgs.offs, b"".join(s), b"".join(R),
                              O.ds_serialize(ds_l))
            with pytest.raises(poslo.PosloError) as e:
                cx.distill(b)
            assert e.value.code == -1
        assert cx.key_cache_stats() == (0, 2)       # missed both times: never kept
        _distill(cx, (Y, msgs, s, R, ds_l, n2))


def _multi(cx, parts):
    cat = synth.pack([m for p in parts for m in p[1].as_list()])
    s = b"".join(b"".join(p[2]) for p in parts)
    R = b"".join(b"".join(p[3]) for p in parts)
    return cx.aver_multi([p[0] for p in parts], [p[1].n for p in parts], [0] * len(parts), [p[5] for p in parts],
                         [O.ds_serialize(p[4]) for p in parts], cat.data, cat.offs, s, R)


def _want(parts):
    return O.verify_multi([(p[0], p[1].as_list(), 0, p[5], p[2], p[3], p[4]) for p in parts])


def test_multi_cache_duplicates_and_fallback():
    import __graft_entry__
    __graft_entry__.build()
    base = [_signer(320 + k, 6 + 3 * k, tamper=1 if k == 2 else 0) for k in range(4)]
    # devices 4 and 5 sign under the keys of devices 0 and 2 (same key, other logs)
    dup = []
    for k, src in [(4, 0), (5, 2)]:
        km = synth.key_material(320 + src, v=16)
        sk, Y = O.kg_f(km.y, km.root, 3, 8, km.bpv_r.tobytes())
        msgs = synth.messages(400 + k, 9, 1, 40)
        subsets = synth.bpv_subsets(400 + k, 9, v=16, k=4)
        sig = [O.sig_f(sk, t, msgs.entry(t), subsets[t]) for t in range(9)]
        if k == 5:
            msgs = synth.apply_tamper(msgs, synth.tamper_plan(400 + k, msgs, 1))
        dup.append((Y, msgs, [x[0] for x in sig], [x[1] for x in sig], O.ds_root(km.root, 3), 8))
    parts = base + dup
    want_acc, want_pairs = _want(parts)
    with poslo.Context(device=0) as cx:
        for _ in range(3):
            acc, pairs = _multi(cx, parts)
            assert list(acc) == want_acc
            assert [tuple(int(x) for x in p) for p in pairs] == want_pairs
        hits, misses = cx.key_cache_stats()
        assert misses == 4 and hits == 2 + 2 * len(parts)
        cx.set_key_cache(3)                          # fewer slots than the call has keys
        acc, pairs = _multi(cx, parts)
        assert list(acc) == want_acc and [tuple(int(x) for x in p) for p in pairs] == want_pairs
        assert cx.key_cache_stats() == (hits, misses)
        # a key that does not decode fails the call and leaves no table behind
        cx.set_key_cache(64)
        badparts = list(parts)
        Y, msgs, s, R, ds_l, n2 = badparts[1]
        badparts[1] = (_undecodable(), msgs, s, R, ds_l, n2)
        with pytest.raises(poslo.PosloError) as e:
            _multi(cx, badparts)
        assert e.value.code == -1
        acc, pairs = _multi(cx, parts)
        assert list(acc) == want_acc


def test_aver_shares_the_cache():
    """AVer takes the key's table from the cache too (unit and weighted, valid and tampered),
    shares it with Distill, and keeps no table of a key that does not decode."""
    import __graft_entry__
    __graft_entry__.build()
    Y, msgs, s, R, ds_l, n2 = sig = _signer(330, 24)
    bad_msgs = synth.apply_tamper(msgs, synth.tamper_plan(330, msgs, 1))
    mk = lambda cx, key, m: cx.make_batch(poslo.VARIANT_F, n2, key, m.data, m.offs, b"".join(s), b"".join(R),
                                          O.ds_serialize(ds_l))
    with poslo.Context(device=0) as cx:
        assert cx.aver(mk(cx, Y, msgs)) is True
        assert cx.aver(mk(cx, Y, msgs), poslo.AGG_WEIGHTED) is True
        assert cx.aver(mk(cx, Y, bad_msgs)) is False
        assert cx.aver(mk(cx, Y, bad_msgs), poslo.AGG_WEIGHTED) is False
        assert cx.key_cache_stats() == (3, 1)
        _distill(cx, sig)
        assert cx.key_cache_stats() == (4, 1)
        bad = _undecodable()
        for _ in range(2):
            with pytest.raises(poslo.PosloError) as e:
                cx.aver(mk(cx, bad, msgs))
            assert e.value.code == -1
        assert cx.key_cache_stats() == (4, 3)
        assert cx.aver(mk(cx, Y, msgs)) is True
        cx.set_key_cache(0)
        assert cx.aver(mk(cx, Y, bad_msgs)) is False
        assert cx.key_cache_stats() == (5, 3)

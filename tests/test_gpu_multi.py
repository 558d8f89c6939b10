"""Multi-device AVer + Distill (many signers in one batch) against the oracle's per-device
definition, through the C ABI."""
import numpy as np
import pytest

from oracle import poslo_oracle as O
from paper_2506_08781_gb300 import poslo, synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctx():
    import __graft_entry__
    __graft_entry__.build()
    c = poslo.Context(device=0, verifier_seed=synth.verifier_seed(123))
    yield c
    c.close()


def _devices(seed, n_dev, lo, hi, tampered, D=4, n2=4, v=16, k=4, empty=()):
    sizes = synth.device_sizes(seed, n_dev, lo, hi)
    for d in empty:
        sizes[d] = 0
    devs, parts = [], []
    bad_devs = set(int(d) for d in synth.choose_without_replacement(seed, "baddev", n_dev, tampered))
    for d in range(n_dev):
        km = synth.key_material(seed * 1000 + d, v=v)
        sk, Y = O.kg_f(km.y, km.root, D, n2, km.bpv_r.tobytes())
        first = int(synth.uniform_int(seed, f"first{d}", 1, 0, 3)[0])
        msgs = synth.messages(seed * 1000 + d, int(sizes[d]), 0, 60)
        subsets = synth.bpv_subsets(seed * 1000 + d, msgs.n, first_index=first, v=v, k=k)
        sig = [O.sig_f(sk, first + t, msgs.entry(t), subsets[t]) for t in range(msgs.n)]
        s = [x[0] for x in sig]
        R = [x[1] for x in sig]
        if d in bad_devs and msgs.n and any(len(m) for m in msgs.as_list()):
            cand = [t for t in range(msgs.n) if len(msgs.entry(t))]
            t = cand[int(synth.uniform_int(seed, f"t{d}", 1, 0, len(cand) - 1)[0])]
            data = msgs.data.copy()
            data[int(msgs.offs[t])] ^= 0x21
            msgs = synth.Messages(data, msgs.offs)
        ds = O.ds_root(km.root, D)
        devs.append((Y, msgs.as_list(), first, n2, s, R, ds))
        parts.append((Y, msgs, first, n2, s, R, O.ds_serialize(ds)))
    return devs, parts


def _concat(parts):
    entries = [m for p in parts for m in p[1].as_list()]
    cat = synth.pack(entries)
    s = b"".join(b"".join(p[4]) for p in parts)
    R = b"".join(b"".join(p[5]) for p in parts)
    return cat, s, R


@pytest.mark.parametrize("seed,n_dev,tampered", [(1, 12, 3), (2, 7, 0), (3, 20, 20)])
def test_multi_matches_per_device_definition(ctx, seed, n_dev, tampered):
    devs, parts = _devices(seed, n_dev, 1, 40, tampered)
    cat, s, R = _concat(parts)
    acc, pairs = ctx.aver_multi([p[0] for p in parts], [p[1].n for p in parts], [p[2] for p in parts],
                                [p[3] for p in parts], [p[6] for p in parts], cat.data, cat.offs, s, R)
    want_acc, want_pairs = O.verify_multi(devs)
    assert list(acc) == want_acc
    assert [tuple(int(x) for x in p) for p in pairs] == want_pairs


def test_multi_cancelling_errors_fall_back(ctx):
    """Two devices whose s-shifts cancel inside every unit aggregate are still localised."""
    devs, parts = _devices(4, 5, 6, 12, 0)
    Y, msgs, first, n2, s, R, ds = parts[2]
    s = list(s)
    s[1] = O.scalar_to_bytes(int.from_bytes(s[1], "little") + 5)
    s[4] = O.scalar_to_bytes(int.from_bytes(s[4], "little") - 5)
    parts[2] = (Y, msgs, first, n2, s, R, ds)
    d = devs[2]
    devs[2] = (d[0], d[1], d[2], d[3], s, d[5], d[6])
    cat, sb, Rb = _concat(parts)
    acc, pairs = ctx.aver_multi([p[0] for p in parts], [p[1].n for p in parts], [p[2] for p in parts],
                                [p[3] for p in parts], [p[6] for p in parts], cat.data, cat.offs, sb, Rb)
    want_acc, want_pairs = O.verify_multi(devs)
    assert list(acc) == want_acc and [tuple(int(x) for x in p) for p in pairs] == want_pairs
    assert want_pairs == [(2, first + 1), (2, first + 4)]


def test_multi_device_inputs_and_empty_device(ctx):
    import torch
    devs, parts = _devices(5, 6, 1, 10, 2, empty=(3,))
    cat, s, R = _concat(parts)
    dev = lambda a: torch.from_numpy(np.ascontiguousarray(a).copy()).cuda()
    acc, pairs = ctx.aver_multi([p[0] for p in parts], [p[1].n for p in parts], [p[2] for p in parts],
                                [p[3] for p in parts], [p[6] for p in parts], dev(cat.data),
                                dev(cat.offs.view(np.int64)), dev(np.frombuffer(s, np.uint8)),
                                dev(np.frombuffer(R, np.uint8)))
    want_acc, want_pairs = O.verify_multi(devs)
    assert list(acc) == want_acc and [tuple(int(x) for x in p) for p in pairs] == want_pairs


def test_multi_malformed_entries_and_capacity(ctx):
    """A non-canonical s_t and an undecodable R_t inside one device are listed like tampered
    entries; a list longer than the caller's room is EBUFSMALL."""
    devs, parts = _devices(6, 4, 3, 10, 1)
    Y, msgs, first, n2, s, R, ds = parts[1]
    s, R = list(s), list(R)
    s[0] = (int.from_bytes(s[0], "little") + O.Q).to_bytes(32, "little")
    y = 2
    while O.decode_point(y.to_bytes(32, "little")) is not None:
        y += 1
    R[2] = y.to_bytes(32, "little")
    parts[1] = (Y, msgs, first, n2, s, R, ds)
    d = devs[1]
    devs[1] = (d[0], d[1], d[2], d[3], s, R, d[6])
    cat, sb, Rb = _concat(parts)
    args = ([p[0] for p in parts], [p[1].n for p in parts], [p[2] for p in parts], [p[3] for p in parts],
            [p[6] for p in parts], cat.data, cat.offs, sb, Rb)
    acc, pairs = ctx.aver_multi(*args)
    want_acc, want_pairs = O.verify_multi(devs)
    assert list(acc) == want_acc and [tuple(int(x) for x in p) for p in pairs] == want_pairs
    assert (1, first) in want_pairs and (1, first + 2) in want_pairs
    with pytest.raises(poslo.PosloError) as e:
        ctx.aver_multi(*args, cap=len(want_pairs) - 1)
    assert e.value.code == -5


def _flip_entry(data, offs, t):
    out = data.copy()
    out[int(offs[t])] ^= 0x5a
    return out


@pytest.mark.parametrize("on_device", [False, True])
def test_multi_graph_replay_reads_each_calls_inputs(on_device):
    """Calls of one shape are captured into a CUDA graph and replayed; every call still reads
    its own message bytes (a different entry is tampered on each call)."""
    import torch
    import __graft_entry__
    __graft_entry__.build()
    devs, parts = _devices(7, 6, 2, 20, 0)
    cat, s, R = _concat(parts)
    starts = np.concatenate([[0], np.cumsum([p[1].n for p in parts])])
    args = ([p[0] for p in parts], [p[1].n for p in parts], [p[2] for p in parts], [p[3] for p in parts],
            [p[6] for p in parts])
    with poslo.Context(device=0, verifier_seed=synth.verifier_seed(7)) as cx:
        if on_device:
            d_msgs = torch.from_numpy(cat.data.copy()).cuda()
            d_offs = torch.from_numpy(cat.offs.view(np.int64).copy()).cuda()
            d_s = torch.from_numpy(np.frombuffer(s, np.uint8).copy()).cuda()
            d_R = torch.from_numpy(np.frombuffer(R, np.uint8).copy()).cuda()
        # trial 1's data first: the localisation of a failing call grows its own workspace
        # once, which would invalidate a graph captured before it; that first call also builds
        # the key tables (a shape of its own), so the second call of the cached shape captures
        for trial in [1] + list(range(5)):
            data = cat.data
            want_devs = [tuple(d) for d in devs]
            if trial:
                dev = trial % len(parts)
                lens = np.diff(cat.offs[starts[dev]:starts[dev + 1] + 1])
                t = int(starts[dev] + int(np.argmax(lens > 0)))
                data = _flip_entry(cat.data, cat.offs, t)
                d = devs[dev]
                ms = list(d[1])
                ms[t - starts[dev]] = bytes(data[int(cat.offs[t]):int(cat.offs[t + 1])])
                want_devs[dev] = (d[0], ms, d[2], d[3], d[4], d[5], d[6])
            if on_device:
                d_msgs.copy_(torch.from_numpy(data))
                torch.cuda.synchronize()
                acc, pairs = cx.aver_multi(*args, d_msgs, d_offs, d_s, d_R)
            else:
                acc, pairs = cx.aver_multi(*args, data, cat.offs, s, R)
            want_acc, want_pairs = O.verify_multi(want_devs)
            assert list(acc) == want_acc, trial
            assert [tuple(int(x) for x in p) for p in pairs] == want_pairs, trial
        captures, replays = cx.graph_stats()
        assert captures == 1 and replays == 3
        # a larger call in between regrows the workspace: the next call of the first shape
        # must not replay the stale graph
        devs2, parts2 = _devices(8, 9, 30, 60, 1)
        cat2, s2, R2 = _concat(parts2)
        acc2, pairs2 = cx.aver_multi([p[0] for p in parts2], [p[1].n for p in parts2], [p[2] for p in parts2],
                                     [p[3] for p in parts2], [p[6] for p in parts2], cat2.data, cat2.offs, s2, R2)
        w2 = O.verify_multi(devs2)
        assert list(acc2) == w2[0]
        if on_device:
            d_msgs.copy_(torch.from_numpy(cat.data))
            torch.cuda.synchronize()
            acc, pairs = cx.aver_multi(*args, d_msgs, d_offs, d_s, d_R)
        else:
            acc, pairs = cx.aver_multi(*args, cat.data, cat.offs, s, R)
        assert list(acc) == [True] * len(parts) and len(pairs) == 0
        assert cx.graph_stats()[1] == 3


def test_multi_graphs_off_same_results():
    import __graft_entry__
    __graft_entry__.build()
    devs, parts = _devices(9, 5, 2, 16, 2)
    cat, s, R = _concat(parts)
    args = ([p[0] for p in parts], [p[1].n for p in parts], [p[2] for p in parts], [p[3] for p in parts],
            [p[6] for p in parts], cat.data, cat.offs, s, R)
    want_acc, want_pairs = O.verify_multi(devs)
    with poslo.Context(device=0) as cx:
        cx.set_graphs(False)
        for _ in range(3):
            acc, pairs = cx.aver_multi(*args)
            assert list(acc) == want_acc and [tuple(int(x) for x in p) for p in pairs] == want_pairs
        assert cx.graph_stats() == (0, 0)


@pytest.mark.parametrize("limit", [0, 1 << 40])
def test_multi_both_check_forms(limit):
    """The combined weighted check with the full weights (limit 0) and window by window (any
    batch below the limit) give the same per-device results: tampered devices, malformed
    entries and cancelling s-shifts."""
    import __graft_entry__
    __graft_entry__.build()
    devs, parts = _devices(11, 9, 1, 30, 3)
    Y, msgs, first, n2, s, R, ds = parts[4]
    s = list(s)
    s[0] = O.scalar_to_bytes(int.from_bytes(s[0], "little") + 9)
    s[-1] = O.scalar_to_bytes(int.from_bytes(s[-1], "little") - 9)
    parts[4] = (Y, msgs, first, n2, s, R, ds)
    d = devs[4]
    devs[4] = (d[0], d[1], d[2], d[3], s, d[5], d[6])
    cat, sb, Rb = _concat(parts)
    want_acc, want_pairs = O.verify_multi(devs)
    with poslo.Context(device=0, verifier_seed=synth.verifier_seed(11)) as cx:
        cx.set_multi_window_limit(limit)
        for _ in range(2):
            acc, pairs = cx.aver_multi([p[0] for p in parts], [p[1].n for p in parts], [p[2] for p in parts],
                                       [p[3] for p in parts], [p[6] for p in parts], cat.data, cat.offs, sb, Rb)
            assert list(acc) == want_acc
            assert [tuple(int(x) for x in p) for p in pairs] == want_pairs
    assert want_acc.count(False) >= 2


def test_multi_devices_across_segment_pieces(ctx):
    """Devices of 0, 1, 2047, 2048, 2049, 4097 and 6500 entries: the per-device sums are taken
    in pieces of 2,048 entries and combined, so devices at and around the piece size, with
    tampered, non-canonical and undecodable entries in later pieces, must still give every
    device's own Distill result (C++ oracle, itself pinned to the Python oracle)."""
    from oracle import cpp_oracle as X
    D, n2 = 16, 4
    sizes = [2049, 0, 1, 2048, 6500, 2047, 4097]
    parts, want_acc, want_pairs = [], [], []
    for d, n in enumerate(sizes):
        km = synth.key_material(900 + d, v=16)
        msgs = synth.messages(900 + d, n, 1, 60)
        sub = synth.bpv_subsets(900 + d, n, v=16, k=4)
        s, R = X.sign_f(km.y, km.root, D, n2, km.bpv_r, sub, msgs.data, msgs.offs, 0)
        s, R = bytearray(s.tobytes()[:32 * n]), bytearray(R.tobytes()[:32 * n])
        if n == 2049:      # non-canonical s in the second piece
            v = int.from_bytes(bytes(s[32 * 2048:32 * 2049]), "little") + O.Q
            s[32 * 2048:32 * 2049] = v.to_bytes(32, "little")
        if n == 6500:      # flips in the third and fourth pieces, an undecodable R in the first
            msgs = synth.apply_tamper(msgs, synth.Tamper(np.array([4500, 6499]), np.zeros(2, np.int64),
                                                         np.array([0x21, 0x80], np.uint8)))
            R[32 * 10:32 * 11] = (O.P + 1).to_bytes(32, "little")
        if n == 4097:      # the entry alone in the last piece
            msgs = synth.apply_tamper(msgs, synth.Tamper(np.array([4096]), np.zeros(1, np.int64),
                                                         np.array([0x01], np.uint8)))
        Y = X.base_mult(int.from_bytes(km.y, "little"))
        ds = O.ds_serialize(O.ds_root(km.root, D))
        inv, _, _ = X.distill_f(Y, msgs.data, msgs.offs, 0, n2, bytes(s), bytes(R), ds)
        want_acc.append(not inv)
        want_pairs += [(d, int(t)) for t in inv]
        parts.append((Y, msgs, bytes(s), bytes(R), ds))
    cat = synth.pack([m for p in parts for m in p[1].as_list()])
    acc, pairs = ctx.aver_multi([p[0] for p in parts], sizes, [0] * len(sizes), [n2] * len(sizes),
                                [p[4] for p in parts], cat.data, cat.offs, b"".join(p[2] for p in parts),
                                b"".join(p[3] for p in parts))
    assert list(acc) == want_acc and [tuple(int(x) for x in p) for p in pairs] == want_pairs
    assert want_acc == [False, True, True, True, False, True, False]
    assert (4, 10) in want_pairs and (4, 4500) in want_pairs and (6, 4096) in want_pairs

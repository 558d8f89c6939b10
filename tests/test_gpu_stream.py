"""Out-of-core AVer + Distill (poslo_distill_stream): chunk by chunk from host memory, with the
same result as Distill over the whole batch (the per-entry definition)."""
import numpy as np
import pytest

from oracle import poslo_oracle as O
from paper_2506_08781_gb300 import poslo, synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def data():
    import __graft_entry__
    __graft_entry__.build()
    D, n2, n = 5, 16, 300
    km = synth.key_material(70, v=32)
    sk, Y = O.kg_f(km.y, km.root, D, n2, km.bpv_r.tobytes())
    msgs = synth.messages(70, n, 0, 120)
    subsets = synth.bpv_subsets(70, n, first_index=5, v=32, k=4)
    sig = [O.sig_f(sk, 5 + t, msgs.entry(t), subsets[t]) for t in range(n)]
    s, R = [x[0] for x in sig], [x[1] for x in sig]
    bad = synth.apply_tamper(msgs, synth.tamper_plan(70, msgs, 9))
    s[40] = (int.from_bytes(s[40], "little") + O.Q).to_bytes(32, "little")    # malformed s
    ds_l = O.ds_root(km.root, D)
    want, _, _ = O.distill_f(Y, bad.as_list(), 5, n2, s, R, ds_l)
    ctx = poslo.Context(device=0)
    yield ctx, Y, bad, s, R, ds_l, n2, want
    ctx.close()


@pytest.mark.parametrize("chunk", [1, 7, 64, 299, 300, 1000])
def test_stream_equals_definition(data, chunk):
    ctx, Y, bad, s, R, ds_l, n2, want = data
    b = ctx.make_batch(poslo.VARIANT_F, n2, Y, bad.data, bad.offs, b"".join(s), b"".join(R), O.ds_serialize(ds_l),
                       first_index=5)
    acc, idx = ctx.distill_stream(b, chunk)
    assert acc is False and list(idx) == want


def test_stream_pinned_inputs_and_capacity(data):
    import torch
    ctx, Y, bad, s, R, ds_l, n2, want = data
    pin = lambda a: torch.from_numpy(np.ascontiguousarray(a).copy()).pin_memory()
    b = ctx.make_batch(poslo.VARIANT_F, n2, Y, pin(bad.data), pin(bad.offs.view(np.int64)),
                       pin(np.frombuffer(b"".join(s), np.uint8)), pin(np.frombuffer(b"".join(R), np.uint8)),
                       O.ds_serialize(ds_l), first_index=5)
    acc, idx = ctx.distill_stream(b, 50)
    assert acc is False and list(idx) == want
    with pytest.raises(poslo.PosloError) as e:
        ctx.distill_stream(b, 50, cap=len(want) - 1)
    assert e.value.code == -5


def test_stream_honest_and_errors(data):
    ctx, Y, bad, s, R, ds_l, n2, want = data
    D, n = 3, 40
    km = synth.key_material(71, v=32)
    sk, Y2 = O.kg_f(km.y, km.root, D, 8, km.bpv_r.tobytes())
    msgs = synth.messages(71, n, 0, 50)
    subsets = synth.bpv_subsets(71, n, v=32, k=4)
    sig = [O.sig_f(sk, t, msgs.entry(t), subsets[t]) for t in range(n)]
    b = ctx.make_batch(poslo.VARIANT_F, 8, Y2, msgs.data, msgs.offs, b"".join(x[0] for x in sig),
                       b"".join(x[1] for x in sig), O.ds_serialize(O.ds_root(km.root, D)))
    acc, idx = ctx.distill_stream(b, 16)
    assert acc is True and len(idx) == 0
    with pytest.raises(poslo.PosloError) as e:
        ctx.distill_stream(b, 0)
    assert e.value.code == -1


def test_stream_empty_batch(data):
    ctx, Y, bad, s, R, ds_l, n2, want = data
    e = synth.pack([])
    b = ctx.make_batch(poslo.VARIANT_F, n2, Y, e.data, e.offs, b"", b"", O.ds_serialize(ds_l))
    acc, idx = ctx.distill_stream(b, 16)
    assert acc is True and len(idx) == 0

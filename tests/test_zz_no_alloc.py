"""The allocation-free hashing entry point (poslo_hash_entries_noalloc).

It serves callers that cannot allocate device memory (their memory belongs to another
allocator, or allocation is forbidden after start-up).  The test calls it through the C ABI
on device-resident batches and checks that its output equals poslo_hash_entries' output
bit for bit, on two calls in a row with different inputs (the second call reuses the same
scratch array the first one left behind), plus its size limit and its error for an
undisclosed seed.  It builds the library itself, so it passes alone in a fresh process and
after the other tests.
"""
import numpy as np
import pytest

from paper_2506_08781_gb300 import poslo, synth

pytestmark = pytest.mark.gpu


def _batch(seed, n, n2, D, first_index):
    import torch
    msgs = synth.messages(seed, n, 0, 200)
    root = synth.random_bytes(seed, "root", 16).tobytes()
    ds = __import__("struct").pack("<II", D, 0) + root
    dev = lambda a: torch.from_numpy(np.ascontiguousarray(a).copy()).cuda()
    zeros = dev(np.zeros(32 * max(n, 1), np.uint8))
    b = poslo.Context.make_batch(poslo.VARIANT_F, n2, bytes(32), dev(msgs.data), dev(msgs.offs.view(np.int64)),
                                 zeros, zeros, ds, first_index=first_index)
    return b


def test_noalloc_matches_hash_entries_twice():
    import torch
    import __graft_entry__
    __graft_entry__.build()
    ctx = poslo.Context(device=0)
    try:
        for seed, n, n2, D, first in [(41, 5000, 256, 6, 77), (42, 1234, 7, 12, 3000)]:
            b = _batch(seed, n, n2, D, first)
            want = torch.zeros(32 * n, dtype=torch.uint8, device="cuda")
            got = torch.full((32 * n,), 0xAB, dtype=torch.uint8, device="cuda")
            torch.cuda.synchronize()
            ctx.hash_entries(b, out=want)
            poslo.hash_entries_noalloc(b, got)
            torch.cuda.synchronize()
            assert torch.equal(got, want)
    finally:
        ctx.close()


def test_noalloc_limits_and_errors():
    import torch
    import __graft_entry__
    __graft_entry__.build()
    # more epochs than the scratch array holds
    b = _batch(43, (1 << 16) + 1, 1, 17, 0)
    out = torch.zeros(32 * b.n, dtype=torch.uint8, device="cuda")
    torch.cuda.synchronize()
    with pytest.raises(poslo.PosloError) as e:
        poslo.hash_entries_noalloc(b, out)
    assert e.value.code == -1
    # a seed the disclosed root does not cover (entries beyond 2^D epochs)
    b = _batch(44, 64, 4, 2, 10)
    out = torch.zeros(32 * 64, dtype=torch.uint8, device="cuda")
    torch.cuda.synchronize()
    with pytest.raises(poslo.PosloError) as e:
        poslo.hash_entries_noalloc(b, out)
    assert e.value.code == -1
    # and a valid call right after the failures still agrees with the context path
    b = _batch(45, 300, 16, 5, 0)
    ctx = poslo.Context(device=0)
    try:
        want = torch.zeros(32 * 300, dtype=torch.uint8, device="cuda")
        got = torch.zeros(32 * 300, dtype=torch.uint8, device="cuda")
        torch.cuda.synchronize()
        ctx.hash_entries(b, out=want)
        poslo.hash_entries_noalloc(b, got)
        torch.cuda.synchronize()
        assert torch.equal(got, want)
    finally:
        ctx.close()


def test_noalloc_on_a_caller_stream_empty_batch_and_poslo_c_rule():
    """The caller's own stream, a batch of no entries, and the whole-epoch rule of POSLO-C
    batches, which poslo_hash_entries applies too."""
    import torch
    import __graft_entry__
    __graft_entry__.build()
    ctx = poslo.Context(device=0)
    try:
        b = _batch(46, 777, 32, 8, 5)
        want = torch.zeros(32 * 777, dtype=torch.uint8, device="cuda")
        got = torch.zeros(32 * 777, dtype=torch.uint8, device="cuda")
        torch.cuda.synchronize()
        ctx.hash_entries(b, out=want)
        st = torch.cuda.Stream()
        poslo.hash_entries_noalloc(b, got, stream=st.cuda_stream)
        st.synchronize()
        assert torch.equal(got, want)
        # no entries: OK, nothing written
        b0 = _batch(47, 0, 4, 3, 0)
        out0 = torch.full((32,), 0x5A, dtype=torch.uint8, device="cuda")
        torch.cuda.synchronize()
        poslo.hash_entries_noalloc(b0, out0)
        torch.cuda.synchronize()
        assert bool((out0 == 0x5A).all())
        # a POSLO-C batch that is not whole epochs is refused by both entry points
        bc = _batch(48, 40, 16, 4, 0)
        bc.variant = poslo.VARIANT_C
        bc.R_count = 1
        out = torch.zeros(32 * 40, dtype=torch.uint8, device="cuda")
        torch.cuda.synchronize()
        with pytest.raises(poslo.PosloError) as e:
            poslo.hash_entries_noalloc(bc, out)
        assert e.value.code == -1
        with pytest.raises(poslo.PosloError) as e:
            ctx.hash_entries(bc, out=out)
        assert e.value.code == -1
    finally:
        ctx.close()

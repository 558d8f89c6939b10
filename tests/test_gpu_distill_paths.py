"""Which localisation path Distill (Fig. 3b semantics, Sec. 4.3) takes, and that each gives the
oracle's list.  After the weighted check of the batch fails, the descent over the segment tree
flags entries by their own checks, and a weighted check of every unflagged entry confirms the
result; only when that confirmation fails (errors hidden inside unit sums) does every entry get
its own check.  The confirmation's sum over the unflagged entries is the whole batch's sum minus
the flagged entries', so a slip there would not change any list (the per-entry fallback would
repair it) but would show as a fallback run: the tests below count the fallback launches.

Batches of up to 2^17 entries are signed and checked by the C++ oracle (the Python oracle's
compiled restatement, pinned to it on the CPU), small ones by the Python oracle as well."""
import numpy as np
import pytest

from oracle import cpp_oracle as X
from oracle import poslo_oracle as O
from paper_2506_08781_gb300 import poslo, synth

pytestmark = pytest.mark.gpu

D, N2 = 16, 4


@pytest.fixture(scope="module")
def ctx():
    import __graft_entry__
    __graft_entry__.build()
    c = poslo.Context(device=0, verifier_seed=synth.verifier_seed(909))
    yield c
    c.close()


def _log(seed, n, lmin=1, lmax=60):
    km = synth.key_material(seed, v=16)
    msgs = synth.messages(seed, n, lmin, lmax)
    sub = synth.bpv_subsets(seed, n, v=16, k=4)
    s, R = X.sign_f(km.y, km.root, D, N2, km.bpv_r, sub, msgs.data, msgs.offs, 0)
    Y = X.base_mult(int.from_bytes(km.y, "little"))
    ds = O.ds_serialize(O.ds_root(km.root, D))
    return Y, msgs, bytearray(s.tobytes()), bytearray(R.tobytes()), ds


def _run(ctx, Y, msgs, s, R, ds, python_too=False):
    b = ctx.make_batch(poslo.VARIANT_F, N2, Y, msgs.data, msgs.offs, bytes(s), bytes(R), ds)
    ctx.set_profiling(True)
    ctx.reset_kernel_times()
    idx, cs, cR = ctx.distill(b)
    fallback = ctx.kernel_time("check")[1]
    ctx.set_profiling(False)
    want, ws, wR = X.distill_f(Y, msgs.data, msgs.offs, 0, N2, bytes(s), bytes(R), ds)
    assert [int(t) for t in idx] == want and cs == ws and cR == wR
    if python_too:
        n = msgs.n
        nodes = [O.Node(D, 0, ds[8:24])]
        pw, _, _ = O.distill_f(Y, msgs.as_list(), 0, N2, [bytes(s[32 * t:32 * t + 32]) for t in range(n)],
                               [bytes(R[32 * t:32 * t + 32]) for t in range(n)], nodes)
        assert pw == want
    return want, fallback


def _shift(s, t, d):
    v = (int.from_bytes(bytes(s[32 * t:32 * t + 32]), "little") + d) % O.Q
    s[32 * t:32 * t + 32] = v.to_bytes(32, "little")


@pytest.mark.parametrize("n,count", [(16385, 1), (20000, 60), (1 << 15, 5), (1 << 15, 300), (1 << 15, 3000)])
def test_tampered_entries_confirmed_without_fallback(ctx, n, count):
    """Sparse to dense one-byte flips above the direct-check size (the descent jumps several
    levels while few nodes fail, one level at a time when many do); the confirmation by
    subtraction accepts at once."""
    Y, msgs, s, R, ds = _log(60 + count, n)
    plan = synth.tamper_plan(count, msgs, count)
    bad = synth.apply_tamper(msgs, plan)
    want, fallback = _run(ctx, Y, bad, s, R, ds)
    assert want == [int(t) for t in plan.idx] and fallback == 0
    assert ctx.kernel_time("bisect")[1] >= 1 and ctx.kernel_time("direct")[1] == 0


@pytest.mark.parametrize("n,count", [(1, 1), (700, 1), (700, 60), (4096, 400), (16384, 30)])
def test_small_batches_checked_entry_by_entry(ctx, n, count):
    """Up to 16,384 entries Distill localises by every entry's own check in one launch (no tree,
    no descent, no confirmation): the list and ccd^v are the oracle's."""
    Y, msgs, s, R, ds = _log(80 + count, n)
    plan = synth.tamper_plan(count, msgs, count)
    bad = synth.apply_tamper(msgs, plan)
    want, fallback = _run(ctx, Y, bad, s, R, ds, python_too=n <= 700)
    assert want == sorted(int(t) for t in plan.idx) and fallback == 0
    assert ctx.kernel_time("direct")[1] == 1 and ctx.kernel_time("bisect")[1] == 0


def test_malformed_and_tampered_confirmed_without_fallback(ctx):
    """Undecodable R_t and non-canonical s_t are flagged before the descent; the subtraction
    leaves out the undecodable points (never in the batch's sum) and takes out the others."""
    n = 20000
    Y, msgs, s, R, ds = _log(71, n)
    s[32 * 10:32 * 11] = (int.from_bytes(bytes(s[32 * 10:32 * 11]), "little") + O.Q).to_bytes(32, "little")
    R[32 * 200:32 * 201] = (O.P + 1).to_bytes(32, "little")
    bad = synth.apply_tamper(msgs, synth.tamper_plan(71, msgs, 3))
    want, fallback = _run(ctx, Y, bad, s, R, ds)
    assert 10 in want and 200 in want and fallback == 0 and ctx.kernel_time("bisect")[1] >= 1


def test_cancelling_pair_in_one_leaf_pair_needs_the_fallback(ctx):
    """s_4 + d and s_5 - d in a batch larger than one step of the descent checks at once (so
    its first step stops above the entries): every tree node holding one of them holds both,
    the unit checks pass; the weighted confirmation fails and every entry gets its own check."""
    n = 1 << 17
    Y, msgs, s, R, ds = _log(72, n)
    _shift(s, 4, 4242)
    _shift(s, 5, -4242)
    want, fallback = _run(ctx, Y, msgs, s, R, ds)
    assert want == [4, 5] and fallback == 1


def test_cancelling_pair_far_apart_found_by_the_descent(ctx):
    """s_3 + d and s_5000 - d sit in different subtrees: the nodes holding one of them fail, so
    the descent flags both and the confirmation accepts the rest."""
    n = 1 << 15
    Y, msgs, s, R, ds = _log(73, n)
    _shift(s, 3, 777)
    _shift(s, 5000, -777)
    want, fallback = _run(ctx, Y, msgs, s, R, ds)
    assert want == [3, 5000] and fallback == 0

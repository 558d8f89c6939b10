"""Serving loop (continuous batching over registered keys) through the C ABI: each result
equals the request verified alone and the oracle's per-entry definition, whether the
request ran alone or mixed with others; admission by memory budget; unknown ids."""
import numpy as np
import pytest

from oracle import poslo_oracle as O
from paper_2506_08781_gb300 import poslo, synth

pytestmark = pytest.mark.gpu


def _requests(seed, n_keys, n_req, D=4, n2=8, v=16, k=4):
    keys = []
    for kk in range(n_keys):
        km = synth.key_material(seed * 100 + kk, v=v)
        sk, Y = O.kg_f(km.y, km.root, D, n2, km.bpv_r.tobytes())
        keys.append((km, sk, Y))
    sizes = synth.log_uniform_int(seed, "rsize", n_req, 1, 60)
    reqs = []
    for r in range(n_req):
        kk = r % n_keys
        km, sk, Y = keys[kk]
        first = int(synth.uniform_int(seed, f"f{r}", 1, 0, 40)[0])
        msgs = synth.messages(seed * 1000 + r, int(sizes[r]), 0, 80)
        sub = synth.bpv_subsets(seed * 1000 + r, msgs.n, first_index=first, v=v, k=k)
        sig = [O.sig_f(sk, first + t, msgs.entry(t), sub[t]) for t in range(msgs.n)]
        s, R = [x[0] for x in sig], [x[1] for x in sig]
        if r % 5 == 1:   # tamper 1..3 non-empty entries
            cand = [t for t in range(msgs.n) if len(msgs.entry(t))]
            if cand:
                pick = synth.choose_without_replacement(seed + r, "tp", len(cand), min(len(cand), 1 + r % 3))
                data = msgs.data.copy()
                for q in pick:
                    data[int(msgs.offs[cand[int(q)]])] ^= 0x40
                msgs = synth.Messages(data, msgs.offs)
        ds = O.ds_root(km.root, D)
        want, _, _ = O.distill_f(Y, msgs.as_list(), first, n2, s, R, ds)
        reqs.append(dict(key=kk, n2=n2, first=first, msgs=msgs, s=b"".join(s), R=b"".join(R),
                         ds=O.ds_serialize(ds), want=want))
    return keys, reqs


def _submit(ctx, kid, q):
    return ctx.submit(kid[q["key"]], q["n2"], q["first"], q["msgs"].data, q["msgs"].offs, q["s"], q["R"], q["ds"])


def test_serving_alone_equals_mix_equals_definition():
    import __graft_entry__
    __graft_entry__.build()
    keys, reqs = _requests(7, 4, 24)
    with poslo.Context(device=0, verifier_seed=synth.verifier_seed(7)) as ctx:
        ctx.serve_start(workers=2, max_batch_devices=8, max_batch_entries=300)
        kid = [ctx.register_key(Y) for _, _, Y in keys]
        alone = []
        for q in reqs:
            t = _submit(ctx, kid, q)
            alone.append(ctx.poll(t, wait_ms=60000))
        tickets = [_submit(ctx, kid, q) for q in reqs]
        mix = [ctx.poll(t, wait_ms=60000) for t in tickets]
        batches, requests, in_use = ctx.serve_stats()
        ctx.serve_stop()
    for q, a, m in zip(reqs, alone, mix):
        assert a is not None and m is not None
        assert (a[0], list(a[1])) == (m[0], list(m[1])) == (not q["want"], q["want"])
    assert requests == 48 and in_use == 0
    assert batches < 48            # the mixed submissions were batched together


def test_serving_budget_and_unknown_ids():
    import __graft_entry__
    __graft_entry__.build()
    keys, reqs = _requests(8, 1, 3)
    with poslo.Context(device=0, mem_budget=60_000) as ctx:
        ctx.serve_start(workers=1)
        # a key that does not decode is refused at registration and takes no id
        y = 2
        while O.decode_point(y.to_bytes(32, "little")) is not None:
            y += 1
        with pytest.raises(poslo.PosloError) as e:
            ctx.register_key(y.to_bytes(32, "little"))
        assert e.value.code == -1                      # EINVAL
        kid = [ctx.register_key(Y) for _, _, Y in keys]
        assert kid == list(range(len(keys)))
        big = dict(reqs[0])
        msgs = synth.messages(99, 200, 100, 100)
        big["msgs"], big["s"], big["R"] = msgs, bytes(32 * 200), bytes(32 * 200)
        with pytest.raises(poslo.PosloError) as e:
            _submit(ctx, kid, big)
        assert e.value.code == -6                      # EBUSY
        small = reqs[1]
        t = _submit(ctx, kid, small)
        res = ctx.poll(t, wait_ms=60000)
        assert res[0] is (not small["want"])
        with pytest.raises(poslo.PosloError) as e:
            ctx.submit(7, 8, 0, small["msgs"].data, small["msgs"].offs, small["s"], small["R"], small["ds"])
        assert e.value.code == -7                      # ENOTFOUND
        with pytest.raises(poslo.PosloError) as e:
            ctx.poll(12345)
        assert e.value.code == -7
        ctx.serve_stop()


def test_serving_borrowed_and_copied_requests_mix():
    """Borrowed requests (POSLO_REQ_BORROW: read from the caller's buffers, offsets absolute
    into a larger message buffer) and copied ones batch together with the same results."""
    import __graft_entry__
    __graft_entry__.build()
    keys, reqs = _requests(9, 3, 18)
    with poslo.Context(device=0, verifier_seed=synth.verifier_seed(9)) as ctx:
        ctx.serve_start(workers=2, max_batch_devices=6, max_batch_entries=200)
        kid = [ctx.register_key(Y) for _, _, Y in keys]
        tickets = []
        for i, q in enumerate(reqs):
            if i % 2:
                # messages at an offset inside a bigger buffer, offsets absolute into it
                pad = 13 + i
                buf = np.concatenate([np.full(pad, 0xEE, np.uint8), q["msgs"].data, np.full(7, 0xEE, np.uint8)])
                offs = q["msgs"].offs.astype(np.uint64) + pad
                s_arr = np.frombuffer(q["s"], np.uint8).copy()
                R_arr = np.frombuffer(q["R"], np.uint8).copy()
                tickets.append(ctx.submit(kid[q["key"]], q["n2"], q["first"], buf, offs, s_arr, R_arr, q["ds"],
                                          borrow=True))
            else:
                tickets.append(_submit(ctx, kid, q))
        res = [ctx.poll(t, wait_ms=60000) for t in tickets]
        ctx.serve_stop()
    for q, r in zip(reqs, res):
        assert (r[0], list(r[1])) == (not q["want"], q["want"])


def test_serving_malformed_request_fails_alone():
    """A request whose disclosed seeds do not cover its epochs fails with EINVAL; the requests
    batched with it still get the per-entry definition's results."""
    import __graft_entry__
    __graft_entry__.build()
    keys, reqs = _requests(11, 3, 8)
    bad = dict(reqs[6])
    bad["ds"] = O.ds_serialize([O.Node(0, 15, bytes(16))])   # epoch 15 only; the request's are 0..12
    reqs[6] = bad
    with poslo.Context(device=0, verifier_seed=synth.verifier_seed(11)) as ctx:
        ctx.serve_start(workers=1, max_batch_devices=8, max_batch_entries=1 << 20)
        kid = [ctx.register_key(Y) for _, _, Y in keys]
        tickets = [_submit(ctx, kid, q) for q in reqs]
        res = []
        for t in tickets:
            try:
                res.append(ctx.poll(t, wait_ms=60000))
            except poslo.PosloError as e:
                res.append(e.code)
        batches, requests, in_use = ctx.serve_stats()
        ctx.serve_stop()
    for k, (q, r) in enumerate(zip(reqs, res)):
        if k == 6:
            assert r == -1                                   # EINVAL
        else:
            assert (r[0], list(r[1])) == (not q["want"], q["want"])
    assert requests == 8 and in_use == 0


def test_serving_timeline_accounts_for_every_batch():
    """The per-batch records: one per batch run, every request counted once, the five times of
    a batch in order, workers named by their index; reading them drains them."""
    import __graft_entry__
    __graft_entry__.build()
    keys, reqs = _requests(12, 3, 20)
    with poslo.Context(device=0, verifier_seed=synth.verifier_seed(12)) as ctx:
        ctx.serve_start(workers=2, max_batch_devices=5, max_batch_entries=150)
        kid = [ctx.register_key(Y) for _, _, Y in keys]
        tickets = [_submit(ctx, kid, q) for q in reqs]
        for t in tickets:
            ctx.poll(t, wait_ms=60000)
        batches, requests, _ = ctx.serve_stats()
        recs = ctx.serve_timeline()
        again = ctx.serve_timeline()
        ctx.serve_stop()
    assert len(recs) == batches and sum(r["requests"] for r in recs) == requests == len(reqs)
    assert sum(r["entries"] for r in recs) == sum(q["msgs"].n for q in reqs)
    for r in recs:
        assert r["t_take_ns"] <= r["t_staged_ns"] <= r["t_verify_ns"] <= r["t_checked_ns"] <= r["t_done_ns"]
        assert r["worker"] in (0, 1) and 1 <= r["requests"] <= 5
    assert again == []


def test_serving_stages_next_batch_while_verifying():
    """One busy worker takes its next batch before verifying the current one and issues that
    batch's copies into its other staging set from a staging thread: consecutive batches
    overlap on the worker's timeline, and every result still equals the definition (tampered
    requests included)."""
    import __graft_entry__
    __graft_entry__.build()
    keys, reqs = _requests(13, 3, 16)
    with poslo.Context(device=0, verifier_seed=synth.verifier_seed(13)) as ctx:
        ctx.serve_start(workers=1, max_batch_devices=2, max_batch_entries=1 << 20)
        kid = [ctx.register_key(Y) for _, _, Y in keys]
        tickets = [_submit(ctx, kid, q) for q in reqs]
        got = [ctx.poll(t, wait_ms=60000) for t in tickets]
        recs = sorted(ctx.serve_timeline(), key=lambda r: r["t_take_ns"])
        ctx.serve_stop()
    for q, (acc, inv) in zip(reqs, got):
        assert (acc, list(inv)) == (not q["want"], q["want"])
    overlapped = sum(1 for a, b in zip(recs, recs[1:]) if b["t_take_ns"] < a["t_checked_ns"])
    assert len(recs) >= 8 and overlapped >= 1


def test_serving_pinned_borrowed_requests_gathered():
    """Borrowed requests in page-locked host memory are staged by the gather kernel that reads
    them in place: messages at every alignment (16-byte vector copies and byte copies), offsets
    absolute into one shared buffer; results equal the definition, mixed with copied requests."""
    import torch
    import __graft_entry__
    __graft_entry__.build()
    keys, reqs = _requests(13, 3, 24)
    pads, chunks, pos = [], [], 0
    for i, q in enumerate(reqs):
        pad = i % 17
        pads.append(pos + pad)
        chunks.append(np.full(pad, 0xEE, np.uint8))
        chunks.append(q["msgs"].data)
        pos += pad + len(q["msgs"].data)
    big = torch.from_numpy(np.concatenate(chunks + [np.zeros(16, np.uint8)])).pin_memory()
    keep = []
    with poslo.Context(device=0, verifier_seed=synth.verifier_seed(13)) as ctx:
        ctx.serve_start(workers=2, max_batch_devices=8, max_batch_entries=300)
        kid = [ctx.register_key(Y) for _, _, Y in keys]
        tickets = []
        for i, q in enumerate(reqs):
            if i % 3 == 2:
                tickets.append(_submit(ctx, kid, q))
                continue
            offs = torch.from_numpy((q["msgs"].offs.astype(np.uint64) + np.uint64(pads[i])).view(np.int64)).pin_memory()
            s_t = torch.from_numpy(np.frombuffer(q["s"], np.uint8).copy()).pin_memory()
            R_t = torch.from_numpy(np.frombuffer(q["R"], np.uint8).copy()).pin_memory()
            keep.append((offs, s_t, R_t))
            req = poslo.Request()
            req.key_id, req.n2, req.first_index = kid[q["key"]], q["n2"], q["first"]
            req.msgs, req.offs, req.n = big.data_ptr(), offs.data_ptr(), q["msgs"].n
            req.s, req.R = s_t.data_ptr(), R_t.data_ptr()
            dsb = (poslo.C.c_uint8 * len(q["ds"])).from_buffer_copy(q["ds"])
            keep.append(dsb)
            req.ds, req.ds_nodes = poslo.C.addressof(dsb), len(q["ds"]) // 24
            req.flags = poslo.REQ_BORROW
            t = poslo.C.c_uint64()
            assert ctx.lib.poslo_submit(ctx.h, poslo.C.byref(req), poslo.C.byref(t)) == 0
            tickets.append(t.value)
        res = [ctx.poll(t, wait_ms=60000) for t in tickets]
        ctx.serve_stop()
    for q, r in zip(reqs, res):
        assert (r[0], list(r[1])) == (not q["want"], q["want"])

"""The C++ oracle (oracle/poslo_oracle.cpp, the timed CPU baseline) against the pinned Python
oracle, on the CPU.

The Python oracle is pinned to FIPS 180-2, RFC 8032, libsodium, the Sec. 4.1 worked example
and brute force (tests/test_oracle_pins.py).  Here the compiled restatement must give the same
e_t (every SHA-256 padding length), the same epoch seeds, the same point decodings and scalar
multiples, and the same accept bits, invalid lists and ccd^v on honest batches, random and
exhaustive single-byte tampering, malformed and non-canonical signatures, torsion components
and the s-shift pair; with one thread or several.
"""
import struct

import numpy as np
import pytest

from oracle import cpp_oracle as X
from oracle import poslo_oracle as O
from paper_2506_08781_gb300 import synth


def _f(seed, n, D=4, n2=4, lmin=0, lmax=48, first=0):
    km = synth.key_material(seed, v=16)
    sk, Y = O.kg_f(km.y, km.root, D, n2, km.bpv_r.tobytes())
    msgs = synth.messages(seed, n, lmin, lmax)
    sub = synth.bpv_subsets(seed, n, first_index=first, v=16, k=4)
    sig = [O.sig_f(sk, first + t, msgs.entry(t), sub[t]) for t in range(n)]
    return sk, Y, msgs, [x[0] for x in sig], [x[1] for x in sig], O.ds_root(km.root, D)


def _same(Y, msgs, first, n2, s, R, ds, threads=(1, 3)):
    want = O.distill_f(Y, msgs.as_list(), first, n2, s, R, ds)
    for th in threads:
        got = X.distill_f(Y, msgs.data, msgs.offs, first, n2, b"".join(s), b"".join(R), O.ds_serialize(ds), th)
        assert got == want, th
    acc = X.aver_f(Y, msgs.data, msgs.offs, first, n2, b"".join(s), b"".join(R), O.ds_serialize(ds))
    assert acc is O.aver_f(Y, msgs.as_list(), first, n2, s, R, ds)
    return want


def test_hash_every_length():
    """Every message length 0..300 (all SHA-256 padding boundaries) against hashlib's."""
    D, n2 = 6, 8
    root = synth.random_bytes(4, "root", 16).tobytes()
    ds = O.ds_root(root, D)
    entries = [synth.random_bytes(4, f"m{L}", L).tobytes() for L in range(0, 301)]
    m = synth.pack(entries)
    got = X.hash_entries(m.data, m.offs, 3, n2, O.ds_serialize(ds))
    assert got == [O.entry_scalar(ds, n2, 3 + t, e) for t, e in enumerate(entries)]


@pytest.mark.parametrize("D", [3, 5])
def test_epoch_seeds_every_ds(D):
    root = synth.random_bytes(D, "root", 16).tobytes()
    leaves = [O.tree_node(root, D, 0, i) for i in range(1 << D)]
    for i in range(1 << D):
        ds = O.ds_serialize(O.ds_after(root, D, i))
        assert X.epoch_seeds(ds, 0, i + 1) == leaves[:i + 1]
        if i + 1 < (1 << D):
            with pytest.raises(ValueError):
                X.epoch_seeds(ds, i + 1, 1)        # not disclosed yet


def test_points_decode_and_multiples():
    for y in list(range(0, 40)) + [O.P - 1, O.P, O.P + 1, (1 << 255) - 1]:
        for sign in (0, 1):
            enc = (y | (sign << 255)).to_bytes(32, "little")
            assert X.decode_ok(enc) is (O.decode_point(enc) is not None), (y, sign)
    for k in [0, 1, 2, 8, O.Q - 1, O.Q, O.Q + 1, (1 << 256) - 1] + \
            [int.from_bytes(synth.random_bytes(9, f"k{i}", 32).tobytes(), "little") for i in range(6)]:
        assert X.base_mult(k) == O.encode_point(O.scalar_mult(k, O.G))
        P = O.encode_point(O.scalar_mult(12345, O.G))
        assert X.scalar_mult(k, P) == O.encode_point(O.scalar_mult(k, O.decode_point(P)))
    # a point with a torsion component: [q]P is not the identity, [8q]P is
    y = 3
    while O.decode_point(y.to_bytes(32, "little")) is None:
        y += 1
    P = y.to_bytes(32, "little")
    assert X.scalar_mult(O.Q, P) == O.encode_point(O.scalar_mult(O.Q, O.decode_point(P)))
    assert X.scalar_mult(8 * O.Q, P) == O.encode_point(O.IDENTITY)


def test_honest_and_tampered_batches():
    sk, Y, msgs, s, R, ds = _f(51, 40, first=0)
    assert _same(Y, msgs, 0, 4, s, R, ds)[0] == []
    plan = synth.tamper_plan(51, msgs, 5)
    bad = synth.apply_tamper(msgs, plan)
    assert _same(Y, bad, 0, 4, s, R, ds)[0] == list(plan.idx)


def test_first_index_and_partial_disclosure():
    sk, Y, msgs, s, R, ds = _f(52, 16, first=5, D=3, n2=4)
    ds2 = O.ds_after(sk.root, sk.D, 5)             # epochs 0..5 disclosed
    _same(Y, msgs, 5, 4, s, R, ds2)
    with pytest.raises(ValueError):               # entry 5 + 15 = 20 lies in epoch 5: fine;
        X.distill_f(Y, msgs.data, msgs.offs, 5 + 8, 4, b"".join(s), b"".join(R),
                    O.ds_serialize(O.ds_after(sk.root, sk.D, 3)))   # epochs beyond 3 are not


def test_bruteforce_single_byte_flips():
    """Every single-byte flip (every position, every mask) of a 3-entry batch of 2-byte
    messages: both oracles list exactly that entry."""
    sk, Y, msgs, s, R, ds = _f(53, 3, lmin=2, lmax=2)
    for t in range(3):
        for pos in range(2):
            for mask in range(1, 256):
                data = msgs.data.copy()
                data[int(msgs.offs[t]) + pos] ^= mask
                m2 = synth.Messages(data, msgs.offs)
                got, _, _ = X.distill_f(Y, m2.data, m2.offs, 0, 4, b"".join(s), b"".join(R), O.ds_serialize(ds), 1)
                assert got == [t]


def test_malformed_noncanonical_torsion_and_s_shift():
    sk, Y, msgs, s, R, ds = _f(54, 24)
    Yp = O.decode_point(Y)
    s, R = list(s), list(R)
    T2 = O.decode_point((O.P - 1).to_bytes(32, "little"))
    e = [O.entry_scalar(ds, 4, t, msgs.entry(t)) for t in range(24)]
    s[1] = (int.from_bytes(s[1], "little") + O.Q).to_bytes(32, "little")           # s >= q
    R[3] = O.encode_point(O.point_add(O.decode_point(R[3]), T2))                    # torsion: valid
    s[5], R[5] = O.scalar_to_bytes(-e[5] * sk.y), (O.P + 1).to_bytes(32, "little")  # O as y = p + 1
    s[7], R[7] = O.scalar_to_bytes(-e[7] * sk.y), (1 | 1 << 255).to_bytes(32, "little")  # x = 0, sign
    s[9], R[9] = O.scalar_to_bytes(-e[9] * sk.y), (1).to_bytes(32, "little")       # O: valid
    R[11] = ((1 << 256) - 1).to_bytes(32, "little")                                 # y = 2^255 - 1
    s[13] = O.Q.to_bytes(32, "little")                                              # s = q, R = eY
    R[13] = O.encode_point(O.scalar_mult(e[13], Yp))
    s[15] = O.scalar_to_bytes(int.from_bytes(s[15], "little") + 77)                 # s-shift pair
    s[16] = O.scalar_to_bytes(int.from_bytes(s[16], "little") - 77)
    want = _same(Y, msgs, 0, 4, s, R, ds)
    assert want[0] == [1, 5, 7, 11, 13, 15, 16]
    # torsion in the key: honest entries still verify
    sk, Y, msgs, s, R, ds = _f(55, 12)
    Yt = O.encode_point(O.point_add(O.decode_point(Y), T2))
    assert _same(Yt, msgs, 0, 4, s, R, ds)[0] == []


def test_undecodable_key_raises():
    sk, Y, msgs, s, R, ds = _f(56, 4)
    with pytest.raises(ValueError):
        X.distill_f((O.P + 1).to_bytes(32, "little"), msgs.data, msgs.offs, 0, 4, b"".join(s), b"".join(R),
                    O.ds_serialize(ds))


def test_empty_batch():
    sk, Y, msgs, s, R, ds = _f(57, 0)
    got = X.distill_f(Y, msgs.data, msgs.offs, 0, 4, b"", b"", O.ds_serialize(ds), 4)
    assert got == ([], O.scalar_to_bytes(0), O.encode_point(O.IDENTITY))
    assert X.aver_f(Y, msgs.data, msgs.offs, 0, 4, b"", b"", O.ds_serialize(ds)) is True


def test_ds_wire_form_matches():
    ds = [O.Node(2, 0, bytes(16)), O.Node(0, 6, bytes(range(16)))]
    assert O.ds_serialize(ds)[:8] == struct.pack("<II", 2, 0)
    assert np.frombuffer(O.ds_serialize(ds), np.uint8).size == 48


def test_signer_matches_python_signer():
    """F.Sig (Fig. 4, BPV Definition 3) byte for byte, with a subset holding repeated indices."""
    D, n2, n, first = 4, 4, 30, 7
    km = synth.key_material(58, v=16)
    sk, Y = O.kg_f(km.y, km.root, D, n2, km.bpv_r.tobytes())
    msgs = synth.messages(58, n, 0, 90)
    sub = synth.bpv_subsets(58, n, first_index=first, v=16, k=5)
    sub[3] = [2, 2, 9, 9, 2]
    for th in (1, 4):
        s, R = X.sign_f(km.y, km.root, D, n2, km.bpv_r, sub, msgs.data, msgs.offs, first, th)
        for t in range(n):
            ws, wR, _ = O.sig_f(sk, first + t, msgs.entry(t), sub[t])
            assert s[32 * t:32 * t + 32].tobytes() == ws and R[32 * t:32 * t + 32].tobytes() == wR, t

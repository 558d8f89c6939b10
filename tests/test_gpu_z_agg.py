"""Agg (Fig. 3a C.Agg, Fig. 4 F.Agg) through the C ABI: s~ against the plain sum of the
scalars mod q (non-canonical encodings included) and R~ against the oracle's group sum and
the closed form sum_{i=1..n} [i]G = [n(n+1)/2]G, from host and from device memory."""
import numpy as np
import pytest

from oracle import poslo_oracle as O
from paper_2506_08781_gb300 import poslo, synth

pytestmark = pytest.mark.gpu


def _multiples(n):
    """[1]G, [2]G, ..., [n]G by repeated addition in the oracle's group law."""
    pts, acc = [], O.IDENTITY
    for _ in range(n):
        acc = O.point_add(acc, O.G)
        pts.append(O.encode_point(acc))
    return pts


def _scalars(seed, n):
    raw = synth.random_bytes(seed, "agg", 32 * n).tobytes()
    sc = [raw[32 * i:32 * i + 32] for i in range(n)]
    if n >= 2:
        sc[0] = b"\xff" * 32                       # 2^256 - 1
        sc[1] = O.Q.to_bytes(32, "little")          # q itself
    return sc


@pytest.fixture(scope="module")
def ctx():
    import __graft_entry__
    __graft_entry__.build()
    c = poslo.Context(device=0)
    yield c
    c.close()


@pytest.mark.parametrize("n", [0, 1, 2, 37, 1000])
def test_agg_sums(ctx, n):
    import torch
    pts, sc = _multiples(n), _scalars(70 + n, n)
    s_host, R_host = ctx.agg(b"".join(sc), b"".join(pts))
    assert s_host == O.agg_scalars(sc)
    assert s_host == (sum(int.from_bytes(x, "little") for x in sc) % O.Q).to_bytes(32, "little")
    assert R_host == O.agg_points(pts)
    assert R_host == O.encode_point(O.scalar_mult(n * (n + 1) // 2, O.G))
    if n:
        d_s = torch.from_numpy(np.frombuffer(b"".join(sc), np.uint8).copy()).cuda()
        d_R = torch.from_numpy(np.frombuffer(b"".join(pts), np.uint8).copy()).cuda()
        torch.cuda.synchronize()
        assert ctx.agg(d_s, d_R, on_device=True) == (s_host, R_host)


def test_agg_undecodable_point_is_einval(ctx):
    pts = _multiples(5)
    y = 2
    while O.decode_point(y.to_bytes(32, "little")) is not None:
        y += 1
    pts[3] = y.to_bytes(32, "little")
    with pytest.raises(poslo.PosloError) as e:
        ctx.agg(bytes(32 * 5), b"".join(pts))
    assert e.value.code == -1
    # the context stays usable
    assert ctx.agg(bytes(32), _multiples(1)[0]) == (bytes(32), O.encode_point(O.G))

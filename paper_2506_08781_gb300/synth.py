"""Seeded synthetic inputs for POSLO batch verification.

This module is the only code shared by the CUDA path's callers (bench, tests) and the
CPU oracle.  It produces random bytes and random integers only; it holds none of the
scheme's arithmetic (no hashing, no field or group operation, no reduction mod q).

Every stream is SplitMix64 (Steele, Lea and Flood, "Fast splittable pseudorandom number
generators", OOPSLA 2014) used in counter mode: word k of stream s is
mix64(s + (k + 1) * GAMMA).  It is vectorised with numpy uint64 arithmetic, so the same
seed gives the same bytes on every machine and numpy version.

Workload shapes follow the paper's cold-storage experiments: epochs of n2 = 2^8 entries
(Sec. 7, Fig. 6 caption), random log entries, and a small fraction of flagged entries
(tau_F, Sec. 7.4).  Message lengths, batch-size distributions and tamper rates are the
parameters of the synthetic workloads the tests and the benchmark build.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

GAMMA = np.uint64(0x9E3779B97F4A7C15)
_M1 = np.uint64(0xBF58476D1CE4E5B9)
_M2 = np.uint64(0x94D049BB133111EB)

# BPV generator parameters (v, k) = (1024, 16) used by the paper's instantiation (Sec. 7.2).
BPV_V = 1024
BPV_K = 16


def _mix64(z: np.ndarray) -> np.ndarray:
    z = (z ^ (z >> np.uint64(30))) * _M1
    z = (z ^ (z >> np.uint64(27))) * _M2
    return z ^ (z >> np.uint64(31))


def _stream_seed(seed: int, tag: str) -> np.uint64:
    """Derive an independent stream id from (seed, tag) with SplitMix64 itself."""
    h = np.uint64(seed & 0xFFFFFFFFFFFFFFFF)
    with np.errstate(over="ignore"):
        for ch in tag.encode():
            h = _mix64(np.array([h ^ np.uint64(ch)], dtype=np.uint64) + GAMMA)[0]
    return h


def words(seed: int, tag: str, n: int, start: int = 0) -> np.ndarray:
    """n uint64 words of stream (seed, tag), counters start .. start+n-1."""
    s = _stream_seed(seed, tag)
    with np.errstate(over="ignore"):
        k = np.arange(start + 1, start + n + 1, dtype=np.uint64)
        return _mix64(s + k * GAMMA)


def random_bytes(seed: int, tag: str, nbytes: int) -> np.ndarray:
    w = words(seed, tag, (nbytes + 7) // 8)
    return w.view(np.uint8)[:nbytes].copy()


def uniform_int(seed: int, tag: str, n: int, lo: int, hi: int) -> np.ndarray:
    """n integers uniform in [lo, hi] (multiply-shift on the top 32 bits)."""
    span = np.uint64(hi - lo + 1)
    w = words(seed, tag, n) >> np.uint64(32)
    return (lo + ((w * span) >> np.uint64(32))).astype(np.int64)


def uniform01(seed: int, tag: str, n: int) -> np.ndarray:
    w = words(seed, tag, n) >> np.uint64(11)
    return w.astype(np.float64) * (1.0 / (1 << 53))


def log_uniform_int(seed: int, tag: str, n: int, lo: int, hi: int) -> np.ndarray:
    """n integers with log-uniform distribution on [lo, hi]."""
    u = uniform01(seed, tag, n)
    v = np.exp(math.log(lo) + u * (math.log(hi + 1) - math.log(lo)))
    return np.clip(np.floor(v).astype(np.int64), lo, hi)


def choose_without_replacement(seed: int, tag: str, n: int, k: int) -> np.ndarray:
    """k distinct indices of [0, n), uniformly, sorted ascending."""
    if k > n:
        raise ValueError("k > n")
    keys = words(seed, tag, n)
    return np.sort(np.argsort(keys, kind="stable")[:k]).astype(np.int64)


@dataclass
class Messages:
    """Log entries packed as one byte buffer plus n+1 offsets (entry t is
    data[offs[t]:offs[t+1]])."""
    data: np.ndarray          # uint8[total]
    offs: np.ndarray          # uint64[n+1]

    @property
    def n(self) -> int:
        return len(self.offs) - 1

    def entry(self, t: int) -> bytes:
        return bytes(self.data[int(self.offs[t]):int(self.offs[t + 1])])

    def as_list(self) -> list[bytes]:
        return [self.entry(t) for t in range(self.n)]


def messages(seed: int, n: int, lmin: int, lmax: int, tag: str = "msg") -> Messages:
    """n random log entries with lengths uniform in [lmin, lmax]."""
    lens = uniform_int(seed, tag + ".len", n, lmin, lmax) if n else np.zeros(0, np.int64)
    offs = np.zeros(n + 1, dtype=np.uint64)
    np.cumsum(lens, out=offs[1:])
    total = int(offs[-1])
    data = random_bytes(seed, tag + ".bytes", total)
    return Messages(data=data, offs=offs)


def pack(entries: list[bytes]) -> Messages:
    lens = np.array([len(m) for m in entries], dtype=np.int64)
    offs = np.zeros(len(entries) + 1, dtype=np.uint64)
    if len(entries):
        np.cumsum(lens, out=offs[1:])
    data = np.frombuffer(b"".join(entries), dtype=np.uint8).copy() if entries else np.zeros(0, np.uint8)
    return Messages(data=data, offs=offs)


@dataclass
class Tamper:
    """Single-byte flips: entry idx[k] gets byte pos[k] XORed with mask[k] (non-zero)."""
    idx: np.ndarray
    pos: np.ndarray
    mask: np.ndarray


def tamper_plan(seed: int, msgs: Messages, count: int, tag: str = "tamper") -> Tamper:
    """Choose `count` distinct entries uniformly; in each, a uniform byte offset and a
    uniform non-zero XOR mask."""
    idx = choose_without_replacement(seed, tag + ".idx", msgs.n, count)
    lens = (msgs.offs[1:] - msgs.offs[:-1]).astype(np.int64)[idx]
    if np.any(lens == 0):
        raise ValueError("cannot tamper an empty entry")
    u = words(seed, tag + ".pos", count) >> np.uint64(32)
    pos = ((u * lens.astype(np.uint64)) >> np.uint64(32)).astype(np.int64)
    mask = uniform_int(seed, tag + ".mask", count, 1, 255).astype(np.uint8)
    return Tamper(idx=idx, pos=pos, mask=mask)


def apply_tamper(msgs: Messages, plan: Tamper) -> Messages:
    data = msgs.data.copy()
    where = msgs.offs[plan.idx].astype(np.int64) + plan.pos
    data[where] ^= plan.mask
    return Messages(data=data, offs=msgs.offs.copy())


@dataclass
class KeyMaterial:
    """Secret randomness for one signer, as raw bytes.

    y and the BPV table scalars are drawn below 2^252 (top nibble cleared), so they are
    already canonical scalars of the edwards25519 group order q > 2^252; r and the root
    are free bytes.  Keygen derives everything else from these."""
    y: bytes                  # 32 B little-endian scalar, 0 < y < 2^252
    r: bytes                  # 32 B (POSLO-C nonce seed)
    root: bytes               # 16 B seed-tree root x_D[0]
    bpv_r: np.ndarray         # uint8[v*32] BPV table scalars (POSLO-F)


def key_material(seed: int, tag: str = "key", v: int = BPV_V) -> KeyMaterial:
    raw = random_bytes(seed, tag, 32 + 32 + 16)
    y = bytearray(raw[:32].tobytes())
    y[31] &= 0x0F
    if not any(y):
        y[0] = 1
    r = raw[32:64].tobytes()
    root = raw[64:80].tobytes()
    bpv = random_bytes(seed, tag + ".bpv", 32 * v).reshape(v, 32)
    bpv[:, 31] &= 0x0F
    return KeyMaterial(y=bytes(y), r=r, root=root, bpv_r=bpv.reshape(-1).copy())


def bpv_subsets(seed: int, n: int, first_index: int = 0, v: int = BPV_V, k: int = BPV_K,
                tag: str = "bpv") -> np.ndarray:
    """BPV online subsets for entries first_index .. first_index+n-1: uint16[n, k] with
    indices uniform in [0, v), drawn with replacement: a repeated index adds the same
    table element twice to both r_t and R_t, so the signature stays valid."""
    w = words(seed, tag, n * k, start=first_index * k) >> np.uint64(32)
    return ((w * np.uint64(v)) >> np.uint64(32)).astype(np.uint16).reshape(n, k)


def verifier_seed(seed: int, tag: str = "verifier") -> bytes:
    return random_bytes(seed, tag, 32).tobytes()


@dataclass
class DeviceBatches:
    """Multi-device workload: device d owns entries [starts[d], starts[d+1]) of msgs."""
    sizes: np.ndarray
    starts: np.ndarray
    msgs: Messages
    tampered_devices: np.ndarray = field(default_factory=lambda: np.zeros(0, np.int64))


def device_sizes(seed: int, n_dev: int, lo: int, hi: int, tag: str = "devsize") -> np.ndarray:
    return log_uniform_int(seed, tag, n_dev, lo, hi)


def poisson_arrivals(seed: int, n: int, rate: float, tag: str = "arrive") -> np.ndarray:
    """n arrival times (seconds) of a Poisson process with the given rate."""
    u = uniform01(seed, tag, n)
    gaps = -np.log1p(-u) / rate
    return np.cumsum(gaps)

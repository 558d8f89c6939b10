"""ctypes binding of the C++ oracle (oracle/poslo_oracle.cpp), test infrastructure only.

The C++ oracle states the same definitions as poslo_oracle.py (SHA-256 instantiation) in a
compiled language, so that the timed CPU baseline is not bound by the Python interpreter.
It is imported by the tests and by the benchmark's CPU-baseline leg, never by the product.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

from oracle import build as _build

_lib = None


def load() -> C.CDLL:
    global _lib
    if _lib is None:
        lib = C.CDLL(_build.build())
        vp, u64, u32 = C.c_void_p, C.c_uint64, C.c_uint32
        lib.oracle_hash_entries.argtypes = [vp, vp, u64, u64, u32, vp, u32, vp]
        lib.oracle_epoch_seeds.argtypes = [vp, u32, u64, u64, vp]
        lib.oracle_decode_ok.argtypes = [vp]
        lib.oracle_scalar_mult.argtypes = [vp, vp, vp]
        lib.oracle_base_mult.argtypes = [vp, vp]
        lib.oracle_distill_f.argtypes = [vp, vp, vp, u64, u64, u32, vp, vp, vp, u32, C.c_int, vp,
                                         C.POINTER(u64), vp, vp]
        lib.oracle_aver_f.argtypes = [vp, vp, vp, u64, u64, u32, vp, vp, vp, u32, vp]
        lib.oracle_sign_f.argtypes = [vp, vp, u32, u32, vp, u32, u32, vp, vp, vp, u64, u64, C.c_int, vp, vp]
        _lib = lib
    return _lib


def _buf(b) -> np.ndarray:
    if isinstance(b, (bytes, bytearray)):
        return np.frombuffer(bytes(b), np.uint8).copy() if len(b) else np.zeros(1, np.uint8)
    a = np.ascontiguousarray(b)
    return a if a.size else np.zeros(1, a.dtype)


def _p(a: np.ndarray):
    return a.ctypes.data


def _check(rc: int, what: str):
    if rc != 0:
        raise ValueError(f"C++ oracle: {what} failed ({rc})")


def hash_entries(msgs, offs, first_index: int, n2: int, ds: bytes) -> list:
    lib = load()
    offs = np.ascontiguousarray(offs, np.uint64)
    n = len(offs) - 1
    m, d = _buf(msgs), _buf(ds)
    out = np.zeros(32 * max(n, 1), np.uint8)
    _check(lib.oracle_hash_entries(_p(m), _p(offs), n, first_index, n2, _p(d), len(ds) // 24, _p(out)), "hash")
    return [int.from_bytes(out[32 * k:32 * k + 32].tobytes(), "little") for k in range(n)]


def epoch_seeds(ds: bytes, first: int, count: int) -> list:
    lib = load()
    d = _buf(ds)
    out = np.zeros(16 * max(count, 1), np.uint8)
    _check(lib.oracle_epoch_seeds(_p(d), len(ds) // 24, first, count, _p(out)), "epoch seeds")
    return [out[16 * k:16 * k + 16].tobytes() for k in range(count)]


def decode_ok(b: bytes) -> bool:
    bb = _buf(b)
    return bool(load().oracle_decode_ok(_p(bb)))


def scalar_mult(k: int, P: bytes) -> bytes:
    kb, Pb, out = _buf(k.to_bytes(32, "little")), _buf(P), np.zeros(32, np.uint8)
    _check(load().oracle_scalar_mult(_p(kb), _p(Pb), _p(out)), "scalar mult")
    return out.tobytes()


def base_mult(k: int) -> bytes:
    kb, out = _buf(k.to_bytes(32, "little")), np.zeros(32, np.uint8)
    _check(load().oracle_base_mult(_p(kb), _p(out)), "base mult")
    return out.tobytes()


def distill_f(Y: bytes, msgs, offs, first_index: int, n2: int, s, R, ds: bytes, threads: int = 0):
    """(sorted invalid global indices, ccd^v s bytes, ccd^v R bytes), as poslo_oracle.distill_f."""
    lib = load()
    offs = np.ascontiguousarray(offs, np.uint64)
    n = len(offs) - 1
    m, sb, Rb, d, Yb = _buf(msgs), _buf(s), _buf(R), _buf(ds), _buf(Y)
    inv = np.zeros(max(n, 1), np.uint64)
    cnt = C.c_uint64()
    cs, cR = np.zeros(32, np.uint8), np.zeros(32, np.uint8)
    _check(lib.oracle_distill_f(_p(Yb), _p(m), _p(offs), n, first_index, n2, _p(sb), _p(Rb), _p(d), len(ds) // 24,
                                threads, _p(inv), C.byref(cnt), _p(cs), _p(cR)), "distill")
    return [int(x) for x in inv[:cnt.value]], cs.tobytes(), cR.tobytes()


def aver_f(Y: bytes, msgs, offs, first_index: int, n2: int, s, R, ds: bytes) -> bool:
    lib = load()
    offs = np.ascontiguousarray(offs, np.uint64)
    n = len(offs) - 1
    m, sb, Rb, d, Yb = _buf(msgs), _buf(s), _buf(R), _buf(ds), _buf(Y)
    acc = np.zeros(1, np.uint8)
    _check(lib.oracle_aver_f(_p(Yb), _p(m), _p(offs), n, first_index, n2, _p(sb), _p(Rb), _p(d), len(ds) // 24,
                             _p(acc)), "aver")
    return bool(acc[0])


def sign_f(y: bytes, root: bytes, D: int, n2: int, bpv_r, subsets, msgs, offs, first_index: int = 0,
           threads: int = 0):
    """POSLO-F.Sig of every entry (BPV subsets uint16[n, k]); returns (s, R) as n*32-byte arrays."""
    lib = load()
    offs = np.ascontiguousarray(offs, np.uint64)
    n = len(offs) - 1
    sub = np.ascontiguousarray(subsets, np.uint16).reshape(n, -1) if n else np.zeros((0, 1), np.uint16)
    k = sub.shape[1]
    rb = _buf(np.ascontiguousarray(bpv_r, np.uint8).reshape(-1))
    yb, rootb, m, subb = _buf(y), _buf(root), _buf(msgs), _buf(sub)
    s = np.zeros(32 * max(n, 1), np.uint8)
    R = np.zeros(32 * max(n, 1), np.uint8)
    _check(lib.oracle_sign_f(_p(yb), _p(rootb), D, n2, _p(rb), rb.size // 32, k, _p(subb), _p(m), _p(offs), n,
                             first_index, threads, _p(s), _p(R)), "sign")
    return s[:32 * n], R[:32 * n]

"""ctypes binding of libposlo (include/poslo.h): argument marshalling only.

Every computation of the verification path runs in the CUDA library.  Arrays may be numpy
arrays (host memory) or torch CUDA tensors (device memory; the call then passes
on_device = 1).  Loading fails loudly when the library has not been built: there is no
CPU fallback.
"""
from __future__ import annotations

import ctypes as C
import os
from dataclasses import dataclass

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libposlo.so")

POSLO_OK = 0
STATUS = {0: "OK", -1: "EINVAL", -2: "ENOMEM", -3: "EDEVICE", -4: "ETIMEOUT", -5: "EBUFSMALL", -6: "EBUSY",
          -7: "ENOTFOUND"}
VARIANT_C, VARIANT_F = 0, 1
AGG_UNIT, AGG_WEIGHTED = 0, 1
INST_SHA256, INST_AES = 0, 1          # POSLO and POSLO+ (Sec. 7.2)

# Every entry point declared in include/poslo.h.
EXPORTS = [
    "poslo_create", "poslo_destroy", "poslo_last_error", "poslo_stream",
    "poslo_keygen_c", "poslo_keygen_f", "poslo_sign_c", "poslo_sign_f", "poslo_disclose",
    "poslo_agg", "poslo_aver", "poslo_distill", "poslo_epoch_seeds", "poslo_hash_entries", "poslo_msm", "poslo_msm_autotune",
    "poslo_msm_get_plan", "poslo_msm_set_plan",
    "poslo_set_profiling", "poslo_kernel_time", "poslo_reset_kernel_times", "poslo_set_graphs", "poslo_graph_stats",
    "poslo_set_multi_window_limit", "poslo_set_key_cache", "poslo_key_cache_stats",
    "poslo_hash_entries_noalloc", "poslo_aver_multi", "poslo_distill_c", "poslo_sebver_c", "poslo_distill_stream",
    "poslo_serve_start", "poslo_serve_stop", "poslo_register_key", "poslo_submit", "poslo_poll",
    "poslo_serve_stats", "poslo_aver_partial", "poslo_combine_check", "poslo_serve_timeline",
]
POSLO_PENDING = 1
POSLO_EBUFSMALL = -5


class PosloError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"{STATUS.get(code, code)}: {msg}")
        self.code = code


class Params(C.Structure):
    _fields_ = [("device", C.c_int), ("msm_window", C.c_uint32), ("mem_budget", C.c_uint64),
                ("verifier_seed", C.c_uint8 * 32), ("instantiation", C.c_uint32)]


class MultiBatch(C.Structure):
    _fields_ = [("n_dev", C.c_uint32), ("Y", C.c_void_p), ("dev_start", C.c_void_p), ("first_index", C.c_void_p),
                ("n2", C.c_void_p), ("ds", C.c_void_p), ("ds_off", C.c_void_p), ("msgs", C.c_void_p),
                ("offs", C.c_void_p), ("s", C.c_void_p), ("R", C.c_void_p), ("on_device", C.c_uint32)]


class Partial(C.Structure):
    """poslo_partial: one shard's aggregate record (216 bytes)."""
    _fields_ = [("e", C.c_uint8 * 32), ("s", C.c_uint8 * 32), ("R", C.c_uint8 * 128), ("first_index", C.c_uint64),
                ("n", C.c_uint64), ("malformed", C.c_uint32), ("agg_mode", C.c_uint32)]

    def to_bytes(self) -> bytes:
        return bytes(memoryview(self).cast("B"))

    @classmethod
    def from_bytes(cls, b: bytes) -> "Partial":
        if len(b) != C.sizeof(cls):
            raise ValueError("a poslo_partial record is 216 bytes")
        return cls.from_buffer_copy(b)


class BatchRecord(C.Structure):
    """poslo_batch_record: one served batch on the service's clock (ns)."""
    _fields_ = [("worker", C.c_uint32), ("requests", C.c_uint32), ("entries", C.c_uint64),
                ("t_take_ns", C.c_uint64), ("t_staged_ns", C.c_uint64), ("t_verify_ns", C.c_uint64),
                ("t_checked_ns", C.c_uint64), ("t_done_ns", C.c_uint64)]


class Request(C.Structure):
    _fields_ = [("key_id", C.c_uint32), ("n2", C.c_uint32), ("first_index", C.c_uint64), ("msgs", C.c_void_p),
                ("offs", C.c_void_p), ("n", C.c_uint64), ("s", C.c_void_p), ("R", C.c_void_p), ("ds", C.c_void_p),
                ("ds_nodes", C.c_uint32), ("flags", C.c_uint32)]


REQ_BORROW = 1


class CcdC(C.Structure):
    _fields_ = [("s_v", C.c_void_p), ("R_v", C.c_void_p), ("umbrellas", C.c_void_p), ("invalid", C.c_void_p),
                ("cap", C.c_uint64), ("n_invalid", C.c_uint64)]


class Batch(C.Structure):
    _fields_ = [("variant", C.c_uint32), ("n2", C.c_uint32), ("Y", C.c_void_p), ("msgs", C.c_void_p),
                ("offs", C.c_void_p), ("n", C.c_uint64), ("first_index", C.c_uint64), ("s", C.c_void_p),
                ("R", C.c_void_p), ("R_count", C.c_uint64), ("ds", C.c_void_p), ("ds_nodes", C.c_uint32),
                ("on_device", C.c_uint32)]


_lib = None


def load_library(path: str = LIB_PATH) -> C.CDLL:
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise ImportError(f"libposlo.so is not built ({path}); run __graft_entry__.build() "
                          "or python -m paper_2506_08781_gb300.build — there is no CPU fallback")
    lib = C.CDLL(path)
    vp, u8p, u64, u32 = C.c_void_p, C.c_void_p, C.c_uint64, C.c_uint32
    sig = {
        "poslo_create": ([C.POINTER(Params), C.POINTER(vp)], C.c_int),
        "poslo_destroy": ([vp], None),
        "poslo_last_error": ([vp], C.c_char_p),
        "poslo_stream": ([vp], vp),
        "poslo_keygen_c": ([vp, u8p, u8p, u32, u32, u8p, u8p], C.c_int),
        "poslo_keygen_f": ([vp, u8p, u8p, u32, u8p, u8p], C.c_int),
        "poslo_sign_c": ([vp, u8p, u8p, u8p, u32, u32, u8p, vp, u64, u64, u8p], C.c_int),
        "poslo_sign_f": ([vp, u8p, u8p, u32, u32, u8p, u8p, u32, u32, vp, u8p, vp, u64, u64, u8p, u8p, u8p],
                         C.c_int),
        "poslo_disclose": ([vp, u8p, u32, u64, u8p, u32, C.POINTER(u32)], C.c_int),
        "poslo_agg": ([vp, u8p, u8p, u64, u32, u8p, u8p], C.c_int),
        "poslo_aver": ([vp, C.POINTER(Batch), u32, u8p], C.c_int),
        "poslo_distill": ([vp, C.POINTER(Batch), vp, u64, C.POINTER(u64), u8p, u8p], C.c_int),
        "poslo_epoch_seeds": ([vp, u8p, u32, u64, u64, u8p], C.c_int),
        "poslo_hash_entries": ([vp, C.POINTER(Batch), u8p], C.c_int),
        "poslo_msm": ([vp, u8p, u8p, u64, u32, u8p], C.c_int),
        "poslo_msm_autotune": ([vp, u64, u32, C.POINTER(u32)], C.c_int),
        "poslo_msm_get_plan": ([vp, u64, u32, C.POINTER(u32), C.POINTER(u32)], C.c_int),
        "poslo_msm_set_plan": ([vp, u64, u32, u32, u32], C.c_int),
        "poslo_set_profiling": ([vp, C.c_int], C.c_int),
        "poslo_set_graphs": ([vp, C.c_int], C.c_int),
        "poslo_set_multi_window_limit": ([vp, u64], C.c_int),
        "poslo_set_key_cache": ([vp, u32], C.c_int),
        "poslo_key_cache_stats": ([vp, C.POINTER(u64), C.POINTER(u64)], C.c_int),
        "poslo_graph_stats": ([vp, C.POINTER(u64), C.POINTER(u64)], C.c_int),
        "poslo_kernel_time": ([vp, C.c_char_p, C.POINTER(C.c_double), C.POINTER(u64)], C.c_int),
        "poslo_reset_kernel_times": ([vp], None),
        "poslo_hash_entries_noalloc": ([C.POINTER(Batch), u8p, vp], C.c_int),
        "poslo_aver_multi": ([vp, C.POINTER(MultiBatch), u8p, vp, u64, C.POINTER(u64)], C.c_int),
        "poslo_distill_c": ([vp, C.POINTER(Batch), u32, u8p, C.POINTER(CcdC)], C.c_int),
        "poslo_distill_stream": ([vp, C.POINTER(Batch), u64, u8p, vp, u64, C.POINTER(u64)], C.c_int),
        "poslo_sebver_c": ([vp, C.POINTER(Batch), u32, C.POINTER(CcdC), u32, u8p], C.c_int),
        "poslo_serve_start": ([vp, u32, u32, u64], C.c_int),
        "poslo_serve_stop": ([vp], C.c_int),
        "poslo_register_key": ([vp, u8p, C.POINTER(u32)], C.c_int),
        "poslo_submit": ([vp, C.POINTER(Request), C.POINTER(u64)], C.c_int),
        "poslo_poll": ([vp, u64, u32, u8p, vp, u64, C.POINTER(u64), C.POINTER(u64)], C.c_int),
        "poslo_serve_stats": ([vp, C.POINTER(u64), C.POINTER(u64), C.POINTER(u64)], C.c_int),
        "poslo_aver_partial": ([vp, C.POINTER(Batch), u32, C.POINTER(Partial)], C.c_int),
        "poslo_serve_timeline": ([vp, vp, u64, C.POINTER(u64)], C.c_int),
        "poslo_combine_check": ([vp, u8p, vp, u32, u8p, C.POINTER(Partial)], C.c_int),
    }
    for name in EXPORTS:
        f = getattr(lib, name)
        f.argtypes, f.restype = sig[name]
    _lib = lib
    return lib


def _is_torch(x) -> bool:
    return type(x).__module__.startswith("torch")


def _ptr(x):
    """Host or device address of a numpy array, bytes, or torch tensor (None -> NULL)."""
    if x is None:
        return None
    if _is_torch(x):
        return x.data_ptr()
    if isinstance(x, (bytes, bytearray)):
        buf = (C.c_uint8 * len(x)).from_buffer_copy(x)
        _keep.append(buf)
        return C.addressof(buf)
    arr = np.ascontiguousarray(x)
    _keep.append(arr)          # alive until the call returns (temporaries included)
    return arr.ctypes.data


_keep: list = []


def _u8(x) -> np.ndarray:
    if isinstance(x, (bytes, bytearray)):
        return np.frombuffer(bytes(x), dtype=np.uint8).copy()
    return np.ascontiguousarray(x, dtype=np.uint8).reshape(-1)


@dataclass
class BatchData:
    """A batch as the caller holds it (numpy arrays or torch CUDA tensors)."""
    variant: int
    n2: int
    Y: bytes
    msgs: object
    offs: object
    n: int
    first_index: int
    s: object
    R: object
    R_count: int
    ds: bytes
    ds_nodes: int


def hash_entries_noalloc(b: BatchData, e_out, stream: int = 0) -> None:
    """poslo_hash_entries_noalloc: e_t for every entry of a device-resident batch into the
    device tensor e_out (n*32 bytes), without a context and without device allocation."""
    lib = load_library()
    if not (_is_torch(b.offs) and b.offs.is_cuda and _is_torch(e_out) and e_out.is_cuda):
        raise ValueError("hash_entries_noalloc takes device tensors only")
    cb = Context._cbatch(None, b)
    rc = lib.poslo_hash_entries_noalloc(C.byref(cb), _ptr(e_out), stream or None)
    _keep.clear()
    if rc != POSLO_OK:
        raise PosloError(rc, "poslo_hash_entries_noalloc failed")


class Context:
    """A libposlo context on one device."""

    def __init__(self, device: int = 0, msm_window: int = 0, mem_budget: int = 0,
                 verifier_seed: bytes = bytes(32), instantiation: int = INST_SHA256):
        self.lib = load_library()
        p = Params()
        p.device = device
        p.msm_window = msm_window
        p.mem_budget = mem_budget
        p.instantiation = instantiation
        for i, b in enumerate(verifier_seed[:32]):
            p.verifier_seed[i] = b
        h = C.c_void_p()
        rc = self.lib.poslo_create(C.byref(p), C.byref(h))
        if rc != POSLO_OK:
            raise PosloError(rc, "poslo_create failed (needs an sm_103 GPU)")
        self.h = h
        self._borrowed = {}

    def close(self):
        if getattr(self, "h", None):
            self.lib.poslo_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    def _check(self, rc: int):
        _keep.clear()
        if rc != POSLO_OK:
            raise PosloError(rc, self.lib.poslo_last_error(self.h).decode())

    @property
    def stream(self) -> int:
        return self.lib.poslo_stream(self.h) or 0

    # ------------------------------------------------------------------ signer side
    def keygen_c(self, y: bytes, r: bytes, D: int, n2: int):
        Y = np.zeros(32, np.uint8)
        R = np.zeros(32 << D, np.uint8)
        self._check(self.lib.poslo_keygen_c(self.h, _ptr(y), _ptr(r), D, n2, _ptr(Y), _ptr(R)))
        return Y.tobytes(), R

    def keygen_f(self, y: bytes, bpv_r):
        bpv_r = _u8(bpv_r)
        v = len(bpv_r) // 32
        Y = np.zeros(32, np.uint8)
        R = np.zeros(32 * v, np.uint8)
        self._check(self.lib.poslo_keygen_f(self.h, _ptr(y), _ptr(bpv_r), v, _ptr(Y), _ptr(R)))
        return Y.tobytes(), R

    def sign_c(self, y: bytes, r: bytes, root: bytes, D: int, n2: int, msgs, offs, first_epoch: int,
               n_epochs: int):
        s = np.zeros(32 * n_epochs, np.uint8)
        offs = np.ascontiguousarray(offs, dtype=np.uint64)
        self._check(self.lib.poslo_sign_c(self.h, _ptr(y), _ptr(r), _ptr(root), D, n2, _ptr(_u8(msgs)),
                                          _ptr(offs), first_epoch, n_epochs, _ptr(s)))
        return s

    def sign_f(self, y: bytes, root: bytes, D: int, n2: int, bpv_r, bpv_R, subsets, msgs, offs,
               first_index: int = 0, want_x: bool = False):
        offs = np.ascontiguousarray(offs, dtype=np.uint64)
        n = len(offs) - 1
        subsets = np.ascontiguousarray(subsets, dtype=np.uint16)
        k = subsets.shape[1] if subsets.ndim == 2 else 0
        bpv_r, bpv_R = _u8(bpv_r), _u8(bpv_R)
        s = np.zeros(32 * n, np.uint8)
        R = np.zeros(32 * n, np.uint8)
        x = np.zeros(16 * n, np.uint8) if want_x else None
        self._check(self.lib.poslo_sign_f(self.h, _ptr(y), _ptr(root), D, n2, _ptr(bpv_r), _ptr(bpv_R),
                                          len(bpv_r) // 32, k, _ptr(subsets), _ptr(_u8(msgs)), _ptr(offs), n,
                                          first_index, _ptr(s), _ptr(R), _ptr(x)))
        return (s, R, x) if want_x else (s, R)

    def disclose(self, root: bytes, D: int, i: int) -> bytes:
        cap = D + 2
        out = np.zeros(24 * cap, np.uint8)
        nodes = C.c_uint32()
        self._check(self.lib.poslo_disclose(self.h, _ptr(root), D, i, _ptr(out), cap, C.byref(nodes)))
        return out[:24 * nodes.value].tobytes()

    # ------------------------------------------------------------------ verifier side
    @staticmethod
    def make_batch(variant: int, n2: int, Y: bytes, msgs, offs, s, R, ds: bytes, first_index: int = 0,
                   R_count: int | None = None) -> BatchData:
        if _is_torch(offs):
            n = offs.numel() - 1
        else:
            offs = np.ascontiguousarray(offs, dtype=np.uint64)
            n = len(offs) - 1
            msgs, s, R = _u8(msgs), _u8(s), _u8(R)
        if R_count is None:
            R_count = n if variant == VARIANT_F else (len(R) // 32 if not _is_torch(R) else R.numel() // 32)
        return BatchData(variant, n2, bytes(Y), msgs, offs, n, first_index, s, R, R_count, bytes(ds), len(ds) // 24)

    def _cbatch(self, b: BatchData) -> Batch:
        cb = Batch()
        cb.variant, cb.n2 = b.variant, b.n2
        cb.Y = _ptr(b.Y)
        on_dev = _is_torch(b.offs) and b.offs.is_cuda
        cb.msgs, cb.offs, cb.s, cb.R = _ptr(b.msgs), _ptr(b.offs), _ptr(b.s), _ptr(b.R)
        cb.n, cb.first_index, cb.R_count = b.n, b.first_index, b.R_count
        cb.ds, cb.ds_nodes = _ptr(b.ds), b.ds_nodes
        cb.on_device = 1 if on_dev else 0
        return cb

    def aver(self, b: BatchData, agg_mode: int = AGG_UNIT) -> bool:
        acc = np.zeros(1, np.uint8)
        cb = self._cbatch(b)
        self._check(self.lib.poslo_aver(self.h, C.byref(cb), agg_mode, _ptr(acc)))
        return bool(acc[0])

    def aver_partial(self, b: BatchData, agg_mode: int = AGG_UNIT) -> Partial:
        """The shard record of poslo_aver_partial (aggregate before the group check)."""
        out = Partial()
        cb = self._cbatch(b)
        self._check(self.lib.poslo_aver_partial(self.h, C.byref(cb), agg_mode, C.byref(out)))
        return out

    def combine_check(self, Y: bytes, parts) -> tuple:
        """poslo_combine_check over shard records (Partial objects or 216-byte strings, in
        index order): returns (accept, summed record)."""
        recs = b"".join(p.to_bytes() if isinstance(p, Partial) else bytes(p) for p in parts)
        arr = np.frombuffer(recs, np.uint8).copy()
        acc = np.zeros(1, np.uint8)
        total = Partial()
        self._check(self.lib.poslo_combine_check(self.h, _ptr(bytes(Y)), _ptr(arr), len(recs) // C.sizeof(Partial),
                                                 _ptr(acc), C.byref(total)))
        return bool(acc[0]), total

    def distill(self, b: BatchData, cap: int | None = None):
        cap = b.n if cap is None else cap
        idx = np.zeros(max(cap, 1), np.uint64)
        cnt = C.c_uint64()
        cs = np.zeros(32, np.uint8)
        cR = np.zeros(32, np.uint8)
        cb = self._cbatch(b)
        self._check(self.lib.poslo_distill(self.h, C.byref(cb), _ptr(idx), cap, C.byref(cnt), _ptr(cs), _ptr(cR)))
        return idx[:cnt.value].copy(), cs.tobytes(), cR.tobytes()

    def aver_multi(self, Ys, dev_sizes, first_index, n2, ds_list, msgs, offs, s, R, cap: int | None = None):
        """Multi-device AVer + Distill.  Ys: per-device 32-byte keys; dev_sizes: entries per
        device; msgs/offs/s/R: the concatenated batch (numpy, or torch CUDA tensors)."""
        nd = len(Ys)
        dev_start = np.zeros(nd + 1, np.uint64)
        dev_start[1:] = np.cumsum(np.asarray(dev_sizes, dtype=np.uint64))
        ds_off = np.zeros(nd + 1, np.uint32)
        ds_off[1:] = np.cumsum([len(d) // 24 for d in ds_list])
        Yb = np.frombuffer(b"".join(bytes(y) for y in Ys), np.uint8).copy()
        dsb = np.frombuffer(b"".join(ds_list), np.uint8).copy()
        fi = np.ascontiguousarray(first_index, dtype=np.uint64)
        n2a = np.ascontiguousarray(n2, dtype=np.uint32)
        on_dev = _is_torch(offs) and offs.is_cuda
        if not _is_torch(offs):
            offs = np.ascontiguousarray(offs, dtype=np.uint64)
            msgs, s, R = _u8(msgs), _u8(s), _u8(R)
        mb = MultiBatch()
        mb.n_dev = nd
        mb.Y, mb.dev_start, mb.first_index, mb.n2 = _ptr(Yb), _ptr(dev_start), _ptr(fi), _ptr(n2a)
        mb.ds, mb.ds_off = _ptr(dsb), _ptr(ds_off)
        mb.msgs, mb.offs, mb.s, mb.R = _ptr(msgs), _ptr(offs), _ptr(s), _ptr(R)
        mb.on_device = 1 if on_dev else 0
        total = int(dev_start[-1])
        cap = total if cap is None else cap
        acc = np.zeros(nd, np.uint8)
        pairs = np.zeros(2 * max(cap, 1), np.uint64)
        cnt = C.c_uint64()
        self._check(self.lib.poslo_aver_multi(self.h, C.byref(mb), _ptr(acc), _ptr(pairs), cap, C.byref(cnt)))
        return acc.astype(bool), pairs[:2 * cnt.value].reshape(-1, 2).copy()

    def distill_stream(self, b: BatchData, chunk_entries: int, cap: int | None = None):
        """Out-of-core AVer + Distill of a host-resident POSLO-F batch; returns (accept, indices)."""
        cap = b.n if cap is None else cap
        idx = np.zeros(max(cap, 1), np.uint64)
        acc = np.zeros(1, np.uint8)
        cnt = C.c_uint64()
        cb = self._cbatch(b)
        self._check(self.lib.poslo_distill_stream(self.h, C.byref(cb), chunk_entries, _ptr(acc), _ptr(idx), cap,
                                                  C.byref(cnt)))
        return bool(acc[0]), idx[:cnt.value].copy()

    # ------------------------------------------------------------------ POSLO-C ccd (Fig. 3b)
    def distill_c(self, b: BatchData, n_umbrella: int, cap: int | None = None):
        """C.Distill: returns (valid per epoch, ccd) with ccd = dict(s_v, R_v, umbrellas=[(s, R)],
        invalid=[global epoch indices])."""
        n1 = b.n // b.n2
        cap = n1 if cap is None else cap
        valid = np.zeros(max(n1, 1), np.uint8)
        sv, Rv = np.zeros(32, np.uint8), np.zeros(32, np.uint8)
        umb = np.zeros(64 * max(n_umbrella, 1), np.uint8)
        inv = np.zeros(max(cap, 1), np.uint64)
        c = CcdC(_ptr(sv), _ptr(Rv), _ptr(umb), _ptr(inv), cap, 0)
        cb = self._cbatch(b)
        self._check(self.lib.poslo_distill_c(self.h, C.byref(cb), n_umbrella, _ptr(valid), C.byref(c)))
        ccd = dict(s_v=sv.tobytes(), R_v=Rv.tobytes(),
                   umbrellas=[(umb[64 * l:64 * l + 32].tobytes(), umb[64 * l + 32:64 * l + 64].tobytes())
                              for l in range(n_umbrella)],
                   invalid=[int(x) for x in inv[:c.n_invalid]])
        return [bool(v) for v in valid[:n1]], ccd

    def sebver_c(self, b: BatchData, n_umbrella: int, ccd: dict, mode: str):
        """SeBVer in mode 'V', 'U' or 'I' against a ccd from distill_c; returns the bits."""
        sv = np.frombuffer(ccd["s_v"], np.uint8).copy()
        Rv = np.frombuffer(ccd["R_v"], np.uint8).copy()
        umb = np.frombuffer(b"".join(s + R for s, R in ccd["umbrellas"]) or bytes(64), np.uint8).copy()
        inv = np.asarray(ccd["invalid"] or [0], np.uint64)
        c = CcdC(_ptr(sv), _ptr(Rv), _ptr(umb), _ptr(inv), len(ccd["invalid"]), len(ccd["invalid"]))
        n = {"V": 1, "U": n_umbrella, "I": len(ccd["invalid"])}[mode]
        bits = np.zeros(max(n, 1), np.uint8)
        cb = self._cbatch(b)
        self._check(self.lib.poslo_sebver_c(self.h, C.byref(cb), n_umbrella, C.byref(c), ord(mode), _ptr(bits)))
        return [bool(x) for x in bits[:n]]

    # ------------------------------------------------------------------ serving
    def serve_start(self, workers: int = 2, max_batch_devices: int = 4096, max_batch_entries: int = 1 << 22):
        self._check(self.lib.poslo_serve_start(self.h, workers, max_batch_devices, max_batch_entries))

    def serve_stop(self):
        self._check(self.lib.poslo_serve_stop(self.h))

    def register_key(self, Y: bytes) -> int:
        kid = C.c_uint32()
        self._check(self.lib.poslo_register_key(self.h, _ptr(bytes(Y)), C.byref(kid)))
        return kid.value

    def submit(self, key_id: int, n2: int, first_index: int, msgs, offs, s, R, ds: bytes,
               borrow: bool = False) -> int:
        """Queue one request (host arrays; copied by the library unless borrow, in which case
        the arrays must stay alive and unchanged until the result is polled).  Raises
        PosloError EBUSY when the memory budget is exhausted."""
        offs = np.ascontiguousarray(offs, dtype=np.uint64)
        arrays = (_u8(msgs), offs, _u8(s), _u8(R))
        q = Request()
        q.key_id, q.n2, q.first_index = key_id, n2, first_index
        q.msgs, q.offs, q.n = _ptr(arrays[0]), _ptr(offs), len(offs) - 1
        q.s, q.R, q.ds, q.ds_nodes = _ptr(arrays[2]), _ptr(arrays[3]), _ptr(bytes(ds)), len(ds) // 24
        q.flags = REQ_BORROW if borrow else 0
        t = C.c_uint64()
        self._check(self.lib.poslo_submit(self.h, C.byref(q), C.byref(t)))
        if borrow:
            self._borrowed[t.value] = arrays     # alive until the result has been polled
        return t.value

    def poll(self, ticket: int, wait_ms: int = 0, cap: int = 1 << 16, with_latency: bool = False):
        """None while pending, else (accept, invalid indices[, seconds spent in the service])."""
        acc = np.zeros(1, np.uint8)
        idx = np.zeros(max(cap, 1), np.uint64)
        cnt = C.c_uint64()
        lat = C.c_uint64()
        rc = self.lib.poslo_poll(self.h, ticket, wait_ms, _ptr(acc), _ptr(idx), cap, C.byref(cnt), C.byref(lat))
        if rc == POSLO_PENDING:
            _keep.clear()
            return None
        if rc != POSLO_EBUFSMALL:
            self._borrowed.pop(ticket, None)
        self._check(rc)
        res = (bool(acc[0]), idx[:cnt.value].copy())
        return res + (lat.value * 1e-9,) if with_latency else res

    def serve_stats(self):
        b, r, u = C.c_uint64(), C.c_uint64(), C.c_uint64()
        self._check(self.lib.poslo_serve_stats(self.h, C.byref(b), C.byref(r), C.byref(u)))
        return b.value, r.value, u.value

    def serve_timeline(self, cap: int = 1 << 16) -> list:
        """The service's per-batch records since the last read (oldest first), as dicts."""
        out = (BatchRecord * max(cap, 1))()
        n = C.c_uint64()
        self._check(self.lib.poslo_serve_timeline(self.h, C.cast(out, C.c_void_p), cap, C.byref(n)))
        return [{f: getattr(out[i], f) for f, _ in BatchRecord._fields_} for i in range(n.value)]

    def epoch_seeds(self, ds: bytes, first_epoch: int, n_epochs: int) -> np.ndarray:
        out = np.zeros(16 * max(n_epochs, 1), np.uint8)
        self._check(self.lib.poslo_epoch_seeds(self.h, _ptr(ds), len(ds) // 24, first_epoch, n_epochs, _ptr(out)))
        return out[:16 * n_epochs].reshape(n_epochs, 16)

    def hash_entries(self, b: BatchData, out=None):
        cb = self._cbatch(b)
        if out is None:
            out = np.zeros(32 * max(b.n, 1), np.uint8)
        self._check(self.lib.poslo_hash_entries(self.h, C.byref(cb), _ptr(out)))
        return out

    def agg(self, scalars, points, on_device: bool = False):
        """Agg: (sum of the scalars mod q, sum of the points), 32 bytes each."""
        s_out = np.zeros(32, np.uint8)
        R_out = np.zeros(32, np.uint8)
        if on_device:
            n = points.numel() // 32
        else:
            points, scalars = _u8(points), _u8(scalars)
            n = len(points) // 32
        self._check(self.lib.poslo_agg(self.h, _ptr(scalars), _ptr(points), n, 1 if on_device else 0, _ptr(s_out),
                                       _ptr(R_out)))
        return s_out.tobytes(), R_out.tobytes()

    def msm(self, points, scalars, on_device: bool = False) -> bytes:
        out = np.zeros(32, np.uint8)
        if on_device:
            n = points.numel() // 32
        else:
            points, scalars = _u8(points), _u8(scalars)
            n = len(points) // 32
        self._check(self.lib.poslo_msm(self.h, _ptr(points), _ptr(scalars), n, 1 if on_device else 0, _ptr(out)))
        return out.tobytes()

    def msm_autotune(self, n: int, scalar_words: int = 4) -> int:
        """Time the bucket MSM's window widths at size n; later MSMs of that size class use the
        fastest.  Returns the chosen width."""
        c = C.c_uint32(0)
        self._check(self.lib.poslo_msm_autotune(self.h, n, scalar_words, C.byref(c)))
        return int(c.value)

    def msm_get_plan(self, n: int, scalar_words: int = 4):
        """(window c, range log2) the next MSM of n entries would use."""
        c, r = C.c_uint32(0), C.c_uint32(0)
        self._check(self.lib.poslo_msm_get_plan(self.h, n, scalar_words, C.byref(c), C.byref(r)))
        return int(c.value), int(r.value)

    def msm_set_plan(self, n: int, window: int, range_log2: int, scalar_words: int = 4):
        """Store a plan for the size class of n."""
        self._check(self.lib.poslo_msm_set_plan(self.h, n, scalar_words, window, range_log2))

    # ------------------------------------------------------------------ profiling
    def set_profiling(self, on: bool):
        self._check(self.lib.poslo_set_profiling(self.h, 1 if on else 0))

    def set_graphs(self, on: bool):
        """Replay repeated call shapes of aver_multi / distill from CUDA graphs (default on)."""
        self._check(self.lib.poslo_set_graphs(self.h, 1 if on else 0))

    def set_multi_window_limit(self, max_entries: int):
        """Multi-device batches up to max_entries check window by window (default 2^21)."""
        self._check(self.lib.poslo_set_multi_window_limit(self.h, max_entries))

    def set_key_cache(self, capacity: int):
        """Drop every cached key table and keep at most `capacity` keys' tables (0: off)."""
        self._check(self.lib.poslo_set_key_cache(self.h, capacity))

    def key_cache_stats(self):
        """(hits, misses) of the key-table cache."""
        h, m = C.c_uint64(0), C.c_uint64(0)
        self._check(self.lib.poslo_key_cache_stats(self.h, C.byref(h), C.byref(m)))
        return int(h.value), int(m.value)

    def graph_stats(self):
        """(graphs captured, replays run) on this context."""
        c, r = C.c_uint64(0), C.c_uint64(0)
        self._check(self.lib.poslo_graph_stats(self.h, C.byref(c), C.byref(r)))
        return int(c.value), int(r.value)

    def kernel_time(self, name: str):
        ms = C.c_double()
        n = C.c_uint64()
        self.lib.poslo_kernel_time(self.h, name.encode(), C.byref(ms), C.byref(n))
        return ms.value, n.value

    def reset_kernel_times(self):
        self.lib.poslo_reset_kernel_times(self.h)

"""Benchmark: verified POSLO log entries per second on GB300 (AVer + Distill).

The workload is one signer's log: 2^20 POSLO-F entries per GPU, message lengths uniform in
[32, 256] bytes, epochs of n2 = 256 (the seed tree's root disclosed), all entries valid.  With
N GPUs (one process each) the log holds N * 2^20 entries and rank r verifies the contiguous
shard of global indices [r 2^20, (r + 1) 2^20).

One step is AVer + Distill of the whole log: every rank reduces its shard to the weighted
aggregate record of poslo_aver_partial (epoch seeds, per-entry PRF and H, the weights z_t,
the scalar sums mod q, decoding of the 2^20 commitments R_t and their bucket MSM), the ranks
exchange the 216-byte records (all-gather), and each runs the cofactored check of the whole
log on its device (poslo_combine_check); only when the log is rejected does every rank run
Distill on its shard and the ranks gather the ascending invalid lists.  On one GPU the same
calls run without the exchange.

Inputs are resident in HBM when the timed region starts (value); the e2e figure repeats the
step through the same C-ABI calls with pinned host buffers, so the host-to-device copies of
the inputs and the device-to-host copies of the results are inside its timed region.  The
inputs (151 MB of messages + 64 MB of signatures) exceed the 129 MB L2 between steps.

Further objects in the line: the shard's own poslo_distill call, Distill with 0.1 % of the
entries tampered, the 4,096-device batch, serving, the hash-bound POSLO-C workloads, out of
core, and the 1,024-entry latencies.

--impl reference times the C++ oracle (the plain per-entry definition) on a bounded sample of
the same workload on this machine's host cores.
"""
from __future__ import annotations

import argparse
import collections
import ctypes as C
import json
import os
import statistics
import struct
import subprocess
import tempfile
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

N_ENTRIES = 1 << 20
N2 = 256
D = 12
LMIN, LMAX = 32, 256
SEED = 2

WORKLOAD = ("POSLO-F AVer+Distill, single signer: N=2^20 entries per GPU (one log of N_gpus x 2^20 entries, "
            "contiguous shards), |m|~U[32,256] B, n2=256 (root disclosed), all valid, edwards25519 + SHA-256")


# ------------------------------------------------------------------------------ helpers

def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


def shard_plan(rank: int, world: int, n_per_rank: int = N_ENTRIES) -> tuple[int, int]:
    """One log of world * n_per_rank entries of one signer, split into contiguous shards: rank r
    verifies global indices [r n, (r + 1) n).  Returns (first index of the shard, depth of the
    signer's seed tree), the tree deep enough for every epoch of the whole log (n2 = 256)."""
    return rank * n_per_rank, D + (world - 1).bit_length()


def max_over_ranks(ms: float, world: int) -> float:
    """The slowest rank's time per step (the job's time): all-reduce MAX over the ranks."""
    if world <= 1:
        return ms
    import torch
    t = torch.tensor([ms], dtype=torch.float64)
    torch.distributed.all_reduce(t, op=torch.distributed.ReduceOp.MAX)
    return float(t.item())


def job_throughput(entries_per_rank: int, world: int, ms: float) -> float:
    """Whole-job entries/s: every rank's entries over the slowest rank's step time."""
    return world * entries_per_rank / (ms * 1e-3)


class ClockSampler:
    """nvidia-smi clock and throttle-reason samples during the timed region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, device: int):
        self.device = device
        self.proc = None
        # the raw samples go to POSLO_CLOCKS_DIR (default: the system's temporary directory)
        out_dir = os.environ.get("POSLO_CLOCKS_DIR", tempfile.gettempdir())
        self.path = os.path.join(out_dir, f"poslo_clocks_{os.getpid()}.csv")

    def __enter__(self):
        os.makedirs(os.path.dirname(self.path), exist_ok=True)
        try:
            self.f = open(self.path, "w")
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={self.device}", f"--query-gpu={self.FIELDS}",
                                          "--format=csv,noheader,nounits", "-lms", "100"],
                                         stdout=self.f, stderr=subprocess.DEVNULL)
            time.sleep(0.3)
        except (OSError, FileNotFoundError):
            self.proc = None
        return self

    def __exit__(self, *a):
        if self.proc:
            self.proc.terminate()
            self.proc.wait()
            self.f.close()

    def summary(self):
        if not self.proc:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        rows = []
        for line in open(self.path):
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                rows.append((float(parts[1]), float(parts[2]), parts[5:9]))
            except ValueError:
                continue
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[k] for _, _, r in rows for k in range(4) if r[k].lower() == "active"})
        return {"sm_mhz": statistics.median(r[0] for r in rows), "sm_max_mhz": max(r[1] for r in rows),
                "reasons": reasons, "samples": len(rows)}


def probe_int_peaks(device: int) -> dict:
    from paper_2506_08781_gb300 import build
    lib = C.CDLL(build.PROBE_LIB)
    out = (C.c_double * 5)()
    rc = lib.poslo_probe_int_peaks(device, out)
    if rc != 0:
        return {}
    return {"imad_lo_ops": out[0], "imad_hi_ops": out[1], "lop3_ops": out[2], "iadd_ops": out[3],
            "shf_ops": out[4]}


# Algorithmic integer work per entry for the roofline (counted from the algorithms, not
# from the compiled code):
#   decoding R_t (k_points): 255 squarings and 21 multiplications in F_p, plus the 7
#     multiplications of its mixed addition into the unit sum.  Counted per half of a
#     32x32-bit product: a squaring has 28 cross products and 8 diagonal squares (low and
#     high halves) and a fold by 38 (8 low + 8 high + 1 low): 45 low, 44 high; a
#     multiplication has 64 products and the fold: 73 low, 72 high.
#   mad.hi issues at half the rate of mad.lo on this GPU (probed), so the work is expressed
#     in mad.lo issue slots: low + high x (mad.lo rate / mad.hi rate).
#   SHA-256: 1,384 ALU instructions per compression with 3-input LOP3/IADD3 and funnel
#     shifts (64 rounds x 14 + 48 schedule words x 10 + 8); compressions per entry =
#     1 (PRF) + ceil((L + 25) / 64) (H)
SQ_LO, SQ_HI, MUL_LO, MUL_HI = 45, 44, 73, 72
DECODE_SQ, DECODE_MUL = 255, 21 + 7
IMAD_LO_PER_DECODE = DECODE_SQ * SQ_LO + DECODE_MUL * MUL_LO    # 13,519
IMAD_HI_PER_DECODE = DECODE_SQ * SQ_HI + DECODE_MUL * MUL_HI    # 13,236
ALU_PER_COMPRESSION = 64 * 14 + 48 * 10 + 8
# DRAM bytes (read + write) of one k_points launch over 2^20 entries, from an ncu capture:
# the 32 MB of encodings read once; of the 100 MB of decoded points written, the part that has
# left L2 by the end of the launch.
POINTS_DRAM_BYTES_2P20 = 33_746_176 + 44_258_304


def make_workload(n=N_ENTRIES, seed=SEED, tamper=0, rank=0, world=1):
    """Shard `rank` of the log: the one signer's key material, the shard's messages (rank 0's
    are the single-GPU workload's) and the BPV subsets at the shard's global indices."""
    from paper_2506_08781_gb300 import synth
    km = synth.key_material(seed)
    first, _ = shard_plan(rank, world, n)
    msgs = synth.messages(seed, n, LMIN, LMAX, tag="msg" if rank == 0 else f"msg.shard{rank}")
    subsets = synth.bpv_subsets(seed, n, first_index=first)
    plan = synth.tamper_plan(seed, msgs, tamper) if tamper else None
    return km, msgs, subsets, plan


def sign_workload(ctx, km, msgs, subsets, first_index=0, depth=D):
    Y, bpv_R = ctx.keygen_f(km.y, km.bpv_r)
    s, R = ctx.sign_f(km.y, km.root, depth, N2, km.bpv_r, bpv_R, subsets, msgs.data, msgs.offs,
                      first_index=first_index)
    return Y, s, R


def compressions(msgs) -> int:
    L = (msgs.offs[1:] - msgs.offs[:-1]).astype(np.int64)
    return int(np.sum(1 + (L + 16 + 9 + 63) // 64))


# ------------------------------------------------------------------------------ many devices (4,096 signers)

MULTI_DEVICES = 4096
MULTI_LO, MULTI_HI = 16, 65536
MULTI_TAMPER_FRAC = 0.005
MULTI_D, MULTI_N2 = 9, 256          # n1 = 512 epochs of 256 entries per device (>= 65,536 entries)


def make_multi_workload(ctx, n_dev=MULTI_DEVICES, lo=MULTI_LO, hi=MULTI_HI, seed=4):
    """4,096 devices, sizes log-uniform in [16, 65536], messages U[32, 256] bytes, 0.5 % of the
    devices with one entry flipped by one byte.  Keys and signatures come from the library's
    signer (BPV table of 64 entries, 4 per subset: the verifier does not depend on them)."""
    from paper_2506_08781_gb300 import synth
    sizes = synth.device_sizes(seed, n_dev, lo, hi)
    total = int(sizes.sum())
    msgs = synth.messages(seed, total, LMIN, LMAX, tag="multi")
    start = np.zeros(n_dev + 1, np.int64)
    start[1:] = np.cumsum(sizes)
    Ys, ss, Rs, dss = [], [], [], []
    for d in range(n_dev):
        km = synth.key_material(seed * 100000 + d, v=64)
        Y, bpv_R = ctx.keygen_f(km.y, km.bpv_r)
        lo_, hi_ = int(start[d]), int(start[d + 1])
        offs = msgs.offs[lo_:hi_ + 1]
        sub = synth.bpv_subsets(seed * 100000 + d, hi_ - lo_, v=64, k=4)
        s, R = ctx.sign_f(km.y, km.root, MULTI_D, MULTI_N2, km.bpv_r, bpv_R, sub, msgs.data, offs)
        Ys.append(Y)
        ss.append(s)
        Rs.append(R)
        dss.append(struct.pack("<II", MULTI_D, 0) + km.root)
    bad_devs = synth.choose_without_replacement(seed, "baddev", n_dev, round(MULTI_TAMPER_FRAC * n_dev))
    data = msgs.data.copy()
    pairs = []
    for d in bad_devs:
        d = int(d)
        t = int(start[d]) + int(synth.uniform_int(seed, f"t{d}", 1, 0, int(sizes[d]) - 1)[0])
        L = int(msgs.offs[t + 1] - msgs.offs[t])
        pos = int(synth.uniform_int(seed, f"p{d}", 1, 0, L - 1)[0])
        data[int(msgs.offs[t]) + pos] ^= int(synth.uniform_int(seed, f"m{d}", 1, 1, 255)[0])
        pairs.append((d, t - int(start[d])))
    return dict(sizes=sizes, msgs=synth.Messages(data, msgs.offs), Y=Ys, s=np.concatenate(ss),
                R=np.concatenate(Rs), ds=dss, pairs=sorted(pairs), total=total)


MULTI_ORACLE_EVERY = 64                # the C++ oracle verifies every 64th device of the workload


def multi_oracle_subsample(w, every: int = MULTI_ORACLE_EVERY) -> dict:
    """The C++ oracle's per-device Distill (the definition) on every `every`-th device of the
    4,096-device workload, entries split over all host cores; its lists are checked against
    the tamper plan's pairs of those devices."""
    from oracle import cpp_oracle as X
    cores = host_cores()
    sizes = w["sizes"]
    start = np.zeros(len(sizes) + 1, np.int64)
    start[1:] = np.cumsum(sizes)
    devices = list(range(0, len(sizes), every))
    n, found = 0, []
    t0 = time.perf_counter()
    for d in devices:
        lo, hi = int(start[d]), int(start[d + 1])
        inv, _, _ = X.distill_f(w["Y"][d], w["msgs"].data, w["msgs"].offs[lo:hi + 1], 0, MULTI_N2,
                                w["s"][32 * lo:32 * hi], w["R"][32 * lo:32 * hi], w["ds"][d], cores)
        found += [(d, int(t)) for t in inv]
        n += hi - lo
    sec = time.perf_counter() - t0
    assert found == [p for p in w["pairs"] if p[0] % every == 0], "the C++ oracle's lists differ from the plan"
    rate = n / sec
    return {"value": rate, "unit": "entries/s", "cores": cores, "kind": "oracle",
            "implementation": "C++ oracle (oracle/poslo_oracle.cpp)",
            "sample": f"every {every}th device ({len(devices)} devices, {n} of the {w['total']} entries) verified "
                      f"by the C++ oracle's per-device Distill on {cores} std::thread workers in {sec:.1f} s; "
                      f"the whole workload at this rate: {w['total'] / rate / 60:.0f} min"}


def bench_multi(ctx, steps: int, warmup: int, cpu: bool = False) -> dict:
    import torch
    from paper_2506_08781_gb300 import poslo
    t0 = time.perf_counter()
    w = make_multi_workload(ctx)
    setup_s = time.perf_counter() - t0
    dev = lambda a: torch.from_numpy(np.ascontiguousarray(a)).cuda()
    d_msgs, d_offs = dev(w["msgs"].data), dev(w["msgs"].offs.view(np.int64))
    d_s, d_R = dev(w["s"]), dev(w["R"])
    nd = len(w["Y"])
    args = (w["Y"], w["sizes"], np.zeros(nd, np.uint64), np.full(nd, MULTI_N2, np.uint32), w["ds"],
            d_msgs, d_offs, d_s, d_R)
    torch.cuda.synchronize()
    msm_window = ctx.msm_autotune(w["total"], 4)
    msm_range = ctx.msm_get_plan(w["total"], 4)[1]
    for _ in range(warmup):
        acc, pairs = ctx.aver_multi(*args)
    got = [(int(a), int(b)) for a, b in pairs]
    assert got == w["pairs"], "multi-device localisation differs from the tamper plan"
    assert int((~acc).sum()) == len({d for d, _ in w["pairs"]})
    stream = torch.cuda.ExternalStream(ctx.stream)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(steps):
        ctx.aver_multi(*args)
    e1.record(stream)
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1) / steps
    # stage times from one more (untimed) call with the context's kernel timers on
    ctx.set_profiling(True)
    ctx.reset_kernel_times()
    ctx.aver_multi(*args)
    torch.cuda.synchronize()
    stages = {}
    for name in ("seeds", "hash", "points", "msm", "msm_sort", "msm_bucket", "msm_reduce", "msm_final", "table",
                 "prep", "segment_sums", "check", "finalize", "tree", "bisect", "localise"):
        tot, cnt = ctx.kernel_time(name)
        if cnt:
            stages[name] = {"ms": tot, "launches": cnt}
    ctx.set_profiling(False)
    return {"workload": f"{nd} devices, sizes log-uniform [{MULTI_LO}, {MULTI_HI}] (total {w['total']} entries), "
                        f"|m|~U[32,256], {len(w['pairs'])} devices with one flipped byte",
            "value": w["total"] / (ms * 1e-3), "unit": "entries/s", "ms_per_step": ms, "steps": steps,
            "invalid_found": len(got), "setup_s": setup_s, "msm_window": msm_window, "msm_range_log2": msm_range,
            "stages": stages, "cpu_baseline": multi_oracle_subsample(w) if cpu else None}


# ------------------------------------------------------------------------------ Distill with tampered entries

TAMPER_FRAC = 0.001
TAMPER_SEED = 3


def bench_distill_tampered(ctx, msgs, Y, s, R, ds, steps: int, warmup: int) -> dict:
    """The localisation workload: the same 2^20 signed entries with round(0.001 * 2^20) = 1,049
    of them flipped by one byte (uniform entries, offsets and non-zero masks), inputs resident
    in HBM; then the same calls from pinned host memory.  Asserts that the invalid list equals
    the tamper plan."""
    import torch
    from paper_2506_08781_gb300 import poslo, synth
    n = msgs.n
    plan = synth.tamper_plan(TAMPER_SEED, msgs, round(TAMPER_FRAC * n))
    bad = synth.apply_tamper(msgs, plan)
    want = [int(t) for t in plan.idx]
    d_msgs = torch.from_numpy(bad.data).cuda()
    d_offs = torch.from_numpy(bad.offs.view(np.int64)).cuda()
    d_s, d_R = torch.from_numpy(s).cuda(), torch.from_numpy(R).cuda()
    torch.cuda.synchronize()
    batch = ctx.make_batch(poslo.VARIANT_F, N2, Y, d_msgs, d_offs, d_s, d_R, ds)
    for _ in range(warmup):
        idx, _, _ = ctx.distill(batch)
    assert [int(t) for t in idx] == want, "tampered Distill differs from the tamper plan"
    stream = torch.cuda.ExternalStream(ctx.stream)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    e0.record(stream)
    for _ in range(steps):
        idx, _, _ = ctx.distill(batch)
    e1.record(stream)
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1) / steps
    assert [int(t) for t in idx] == want
    # stage times from further (untimed) calls with the context's kernel timers on
    ctx.set_profiling(True)
    ctx.reset_kernel_times()
    prof_calls = 3
    for _ in range(prof_calls):
        ctx.distill(batch)
    torch.cuda.synchronize()
    stages = {}
    for name in ("table", "seeds", "hash", "points", "msm", "msm_sort", "msm_bucket", "msm_reduce", "msm_final",
                 "finalize", "tree", "bisect", "check"):
        tot, cnt = ctx.kernel_time(name)
        if cnt:
            stages[name] = {"ms_per_call": tot / prof_calls, "launches_per_call": cnt / prof_calls}
    ctx.set_profiling(False)
    # end to end from pinned host memory
    p = [torch.from_numpy(a).pin_memory() for a in (bad.data, bad.offs.view(np.int64), s, R)]
    hbatch = ctx.make_batch(poslo.VARIANT_F, N2, Y, p[0], p[1], p[2], p[3], ds)
    for _ in range(2):
        ctx.distill(hbatch)
    t0 = time.perf_counter()
    for _ in range(steps):
        idx, _, _ = ctx.distill(hbatch)
    e2e_s = (time.perf_counter() - t0) / steps
    assert [int(t) for t in idx] == want
    del d_msgs, d_offs, d_s, d_R
    return {"workload": f"POSLO-F Distill, single signer: N=2^20 entries, |m|~U[32,256] B, n2=256, "
                        f"{len(want)} entries ({TAMPER_FRAC:.1%}) flipped by one byte at seeded uniform positions",
            "value": n / (ms * 1e-3), "unit": "entries/s", "ms_per_step": ms, "steps": steps,
            "invalid_found": len(want), "list_equals_plan": True,
            "stages": stages,
            "e2e": {"value": n / e2e_s, "unit": "entries/s",
                    "h2d_bytes_per_step": int(bad.data.nbytes + bad.offs.nbytes + s.nbytes + R.nbytes + 32 + len(ds)),
                    "d2h_bytes_per_step": 8 * len(want) + 72}}


# ------------------------------------------------------------------------------ graph replay

REPLAY_DEVICES, REPLAY_LO, REPLAY_HI, REPLAY_CALLS = 64, 16, 1024, 40


def bench_graph_replay(ctx) -> dict:
    """A small multi-device batch verified again and again with the same layout (a gateway
    re-checking a fixed fleet): per-call wall time with the launch sequence replayed from a
    CUDA graph against the same calls launched kernel by kernel."""
    import torch
    w = make_multi_workload(ctx, n_dev=REPLAY_DEVICES, lo=REPLAY_LO, hi=REPLAY_HI, seed=6)
    dev = lambda a: torch.from_numpy(np.ascontiguousarray(a)).cuda()
    args = (w["Y"], w["sizes"], np.zeros(REPLAY_DEVICES, np.uint64), np.full(REPLAY_DEVICES, MULTI_N2, np.uint32),
            w["ds"], dev(w["msgs"].data), dev(w["msgs"].offs.view(np.int64)), dev(w["s"]), dev(w["R"]))
    torch.cuda.synchronize()
    out = {"workload": f"{REPLAY_DEVICES} devices, sizes log-uniform [{REPLAY_LO}, {REPLAY_HI}] "
                       f"(total {w['total']} entries), device-resident, {len(w['pairs'])} tampered devices",
           "calls": REPLAY_CALLS}
    for mode in ("launched", "graph"):
        ctx.set_graphs(mode == "graph")
        for _ in range(3):
            ctx.aver_multi(*args)
        c0 = ctx.graph_stats()
        times = []
        for _ in range(REPLAY_CALLS):
            t0 = time.perf_counter()
            acc, pairs = ctx.aver_multi(*args)
            times.append(time.perf_counter() - t0)
        assert [(int(a), int(b)) for a, b in pairs] == w["pairs"]
        c1 = ctx.graph_stats()
        out[mode] = {"ms_per_call_p50": float(np.percentile(times, 50) * 1e3),
                     "ms_per_call_mean": float(np.mean(times) * 1e3), "replays": c1[1] - c0[1]}
    ctx.set_graphs(True)
    return out


# ------------------------------------------------------------------------------ out of core

STREAM_CHUNKS = 8                      # 8 x 2^20 entries (1.2 GB of messages) from pinned host memory
STREAM_D = 15                          # n1 = 32,768 epochs of 256 entries


# ------------------------------------------------------------------------------ 1,024 entries of 64 bytes (latency)

SMALL_N, SMALL_L, SMALL_D, SMALL_CALLS = 1024, 64, 2, 200     # n1 = 4 epochs of n2 = 256


def bench_small_latency(device: int, calls: int = SMALL_CALLS) -> dict:
    """The smallest workload: 1,024 entries of 64-byte messages under POSLO-C (n1 = 4, n2 = 256)
    and POSLO-F, a valid copy and a copy with one flipped byte.  Per-call wall time of the
    synchronous calls a user makes with host buffers (inputs copied in, results read back),
    p50 and p99 in microseconds over `calls` calls after 5 warm-up calls."""
    from paper_2506_08781_gb300 import poslo, synth
    km = synth.key_material(SEED + 11, v=64)
    msgs = synth.messages(SEED + 11, SMALL_N, SMALL_L, SMALL_L)
    plan = synth.tamper_plan(SEED + 11, msgs, 1)
    bad = synth.apply_tamper(msgs, plan)
    ctx = poslo.Context(device=device, verifier_seed=synth.verifier_seed(11))
    ds = struct.pack("<II", SMALL_D, 0) + km.root
    Yc, epoch_R = ctx.keygen_c(km.y, km.r, SMALL_D, N2)
    s_ep = ctx.sign_c(km.y, km.r, km.root, SMALL_D, N2, msgs.data, msgs.offs, 0, 1 << SMALL_D).reshape(-1, 32)
    # C.Agg of the epochs' signatures (test-data side, outside the timed calls)
    s_agg, _ = ctx.agg(s_ep.tobytes(), np.asarray(epoch_R, np.uint8).tobytes())
    Yf, bpv_R = ctx.keygen_f(km.y, km.bpv_r)
    sub = synth.bpv_subsets(SEED + 11, SMALL_N, v=64, k=4)
    s_f, R_f = ctx.sign_f(km.y, km.root, SMALL_D, N2, km.bpv_r, bpv_R, sub, msgs.data, msgs.offs)
    mk = lambda v, Y, m, s_, R_: ctx.make_batch(v, N2, Y, m.data, m.offs, s_, R_, ds)
    bc, bc_bad = mk(poslo.VARIANT_C, Yc, msgs, s_agg, epoch_R), mk(poslo.VARIANT_C, Yc, bad, s_agg, epoch_R)
    bf, bf_bad = mk(poslo.VARIANT_F, Yf, msgs, s_f, R_f), mk(poslo.VARIANT_F, Yf, bad, s_f, R_f)
    assert ctx.aver(bc) is True and ctx.aver(bc_bad) is False
    assert ctx.aver(bf) is True and ctx.aver(bf_bad) is False
    assert len(ctx.distill(bf)[0]) == 0 and list(ctx.distill(bf_bad)[0]) == list(plan.idx)

    def lat(fn):
        for _ in range(5):
            fn()
        ts = []
        for _ in range(calls):
            t0 = time.perf_counter()
            fn()
            ts.append(time.perf_counter() - t0)
        ts = np.array(ts) * 1e6
        return {"p50_us": float(np.percentile(ts, 50)), "p99_us": float(np.percentile(ts, 99))}

    out = {"workload": f"{SMALL_N} entries of {SMALL_L}-byte messages, n2 = {N2}, n1 = {1 << SMALL_D} "
                       "(root disclosed), host buffers, one flipped byte in the tampered copy",
           "calls": calls,
           "poslo_c_aver_valid": lat(lambda: ctx.aver(bc)),
           "poslo_c_aver_tampered": lat(lambda: ctx.aver(bc_bad)),
           "poslo_f_aver_valid": lat(lambda: ctx.aver(bf)),
           "poslo_f_aver_tampered": lat(lambda: ctx.aver(bf_bad)),
           "poslo_f_distill_valid": lat(lambda: ctx.distill(bf)),
           "poslo_f_distill_tampered": lat(lambda: ctx.distill(bf_bad))}
    ctx.close()
    return out


def bench_stream(device: int) -> dict:
    """Out-of-core AVer + Distill (poslo_distill_stream) of 8 x 2^20 POSLO-F entries held in
    pinned host memory, verified 2^20 entries at a time while the next chunk is copied; the
    per-chunk workload is the 2^20-entry single-signer one (the messages repeat, the signatures do not: each chunk
    is signed at its own global indices)."""
    import torch
    from paper_2506_08781_gb300 import poslo, synth
    ctx = poslo.Context(device=device)
    km, msgs, subsets, _ = make_workload()
    Y, bpv_R = ctx.keygen_f(km.y, km.bpv_r)
    n = STREAM_CHUNKS * N_ENTRIES
    s_all = np.empty((STREAM_CHUNKS, 32 * N_ENTRIES), np.uint8)
    R_all = np.empty((STREAM_CHUNKS, 32 * N_ENTRIES), np.uint8)
    for k in range(STREAM_CHUNKS):
        s_all[k], R_all[k] = ctx.sign_f(km.y, km.root, STREAM_D, N2, km.bpv_r, bpv_R, subsets, msgs.data, msgs.offs,
                                        first_index=k * N_ENTRIES)
    L = int(msgs.offs[-1])
    offs = np.concatenate([msgs.offs[:-1].astype(np.int64) + k * L for k in range(STREAM_CHUNKS)] +
                          [np.array([STREAM_CHUNKS * L], np.int64)])
    p_msgs = torch.from_numpy(np.tile(msgs.data, STREAM_CHUNKS)).pin_memory()
    p_offs = torch.from_numpy(offs).pin_memory()
    p_s = torch.from_numpy(s_all.reshape(-1)).pin_memory()
    p_R = torch.from_numpy(R_all.reshape(-1)).pin_memory()
    b = ctx.make_batch(poslo.VARIANT_F, N2, Y, p_msgs, p_offs, p_s, p_R, struct.pack("<II", STREAM_D, 0) + km.root)
    acc, idx = ctx.distill_stream(b, N_ENTRIES)           # warm-up
    assert acc and len(idx) == 0
    t0 = time.perf_counter()
    acc, idx = ctx.distill_stream(b, N_ENTRIES)
    wall = time.perf_counter() - t0
    ctx.close()
    host_bytes = int(p_msgs.numel() + p_offs.numel() * 8 + p_s.numel() + p_R.numel())
    per_entry = host_bytes / n
    return {"workload": f"{n} POSLO-F entries (|m|~U[32,256] B) in pinned host memory, chunks of {N_ENTRIES}",
            "entries_per_s": n / wall, "wall_s": wall, "host_GB_per_s": host_bytes / wall / 1e9,
            "bytes_per_entry": per_entry, "s_per_TB_of_log_data": 1e12 / per_entry / (n / wall)}


# ------------------------------------------------------------------------------ POSLO-C, hash-bound

# Thread instructions per AES-128 of the table cipher with its on-the-fly key schedule, counted
# from the algorithm (not the compiled code): each of the 16 round lookups and 4 key-schedule
# S-box lookups is a byte extract, an address computation and a shared-memory read (3); a full
# round adds 12 rotations, 8 three-input XORs and 15 key-schedule operations (masks, shifts,
# the XOR chain, Rcon): 9 x (60 + 12 + 8 + 15) = 855; the last round's 16 S-box reads with their
# masks and shifts (4 x 20) + 4 XORs + its key schedule (27) = 111; the initial AddRoundKey 4;
# the MMO/MDC-2 feed-forward XOR 4: about 974.  The kernel is bound by instruction issue (the
# ALU and shared-memory pipes share the 4 schedulers of an SM), so this count is its roofline.
AES_INSTR = 9 * (16 * 3 + 4 * 3 + 12 + 8 + 15) + (4 * 20 + 4 + 27) + 4 + 4


CCD_UMBRELLAS = 64


def bench_distill_c(ctx_inst, device, km, msgs, Y, epoch_R, s_ep, steps, warmup) -> dict:
    """C.Distill (Fig. 3b) of the same 2^20 entries with 0.1 % of them flipped by one byte
    (0.1 % of the entries, one flipped byte each), 64 umbrellas, then SeBVer in each mode."""
    import torch
    from paper_2506_08781_gb300 import poslo, synth
    plan = synth.tamper_plan(SEED + 8, msgs, round(0.001 * msgs.n))
    bad = synth.apply_tamper(msgs, plan)
    want = sorted({int(t) // N2 for t in plan.idx})
    ctx = poslo.Context(device=device, instantiation=ctx_inst)
    b = ctx.make_batch(poslo.VARIANT_C, N2, Y, torch.from_numpy(bad.data).cuda(),
                       torch.from_numpy(bad.offs.view(np.int64)).cuda(),
                       torch.from_numpy(np.ascontiguousarray(s_ep).reshape(-1).copy()).cuda(),
                       torch.from_numpy(np.asarray(epoch_R, np.uint8).copy()).cuda(), struct.pack("<II", D, 0) + km.root)
    torch.cuda.synchronize()
    for _ in range(warmup):
        valid, ccd = ctx.distill_c(b, CCD_UMBRELLAS)
    assert ccd["invalid"] == want, "C.Distill differs from the tamper plan"
    t0 = time.perf_counter()
    for _ in range(steps):
        ctx.distill_c(b, CCD_UMBRELLAS)
    dms = (time.perf_counter() - t0) / steps * 1e3
    out = {"invalid_epochs": len(want), "umbrellas": CCD_UMBRELLAS, "ms_distill": dms,
           "entries_per_s_distill": N_ENTRIES / (dms * 1e-3)}
    for mode in "VUI":
        bits = ctx.sebver_c(b, CCD_UMBRELLAS, ccd, mode)
        assert all(bits) if mode != "I" else not any(bits)
        t0 = time.perf_counter()
        for _ in range(steps):
            ctx.sebver_c(b, CCD_UMBRELLAS, ccd, mode)
        out[f"ms_sebver_{mode}"] = (time.perf_counter() - t0) / steps * 1e3
    ctx.close()
    return out


def bench_hash_bound(device: int, steps: int, warmup: int) -> dict:
    """POSLO-C AVer (Fig. 3a with the epochs' R~_i from pk): hashing of every entry, one
    aggregate check, no per-entry group work -- the paper's PAVer workload -- at 2^20 entries
    (n2 = 256, n1 = 4096), under POSLO (SHA-256) and POSLO+ (AES: MMO PRF, MDC-2 H), for the
    bench's U[32, 256] messages and for the paper's 16-byte messages (Table 6)."""
    import torch
    from paper_2506_08781_gb300 import poslo, synth
    out = {}
    for label, lmin, lmax in (("U[32,256] B", LMIN, LMAX), ("16 B", 16, 16)):
        km = synth.key_material(SEED + 7)
        msgs = synth.messages(SEED + 7, N_ENTRIES, lmin, lmax)
        L = (msgs.offs[1:] - msgs.offs[:-1]).astype(np.int64)
        d_msgs = torch.from_numpy(msgs.data).cuda()
        d_offs = torch.from_numpy(msgs.offs.view(np.int64)).cuda()
        row = {}
        for name, inst in (("POSLO", poslo.INST_SHA256), ("POSLO+", poslo.INST_AES)):
            ctx = poslo.Context(device=device, instantiation=inst)
            Y, epoch_R = ctx.keygen_c(km.y, km.r, D, N2)
            s_ep = ctx.sign_c(km.y, km.r, km.root, D, N2, msgs.data, msgs.offs, 0, 1 << D).reshape(-1, 32)
            s_agg, _ = ctx.agg(s_ep.tobytes(), np.asarray(epoch_R, np.uint8).tobytes())   # C.Agg, test data
            d_s = torch.from_numpy(np.frombuffer(s_agg, np.uint8).copy()).cuda()
            d_R = torch.from_numpy(np.asarray(epoch_R, np.uint8).copy()).cuda()
            ds = struct.pack("<II", D, 0) + km.root
            torch.cuda.synchronize()
            b = ctx.make_batch(poslo.VARIANT_C, N2, Y, d_msgs, d_offs, d_s, d_R, ds)
            for _ in range(warmup):
                assert ctx.aver(b) is True
            stream = torch.cuda.ExternalStream(ctx.stream)
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            ctx.set_profiling(True)
            ctx.reset_kernel_times()
            e0.record(stream)
            for _ in range(steps):
                ctx.aver(b)
            e1.record(stream)
            torch.cuda.synchronize()
            ms = e0.elapsed_time(e1) / steps
            tot, cnt = ctx.kernel_time("hash")
            hash_ms = tot / cnt
            ctx.set_profiling(False)
            ctx.close()
            if inst == poslo.INST_AES:
                aes = int(np.sum(2 * ((L + 32) // 16) + 2))           # MDC-2 blocks x 2 + the PRF's 2
                work = {"unit": "G thread-instructions/s", "per_launch": aes * AES_INSTR, "pipe": "issue",
                        "peak_note": "4 warp instructions per clock per SM (32 threads each)",
                        "aes_calls": aes, "instr_per_aes": AES_INSTR}
                peak = 4 * 32 * 152 * 2.07e9
            else:
                work = {"unit": "G ALU ops/s", "per_launch": compressions(msgs) * ALU_PER_COMPRESSION,
                        "pipe": "ALU (LOP3/SHF/IADD3)", "peak_note": "64 ops per clock per SM"}
                peak = 64 * 152 * 2.07e9
            ach = work["per_launch"] / (hash_ms * 1e-3)
            row[name] = {"entries_per_s": N_ENTRIES / (ms * 1e-3), "ms_per_aver": ms, "hash_kernel_ms": hash_ms,
                         "hash_roofline": {"bound": work["pipe"], "achieved": ach / 1e9, "peak": peak / 1e9,
                                           "unit": work["unit"], "frac": ach / peak,
                                           "peak_source": work["peak_note"] + " at 2070 MHz, 152 SMs"}}
            if label.startswith("U"):
                row[name]["distill_c"] = bench_distill_c(ctx_inst=inst, device=device, km=km, msgs=msgs, Y=Y,
                                                         epoch_R=epoch_R, s_ep=s_ep, steps=steps, warmup=warmup)
        out[label] = row
    return {"workload": "POSLO-C AVer, 2^20 entries, n2 = 256, n1 = 4096 (root disclosed), R~_i from pk, "
                        "device-resident inputs", "results": out}


# ------------------------------------------------------------------------------ serving (10,000 resident keys)

SERVE_KEYS = 10000
SERVE_REQUESTS = 1500
SERVE_LO, SERVE_HI = 1, 65536
SERVE_TAMPER_FRAC = 0.01
SERVE_BUDGET = 64 << 30
SERVE_WORKERS = 2                      # each stages its next batch while verifying the current one
SERVE_MAX_BATCH = 1 << 22              # entries per served batch at most
SERVE_PER_LEVEL = 20000                # requests per load level, drawn from the SERVE_REQUESTS payloads


def make_serving_workload(ctx, seed=5):
    """10,000 resident keys; SERVE_REQUESTS requests (request r signed under key r) with
    sizes log-uniform in [1, 65536], messages U[32, 256] bytes, 1 % of them with 1-4
    flipped entries.  Returns the request arrays and the expected invalid lists."""
    from paper_2506_08781_gb300 import synth
    sizes = synth.log_uniform_int(seed, "reqsize", SERVE_REQUESTS, SERVE_LO, SERVE_HI)
    total = int(sizes.sum())
    msgs = synth.messages(seed, total, LMIN, LMAX, tag="serve")
    start = np.zeros(SERVE_REQUESTS + 1, np.int64)
    start[1:] = np.cumsum(sizes)
    bad_req = set(int(r) for r in synth.choose_without_replacement(seed, "badreq", SERVE_REQUESTS,
                                                                    round(SERVE_TAMPER_FRAC * SERVE_REQUESTS)))
    data = msgs.data.copy()
    reqs = []
    for r in range(SERVE_REQUESTS):
        km = synth.key_material(seed * 1000000 + r, v=64)
        Y, bpv_R = ctx.keygen_f(km.y, km.bpv_r)
        lo, hi = int(start[r]), int(start[r + 1])
        offs = msgs.offs[lo:hi + 1]
        sub = synth.bpv_subsets(seed * 1000000 + r, hi - lo, v=64, k=4)
        sv, Rv = ctx.sign_f(km.y, km.root, MULTI_D, MULTI_N2, km.bpv_r, bpv_R, sub, msgs.data, offs)
        want = []
        if r in bad_req:
            nflip = min(hi - lo, 1 + int(synth.uniform_int(seed, f"nf{r}", 1, 0, 3)[0]))
            for t in synth.choose_without_replacement(seed, f"ft{r}", hi - lo, nflip):
                t = int(t)
                o = int(offs[t])
                data[o] ^= 0x5A       # lengths are >= 32: the first byte exists
                want.append(t)
        reqs.append(dict(Y=Y, offs=(offs - offs[0]).astype(np.uint64), lo=int(offs[0]), hi=int(offs[-1]),
                         s=sv, R=Rv, ds=struct.pack("<II", MULTI_D, 0) + km.root, want=sorted(want), n=hi - lo))
    for r in reqs:
        r["msgs"] = data[r["lo"]:r["hi"]].copy()
    idle = []
    for k in range(SERVE_REQUESTS, SERVE_KEYS):
        y = bytearray(synth.random_bytes(seed, f"idle{k}", 32).tobytes())
        y[31] &= 0x0F
        Y, _ = ctx.keygen_f(bytes(y), np.zeros(0, np.uint8))
        idle.append(Y)
    return reqs, idle, total


def bench_serving(ctx_factory, workers: int = SERVE_WORKERS, max_batch_entries: int = SERVE_MAX_BATCH,
                  workload=None, plain_path: bool = True) -> dict:
    import ctypes as C
    from paper_2506_08781_gb300 import poslo, synth
    t0 = time.perf_counter()
    if workload is None:
        gen_ctx = ctx_factory()
        workload = make_serving_workload(gen_ctx)
        gen_ctx.close()
    reqs, idle, total = workload
    setup_s = time.perf_counter() - t0
    import torch
    svc = poslo.Context(device=0, mem_budget=SERVE_BUDGET, verifier_seed=synth.verifier_seed(55))
    svc.serve_start(workers=workers, max_batch_devices=4096, max_batch_entries=max_batch_entries)
    kid = [svc.register_key(r["Y"]) for r in reqs] + [svc.register_key(Y) for Y in idle]
    lib = svc.lib
    # the clients' data sit in pinned host memory and are lent to the service (POSLO_REQ_BORROW):
    # each request's inputs go by DMA straight into the batch's device staging
    mbase = np.cumsum([0] + [len(r["msgs"]) for r in reqs])
    ebase = np.cumsum([0] + [r["n"] for r in reqs])
    p_msgs = torch.from_numpy(np.concatenate([r["msgs"] for r in reqs])).pin_memory()
    p_offs = torch.from_numpy(np.concatenate([r["offs"].astype(np.int64) + mbase[i]
                                              for i, r in enumerate(reqs)])).pin_memory()
    p_s = torch.from_numpy(np.concatenate([r["s"] for r in reqs])).pin_memory()
    p_R = torch.from_numpy(np.concatenate([r["R"] for r in reqs])).pin_memory()
    obase = np.cumsum([0] + [r["n"] + 1 for r in reqs])
    structs = []
    for i, (r, k) in enumerate(zip(reqs, kid)):
        q = poslo.Request()
        q.key_id, q.n2, q.first_index = k, MULTI_N2, 0
        q.msgs, q.offs, q.n = p_msgs.data_ptr(), p_offs.data_ptr() + 8 * int(obase[i]), r["n"]
        q.s, q.R = p_s.data_ptr() + 32 * int(ebase[i]), p_R.data_ptr() + 32 * int(ebase[i])
        dsb = (C.c_uint8 * len(r["ds"])).from_buffer_copy(r["ds"])
        r["_ds"] = dsb
        q.ds, q.ds_nodes = C.addressof(dsb), 1
        q.flags = poslo.REQ_BORROW
        structs.append(q)
    acc = np.zeros(1, np.uint8)
    idx = np.zeros(1 << 16, np.uint64)

    # each load level submits SERVE_PER_LEVEL requests, each one of the distinct signed payloads
    # drawn uniformly (with replacement): a payload may be in flight in several requests at once
    order = synth.uniform_int(5, "serve.order", SERVE_PER_LEVEL, 0, len(reqs) - 1)
    seq = [structs[int(i)] for i in order]
    seq_reqs = [reqs[int(i)] for i in order]
    seq_total = int(sum(r["n"] for r in seq_reqs))

    def run(arrivals):
        """Submit the requests at their arrival times.  The budget a request holds is released
        when its result is read, so when the service refuses a request (EBUSY) the oldest
        outstanding result is read first; the rest are read after the last submission."""
        outstanding = collections.deque()
        lat, results = [None] * len(seq), [None] * len(seq)
        tk = C.c_uint64()
        cnt, ln = C.c_uint64(), C.c_uint64()

        def read_oldest():
            i, t = outstanding.popleft()
            rc = lib.poslo_poll(svc.h, t, 600000, acc.ctypes.data, idx.ctypes.data, len(idx), C.byref(cnt),
                                C.byref(ln))
            assert rc == 0, rc
            lat[i] = ln.value * 1e-9
            results[i] = (bool(acc[0]), idx[:cnt.value].tolist())

        base = time.perf_counter()
        for i, (q, at) in enumerate(zip(seq, arrivals)):
            now = time.perf_counter() - base
            if at > now:
                time.sleep(at - now)
            while True:
                rc = lib.poslo_submit(svc.h, C.byref(q), C.byref(tk))
                if rc != -6:        # EBUSY: over the memory budget
                    break
                assert outstanding, "a single request exceeds the memory budget"
                read_oldest()
            assert rc == 0, rc
            outstanding.append((i, tk.value))
        while outstanding:
            read_oldest()
        wall = time.perf_counter() - base
        return np.array(lat), results, wall

    def timeline(wall):
        """Where the workers' time went in the last run, from the service's batch records."""
        recs = svc.serve_timeline(1 << 20)
        if not recs:
            return None
        issue = sum(r["t_staged_ns"] - r["t_take_ns"] for r in recs) * 1e-9
        # a worker waits for a batch's copies only once it has nothing else to do: after the
        # batch's own issue, the end of its previous batch and the issue of its next one (the
        # copies run while the previous batch is verified)
        wait = 0.0
        for w in {r["worker"] for r in recs}:
            mine = sorted((r for r in recs if r["worker"] == w), key=lambda r: r["t_take_ns"])
            for k, r in enumerate(mine):
                busy_until = r["t_staged_ns"]
                if k:
                    busy_until = max(busy_until, mine[k - 1]["t_done_ns"])
                if k + 1 < len(mine) and mine[k + 1]["t_take_ns"] < r["t_verify_ns"]:
                    busy_until = max(busy_until, mine[k + 1]["t_staged_ns"])
                wait += max(0, r["t_verify_ns"] - busy_until) * 1e-9
        check = sum(r["t_checked_ns"] - r["t_verify_ns"] for r in recs) * 1e-9
        publish = sum(r["t_done_ns"] - r["t_checked_ns"] for r in recs) * 1e-9
        busy = wait + check + publish
        # steady state: the rate between the times 10 % and 90 % of the entries were done (the
        # ramp while the first requests arrive and the drain of the last batches left out)
        done = sorted(recs, key=lambda r: r["t_done_ns"])
        cum = np.cumsum([r["entries"] for r in done])
        t10 = done[int(np.searchsorted(cum, 0.1 * cum[-1]))]["t_done_ns"]
        k90 = int(np.searchsorted(cum, 0.9 * cum[-1]))
        t90 = done[k90]["t_done_ns"]
        e10 = cum[int(np.searchsorted(cum, 0.1 * cum[-1]))]
        steady = (cum[k90] - e10) / ((t90 - t10) * 1e-9) if t90 > t10 else None
        return {"batches": len(recs), "requests_per_batch": float(np.mean([r["requests"] for r in recs])),
                "entries_per_batch": float(np.mean([r["entries"] for r in recs])),
                "staging_s_issuing_copies": issue, "worker_s_waiting_for_copies": wait,
                "worker_s_verifying": check, "worker_s_publishing": publish,
                "worker_idle_frac": max(0.0, 1.0 - busy / (workers * wall)),
                "steady_entries_per_s": steady}

    svc.serve_timeline(1 << 20)      # drop the records of the warm-up
    # saturated (every request at t = 0): the service's peak
    lat, results, wall = run(np.zeros(len(seq)))
    sat_timeline = timeline(wall)
    for r, (a, inv) in zip(seq_reqs, results):
        assert inv == r["want"] and a == (not r["want"]), "served result differs from the expected one"
    peak = seq_total / wall
    mean_size = seq_total / len(seq)
    levels = []
    for load in (0.5, 0.8, 0.95):
        rate = load * peak / mean_size
        arr = synth.poisson_arrivals(int(load * 100), len(seq), rate)
        lat, results, wall = run(arr)
        assert all(inv == r["want"] for r, (a, inv) in zip(seq_reqs, results))
        levels.append({"load": load, "offered_requests_per_s": rate, "achieved_entries_per_s": seq_total / wall,
                       "requests": len(seq), "p50_ms": float(np.percentile(lat, 50) * 1e3),
                       "p99_ms": float(np.percentile(lat, 99) * 1e3), "timeline": timeline(wall)})
    batches, nreq, _ = svc.serve_stats()
    svc.serve_stop()
    svc.close()
    head = {"workload": f"{SERVE_KEYS} resident keys; per load level {len(seq)} requests ({seq_total} entries), "
                        f"each one of {len(reqs)} distinct signed payloads of log-uniform [{SERVE_LO}, {SERVE_HI}] "
                        f"entries drawn uniformly; |m|~U[32,256], 1 % of payloads tampered, 64 GB budget, {workers} workers, "
                        f"batches of at most {max_batch_entries} entries, request data lent from pinned host "
                        "memory (POSLO_REQ_BORROW)",
            "peak_entries_per_s": peak,
            "steady_entries_per_s": sat_timeline["steady_entries_per_s"] if sat_timeline else None,
            "peak_timeline": sat_timeline, "levels": levels, "batches": batches,
            "requests_served": nreq,
            "setup_s": setup_s}
    if not plain_path:
        return head
    # the plain path for comparison: one request at a time through poslo_distill on one
    # context, from the same pinned buffers, no batching
    one = poslo.Context(device=0, verifier_seed=synth.verifier_seed(56))
    single_lat = []
    t_all = time.perf_counter()
    for i, r in enumerate(reqs):
        lo, hi = int(ebase[i]), int(ebase[i + 1])
        b = one.make_batch(poslo.VARIANT_F, MULTI_N2, r["Y"], p_msgs, p_offs[int(obase[i]):int(obase[i + 1])],
                           p_s[32 * lo:32 * hi], p_R[32 * lo:32 * hi], r["ds"])
        t0 = time.perf_counter()
        inv, _, _ = one.distill(b)
        single_lat.append(time.perf_counter() - t0)
        assert list(inv) == r["want"]
    single_wall = time.perf_counter() - t_all
    one.close()
    single_lat = np.array(single_lat)
    head["one_request_at_a_time"] = {"entries_per_s": total / single_wall,
                                     "p50_ms": float(np.percentile(single_lat, 50) * 1e3),
                                     "p99_ms": float(np.percentile(single_lat, 99) * 1e3),
                                     "note": "poslo_distill per request, sequential, same pinned inputs; "
                                             "latency = its own verification time (no queue)"}
    return head


# ------------------------------------------------------------------------------ CPU oracle arm

def host_cores() -> int:
    try:
        return len(os.sched_getaffinity(0))
    except AttributeError:
        return os.cpu_count() or 1


class OracleSample:
    """A bounded sample of the workload (the same message generator, lengths U[32, 256],
    n2 = 256 under a D = 12 tree with the root disclosed) signed by the C++ oracle's own
    signer and verified by the C++ oracle's per-entry Distill, which also decides AVer:
    textbook 4 x 64-bit field arithmetic, double-and-add, SHA-256 from FIPS 180-4, entries
    split over std::thread workers (oracle/poslo_oracle.cpp)."""

    def __init__(self, n: int, cores: int):
        from oracle import cpp_oracle as X
        from paper_2506_08781_gb300 import synth
        self.X = X
        self.cores = cores
        km = synth.key_material(SEED, v=64)
        self.msgs = synth.messages(SEED, n, LMIN, LMAX)
        subsets = synth.bpv_subsets(SEED, n, v=64)
        self.Y = X.base_mult(int.from_bytes(km.y, "little"))
        self.s, self.R = X.sign_f(km.y, km.root, D, N2, km.bpv_r, subsets, self.msgs.data, self.msgs.offs, 0,
                                  threads=cores)
        self.ds = struct.pack("<II", D, 0) + km.root

    def run(self, lo: int, count: int, threads: int):
        """Verify entries lo .. lo+count-1; returns (entries, seconds, invalid found)."""
        offs = self.msgs.offs[lo:lo + count + 1]
        t0 = time.perf_counter()
        inv, _, _ = self.X.distill_f(self.Y, self.msgs.data, offs, lo, N2, self.s[32 * lo:32 * (lo + count)],
                                     self.R[32 * lo:32 * (lo + count)], self.ds, threads)
        return count, time.perf_counter() - t0, len(inv)


def cpu_oracle_baseline(per_core: int = 2048):
    cores = host_cores()
    n_all = cores * per_core
    one = max(64, per_core // 4)
    smp = OracleSample(n_all + one, cores)
    n, sec, bad = smp.run(0, n_all, cores)
    n1, sec1, bad1 = smp.run(n_all, one, 1)
    assert bad == 0 and bad1 == 0, "the C++ oracle rejected honest entries"
    return {"value": n / sec, "unit": "entries/s", "cores": cores, "kind": "oracle",
            "implementation": "C++ oracle (oracle/poslo_oracle.cpp)",
            "single_thread_value": n1 / sec1,
            "sample": f"{n} entries of the same workload ({per_core} per core) verified by the C++ oracle's "
                      f"per-entry Distill (the definition) on {cores} std::thread workers in {sec:.1f} s; "
                      f"single thread: {n1} further entries in {sec1:.1f} s"}


def run_reference(args):
    rank, world, _ = dist_env()
    if rank != 0:
        return
    cores = host_cores()
    per_step = max(16, args.cpu_per_core // 8)
    step_n = cores * per_step
    smp = OracleSample(step_n * (args.steps + args.warmup), cores)
    for w in range(args.warmup):
        smp.run(w * step_n, step_n, cores)
    tot_n, tot_t = 0, 0.0
    for k in range(args.steps):
        n, sec, bad = smp.run((args.warmup + k) * step_n, step_n, cores)
        assert bad == 0
        tot_n += n
        tot_t += sec
    n1, sec1, _ = smp.run(0, max(16, per_step // 2), 1)
    value = tot_n / tot_t
    sample = (f"{step_n} entries per step ({per_step} per core) verified by the C++ oracle's per-entry Distill "
              f"(the definition) on {cores} std::thread workers")
    line = {"impl": "reference", "metric": "verified log entries/sec at 1 GB300 (AVer+Distill)",
            "value": value, "unit": "entries/s", "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": 1e3 * tot_t / max(args.steps, 1), "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "u64", "data": "synthetic",
            "config": {"workload": WORKLOAD, "entries_per_gpu": N_ENTRIES, "log_entries": N_ENTRIES * world,
                       "parallelism": f"dp{world}"},
            "cpu_baseline": {"value": value, "unit": "entries/s", "cores": cores, "kind": "oracle",
                             "implementation": "C++ oracle (oracle/poslo_oracle.cpp)",
                             "sample": sample, "single_thread_value": n1 / sec1},
            "e2e": {"value": value, "unit": "entries/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


# ------------------------------------------------------------------------------ GPU arm

def run_ours(args):
    import torch
    import __graft_entry__
    from paper_2506_08781_gb300 import poslo, synth

    from paper_2506_08781_gb300 import shard

    rank, world, local = dist_env()
    device = local
    torch.cuda.set_device(device)
    if world > 1:
        import torch.distributed as dist
        # host-side bookkeeping (timing maxima) over gloo, the shard records over NCCL
        dist.init_process_group("cpu:gloo,cuda:nccl")
    __graft_entry__.build()
    # one verifier: every rank holds the same secret weight seed, so the shards' weighted
    # records combine into the weighted check of the whole log
    ctx = poslo.Context(device=device, verifier_seed=synth.verifier_seed(1000))
    first, depth = shard_plan(rank, world)
    km, msgs, subsets, _ = make_workload(rank=rank, world=world)
    Y, s, R = sign_workload(ctx, km, msgs, subsets, first_index=first, depth=depth)
    ds = struct.pack("<II", depth, 0) + km.root      # final disclosure: the root x_D[0] alone
    n = msgs.n
    exch = f"cuda:{device}"

    # device-resident inputs
    d_msgs = torch.from_numpy(msgs.data).cuda()
    d_offs = torch.from_numpy(msgs.offs.view(np.int64)).cuda()
    d_s = torch.from_numpy(s).cuda()
    d_R = torch.from_numpy(R).cuda()
    torch.cuda.synchronize()
    batch = ctx.make_batch(poslo.VARIANT_F, N2, Y, d_msgs, d_offs, d_s, d_R, ds, first_index=first)
    if args.msm_plan:
        c_fix, r_fix = (int(v) for v in args.msm_plan.split(","))
        ctx.msm_set_plan(n, c_fix, r_fix)
        plan_source = "fixed by --msm-plan"
    else:
        ctx.msm_autotune(n, 4)            # window and range length of the weighted MSM, timed on this GPU
        plan_source = "poslo_msm_autotune"
    msm_window, msm_range = ctx.msm_get_plan(n, 4)

    def step(b):
        """AVer + Distill of the log: this shard's weighted aggregate record, the exchange of the
        records (an all-gather of 216 bytes per rank), the combined check of the whole log on the
        device; only when the log is rejected, Distill of this shard and the gather of the
        shards' invalid lists.  One rank: the same calls without the exchange."""
        rec = ctx.aver_partial(b, poslo.AGG_WEIGHTED)
        recs = shard.all_gather_records(rec.to_bytes(), device=exch) if world > 1 else [rec]
        accepted, _ = ctx.combine_check(Y, recs)
        if accepted:
            return np.zeros(0, np.uint64)
        idx, _, _ = ctx.distill(b)
        return shard.gather_lists(idx, device=exch) if world > 1 else idx

    for _ in range(args.warmup):
        idx = step(batch)
    assert len(idx) == 0, "all-valid workload reported invalid entries"

    stream = torch.cuda.ExternalStream(ctx.stream)
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    if world > 1:
        torch.distributed.barrier()
    torch.cuda.synchronize()
    ctx.set_profiling(True)
    ctx.reset_kernel_times()
    launches0 = ctx.kernel_time("*")[1]
    with ClockSampler(device) as clk:
        ev0.record(stream)
        t0 = time.perf_counter()
        for _ in range(args.steps):
            step(batch)
        ev1.record(stream)
        torch.cuda.synchronize()
        wall = time.perf_counter() - t0
    ms = ev0.elapsed_time(ev1) / args.steps
    gpu_launches = ctx.kernel_time("*")[1] - launches0
    kernels = {}
    for name in ("seeds", "hash", "points", "table", "msm", "msm_sort", "msm_bucket", "msm_reduce", "msm_final",
                 "finalize", "tree", "bisect", "check"):
        tot, cnt = ctx.kernel_time(name)
        if cnt:
            kernels[name] = {"ms_per_launch": tot / cnt, "launches": cnt}
    ctx.set_profiling(False)
    ms = max_over_ranks(ms, world)
    value = job_throughput(n, world, ms)

    # unit AVer (the paper's equation) on the same resident inputs, for context
    for _ in range(2):
        ctx.aver(batch, poslo.AGG_UNIT)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(args.steps):
        ctx.aver(batch, poslo.AGG_UNIT)
    e1.record(stream)
    torch.cuda.synchronize()
    aver_ms = e0.elapsed_time(e1) / args.steps

    # the shard's own Distill on the same resident inputs (its launch sequence replayed from a
    # CUDA graph): the call a single-GPU user makes for AVer + Distill in one
    for _ in range(2):
        ctx.distill(batch)
    g0 = ctx.graph_stats()
    e0.record(stream)
    for _ in range(args.steps):
        idx_d, _, _ = ctx.distill(batch)
    e1.record(stream)
    torch.cuda.synchronize()
    g1 = ctx.graph_stats()
    assert len(idx_d) == 0
    distill_ms = e0.elapsed_time(e1) / args.steps
    distill_step = {"value": n / (distill_ms * 1e-3), "unit": "entries/s", "ms_per_step": distill_ms,
                    "replays": g1[1] - g0[1],
                    "call": "poslo_distill of the shard (weighted check window by window, then localisation "
                            "when it fails), launch sequence replayed from its CUDA graph"}

    tampered = None
    if not args.no_tampered and world == 1:
        tampered = bench_distill_tampered(ctx, msgs, Y, s, R, ds, steps=args.steps, warmup=max(2, args.warmup))

    multi = None
    replay = None
    if not args.no_multi and world == 1:
        multi = bench_multi(ctx, steps=max(2, args.steps // 5), warmup=2, cpu=not args.no_cpu_baseline)
        replay = bench_graph_replay(ctx)
    serving = None
    if not args.no_serving and world == 1:
        serving = bench_serving(lambda: poslo.Context(device=device))
    hash_bound = None
    if not args.no_hash_bound and world == 1:
        hash_bound = bench_hash_bound(device, steps=max(3, args.steps // 2), warmup=2)
    stream = None
    if not args.no_stream and world == 1:
        stream = bench_stream(device)
    small = None
    if not args.no_small and world == 1:
        small = bench_small_latency(device)

    # end to end through the C ABI from pinned host memory
    p_msgs = torch.from_numpy(msgs.data).pin_memory()
    p_offs = torch.from_numpy(msgs.offs.view(np.int64)).pin_memory()
    p_s = torch.from_numpy(s).pin_memory()
    p_R = torch.from_numpy(R).pin_memory()
    hbatch = ctx.make_batch(poslo.VARIANT_F, N2, Y, p_msgs, p_offs, p_s, p_R, ds, first_index=first)
    for _ in range(2):
        step(hbatch)
    t0 = time.perf_counter()
    for _ in range(args.steps):
        idx = step(hbatch)
    e2e_s = (time.perf_counter() - t0) / args.steps
    e2e_s = max_over_ranks(e2e_s * 1e3, world) * 1e-3
    h2d = msgs.data.nbytes + msgs.offs.nbytes + s.nbytes + R.nbytes + 32 + len(ds) + 216 * world
    d2h = 8 * len(idx) + 2 * 216 + 1 + 8

    # roofline of the dominant kernel
    peaks = probe_int_peaks(device)
    # the dominant kernel is the decoding: the largest share of kernel time in the ncu launch list
    # of this step (about half of the Distill step's own kernel time).  The stage timers cannot
    # pick it: they span each stream's interval, including the time a stage's blocks wait for
    # SMs held by the others.
    dom = "points" if "points" in kernels else None
    roof = None
    if dom in ("points", "check") and peaks:
        hi_cost = peaks["imad_lo_ops"] / peaks["imad_hi_ops"]
        work = n * (IMAD_LO_PER_DECODE + IMAD_HI_PER_DECODE * hi_cost)
        ach = work / (kernels[dom]["ms_per_launch"] * 1e-3) / 1e9
        pk = peaks["imad_lo_ops"] / 1e9
        roof = {"bound": "alu", "pipe": "IMAD", "kernel": dom, "achieved": ach, "peak": pk, "unit": "Gop/s",
                "frac": ach / pk, "traffic": POINTS_DRAM_BYTES_2P20 * n / (1 << 20),
                "traffic_source": "ncu dram__bytes_read.sum + dram__bytes_write.sum of one k_points launch "
                                  "at 2^20 entries",
                "peak_source": "probed mad.lo.u32 issue rate on this GPU (probe/peaks.cu)",
                "work": f"{IMAD_LO_PER_DECODE:,} mad.lo + {IMAD_HI_PER_DECODE:,} mad.hi per R_t decode and its "
                        f"unit-sum addition; mad.hi counted as {hi_cost:.2f} mad.lo issue slots (probed rate ratio)",
                "timing": "k_points duration on its own stream during the timed steps (it shares the GPU with "
                          "the hashing and the counting sort, so this understates the kernel alone)"}
    elif dom == "hash" and peaks:
        work = compressions(msgs) * ALU_PER_COMPRESSION
        ach = work / (kernels[dom]["ms_per_launch"] * 1e-3) / 1e9
        pk = peaks["lop3_ops"] / 1e9
        roof = {"bound": "alu", "pipe": "ALU", "kernel": dom, "achieved": ach, "peak": pk, "unit": "Gop/s",
                "frac": ach / pk, "traffic": None, "peak_source": "probed lop3 issue rate on this GPU",
                "work": "1,384 ALU ops per SHA-256 compression"}
    clocks = clk.summary()

    if rank == 0:
        cpu = None
        if world == 1 and not args.no_cpu_baseline:
            cpu = cpu_oracle_baseline(per_core=args.cpu_per_core)
        line = {
            "metric": "verified log entries/sec at 1 GB300 (AVer+Distill)",
            "value": value, "unit": "entries/s", "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": ms, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "u32", "data": "synthetic (seeded SplitMix64 messages; keys and signatures made by "
                                    "poslo_keygen_f/poslo_sign_f)",
            "config": {"workload": WORKLOAD, "entries_per_gpu": n, "log_entries": n * world,
                       "message_bytes": int(msgs.data.nbytes),
                       "l2": "inputs (215 MB) larger than the 129 MB L2; no flush", "parallelism": f"dp{world}",
                       "msm_window": msm_window, "msm_range_log2": msm_range,
                       "msm_plan_source": plan_source},
            "clocks": clocks,
            "gpu_launches": gpu_launches,
            "kernels": kernels,
            "aver_unit": {"value": n / (aver_ms * 1e-3), "ms_per_step": aver_ms},
            "distill_step": distill_step,
            "e2e": {"value": world * n / e2e_s, "unit": "entries/s", "h2d_bytes_per_step": h2d,
                    "d2h_bytes_per_step": d2h},
            "roofline": roof,
            "distill_tampered": tampered,
            "multi_device": multi,
            "small_batch_graph_replay": replay,
            "hash_bound_poslo_c": hash_bound,
            "out_of_core": stream,
            "latency_1024_entries": small,
            "serving": serving,
            "int_peaks": peaks,
            "cpu_baseline": cpu,
            "wall_s_timed": wall,
        }
        print(json.dumps(line), flush=True)
    ctx.close()
    if world > 1:
        torch.distributed.destroy_process_group()


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--cpu-per-core", type=int, default=2048)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-multi", action="store_true", help="skip the 4,096-device measurement")
    ap.add_argument("--no-tampered", action="store_true", help="skip the Distill measurement with 1,049 flipped entries")
    ap.add_argument("--no-serving", action="store_true", help="skip the serving-loop measurement")
    ap.add_argument("--no-hash-bound", action="store_true", help="skip the POSLO-C / POSLO+ hash-bound measurement")
    ap.add_argument("--no-stream", action="store_true", help="skip the out-of-core streaming measurement")
    ap.add_argument("--no-small", action="store_true", help="skip the 1,024-entry latency measurement")
    ap.add_argument("--msm-plan", default=None,
                    help="C,R: fix the Distill MSM plan (window C, ranges of 2^R entries) instead of autotuning it "
                         "(autotuner timings taken under a profiler are distorted)")
    args = ap.parse_args()
    if args.impl == "reference":
        run_reference(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()

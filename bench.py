"""Benchmark: epsilon-cost-sharded VFilter/VFunc construction and 3-probe
queries on GB300, through the C ABI (libvfunc.so).

Default workload (one step = the whole hot path once): build a VFilter over
n = 10^8 distinct uniform 64-bit keys with b = 8 fingerprint bits, then query
the 10^8 members and 10^8 disjoint non-members (false-positive rate ~ 2^-8).
`value` is the construction cost in ns per key (device-resident inputs,
CUDA events on the launching stream); the query rate is reported next to it.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl gpu|reference]
                    [--workload c2|c1|c3|c4|c5|mwhc|fuse4] [--no-extras] [--no-cpu-baseline]

The default run also carries the rest of the metric as sub-objects, each
measured after the headline: "c4" (4096 uneven structures, one batched
graph-captured build against one vf_build per structure), "c5_scale" (one
VFilter of 5e9 keys built by shard group, and its queries against the HBM
random-sector roofline) and "c5_serving" (Poisson builds and queries under a
memory budget, p50/p99 latency). "cpu_baseline" is the oracle on every host
core over the whole workload; "cpu_baseline_1core" one core on a sample.

--impl reference times the plain CPU oracle (the paper's algorithm; shards
solved on every host core) on a bounded sample of the same workload. Under
torchrun every rank builds its own replica (the structure is single-GPU;
replicas only).
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

METRIC = "build ns/key & Gqueries/s on 1 GB300 vs plain GPU path; p50/p99 request latency"
PEAKS_PATH = os.path.join(ROOT, "MEASURED_PEAKS.json")
L2_BYTES = 129e6
FALLBACK_HBM = 6800.0

WORKLOADS = {
    # name: (kind, b, n, key kind, description[, parameter overrides])
    "c2": ("filter", 8, 100_000_000, "u64",
           "VFilter n=1e8 uniform 64-bit keys, b=8, fuse graphs (eps-cost sharding h=3); "
           "query 1e8 members + 1e8 disjoint keys"),
    "c1": ("func", 8, 1 << 20, "u64",
           "VFunc n=2^20 uniform 64-bit keys, 8-bit values, unsharded fuse graph; "
           "query 2^20 members + 2^20 disjoint keys"),
    "c4": ("mixed", 0, 4096, "u64",
           "4096 independent VFunc/VFilter structures, sizes log-uniform in 1e3..1e6 uniform 64-bit keys, "
           "b in {1,8,16,32}, kind 50/50; batched persistent graph-captured build vs one vf_build per structure"),
    "c5": ("serve", 8, 5_000_000_000, "u64",
           "serving: Poisson arrivals of builds (log-uniform 1e4..1e8 keys, b in {8,16}) and query batches "
           "(log-uniform 1e3..1e7 keys, half members) under a device-memory budget, plus one VFilter of 5e9 "
           "uniform 64-bit keys (b=8) generated on the device in chunks and built by shard group"),
    "c3": ("func", 16, 10_000_000, "bytes",
           "VFunc n=1e7 byte strings (length 8..64), 16-bit values, LGE regime shards; "
           "query 1e7 members + 1e7 disjoint strings", {"mode": "lge"}),
    "fuse4": ("filter", 8, 100_000_000, "u64",
              "VFilter n=1e8 uniform 64-bit keys, b=8, 4-uniform fuse graphs (one more probe per query, "
              "c = 1.075); query 1e8 members + 1e8 disjoint keys", {"mode": "fuse", "arity": 4}),
    "mwhc": ("filter", 8, 100_000_000, "u64",
             "VFilter n=1e8 uniform 64-bit keys, b=8, MWHC construction (3-partite random 3-hypergraphs, "
             "c=1.23, eps=0.01, eta=1e-3: 64 shards); query 1e8 members + 1e8 disjoint keys",
             {"mode": "mwhc", "eps": 0.01, "eta": 1e-3}),
}

# Algorithmic DRAM bytes per unit (key, edge or query) of each phase: the
# method's own traffic with shard state off chip, every random access one
# 32-byte sector and every random update a read-modify-write of one (64 B).
# Streams: the key is read by the histogram and again by the scatter pass (hash
# recomputed), the bucketed (local signature, value) pair is written once and
# read once, the data array written once (c cells of b bits per key).
# Random updates: incidence 3 (degree/edge-index words of the three vertices),
# peel 3 (removal from the three vertices), assignment 3 + 1 (the other two
# vertices' values read, the peeled cell written, its word updated).
def _vb(b, kind):
    return 0.0 if kind == "filter" else (1.0 if b <= 8 else 2.0 if b <= 16 else 4.0)


ALGO_BYTES = {
    "hash_hist": lambda b, kind: 8.0,
    "scatter": lambda b, kind: 8.0 + _vb(b, kind) + 8.0 + _vb(b, kind),
    "incidence": lambda b, kind: 8.0 + 3 * 64.0,
    "peel": lambda b, kind: 3 * 64.0,
    "assign": lambda b, kind: _vb(b, kind) + 4 * 64.0 + 1.105 * b / 8,
    "lge": lambda b, kind: 8.0 + _vb(b, kind) + 1.12 * b / 8,   # shard state on chip
    "query": lambda b, kind, k=3: 8.0 + k * 32.0 + (1.0 if kind == "filter" else max(1.0, b / 8)),
}

# The same phases counted by what the kernels here move (the segment sort's
# counting and scatter passes, the asynchronous peel's 16-byte records and queue items, the polled
# value words of the dataflow assignment): a second figure, for comparison.
def _seg_sort_bytes(kind):
    return 24.0 + (0 if kind == "filter" else 8.0)


KERNEL_BYTES = {
    "hash_hist": lambda b, kind: 8.0,
    "scatter": lambda b, kind: 8.0 + 8.0 + (0 if kind == "filter" else 1.0 + 4.0),
    "incidence": lambda b, kind: 8.0 + 3 * 32.0,
    "peel": lambda b, kind: 8 + (0 if kind == "filter" else 4) + 2 * 32 + 16 + 16,
    "assign": lambda b, kind: 16 + 2 * 32 + 32 + 32,
    "lge": lambda b, kind: 8.0 + 8.0 * 3,
    "query": lambda b, kind, k=3: 8.0 + k * 32.0 + 1.0,
}


def reduce_max(vals, dist, device):
    """Element-wise maximum over ranks: the slowest replica sets the job's time."""
    vals = [float(v) for v in vals]
    if dist is None:
        return vals
    import torch

    t = torch.tensor(vals, dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return t.tolist()


def job_rates(b_ms, q_ms, n, world):
    """Whole-job rates of `world` replicas that each built n keys in b_ms and
    queried 2n keys in q_ms (max-over-ranks times): build ns per key over all
    world*n keys, and Gqueries/s over all 2*n*world queries."""
    return b_ms * 1e6 / (n * world), 2 * n * world / (q_ms * 1e-3) / 1e9


def apply_overrides(p, workload, mod):
    """Parameter overrides of a workload (mode by name, eps, eta) on a params struct."""
    ov = WORKLOADS[workload][5] if len(WORKLOADS[workload]) > 5 else {}
    for k, v in ov.items():
        if k == "mode":
            p.mode = {"lge": mod.MODE_LGE, "fuse": mod.MODE_FUSE, "mwhc": mod.MODE_MWHC}[v]
        else:
            setattr(p, k, v)


def peaks():
    try:
        with open(PEAKS_PATH) as f:
            p = json.load(f)
        return float(p["hbm_gbs"]), "measured"
    except Exception:
        return FALLBACK_HBM, "fallback"


class Clocks:
    """nvidia-smi samples during the timed region."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.rows = []
        self.proc = None
        self.thread = None

    def start(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={self.index}", f"--query-gpu={self.Q}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
        except Exception:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            parts = [x.strip() for x in line.split(",")]
            if len(parts) >= 9:
                self.rows.append(parts)

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        self.thread.join(timeout=2)
        sm = [float(r[1]) for r in self.rows if r[1].replace(".", "").isdigit()]
        mx = [float(r[2]) for r in self.rows if r[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in self.rows for i in range(4) if r[5 + i].lower() == "active"})
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": reasons, "samples": len(self.rows)}


def make_inputs(workload: str, seed: int, n_override: int = 0):
    from paper_2503_18397_gb300 import synth

    kind, b, n, kk = WORKLOADS[workload][:4]
    n = n_override or n
    if kk == "u64":
        keys = synth.u64_keys(0, n, seed)
        other = synth.u64_keys(n, n, seed)
        offs = ooffs = None
    else:
        keys, offs = synth.byte_strings(0, n, seed)
        other, ooffs = synth.byte_strings(n, n, seed)
    vals = synth.values(n, b, seed) if kind == "func" else None
    return kind, b, n, keys, offs, vals, other, ooffs


def to_dev(a, torch, pin=False):
    if a is None:
        return None
    if a.dtype == np.uint64:
        t = torch.from_numpy(a.view(np.int64))
    elif a.dtype == np.uint16:
        t = torch.from_numpy(a.view(np.int16))
    elif a.dtype == np.uint32:
        t = torch.from_numpy(a.view(np.int32))
    else:
        t = torch.from_numpy(a)
    if pin:
        return t.pin_memory()
    return t.cuda()


# ----------------------------------------------------------------------- GPU arm

def run_gpu(args):
    import torch

    import paper_2503_18397_gb300 as vf
    from paper_2503_18397_gb300 import build as vbuild

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    dist = None
    if world > 1:
        import torch.distributed as dist

        torch.cuda.set_device(local)
        dist.init_process_group("nccl")
    else:
        torch.cuda.set_device(0)
    if rank == 0 or world > 1:
        vbuild.build()
    vf.lib()

    kind, b, n, keys, offs, vals, other, ooffs = make_inputs(args.workload, 0x5EED + rank, args.n)
    p = vf.vf_params_default(kind=vf.FILTER if kind == "filter" else vf.FUNC, b=b,
                             key_kind=vf.KEYS_BYTES if offs is not None else vf.KEYS_U64, seed=1 + rank)
    apply_overrides(p, args.workload, vf)
    kd, vd, od, xd, xo = (to_dev(a, torch) for a in (keys, vals, offs, other, ooffs))
    stream = torch.cuda.current_stream()

    step_no = [0]

    def step(timing):
        # every step builds with its own seed, so retries (a ~5% event at the
        # paper's eta) show up in the average as often as they occur
        p.seed = 1 + rank + 1000 * step_no[0]
        step_no[0] += 1
        e0, e1, e2 = (torch.cuda.Event(enable_timing=True) for _ in range(3))
        e0.record(stream)
        s = vf.vf_build(kd, vd, offsets=od, params=p, stream=stream)
        e1.record(stream)
        o1 = s.query(kd, offsets=od, stream=stream)
        o2 = s.query(xd, offsets=xo, stream=stream)
        e2.record(stream)
        return s, e0, e1, e2, o1, o2

    for _ in range(args.warmup):
        s, *_rest = step(False)
        torch.cuda.synchronize()
        info = s.info
        s.free()
    # correctness of the last warm-up step (outside the timed region)
    s, e0, e1, e2, o1, o2 = step(False)
    torch.cuda.synchronize()
    info = s.info
    if kind == "func":
        ok = bool((o1.view(torch.int16 if b > 8 else torch.uint8) ==
                   to_dev(vals, torch).view(torch.int16 if b > 8 else torch.uint8)).all().item())
    else:
        ok = bool(o1.bool().all().item())
    fpr = float(o2.float().mean().item()) if kind == "filter" else None
    s.free()

    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    clocks = Clocks(local)
    clocks.start()
    vf.vf_timing_read()
    vf.vf_timing_enable(True)
    # inputs smaller than L2 (129 MB): a 256 MB write before every timed step
    # evicts them, outside the step's events
    in_bytes = keys.nbytes + (offs.nbytes if offs is not None else 0) + (vals.nbytes if vals is not None else 0) + \
        other.nbytes + (ooffs.nbytes if ooffs is not None else 0)
    l2_flush = None if in_bytes > L2_BYTES else torch.empty(256 << 20, dtype=torch.uint8, device=kd.device)
    build_ms, query_ms, step_ms = [], [], []
    t_start = torch.cuda.Event(enable_timing=True)
    t_end = torch.cuda.Event(enable_timing=True)
    t_start.record(stream)
    timed_seeds = []
    for _ in range(args.steps):
        if l2_flush is not None:
            l2_flush.fill_(step_no[0] & 0xFF)
        timed_seeds.append(1 + rank + 1000 * step_no[0])
        s, e0, e1, e2, o1, o2 = step(True)
        torch.cuda.synchronize()
        build_ms.append(e0.elapsed_time(e1))
        query_ms.append(e1.elapsed_time(e2))
        step_ms.append(e0.elapsed_time(e2))
        s.free()
    t_end.record(stream)
    torch.cuda.synchronize()
    vf.vf_timing_enable(False)
    phases = vf.vf_timing_read()
    clk = clocks.stop()
    total_ms = t_start.elapsed_time(t_end)
    total_ms, b_ms, q_ms = reduce_max([total_ms, statistics.mean(build_ms), statistics.mean(query_ms)], dist, "cuda")

    # end to end: the same build and queries from pinned host buffers, host output
    kh, vh, oh, xh, xoh = (None if a is None else to_dev(a, torch, pin=True) for a in (keys, vals, offs, other, ooffs))
    outh = torch.empty(n, dtype=torch.uint8 if (kind == "filter" or b <= 8) else torch.int16).pin_memory()
    # untimed warm-up of the host-buffer path: the first transfers from newly
    # pinned buffers and the first pipelined queries of a process run slower
    # (up to ~60 ms a call measured) than every later one
    for w in range(args.warmup):
        p.seed = 1 + rank + 1000 * (step_no[0] + w)
        s = vf.vf_build(kh, vh, offsets=oh, params=p)
        vf.vf_query(s, kh, offsets=oh, out=outh)
        vf.vf_query(s, xh, offsets=xoh, out=outh)
        s.free()
    e2e_b, e2e_q, e2e_calls = [], [], []
    # one build per timed step with that step's seed, so retries (a property
    # of the seed) weigh the same as in the device-timed steps
    for seed in timed_seeds:
        p.seed = seed
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        s = vf.vf_build(kh, vh, offsets=oh, params=p)
        t1 = time.perf_counter()
        vf.vf_query(s, kh, offsets=oh, out=outh)
        tq = time.perf_counter()
        vf.vf_query(s, xh, offsets=xoh, out=outh)
        t2 = time.perf_counter()
        e2e_b.append((t1 - t0) * 1e3)
        e2e_q.append((t2 - t1) * 1e3)
        e2e_calls.extend([(tq - t1) * 1e3, (t2 - tq) * 1e3])
        s.free()
    key_bytes = keys.nbytes + (offs.nbytes if offs is not None else 0)
    other_bytes = other.nbytes + (ooffs.nbytes if ooffs is not None else 0)
    h2d = key_bytes + (vals.nbytes if vals is not None else 0) + key_bytes + other_bytes
    d2h = 2 * n * outh.element_size()
    e2e_b_ms, e2e_q_ms = reduce_max([statistics.mean(e2e_b), statistics.mean(e2e_q)], dist, "cuda")

    # the host link bounds the end-to-end queries: every key crosses it once
    h2d_gbs = host_to_device_gbs(torch)
    hbm, peak_kind = peaks()
    per_phase, dom, roof = phase_table(phases, n, args.steps, b, kind, hbm, peak_kind, args.workload,
                                       info.regime == vf.REGIME_FUSE, int(info.k))
    launches = sum(v[1] for v in phases.values())
    build_ns, qgps = job_rates(b_ms, q_ms, n, world)
    e2e_ns, e2e_qgps = job_rates(e2e_b_ms, e2e_q_ms, n, world)
    out = {
        "metric": METRIC,
        "value": round(build_ns, 4),
        "unit": "ns/key",
        "n_gpus": world,
        "steps": args.steps,
        "warmup": args.warmup,
        "ms_per_step": round(total_ms / args.steps, 3),
        "higher_is_better": False,
        "scaling": "weak",
        "vs_baseline": None,
        "dtype": "u64",
        "data": "synthetic",
        "config": {"workload": WORKLOADS[args.workload][4] if not args.n else f"{args.workload} with n={n}", "n": n, "b": b, "kind": kind,
                   "l2": "inputs larger than L2 (no flush)" if l2_flush is None else
                   "L2 flushed before every step (256 MB write, outside the step's events)",
                   "parallelism": "replicas" if world > 1 else "single GPU",
                   "shards": int(info.shards), "cells_per_shard": int(info.cells), "lg_seg": int(info.lg_seg),
                   "c": info.c, "space_overhead": round(info.total_cells / n - 1, 4)},
        "build_ms": round(b_ms, 3),
        "query": {"gqps": round(qgps, 3), "ms_per_2n": round(q_ms, 3)},
        "e2e": {"value": round(e2e_ns, 4), "unit": "ns/key", "query_gqps": round(e2e_qgps, 3),
                "h2d_bytes_per_step": int(h2d), "d2h_bytes_per_step": int(d2h),
                "query_link_bound": {"h2d_gbs": round(h2d_gbs, 1),
                                     "gqps": round(h2d_gbs / (key_bytes / n), 3),
                                     "frac": round(e2e_qgps / (h2d_gbs / (key_bytes / n)), 4),
                                     "what": "pinned host-to-device copy rate measured in this run, divided by "
                                             "the bytes of one key: queries from host memory cannot go faster"},
                "query_call_ms": {"min": round(min(e2e_calls), 3), "median": round(statistics.median(e2e_calls), 3),
                                  "max": round(max(e2e_calls), 3), "calls": len(e2e_calls)},
                "build_call_ms": {"min": round(min(e2e_b), 3), "median": round(statistics.median(e2e_b), 3),
                                  "max": round(max(e2e_b), 3)}},
        "gpu_launches": int(launches),
        "phases": per_phase,
        "roofline": roof,
        "clocks": clk,
        "check": {"members_ok": ok, "fpr": fpr, "retries": int(info.retries)},
    }
    # the query's bound: its three random sectors come from L2 while the data
    # array fits there (the key stream and the output from HBM), else from HBM
    qps = 2 * n * world / (q_ms * 1e-3)
    q_hbm = random_sector_roofline(qps / world, b, kind, hbm, peak_kind, int(info.k))
    out["query"]["roofline"] = {"hbm": q_hbm}
    out["build_roofline"] = build_roofline(b_ms, n, b, kind, float(info.c), hbm, peak_kind,
                                           info.regime != vf.REGIME_LGE,
                                           max(1, phases.get("hash_hist", (0, 0))[1]) / args.steps)
    out["query"]["roofline"]["sectors"] = sector_roofline(
        qps / world, int(info.data_bytes), "l2" if info.data_bytes <= L2_BYTES else "hbm", int(info.k))
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        # the oracle on every host core over the whole workload, and on one
        # core over a bounded sample
        full = args.workload in ("c1", "c2", "mwhc") and not args.n
        out["cpu_baseline"] = cpu_baseline(args.workload, quick=True, threads=host_threads(), full=full)
        out["cpu_baseline_1core"] = cpu_baseline(args.workload, quick=True, threads=1)
    if rank == 0 and world == 1 and args.workload == "c2" and not args.n and not args.no_extras:
        # the other parts of the metric, each with its own warm-up and clocks:
        # batched vs plain per-structure builds, the 5e9-key build and its
        # HBM-bound queries, and serving latency percentiles
        del kd, vd, od, xd, xo, kh, vh, oh, xh, xoh, outh, l2_flush
        torch.cuda.empty_cache()
        out["c4"] = measure_c4(3, 3)
        out["c5_scale"] = measure_c5_scale(5_000_000_000, hbm, peak_kind)
        out["c5_serving"] = measure_c5_serving()
    if rank == 0:
        print(json.dumps(out), flush=True)
    if dist:
        dist.barrier()
        dist.destroy_process_group()


# Build attempts run hash+histogram once each; every attempt passes the keys
# through scatter, incidence and peel (or the LGE solver); a successful one also
# through assignment; every step queries 2n keys.
def _algo(ph, b, kind, k):
    """Algorithmic bytes per unit of a phase; a k-uniform graph has k vertex
    updates per edge in incidence and peel, and k - 1 other values to read in
    the assignment (the models above are written for k = 3)."""
    if ph == "query":
        return ALGO_BYTES[ph](b, kind, k)
    extra = (k - 3) * 64.0 if ph in ("incidence", "peel", "assign") else 0.0
    return ALGO_BYTES[ph](b, kind) + extra


def phase_table(phases, n, steps, b, kind, hbm, peak_kind, workload, fuse, k=3):
    attempts = max(1, phases.get("hash_hist", (0, 0))[1])
    units = {"hash_hist": n * attempts, "scatter": n * attempts, "incidence": n * attempts,
             "peel": n * attempts, "lge": n * attempts, "assign": n * steps, "query": 2 * n * steps}
    passes = {"hash_hist": attempts, "scatter": attempts, "incidence": attempts, "peel": attempts,
              "lge": attempts, "assign": steps, "query": 2 * steps}
    total = max(sum(v[0] for v in phases.values()), 1e-9)
    per_phase = {}
    for ph, (ms, cnt) in phases.items():
        if cnt == 0:
            continue
        kb = KERNEL_BYTES[ph](b, kind)
        if ph == "scatter" and fuse:  # segment sort: signatures read twice, written once (values once more)
            kb += _seg_sort_bytes(kind)
        if ph == "incidence" and fuse:  # owner-computes: three signature reads, one vertex-word store
            kb = 3 * 8.0 + 4.0 * 1.105
        per_phase[ph] = {"ms_total": round(ms, 3), "kernels": cnt, "passes": passes[ph],
                         "ms_per_pass": round(ms / passes[ph], 4), "share": round(ms / total, 4),
                         "achieved_gbs": round(_algo(ph, b, kind, k) * units[ph] / (ms * 1e-3) / 1e9, 2),
                         "kernel_model_gbs": round(kb * units[ph] / (ms * 1e-3) / 1e9, 2)}
    dom = max(per_phase, key=lambda k: per_phase[k]["share"]) if per_phase else None
    roof = None
    if dom:
        d = per_phase[dom]
        kb = KERNEL_BYTES[dom](b, kind) + (_seg_sort_bytes(kind) if dom == "scatter" and fuse else 0)
        if dom == "incidence" and fuse:
            kb = 3 * 8.0 + 4.0 * 1.105
        roof = {"bound": "hbm", "kernel": dom, "achieved": d["achieved_gbs"], "peak": hbm, "unit": "GB/s",
                "frac": round(d["achieved_gbs"] / hbm, 4), "traffic": TRAFFIC.get((workload, dom)),
                "peak_source": f"{peak_kind} hbm_gbs", "algorithmic_bytes_per_unit": _algo(dom, b, kind, k),
                "kernel_model": {"bytes_per_unit": kb, "achieved": d["kernel_model_gbs"],
                                 "frac": round(d["kernel_model_gbs"] / hbm, 4)}}
    return per_phase, dom, roof


# Per-launch DRAM traffic (bytes) from ncu captures of the same kernels, scaled
# from the captured case by units processed; absent until a capture of the
# current kernel exists (profiles/ holds the summaries).
TRAFFIC = {("c2", "peel"): round(1120.07e6 / 2e7 * 1e8),   # k_flow_peel, one launch per attempt at 1e8
           ("c2", "query"): round(189.42e6 / 2e7 * 1e8),  # k_query, one launch per 1e8 queries
           ("c3", "lge"): round(788.86e6 + 806.24e6)}     # k_lge medium configuration, full-size capture


# ---------------------------------------------------------------- reference arm

def oracle_sample(workload: str, quick: bool, threads: int = 1):
    """Bounded sample of the workload for the oracle: a few seconds of host
    work per build (more keys, hence several shards, for several threads)."""
    kind, b, n, kk = WORKLOADS[workload][:4]
    if len(WORKLOADS[workload]) > 5 and WORKLOADS[workload][5].get("mode") == "lge":
        # plain Gaussian elimination of every 2-core is cubic: a few shards only
        return kind, b, min(n, 40_000 * threads), kk
    ns = min(n, 25_000_000 if threads > 1 else 4_000_000 if quick else 8_000_000)
    return kind, b, ns, kk


def host_threads() -> int:
    try:
        return max(1, len(os.sched_getaffinity(0)))
    except Exception:
        return max(1, os.cpu_count() or 1)


def cpu_baseline(workload: str, quick: bool = True, threads: int = 1, full: bool = False):
    """The oracle timed on the host: `threads` threads (shards solved side by
    side, queries split), on the whole workload (`full`) or a bounded sample."""
    from oracle import oracle as O
    from paper_2503_18397_gb300 import synth

    kind, b, ns, kk = oracle_sample(workload, quick, threads)
    if full:
        ns = WORKLOADS[workload][2]
    gseed = 0x5EED if full else 3
    if kk == "u64":
        keys, offs = synth.u64_keys(0, ns, gseed), None
        other, ooffs = synth.u64_keys(ns, ns, gseed), None
    else:
        keys, offs = synth.byte_strings(0, ns, gseed)
        other, ooffs = synth.byte_strings(ns, ns, gseed)
    vals = synth.values(ns, b, gseed) if kind == "func" else None
    p = O.default_params(kind=O.FILTER if kind == "filter" else O.FUNC, b=b,
                         key_kind=O.KEYS_BYTES if offs is not None else O.KEYS_U64, seed=1, threads=threads)
    apply_overrides(p, workload, O)
    t0 = time.perf_counter()
    st, info, data = O.build(p, keys, vals, offsets=offs)
    t1 = time.perf_counter()
    O.query(info, data, keys, offsets=offs, threads=threads)
    O.query(info, data, other, offsets=ooffs, threads=threads)
    t2 = time.perf_counter()
    what = "the whole workload" if full else f"a sample of {ns} keys"
    return {"value": round((t1 - t0) * 1e9 / ns, 3), "unit": "ns/key", "cores": threads, "kind": "oracle",
            "query_gqps": round(2 * ns / (t2 - t1) / 1e9, 6), "retries": int(info.retries),
            "sample": f"oracle build of {what} ({ns} keys, {kind}, b={b}, same parameters, seed 1, "
                      f"{info.retries} retries) + query of {2 * ns} keys (members + disjoint), "
                      f"{threads} thread{'s' if threads > 1 else ''} (shards solved side by side)"}


def run_reference(args):
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    from oracle import oracle as O

    O.build_oracle()
    threads = host_threads()
    kind, b, ns, kk = oracle_sample(args.workload, quick=True, threads=threads)
    for _ in range(args.warmup if args.warmup < 1 else 1):
        cpu_baseline(args.workload, quick=True, threads=threads)
    vals = []
    t0 = time.perf_counter()
    for _ in range(args.steps):
        vals.append(cpu_baseline(args.workload, quick=True, threads=threads))
    t1 = time.perf_counter()
    v = statistics.mean(x["value"] for x in vals)
    out = {"impl": "reference", "metric": METRIC, "value": round(v, 3), "unit": "ns/key", "n_gpus": world,
           "steps": args.steps, "warmup": args.warmup, "ms_per_step": round((t1 - t0) * 1e3 / args.steps, 3),
           "higher_is_better": False, "scaling": "weak", "vs_baseline": None, "dtype": "u64",
           "data": "synthetic", "config": {"workload": WORKLOADS[args.workload][4], "n": ns, "b": b, "kind": kind},
           "cpu_baseline": {"value": round(v, 3), "unit": "ns/key", "cores": threads, "kind": "oracle",
                            "sample": vals[0]["sample"]},
           "e2e": {"value": round(v, 3), "unit": "ns/key", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
           "query_gqps": statistics.mean(x["query_gqps"] for x in vals)}
    print(json.dumps(out), flush=True)


def measure_c4(steps: int, warmup: int, count: int = 4096) -> dict:
    """Batched build of `count` uneven structures (one persistent, graph-captured
    solver launch, autotuned options) against the plain per-structure path (one
    vf_build per structure, same seeds and options) on the same GPU."""
    import torch

    import paper_2503_18397_gb300 as vf
    from paper_2503_18397_gb300 import synth

    rng = np.random.default_rng(0xC4)
    sizes = synth.log_uniform_sizes(count, 1e3, 1e6, 0xC4)
    kinds = rng.integers(0, 2, size=count)
    bs = rng.choice([1, 8, 16, 32], size=count)
    items, start = [], 0
    for i in range(count):
        n = int(sizes[i])
        keys = synth.u64_keys_torch(start, n, 0xC4)
        start += n
        vals = synth.values_torch(n, int(bs[i]), 0xC4 + i) if kinds[i] == 0 else None
        items.append((keys, vals, int(kinds[i]), int(bs[i]), 1000 + i))
    total = int(sizes.sum())
    stream = torch.cuda.current_stream()
    t0 = time.perf_counter()
    best, sample_ms = vf.vf_tune_batch(items)
    tune_s = time.perf_counter() - t0
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(2)]
    for _ in range(warmup):
        for s_ in vf.vf_build_batch(items, opts=best):
            s_.free()
    torch.cuda.synchronize()
    clocks = Clocks(torch.cuda.current_device())
    clocks.start()
    vf.vf_timing_read()
    vf.vf_timing_enable(True)
    ms = []
    last = None
    for _ in range(steps):
        ev[0].record(stream)
        structs = vf.vf_build_batch(items, opts=best, stream=stream)
        ev[1].record(stream)
        torch.cuda.synchronize()
        ms.append(ev[0].elapsed_time(ev[1]))
        if last is not None:
            for s_ in last:
                s_.free()
        last = structs
    vf.vf_timing_enable(False)
    phases = vf.vf_timing_read()
    # members of a few structures decode exactly
    ok = True
    for i in range(count - 8, count):
        out = last[i].query(items[i][0])
        if items[i][2] == 0:
            dt = torch.int32 if bs[i] == 32 else torch.int16 if bs[i] > 8 else torch.uint8
            ok &= bool((out.view(dt) == items[i][1].view(dt)).all().item())
        else:
            ok &= bool(out.bool().all().item())
    for s_ in last:
        s_.free()
    # plain per-structure path: one vf_build per structure, same seeds and options
    torch.cuda.synchronize()
    plain = []
    for _ in range(2):
        ev[0].record(stream)
        for (k, v, kind, b, seed) in items:
            p = vf.vf_params_default(kind=kind, b=b, seed=seed, lge_threshold=best.lge_threshold,
                                     lge_target=best.lge_target)
            vf.vf_build(k, v, params=p, stream=stream).free()
        ev[1].record(stream)
        torch.cuda.synchronize()
        plain.append(ev[0].elapsed_time(ev[1]))
    clk = clocks.stop()
    plain_ms = plain[-1]  # the first pass is its warm-up
    b_ms = statistics.mean(ms)
    total_ms = sum(v[0] for v in phases.values())
    del items
    torch.cuda.empty_cache()
    return {
        "workload": WORKLOADS["c4"][4], "structures": count, "total_keys": total,
        "value": round(b_ms * 1e6 / total, 4), "unit": "ns/key", "ms_per_batch": round(b_ms, 3),
        "steps": steps, "warmup": warmup, "tuned": best.as_dict(),
        "plain_path": {"ms": round(plain_ms, 3), "ns_per_key": round(plain_ms * 1e6 / total, 4),
                       "speedup_batched": round(plain_ms / b_ms, 3),
                       "what": "one vf_build per structure, same seeds and options, after one untimed pass"},
        "tuner": {"seconds": round(tune_s, 3), "sample_ms": sample_ms},
        "phases": {k: {"ms": round(v[0], 3), "launches": v[1], "share": round(v[0] / max(total_ms, 1e-9), 4)}
                   for k, v in phases.items() if v[1]},
        "gpu_launches": int(sum(v[1] for v in phases.values())),
        "clocks": clk, "check": {"members_ok": ok},
    }


def build_roofline(build_ms: float, n: int, b: int, kind: str, c: float, hbm: float, peak_kind: str,
                   peeled: bool, attempts: float) -> dict:
    """The whole build against two algorithmic HBM models: streams only (the key
    read twice, the value once, the bucketed local signature and value written
    and read once, the data array written: shard state on chip), and streams
    plus the random 32-byte sector read-modify-writes of a peeled shard whose
    state is in HBM (incidence 3, peel 3, assignment 3 + 1, 64 B each).
    Retries count against the build (attempts per build given)."""
    vb = _vb(b, kind)
    stream = 16.0 + vb + 2 * (8.0 + vb) + c * b / 8
    models = {"streaming": stream}
    if peeled:
        models["streaming_plus_random_sectors"] = stream + 10 * 64.0
    out = {"attempts_per_build": round(attempts, 3), "unit": "GB/s", "peak": hbm,
           "peak_source": f"{peak_kind} hbm_gbs"}
    for name, bpk in models.items():
        bound_ns = bpk / hbm  # bytes per key / (GB/s) = ns per key
        achieved = bpk * n / (build_ms * 1e-3) / 1e9
        out[name] = {"bytes_per_key": round(bpk, 2), "bound_ns_per_key": round(bound_ns, 5),
                     "achieved": round(achieved, 2), "frac": round(achieved / hbm, 4)}
    return out


def random_sector_roofline(qps: float, b: int, kind: str, hbm: float, peak_kind: str, k: int = 3) -> dict:
    """A query against a data array larger than L2: k random 32-byte sectors
    from HBM per key (k = 3, or 4 for 4-uniform fuse graphs), plus its 8-byte
    key and its output."""
    per_q = ALGO_BYTES["query"](b, kind, k)
    sectors = k * qps
    return {"bound": "hbm", "unit": "GB/s", "achieved": round(per_q * qps / 1e9, 2), "peak": hbm,
            "frac": round(per_q * qps / 1e9 / hbm, 4), "peak_source": f"{peak_kind} hbm_gbs",
            "sectors_per_s": round(sectors / 1e9, 3), "sector_peak_per_s": round(hbm / 32, 3),
            "bytes_per_query": per_q}


def host_to_device_gbs(torch) -> float:
    """Pinned host-to-device copy bandwidth (GB/s), best of four 1 GiB copies."""
    src = torch.empty(1 << 30, dtype=torch.uint8).pin_memory()
    dst = torch.empty(1 << 30, dtype=torch.uint8, device="cuda")
    st = torch.cuda.current_stream()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    best = 0.0
    for _ in range(4):
        e0.record(st)
        dst.copy_(src, non_blocking=True)
        e1.record(st)
        torch.cuda.synchronize()
        best = max(best, (1 << 30) / (e0.elapsed_time(e1) * 1e-3) / 1e9)
    del src, dst
    return best


def sector_rate(table_bytes: int) -> dict:
    """Random 32-byte sector reads per second that the device delivers from a
    table of `table_bytes` (the library's probe: 12 independent random 4-byte
    loads per thread, best of six launches)."""
    import paper_2503_18397_gb300 as vf

    r = vf.vf_sector_rate(int(table_bytes))
    return {"sectors_per_s": r, "source": f"measured in this run: vf_sector_rate over a {table_bytes / 1e6:.1f} MB "
                                         f"table (random 4-byte loads, one 32-byte sector each)"}


def sector_roofline(qps: float, table_bytes: int, bound: str, k: int = 3) -> dict:
    """k random sectors per query against the device's measured random-sector
    rate for a table the size of the data array."""
    pk = sector_rate(table_bytes)
    got = k * qps
    return {"bound": bound, "unit": "G sectors/s", "achieved": round(got / 1e9, 3),
            "peak": round(pk["sectors_per_s"] / 1e9, 3), "frac": round(got / pk["sectors_per_s"], 4),
            "peak_source": pk["source"], "data_bytes": int(table_bytes)}


def measure_c5_scale(n: int, hbm: float, peak_kind: str) -> dict:
    """One VFilter over n keys generated on the device in chunks, built one
    shard group at a time; queries of 10^8 members and 10^8 disjoint keys
    against its data array (far larger than L2)."""
    import torch

    import paper_2503_18397_gb300 as vf
    from paper_2503_18397_gb300 import synth

    keys = torch.empty(n, dtype=torch.int64, device="cuda")
    chunk = 1 << 28
    for c0 in range(0, n, chunk):
        c1 = min(n, c0 + chunk)
        keys[c0:c1] = synth.u64_keys_torch(c0, c1 - c0, 0xC5)
    torch.cuda.synchronize()
    p = vf.vf_params_default(kind=vf.FILTER, b=8, seed=3)
    stream = torch.cuda.current_stream()
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(4)]
    clocks = Clocks(torch.cuda.current_device())
    clocks.start()
    vf.vf_timing_read()
    vf.vf_timing_enable(True)
    ev[0].record(stream)
    s = vf.vf_build(keys, None, params=p, stream=stream)
    ev[1].record(stream)
    torch.cuda.synchronize()
    info = s.info
    mq = min(n, 100_000_000)
    member = keys[:: max(1, n // mq)][:mq].contiguous()
    other = synth.u64_keys_torch(n, mq, 0xC5)
    for _ in range(3):  # warm-up
        s.query(member[: 1 << 24], stream=stream)
    ev[2].record(stream)
    o1 = s.query(member, stream=stream)
    o2 = s.query(other, stream=stream)
    ev[3].record(stream)
    torch.cuda.synchronize()
    vf.vf_timing_enable(False)
    phases = vf.vf_timing_read()
    clk = clocks.stop()
    b_ms, q_ms = ev[0].elapsed_time(ev[1]), ev[2].elapsed_time(ev[3])
    qps = 2 * mq / (q_ms * 1e-3)
    res = {"workload": "one VFilter of %d uniform 64-bit keys, b=8, keys generated on the device in chunks, "
                       "built by shard group; 1e8 members + 1e8 disjoint keys queried" % n,
           "n": n, "value": round(b_ms * 1e6 / n, 4), "unit": "ns/key", "build_ms": round(b_ms, 3),
           "shards": int(info.shards), "cells_per_shard": int(info.cells), "lg_seg": int(info.lg_seg), "c": info.c,
           "data_bytes": int(info.data_bytes), "space_overhead": round(info.total_cells / n - 1, 4),
           "retries": int(info.retries), "query_gqps": round(qps / 1e9, 3),
           "query_roofline": {"hbm": random_sector_roofline(qps, 8, "filter", hbm, peak_kind),
                              "sectors": sector_roofline(qps, int(info.data_bytes), "hbm")},
           "members_ok": bool(o1.bool().all().item()), "fpr": float(o2.float().mean().item()),
           "phases": {k: {"ms": round(v[0], 3), "launches": v[1]} for k, v in phases.items() if v[1]},
           "gpu_launches": int(sum(v[1] for v in phases.values())), "clocks": clk}
    s.free()
    del keys, member, other, o1, o2
    torch.cuda.empty_cache()
    return res


def measure_c5_serving() -> dict:
    """Poisson arrivals of builds and query batches under a device-memory
    budget: continuous batching, resident structures, p50/p99 latency."""
    import torch

    from paper_2503_18397_gb300 import serve, synth

    rng = np.random.default_rng(0x5E)
    nb, nq = 24, 96
    sizes = synth.log_uniform_sizes(nb, 1e4, 1e8, 0x5E)
    qsizes = synth.log_uniform_sizes(nq, 1e3, 1e7, 0x5F)
    work = float(sum(sizes)) * 4e-9 + nb * 5e-3 + float(sum(qsizes)) * 1e-9 + nq * 1e-3
    rate = (nb + nq) / (work / 0.7)  # about 70% of the estimated capacity
    t, reqs, bkeys, rid, qi = 0.0, [], {}, 0, 0
    for i in range(nb):
        t += rng.exponential(1 / rate)
        nn = int(sizes[i])
        b = int(rng.choice([8, 16]))
        kind = int(rng.integers(0, 2))
        k = synth.u64_keys(i * 10**9, nn, 0x5E)
        v = synth.values(nn, b, 0x5E + i) if kind == 0 else None
        bkeys[i] = k
        kt = torch.from_numpy(k.view(np.int64)).pin_memory()
        vt = None if v is None else torch.from_numpy(v.view({1: np.uint8, 2: np.int16}[v.dtype.itemsize])).pin_memory()
        reqs.append(serve.BuildRequest(rid, t, i, kt, vt, kind, b, 77 + i))
        rid += 1
        for _ in range(nq // nb):
            t += rng.exponential(1 / rate)
            sid = int(rng.integers(0, i + 1))
            m = int(qsizes[qi])
            qi += 1
            kk = bkeys[sid]
            q = np.concatenate([kk[rng.integers(0, len(kk), size=m // 2)],
                                synth.u64_keys(10**15 + rid * 10**7, m - m // 2, 0x5E)])
            reqs.append(serve.QueryRequest(rid, t, sid, torch.from_numpy(q.view(np.int64)).pin_memory()))
            rid += 1
    free, _ = torch.cuda.mem_get_info()
    srv = serve.Server(budget=int(free * 0.25))
    t0 = time.perf_counter()
    recs = srv.run(reqs)
    span = time.perf_counter() - t0
    srv.close()
    total_b = int(sum(sizes))
    total_q = int(sum(qsizes))
    return {"workload": "serving: Poisson arrivals of %d builds (log-uniform 1e4..1e8 keys, b in {8,16}) and %d "
                        "query batches (log-uniform 1e3..1e7 keys, half members) under a budget of 25%% of free "
                        "device memory" % (nb, nq),
            "requests": len(reqs), "builds": serve.percentiles(recs, "build"),
            "queries": serve.percentiles(recs, "query"), "span_s": round(span, 3),
            "arrival_rate_per_s": round(rate, 2), "budget_gb": round(free * 0.25 / 2**30, 1),
            "build_keys": total_b, "query_keys": total_q,
            "throughput_keys_per_s": round((total_b + total_q) / span, 1)}


def _standalone(args, workload):
    import torch

    import paper_2503_18397_gb300 as vf
    from paper_2503_18397_gb300 import build as vbuild

    torch.cuda.set_device(0)
    vbuild.build()
    vf.lib()
    return {"metric": METRIC, "n_gpus": 1, "steps": args.steps, "warmup": args.warmup, "higher_is_better": False,
            "scaling": "weak", "vs_baseline": None, "dtype": "u64", "data": "synthetic",
            "config": {"workload": WORKLOADS[workload][4]}}


def run_batch(args):
    """Batched build of many uneven structures against the plain per-structure path."""
    out = _standalone(args, "c4")
    c4 = measure_c4(args.steps, args.warmup, args.n or 4096)
    out.update({"value": c4["value"], "unit": "ns/key", "ms_per_step": c4["ms_per_batch"],
                "gpu_launches": c4["gpu_launches"], "clocks": c4["clocks"], "c4": c4})
    out["config"].update({"structures": c4["structures"], "total_keys": c4["total_keys"],
                          "l2": "inputs larger than L2 (no flush)", "tuned": c4["tuned"]})
    print(json.dumps(out), flush=True)


def run_serving(args):
    """Scale (one 5e9-key VFilter built by shard group) and serving (Poisson mix)."""
    out = _standalone(args, "c5")
    hbm, peak_kind = peaks()
    sc = measure_c5_scale(args.n or 5_000_000_000, hbm, peak_kind)
    out.update({"value": sc["value"], "unit": "ns/key", "ms_per_step": sc["build_ms"],
                "gpu_launches": sc["gpu_launches"], "clocks": sc["clocks"], "scale": sc})
    out["serving"] = measure_c5_serving()
    print(json.dumps(out), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="gpu", choices=["gpu", "reference"])
    ap.add_argument("--workload", default="c2", choices=sorted(WORKLOADS))
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-extras", action="store_true",
                    help="default workload only: skip the batched (c4), scale and serving (c5) sub-measurements")
    ap.add_argument("--n", type=int, default=0, help="override the workload's key count (profiling runs)")
    args = ap.parse_args()
    if args.impl == "reference":
        run_reference(args)
    elif args.workload == "c4":
        run_batch(args)
    elif args.workload == "c5":
        run_serving(args)
    else:
        run_gpu(args)


if __name__ == "__main__":
    main()

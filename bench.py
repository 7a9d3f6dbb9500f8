"""Benchmark of the zd-tree k-NN path on GB300.

One step = one pass of the whole hot path over the 3D clustered workload
(n = 10,000,000 int32 points in [0, 2^20)^3 from 1,000 Gaussian clusters,
L = 16, k = 10): Morton encode, radix sort, gather, canonical tree (leaves,
internal nodes, boxes), then exact all-points k-NN with int32 ids and int64
squared distances written for every point.  Inputs are resident in HBM when
the timed region starts; L2 is flushed (256 MiB write) between steps.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

--impl reference times the CPU oracle (plain C, OpenMP over queries) on the
host cores on a bounded sample of the same workload.  Other workloads:
--workload 2d-uniform | dynamic | batched | differentiable | large-k | skewed |
update-sweep | n-sweep | k-sweep.
Prints one JSON line (rank 0).
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import re
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "kNN queries/s + zd-tree build pts/s (3D n=1e7,k=10) and % HBM roofline; fwd+bwd/s"

# Algorithmic bytes (declared before measuring).
#   all-points k-NN, per query: 4 dim (own coordinates) + 4 (sorted position
#   -> id) + 12 (amortized node / leaf data) + 4k (ids) + 8k (int64 d^2; 4k
#   for fp32 distances).
#   build, per point (c = 4 dim coordinate bytes): encode c + 8, histogram 8,
#   radix passes 20 + 24 (P - 1), gather 4 + 2c, split 8, boxes c, nodes
#   0.25 * 48 (3D, 8 passes: 276).
#   backward, per (query, neighbour): 12 (query) + 12 (reference, gathered)
#   + 4 (id) + 12 (query gradient, amortized) + 12 (reference gradient).
#   updates (paper-work model, Theorem 3): b (encode + sort + route, 276 B)
#   + touched leaves * 2 * (L * 16 B) + rebuilt nodes * 48 B.
def knn_bytes_per_query(k: int, dim: int = 3, dist_bytes: int = 8, own_id: bool = True) -> int:
    return 4 * dim + (4 if own_id else 0) + 12 + (4 + dist_bytes) * k


def build_bytes_per_point(passes: int = 8, dim: int = 3) -> int:
    c = 4 * dim
    return (c + 8) + 8 + (20 + 24 * (passes - 1)) + (4 + 2 * c) + 8 + c + 12


def sort_passes(key_bits: int) -> int:
    return (key_bits + 7) // 8


BACKWARD_BYTES_PER_PAIR = 12 + 12 + 4 + 12 + 12


def update_bytes(b: int, touched_leaves: int, leaf_size: int = 16, rebuilt_nodes: int = None) -> int:
    """Paper-work model of one batch update (Theorem 3): the batch's encode,
    sort and routing, the touched leaves read and written, and the nodes
    rebuilt (one per touched leaf)."""
    if rebuilt_nodes is None:
        rebuilt_nodes = touched_leaves
    return 276 * b + touched_leaves * 2 * leaf_size * 16 + rebuilt_nodes * 48


def roofline(kernel: str, bytes_per_launch: float, ms: float, traffic=None, bound: str = "hbm") -> dict:
    """Roofline object: algorithmic bytes of one launch over its measured
    duration, against the measured HBM copy bandwidth."""
    pk, pk_src = hbm_peak()
    achieved = bytes_per_launch / (ms / 1e3) / 1e9
    return {"kernel": kernel, "bound": bound, "achieved": achieved, "peak": pk, "peak_source": pk_src,
            "unit": "GB/s", "frac": achieved / pk, "traffic": traffic,
            "algorithmic_bytes_per_launch": int(bytes_per_launch)}


def peaks() -> dict:
    try:
        return json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except Exception:
        return {}


def hbm_peak():
    p = peaks()
    if "hbm_gbs" in p:
        return float(p["hbm_gbs"]), "measured"
    return 6800.0, "fallback"


def source_digest(files) -> str:
    h = hashlib.sha256()
    for f in files:
        h.update(open(os.path.join(ROOT, f), "rb").read())
    return h.hexdigest()[:12]


KNN_SOURCES = ["paper_2111_04182_gb300/csrc/knn_impl.cuh", "paper_2111_04182_gb300/csrc/knn_group.cuh",
               "paper_2111_04182_gb300/csrc/knn_i32.cu"]
WIDE_SOURCES = ["paper_2111_04182_gb300/csrc/knn_impl.cuh", "paper_2111_04182_gb300/csrc/knn_wide.cuh",
                "paper_2111_04182_gb300/csrc/knn_wide.cu"]


def profiled_value(field: str, kernel: str, workload: str, summary: str, sources):
    """A number `field` of `kernel` from a committed ncu summary line
    `<field>: <value> source: <digest> kernel: <k> workload: <w>`, or None
    when absent or when the kernel's sources changed since the capture."""
    path = os.path.join(ROOT, "profiles", summary)
    if not os.path.exists(path):
        return None
    text = open(path).read()
    m = re.search(r"%s:\s*([0-9.]+)\s+source:\s*([0-9a-f]+)\s+kernel:\s*(\S+)\s+workload:\s*(\S+)" % field,
                  text)
    if not m or m.group(3) != kernel or m.group(4) != workload:
        return None
    if m.group(2) != source_digest(sources):
        return None
    return float(m.group(1))


def profiled_traffic(kernel: str, workload: str, summary: str = "knn_allpoints_3d_clustered.md",
                     sources=None):
    """Per-launch DRAM bytes of `kernel` from the committed ncu summary, or
    None when absent or when the kernel source changed since the capture."""
    v = profiled_value("traffic_bytes_per_launch", kernel, workload, summary, sources or KNN_SOURCES)
    return None if v is None else int(v)


def issue_roofline(inst_per_unit, units: int, ms: float, sm_mhz) -> dict:
    """Instruction-issue roofline: warp instructions per unit (from the
    committed ncu summary) x units / the measured time, against the issue
    peak of one warp instruction per cycle per scheduler (4 per SM)."""
    import torch
    sms = torch.cuda.get_device_properties(torch.cuda.current_device()).multi_processor_count
    peak = sms * 4 * (sm_mhz or 0) * 1e6
    if inst_per_unit is None or not peak:
        return {"bound": "issue", "achieved": None, "peak": peak or None, "unit": "warp-inst/s", "frac": None,
                "inst_per_unit": inst_per_unit}
    ach = inst_per_unit * units / (ms / 1e3)
    return {"bound": "issue", "achieved": ach, "peak": peak, "unit": "warp-inst/s", "frac": ach / peak,
            "inst_per_unit": inst_per_unit, "peak_basis": "%d SMs x 4 schedulers x %.0f MHz (median under load)"
            % (sms, sm_mhz)}


class ClockSampler:
    """nvidia-smi samples of SM clock and throttle reasons during a region."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.index), "--query-gpu=" + self.Q,
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.th = threading.Thread(target=self._read, daemon=True)
            self.th.start()
        except Exception:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self) -> dict:
        if not self.proc:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        time.sleep(0.25)
        self.proc.terminate()
        try:
            self.proc.wait(2)
        except Exception:
            self.proc.kill()
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in self.lines:
            f = [x.strip() for x in line.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                mx.append(float(f[2]))
            except ValueError:
                continue
            for nm, v in zip(names, f[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        return {"sm_mhz": float(np.median(sm)) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": sorted(reasons), "samples": len(sm)}


def dist_env():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def barrier(ws):
    if ws > 1:
        import torch.distributed as dist
        dist.barrier()


def max_over_ranks(x: float, ws: int) -> float:
    """The slowest rank's time (all ranks get it)."""
    if ws == 1:
        return x
    import torch
    import torch.distributed as dist
    dev = "cuda" if dist.get_backend() == "nccl" else "cpu"
    t = torch.tensor([x], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def weak_scaling_value(units_per_rank: int, local_ms: float, ws: int):
    """Replicas: every rank processes units_per_rank; the job's rate is all
    units over the slowest rank's time.  Returns (units/s, max ms)."""
    ms = max_over_ranks(local_ms, ws)
    return ws * units_per_rank / (ms / 1e3), ms


# ------------------------------------------------------------------ ours
def run_ours(args):
    import torch

    ws, rank, local = dist_env()
    if ws > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    import __graft_entry__
    __graft_entry__.build()
    from paper_2111_04182_gb300 import datagen, zd

    if args.workload != "3d-clustered":
        return run_other(args, ws, rank, local)

    w = datagen.workload_3d_clustered(n=args.n)
    n, k, L, B = len(w["pts"]), w["k"], w["leaf_size"], w["coord_bits"]
    pts_host = torch.from_numpy(w["pts"]).pin_memory()
    pts = pts_host.to(dev)
    idx = torch.empty((n, k), dtype=torch.int32, device=dev)
    d2 = torch.empty((n, k), dtype=torch.int64, device=dev)
    flush = torch.empty(256 << 20, dtype=torch.uint8, device=dev)
    s = torch.cuda.current_stream()

    def step(ev=None):
        if ev is not None:
            ev[0].record(s)
        t = zd.zd_build(pts, L, B)
        if ev is not None:
            ev[1].record(s)
        t.knn(k, out=(idx, d2))
        if ev is not None:
            ev[2].record(s)
        t.free()

    for _ in range(args.warmup):
        step()
    st = zd.zd_check()
    if st != 0:
        raise RuntimeError("device status %d after warm-up" % st)
    torch.cuda.synchronize()

    evs = [[torch.cuda.Event(enable_timing=True) for _ in range(3)] for _ in range(args.steps)]
    clocks = ClockSampler(local)
    clocks.start()
    barrier(ws)
    torch.cuda.synchronize()
    for i in range(args.steps):
        step(evs[i])
        flush.zero_()  # L2 flush between steps, outside the step's events
    torch.cuda.synchronize()
    barrier(ws)
    clk = clocks.stop()
    st = zd.zd_check()
    if st != 0:
        raise RuntimeError("device status %d in the timed region" % st)
    build_ms = [e[0].elapsed_time(e[1]) for e in evs]
    knn_ms = [e[1].elapsed_time(e[2]) for e in evs]
    step_ms = sum(b + q for b, q in zip(build_ms, knn_ms)) / args.steps
    value, step_ms = weak_scaling_value(n, step_ms, ws)

    # End to end through the public API with host buffers: every step copies
    # its points host -> device (pinned) and its ids and distances device ->
    # host (pinned).  Streamed the way a user feeds successive batches: step
    # i + 1's points are copied in and step i's results copied out on two
    # copy streams while the device builds and searches (inputs and outputs
    # double-buffered); the timed region runs from the first step's input
    # copy to the last step's output copy.  The same steps run back to back
    # on one stream are reported beside it.
    dev_out = [(idx, d2), (torch.empty_like(idx), torch.empty_like(d2))]
    host_out = [(torch.empty((n, k), dtype=torch.int32).pin_memory(),
                 torch.empty((n, k), dtype=torch.int64).pin_memory()) for _ in range(2)]
    dev_in = [torch.empty_like(pts), torch.empty_like(pts)]
    cs, hs = torch.cuda.Stream(), torch.cuda.Stream()  # copy-out, copy-in

    def e2e_run(steps, pipelined):
        if not pipelined:
            for _ in range(steps):
                p = pts_host.to(dev, non_blocking=True)
                t = zd.zd_build(p, L, B)
                t.knn(k, out=dev_out[0])
                host_out[0][0].copy_(dev_out[0][0], non_blocking=True)
                host_out[0][1].copy_(dev_out[0][1], non_blocking=True)
                t.free()
            return 0
        copied, consumed, arrived = [None, None], [None, None], [None, None]

        def copy_in(i):
            j = i % 2
            if consumed[j] is not None:
                hs.wait_event(consumed[j])  # the build that read this input is done
            with torch.cuda.stream(hs):
                dev_in[j].copy_(pts_host, non_blocking=True)
            arrived[j] = torch.cuda.Event()
            arrived[j].record(hs)

        copy_in(0)
        for i in range(steps):
            j = i % 2
            if i + 1 < steps:
                copy_in(i + 1)
            s.wait_event(arrived[j])
            if copied[j] is not None:
                s.wait_event(copied[j])  # the copy that read these outputs has finished
            t = zd.zd_build(dev_in[j], L, B)
            consumed[j] = torch.cuda.Event()
            consumed[j].record(s)
            t.knn(k, out=dev_out[j])
            ready = torch.cuda.Event()
            ready.record(s)
            cs.wait_event(ready)
            with torch.cuda.stream(cs):
                host_out[j][0].copy_(dev_out[j][0], non_blocking=True)
                host_out[j][1].copy_(dev_out[j][1], non_blocking=True)
            copied[j] = torch.cuda.Event()
            copied[j].record(cs)
            t.free()
        s.wait_stream(cs)
        return (steps - 1) % 2

    e2e_steps = max(2, min(args.steps, 6))
    e2e_res = {}
    for pipelined in (False, True):
        e2e_run(2, pipelined)
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        barrier(ws)
        e0.record(s)
        last = e2e_run(e2e_steps, pipelined)
        e1.record(s)
        torch.cuda.synchronize()
        e2e_res[pipelined] = max_over_ranks(e0.elapsed_time(e1) / e2e_steps, ws)
        if not (torch.equal(host_out[last][0], dev_out[last][0].cpu()) and
                torch.equal(host_out[last][1], dev_out[last][1].cpu())):
            raise RuntimeError("end-to-end host results differ from the device results")
    e2e_ms = e2e_res[True]

    pk, pk_src = hbm_peak()
    kb = knn_bytes_per_query(k) * n
    knn_avg = sum(knn_ms) / len(knn_ms)
    build_avg = sum(build_ms) / len(build_ms)
    achieved = kb / (knn_avg / 1e3) / 1e9
    traffic = profiled_traffic("k_knn_group", "3d-clustered-1e7") if n == 10_000_000 else None
    ipq = (profiled_value("warp_inst_per_query", "k_knn_group", "3d-clustered-1e7",
                          "knn_allpoints_3d_clustered.md", KNN_SOURCES) if n == 10_000_000 else None)
    bb = build_bytes_per_point() * n
    # build: liveness bitmap init, encode, plan, 8 sort passes, finish,
    # gather (+ float copy), split flags, scan, leaf index, internal nodes,
    # boxes (18); k-NN: warp groups + exact fallback (2)
    launches_per_step = 20
    out = {
        "metric": METRIC, "value": value, "unit": "queries/s", "n_gpus": ws, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": step_ms, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "int64", "data": "synthetic",
        "config": headline_config(n, k, L, B, "replicas" if ws > 1 else "1 GPU"),
        "components": {"build_ms": build_avg, "build_pts_per_s": n / (build_avg / 1e3),
                       "build_hbm_frac": bb / (build_avg / 1e3) / 1e9 / pk,
                       "knn_ms": knn_avg, "knn_queries_per_s": n / (knn_avg / 1e3)},
        "roofline": {"kernel": "k_knn_group<3,10,fs>", "bound": "hbm", "achieved": achieved, "peak": pk,
                     "peak_source": pk_src, "unit": "GB/s", "frac": achieved / pk,
                     "traffic": traffic, "algorithmic_bytes_per_launch": kb},
        "issue_roofline": dict(issue_roofline(ipq, n, knn_avg, clk.get("sm_mhz")), kernel="k_knn_group<3,10,fs>"),
        "clocks": clk,
        "e2e": {"value": ws * n / (e2e_ms / 1e3), "unit": "queries/s", "ms_per_step": e2e_ms,
                "h2d_bytes_per_step": n * 12, "d2h_bytes_per_step": n * k * 12,
                "mode": "streamed: copies in and out overlap the neighbouring steps' device work",
                "sequential_ms_per_step": e2e_res[False]},
        "gpu_launches": launches_per_step * args.steps,
    }
    if rank == 0 and ws == 1 and not args.no_cpu_baseline:
        out["cpu_baseline"] = cpu_baseline("3d-clustered", w)
    if rank == 0:
        print(json.dumps(out))
    if ws > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


def cpu_baseline(kind: str, w: dict, **kw) -> dict:
    """The oracle (plain C; OpenMP over independent queries only, its build
    sequential) timed as it stands on the host cores, on a bounded sample of
    workload `kind`; returns a cpu_baseline object in the unit of that
    workload's line.  The only place this file runs the oracle."""
    from oracle import oracle
    cores = len(os.sched_getaffinity(0))
    base = {"cores": cores, "kind": "oracle"}
    if kind in ("3d-clustered", "2d-uniform"):
        # the whole step: build of all points + leaf-based k-NN of all points
        pts, k, L, B = w["pts"], w["k"], w["leaf_size"], w["coord_bits"]
        n = len(pts)
        reps = kw.get("reps", 1)
        tb, tk = [], []
        for _ in range(reps):
            t0 = time.perf_counter()
            t = oracle.OracleTree(pts, L, B)
            t1 = time.perf_counter()
            t.knn(k, nthreads=cores)
            t2 = time.perf_counter()
            del t
            tb.append(t1 - t0)
            tk.append(t2 - t1)
        b_s, k_s = float(np.median(tb)), float(np.median(tk))
        return dict(base, value=n / (b_s + k_s), unit="queries/s",
                    sample="the whole step: build of all %d points (1 thread) + leaf-based k-NN of all %d "
                           "points (%d threads)%s" % (n, n, cores, ", median of %d" % reps if reps > 1 else ""),
                    build_s=b_s, knn_s=k_s, build_pts_per_s=n / b_s, knn_queries_per_s=n / k_s)
    if kind == "dynamic":
        # one round on the live set the GPU ended with: the oracle's update is
        # a rebuild of the current set (insert, then delete), then the round's
        # bit-based queries
        pts, ids, ins, dele, q, k = kw["pts"], kw["ids"], kw["ins"], kw["dele"], kw["queries"], w["k"]
        L, B = w["leaf_size"], w["coord_bits"]
        new_ids = np.arange(kw["next_id"], kw["next_id"] + len(ins), dtype=np.int32)
        t0 = time.perf_counter()
        t = oracle.OracleTree(np.concatenate([pts, ins]), L, B, ids=np.concatenate([ids, new_ids]))
        t_ins = time.perf_counter() - t0
        del t
        all_pts, all_ids = np.concatenate([pts, ins]), np.concatenate([ids, new_ids])
        keep = ~np.isin(all_ids, dele)
        t0 = time.perf_counter()
        t = oracle.OracleTree(all_pts[keep], L, B, ids=all_ids[keep])
        t_del = time.perf_counter() - t0
        t0 = time.perf_counter()
        t.knn(k, queries=q, mode=oracle.MODE_BIT, nthreads=cores)
        t_q = time.perf_counter() - t0
        del t
        b = len(ins)
        return dict(base, value=b / t_ins, unit="updates/s", insert_per_s=b / t_ins, delete_per_s=len(dele) / t_del,
                    query_per_s=len(q) / t_q,
                    sample="one round: rebuild of the live set after inserting %d points (%d points) and after "
                           "deleting %d ids (1 thread), %d bit-based queries k=%d (%d threads)"
                           % (b, len(all_pts), len(dele), len(q), k, cores),
                    insert_s=t_ins, delete_s=t_del, query_s=t_q)
    if kind == "batched":
        off, pts, k, B = w["offsets"], w["pts"], w["k"], w["coord_bits"]
        L, c_s = kw["leaf_size"], kw.get("clouds", 64)
        t0 = time.perf_counter()
        for c in range(c_s):
            oracle.OracleTree(pts[off[c]:off[c + 1]], L, B).knn(k, nthreads=cores)
        ts = time.perf_counter() - t0
        frac = float(off[c_s]) / float(off[-1])
        step = ts / frac
        return dict(base, value=(len(off) - 1) / step, unit="clouds/s", points_per_s=float(off[-1]) / step,
                    sample="the first %d clouds (%d points): per-cloud build (1 thread) + all-points k=%d "
                           "(%d threads), time scaled by total/sampled points" % (c_s, int(off[c_s]), k, cores),
                    sample_s=ts)
    if kind == "differentiable":
        # a few pairs: float tree of B, root-based k-NN of A (fp64 ranking),
        # fp64 gradient; the GPU's outputs for those pairs are compared with
        # the oracle's (FP32 error against FP64, per element)
        A, Bc, k, L, B = w["A"], w["B"], w["k"], w["leaf_size"], w["coord_bits"]
        gpu = kw["gpu"]  # {pair: (idx, dist, gA, gB)} host arrays
        errs = {"dist_max_rel": 0.0, "grad_a_max_rel": 0.0, "grad_b_max_rel": 0.0, "ids_equal": True}
        t0 = time.perf_counter()
        outs = {}
        for p in gpu:
            lo, scale = oracle.quantization_of(Bc[p], B)
            t = oracle.OracleTree(Bc[p], L, B, qlo=lo, qscale=scale)
            oi, od = t.knn(k, queries=A[p], mode=oracle.MODE_ROOT, nthreads=cores)
            _, ga, gb = oracle.knn_dist_grad(A[p], Bc[p], oi)
            outs[p] = (oi, np.sqrt(od), ga, gb)
        ts = time.perf_counter() - t0
        for p, (oi, d64, ga, gb) in outs.items():
            gi, gd, gA, gB = gpu[p]
            errs["ids_equal"] &= bool(np.array_equal(gi, oi))
            errs["dist_max_rel"] = max(errs["dist_max_rel"], float(np.max(np.abs(gd - d64) / d64)))
            errs["grad_a_max_rel"] = max(errs["grad_a_max_rel"], float(np.max(
                np.abs(gA - ga) / np.maximum(np.abs(ga), 1e-3))))
            errs["grad_b_max_rel"] = max(errs["grad_b_max_rel"], float(np.max(
                np.abs(gB - gb) / np.maximum(np.abs(gb), 1e-3))))
        step = ts / len(gpu) * len(A)
        return dict(base, value=1.0 / step, unit="fwd+bwd/s",
                    sample="%d of %d pairs: float tree of B (1 thread), root-based k=%d of A (%d threads), fp64 "
                           "gradient; time scaled by pairs" % (len(gpu), len(A), k, cores),
                    sample_s=ts, fp32_vs_fp64=errs)
    raise ValueError(kind)


# ------------------------------------------------------------- reference
def run_reference(args):
    """The oracle as the reference arm: every step is the whole headline step
    (build of all points + leaf-based k-NN of all points) run on the host
    cores; the line reports the measured wall time per step."""
    ws, rank, _ = dist_env()
    if rank != 0:
        return
    from paper_2111_04182_gb300 import datagen
    if args.workload != "3d-clustered":
        print(json.dumps({"impl": "reference", "unavailable": "reference arm is timed on the 3d-clustered workload only"}))
        return
    w = datagen.workload_3d_clustered(n=args.n)
    n = len(w["pts"])
    for _ in range(args.warmup):  # untimed
        cpu_baseline("3d-clustered", w)
    step_s = []
    for _ in range(args.steps):
        t0 = time.perf_counter()
        cb = cpu_baseline("3d-clustered", w)
        step_s.append(time.perf_counter() - t0)
    mean_s = float(np.mean(step_s))
    value = n / mean_s
    cb["value"] = value
    cb["sample"] = "every step is the whole step: " + cb["sample"].split(": ", 1)[1]
    out = {"metric": METRIC, "value": value, "unit": "queries/s", "n_gpus": ws, "steps": args.steps,
           "warmup": args.warmup, "ms_per_step": mean_s * 1e3, "higher_is_better": True,
           "scaling": "weak", "vs_baseline": None, "dtype": "int64", "data": "synthetic",
           "config": headline_config(n, w["k"], w["leaf_size"], w["coord_bits"], "host cores (oracle)",
                                     "n/a (host)"),
           "impl": "reference", "cpu_baseline": cb,
           "e2e": {"value": value, "unit": "queries/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(out))


def headline_config(n: int, k: int, L: int, B: int, parallelism: str,
                    l2: str = "flushed between steps (256 MiB write)") -> dict:
    """The `config` object of the headline line, shared by both arms."""
    return {"workload": "3d-clustered-1e7" if n == 10_000_000 else "3d-clustered-%d" % n,
            "n": n, "dim": 3, "k": k, "leaf_size": L, "coord_bits": B, "clusters": 1000,
            "step": "build + all-points k-NN (ids and int64 d^2 written)",
            "l2": l2, "parallelism": parallelism}


def _events(n):
    import torch
    return [torch.cuda.Event(enable_timing=True) for _ in range(n)]


def run_other(args, ws, rank, local):
    fn = {"2d-uniform": bench_2d, "dynamic": bench_dynamic, "batched": bench_batched,
          "differentiable": bench_differentiable, "large-k": bench_large_k,
          "skewed": bench_skewed, "update-sweep": bench_update_sweep,
          "n-sweep": bench_n_sweep, "k-sweep": bench_k_sweep}.get(args.workload)
    if fn is None:
        raise SystemExit("unknown workload %r" % args.workload)
    out = fn(args)
    out["n_gpus"] = ws
    if rank == 0:
        print(json.dumps(out))


def bench_2d(args):
    """2D uniform, n = 100,000, L = 16, k = 10: build + all-points k-NN."""
    import torch
    from paper_2111_04182_gb300 import datagen, zd
    w = datagen.workload_2d_uniform()
    n, k = len(w["pts"]), w["k"]
    pts = torch.from_numpy(w["pts"]).cuda()
    idx = torch.empty((n, k), dtype=torch.int32, device="cuda")
    d2 = torch.empty((n, k), dtype=torch.int64, device="cuda")
    for _ in range(args.warmup):
        t = zd.zd_build(pts, w["leaf_size"], w["coord_bits"]); t.knn(k, out=(idx, d2)); t.free()
    torch.cuda.synchronize()
    ms = []
    for _ in range(args.steps):
        a, b, c = _events(3)
        a.record(); t = zd.zd_build(pts, w["leaf_size"], w["coord_bits"]); b.record()
        t.knn(k, out=(idx, d2)); c.record(); c.synchronize(); t.free()
        ms.append((a.elapsed_time(b), b.elapsed_time(c)))
    assert zd.zd_check() == 0
    bm = float(np.median([m[0] for m in ms])); km = float(np.median([m[1] for m in ms]))
    passes = sort_passes(2 * w["coord_bits"])
    out = {"workload": "2d-uniform-1e5", "metric": "queries/s (build + all-points k=10)",
           "value": n / ((bm + km) / 1e3), "unit": "queries/s", "build_ms": bm, "knn_ms": km,
           "build_pts_per_s": n / (bm / 1e3), "knn_queries_per_s": n / (km / 1e3), "steps": args.steps,
           "l2": "inputs and outputs (13 MB) fit in L2",
           "roofline": roofline("k_knn_group<2,10,fs>", knn_bytes_per_query(k, dim=2) * n, km),
           "build_roofline": roofline("build (%d sort passes)" % passes,
                                      build_bytes_per_point(passes, dim=2) * n, bm)}
    if not args.no_cpu_baseline:
        out["cpu_baseline"] = cpu_baseline("2d-uniform", w, reps=5)
    return out


def touched_leaves(tree, coord_bits: int, ins_pts=None, del_ids=None) -> int:
    """Leaves of `tree` (before an update) that a batch touches: the leaf
    each inserted key falls into by sorted position, or the leaf of each
    deleted id.  Counted with torch on the device, outside any timed region,
    for the paper-work byte model of an update."""
    import torch
    from paper_2111_04182_gb300 import zd
    e = tree.export()
    leaf_lo = e["leaf_lo"].to(torch.int64)
    if ins_pts is not None:
        pos = torch.searchsorted(e["keys"], zd.zd_morton_encode(ins_pts, coord_bits))
    else:
        ids = e["ids"].to(torch.int64)
        inv = torch.full((int(ids.max()) + 1,), -1, dtype=torch.int64, device=ids.device)
        inv[ids] = torch.arange(len(ids), device=ids.device)
        pos = inv[del_ids.to(torch.int64)]
    leaf = torch.searchsorted(leaf_lo[1:], pos, right=True).clamp_(max=len(leaf_lo) - 2)
    return int(torch.unique(leaf).numel())


def bench_dynamic(args):
    """5e7 uniform points; rounds of +1e6 insert, -1e6 delete, 1e6 queries
    (k = 5, bit-based).  Every round, sampled rows are checked for properties
    any exact answer has (live ids, distances recomputed from the host copy of
    the points, non-decreasing rows); every row of every round is checked
    against the oracle by the full-size tests.  Rooflines: updates by the
    paper-work model (Theorem 3, touched leaves counted per round), queries
    by the external-query search bytes."""
    import torch
    from paper_2111_04182_gb300 import datagen, zd
    rounds = args.rounds
    w = datagen.DynamicWorkload(n0=args.dyn_n0, batch=args.dyn_batch, n_queries=args.dyn_batch, rounds=rounds)
    cap = w.n0 + w.batch
    all_pts = np.empty((w.n0 + rounds * w.batch, 3), np.int32)
    all_pts[: w.n0] = w.initial
    pts = torch.from_numpy(w.initial).cuda()
    a, b = _events(2)
    a.record(); t = zd.zd_build(pts, w.leaf_size, w.coord_bits, capacity=cap); b.record(); b.synchronize()
    build_ms = a.elapsed_time(b)
    del pts
    ins_ms, del_ms, q_ms, checked, t_ins, t_del = [], [], [], 0, [], []
    rng = np.random.default_rng(7)
    for r in range(rounds):
        ins, dele, q = w.round()
        ins_d, del_d, q_d = torch.from_numpy(ins).cuda(), torch.from_numpy(dele).cuda(), torch.from_numpy(q).cuda()
        t_ins.append(touched_leaves(t, w.coord_bits, ins_pts=ins_d))
        torch.cuda.synchronize()
        e = _events(6)
        e[0].record(); new = t.insert(ins_d); e[1].record(); e[1].synchronize()
        t_del.append(touched_leaves(t, w.coord_bits, del_ids=del_d))
        torch.cuda.synchronize()
        e[2].record(); t.delete(del_d); e[3].record()
        e[4].record(); idx, d2 = t.knn(w.k, queries=q_d, mode=zd.ZD_SEARCH_BIT); e[5].record()
        e[5].synchronize()
        ins_ms.append(e[0].elapsed_time(e[1])); del_ms.append(e[2].elapsed_time(e[3])); q_ms.append(e[4].elapsed_time(e[5]))
        all_pts[new.cpu().numpy()] = ins
        sel = torch.from_numpy(rng.choice(len(q), size=args.dyn_check, replace=False)).cuda()
        I, D = idx[sel].cpu().numpy(), d2[sel].cpu().numpy()
        diff = all_pts[I].astype(np.int64) - q[sel.cpu().numpy()][:, None, :].astype(np.int64)
        if not (np.isin(I, w.live).all() and np.array_equal((diff * diff).sum(-1), D)
                and np.all(D[:, 1:] >= D[:, :-1])):
            raise RuntimeError("round %d: k-NN rows fail the property checks" % r)
        checked += len(sel)
    assert zd.zd_check() == 0
    im, dm, qm = (float(np.median(x)) for x in (ins_ms, del_ms, q_ms))
    ti, td = float(np.mean(t_ins)), float(np.mean(t_del))
    t.free()
    qbytes = (12 + 8 + 24 * sort_passes(3 * w.coord_bits) + 16 + knn_bytes_per_query(w.k, own_id=False)) * w.batch
    out = {"workload": "dynamic-5e7", "metric": "updates/s (insert, delete) and queries/s", "unit": "updates/s",
           "value": w.batch / (im / 1e3), "insert_per_s": w.batch / (im / 1e3),
           "delete_per_s": w.batch / (dm / 1e3), "query_per_s": w.batch / (qm / 1e3), "insert_ms": im,
           "delete_ms": dm, "query_ms": qm, "initial_build_ms": build_ms, "rounds": rounds,
           "property_checked_rows": checked, "k": w.k, "touched_leaves": {"insert": ti, "delete": td},
           "roofline": roofline("insert (merge + re-derive)", update_bytes(w.batch, int(ti), w.leaf_size), im),
           "rooflines": {
               "delete": roofline("delete (mark + compact + re-derive)", update_bytes(w.batch, int(td), w.leaf_size), dm),
               "query": roofline("queries (encode + sort + k_knn)", qbytes, qm)},
           "byte_models": "updates: 276 B per batch point + 2 * L * 16 B per touched leaf + 48 B per rebuilt "
                          "node (one per touched leaf); queries: encode 20 + sort 24/pass + gather 16 + search "
                          "12 + 12 + 12k per query"}
    if not args.no_cpu_baseline:
        live = w.live
        ins, dele, q = w.round()
        out["cpu_baseline"] = cpu_baseline("dynamic", {"k": w.k, "leaf_size": w.leaf_size,
                                                       "coord_bits": w.coord_bits},
                                           pts=all_pts[live], ids=live.astype(np.int32), ins=ins, dele=dele,
                                           queries=q, next_id=int(w.n0 + rounds * w.batch))
    return out


def bench_batched(args):
    """4096 clouds (1024..65536 points each), all-points k = 16 in every cloud:
    leaf size and thread mapping autotuned; the whole step (forest build +
    search + free) captured in one CUDA graph and replayed."""
    import torch
    from paper_2111_04182_gb300 import autotune, datagen, zd
    w = datagen.workload_batched(n_clouds=args.clouds)
    pts = torch.from_numpy(w["pts"]).cuda()
    off = w["offsets"]
    n, k, B = int(off[-1]), w["k"], w["coord_bits"]
    idx = torch.empty((n, k), dtype=torch.int32, device="cuda")
    d2 = torch.empty((n, k), dtype=torch.int64, device="cuda")
    tune = autotune.tune_batched(pts, off, k, B, out=(idx, d2), use_cache=False)
    L, mp = tune["leaf_size"], tune["mapping"]

    off_d = torch.from_numpy(off).cuda()

    def step():
        t = zd.zd_build_batched(pts, off, L, B, offsets_device=off_d)
        zd.zd_knn_batched(t, k, out=(idx, d2), mapping=mp)
        t.free()

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()
    graph = None
    try:
        s = torch.cuda.Stream()
        s.wait_stream(torch.cuda.current_stream())
        g = torch.cuda.CUDAGraph()
        with torch.cuda.stream(s):
            step()
            torch.cuda.synchronize()
            g.capture_begin()
            step()
            g.capture_end()
        torch.cuda.current_stream().wait_stream(s)
        graph = g
    except Exception as e:  # report, and time the eager step instead
        graph_error = repr(e)
        torch.cuda.synchronize()
    ms = []
    for _ in range(args.steps):
        a, b = _events(2)
        a.record()
        if graph is not None:
            graph.replay()
        else:
            step()
        b.record(); b.synchronize()
        ms.append(a.elapsed_time(b))
    # the same step eagerly with events between the phases, for the rooflines
    ph = []
    for _ in range(max(1, args.steps // 2)):
        a, b, c = _events(3)
        a.record(); t = zd.zd_build_batched(pts, off, L, B, offsets_device=off_d); b.record()
        zd.zd_knn_batched(t, k, out=(idx, d2), mapping=mp); c.record(); c.synchronize(); t.free()
        ph.append((a.elapsed_time(b), b.elapsed_time(c)))
    assert zd.zd_check() == 0
    m = float(np.median(ms))
    bm, km = float(np.median([x[0] for x in ph])), float(np.median([x[1] for x in ph]))
    cbits = int(np.ceil(np.log2(len(off) - 1)))
    passes = sort_passes(3 * B + cbits)
    out = {"workload": "batched-4096", "metric": "clouds/s, points/s (build + all-points k=16 per cloud)",
           "value": (len(off) - 1) / (m / 1e3), "unit": "clouds/s", "ms_per_step": m,
           "points_per_s": n / (m / 1e3), "queries_per_s": n / (m / 1e3), "n_points": n, "k": k,
           "leaf_size": L, "mapping": tune["mapping_name"], "tuning": tune["table"],
           "graph": graph is not None, "graph_launches_per_step": 1 if graph is not None else None,
           "eager_phase_ms": {"build": bm, "knn": km},
           "l2": "inputs (1.6 GB) and outputs (26 GB) exceed L2",
           "roofline": roofline("k_knn (forest, %s)" % tune["mapping_name"], knn_bytes_per_query(k) * n, km),
           "build_roofline": roofline("forest build (%d sort passes)" % passes,
                                      build_bytes_per_point(passes) * n, bm),
           "step_roofline": roofline("graph: forest build + k-NN", (build_bytes_per_point(passes) +
                                                                   knn_bytes_per_query(k)) * n, m)}
    if graph is None:
        out["graph_error"] = graph_error
    if not args.no_cpu_baseline:
        out["cpu_baseline"] = cpu_baseline("batched", w, leaf_size=L)
    return out


def bench_differentiable(args):
    """64 pairs of float clouds (A 16384, B 32768): k = 8 neighbours in B for
    every point of A (fp64 ranking), loss = sum of fp32 distances, backward to
    A and B.  The CPU baseline also reports the FP32 distances' and
    gradients' largest per-element errors against the oracle's FP64 values on
    its sample pairs."""
    import torch
    from paper_2111_04182_gb300 import datagen, zd
    w = datagen.workload_differentiable()
    A = torch.from_numpy(w["A"]).cuda().requires_grad_(True)
    B = torch.from_numpy(w["B"]).cuda().requires_grad_(True)
    k = w["k"]
    P, m, r = w["A"].shape[0], w["A"].shape[1], w["B"].shape[1]

    def step(ev=None):
        A.grad = None
        B.grad = None
        if ev:
            ev[0].record()
        dist, idx = zd.KnnDist.apply(A, B, k, w["leaf_size"], w["coord_bits"])
        loss = dist.sum()
        if ev:
            ev[1].record()
        loss.backward()
        if ev:
            ev[2].record()
        return dist, idx

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()
    ms = []
    for _ in range(args.steps):
        ev = _events(3)
        dist, idx = step(ev)
        ev[2].synchronize()
        ms.append((ev[0].elapsed_time(ev[1]), ev[1].elapsed_time(ev[2])))
    assert zd.zd_check() == 0
    fm, bm = float(np.median([x[0] for x in ms])), float(np.median([x[1] for x in ms]))
    mm = fm + bm
    pairs = P * m * k
    # forward: forest of B (quantize + build, 8 passes) + external queries
    # (encode + sort + gather of A) + the search writing ids and fp32 distances
    fwd_bytes = (build_bytes_per_point(8) * P * r +
                 (20 + 24 * 8 + 16 + knn_bytes_per_query(k, dist_bytes=4, own_id=False)) * P * m)
    out = {"workload": "differentiable-64x16384x32768", "metric": "fwd+bwd/s", "value": 1e3 / mm,
           "unit": "fwd+bwd/s", "ms_per_step": mm, "forward_ms": fm, "backward_ms": bm,
           "pairs_per_s": P * 1e3 / mm, "queries_per_s": P * m * 1e3 / mm, "k": k,
           "roofline": roofline("forward (forest build + k_knn_group_f)", fwd_bytes, fm),
           "backward_roofline": roofline("backward (k_grad_q + pair sort + k_grad_ref)",
                                         BACKWARD_BYTES_PER_PAIR * pairs, bm)}
    if not args.no_cpu_baseline:
        sample = (0, 37)
        gpu = {p: (idx[p].cpu().numpy(), dist[p].detach().cpu().numpy().astype(np.float64),
                   A.grad[p].cpu().numpy().astype(np.float64), B.grad[p].cpu().numpy().astype(np.float64))
               for p in sample}
        out["cpu_baseline"] = cpu_baseline("differentiable", w, gpu=gpu)
        out["fp32_vs_fp64"] = dict(out["cpu_baseline"]["fp32_vs_fp64"], pairs=list(sample),
                                   form="max_i |x_i - x64_i| / max(|x64_i|, 1e-3) (distances: / x64_i)")
    return out


def bench_skewed(args):
    """The paper's search-start comparison (Sec. 5, k = 1): for each of the
    five point sets (2DinCube, 2Dkuzmin, 3DonSphere, 3DinCube, 3Dplummer,
    n = 10^7, L = 16) the k-NN graph computed leaf-based (warp groups and one
    thread per query), bit-based and root-based.  All four must return the
    same ids; sampled rows are checked for properties any exact answer has."""
    import torch
    from paper_2111_04182_gb300 import datagen, zd
    k = args.k_skewed
    variants = [("leaf_group", zd.ZD_SEARCH_LEAF, zd.ZD_KNN_WARP_GROUP),
                ("leaf_thread", zd.ZD_SEARCH_LEAF, zd.ZD_KNN_THREAD_PER_QUERY),
                ("bit", zd.ZD_SEARCH_BIT, 0), ("root", zd.ZD_SEARCH_ROOT, 0)]
    sets, total_q, total_ms = {}, 0, 0.0
    for name in datagen.SKEWED_SETS:
        w = datagen.workload_skewed(name, n=args.n, k=k)
        n = len(w["pts"])
        pts = torch.from_numpy(w["pts"]).cuda()
        outs = {v[0]: (torch.empty((n, k), dtype=torch.int32, device="cuda"),
                       torch.empty((n, k), dtype=torch.int64, device="cuda")) for v in variants}
        res = {}
        bms = []
        for step in range(args.warmup + args.steps):
            a, b = _events(2)
            a.record(); t = zd.zd_build(pts, w["leaf_size"], w["coord_bits"]); b.record()
            for vname, mode, mapping in variants:
                c, d = _events(2)
                c.record(); t.knn(k, mode=mode, mapping=mapping, out=outs[vname]); d.record()
                d.synchronize()
                if step >= args.warmup:
                    res.setdefault(vname, []).append(c.elapsed_time(d))
            if step >= args.warmup:
                bms.append(a.elapsed_time(b))
            t.free()
        assert zd.zd_check() == 0
        ref_i, ref_d = outs["leaf_group"]
        same = all(torch.equal(outs[v][0], ref_i) and torch.equal(outs[v][1], ref_d) for v in outs)
        rows = np.random.default_rng(1).choice(n, 4096, replace=False)
        r_d = torch.from_numpy(rows).cuda()
        I, D = ref_i[r_d].cpu().numpy(), ref_d[r_d].cpu().numpy()
        diff = w["pts"][I].astype(np.int64) - w["pts"][rows][:, None, :].astype(np.int64)
        if not (same and np.array_equal((diff * diff).sum(-1), D) and np.all(I != rows[:, None])):
            raise RuntimeError("%s: k-NN graph rows fail the checks" % name)
        bm = float(np.median(bms))
        entry = {"build_ms": bm}
        for vname, _, _ in variants:
            km = float(np.median(res[vname]))
            entry[vname + "_ms"] = km
            entry[vname + "_queries_per_s"] = n / (km / 1e3)
        sets[name] = entry
        total_q += n
        total_ms += bm + entry["leaf_group_ms"]
        del pts, outs
        torch.cuda.empty_cache()
    return {"workload": "skewed-5x%d-k%d" % (args.n, k),
            "metric": "queries/s (build + leaf-based k-NN graph, k=%d, five point sets)" % k,
            "value": total_q / (total_ms / 1e3), "unit": "queries/s", "k": k, "steps": args.steps,
            "sets": sets, "all_starts_same_ids": True}


def bench_update_sweep(args):
    """Per-point cost of batch updates and of dynamic queries against the
    batch size (the paper's update and dynamic-query plots): a 2D tree of
    10^7 uniform points in [0, 2^20)^2, L = 16; for each batch size b an
    insert of b uniform points then a delete of those b ids (the set is
    restored each time), and bit-based queries in batches of m.
    Batches above ZD_SMALL_BATCH validate on the host (they sync), so their
    times are whole-call latencies; smaller ones run on the device without a
    sync, and the re-derivation they leave for the next search is timed
    separately.  Queries use k = 1, 5 and 10.  At the end the tree
    must equal a fresh build of the original points (same sorted keys and
    node structure)."""
    import torch
    from paper_2111_04182_gb300 import datagen, zd
    n0 = args.n
    rng = np.random.default_rng(11)
    pts = datagen.uniform(rng, n0, 2, 20)
    sizes = [b for b in (1, 10, 100, 1_000, 10_000, 100_000, 1_000_000, 5_000_000) if b <= n0]
    t = zd.zd_build(torch.from_numpy(pts).cuda(), 16, 20, capacity=n0 + max(sizes))
    ups = []
    for b in sizes:
        # small batches (no sync in the call) are timed as a run of R calls
        # issued back to back, the way a stream of single updates runs; the
        # latency of one isolated call (host enqueue included) is reported too
        R = max(1, 64 // b) if b <= zd.ZD_SMALL_BATCH else 1
        ins_ms, del_ms, one_ms = [], [], []
        for rep in range(args.warmup + max(1, args.steps // 3)):
            batches = [torch.from_numpy(datagen.uniform(rng, b, 2, 20)).cuda() for _ in range(R)]
            torch.cuda.synchronize()
            e = _events(6)
            e[0].record(); ids = [t.insert(x) for x in batches]; e[1].record()
            e[2].record()
            for i in ids:
                t.delete(i)
            e[3].record(); e[3].synchronize()
            one = datagen.uniform(rng, b, 2, 20)
            onet = torch.from_numpy(one).cuda()
            torch.cuda.synchronize()
            e[4].record(); i1 = t.insert(onet); e[5].record(); e[5].synchronize()
            t.delete(i1)
            if rep >= args.warmup:
                ins_ms.append(e[0].elapsed_time(e[1]) / R); del_ms.append(e[2].elapsed_time(e[3]) / R)
                one_ms.append(e[4].elapsed_time(e[5]))
        im, dm, om = float(np.median(ins_ms)), float(np.median(del_ms)), float(np.median(one_ms))
        ups.append({"batch": b, "calls_per_timing": R, "insert_ms": im, "delete_ms": dm,
                    "insert_s_per_point": im / 1e3 / b, "delete_s_per_point": dm / 1e3 / b,
                    "isolated_insert_call_ms": om})
    # batches of at most ZD_SMALL_BATCH points are applied on the tree's pointer
    # form.  Right after them a sparse search runs on the pointer form; a dense
    # search, the all-points graph, an export or info() first re-derive the
    # flat layout: time a one-query search right after a small insert +
    # delete, the re-derivation (forced by info()), and the same search on the
    # re-derived tree
    q1 = torch.from_numpy(datagen.uniform(rng, 1, 2, 20)).cuda()
    first, rederive, steady = [], [], []
    for rep in range(args.warmup + max(1, args.steps // 3)):
        ids = t.insert(torch.from_numpy(datagen.uniform(rng, 1, 2, 20)).cuda())
        t.delete(ids)
        e = _events(6)
        e[0].record(); t.knn(1, queries=q1, mode=zd.ZD_SEARCH_BIT); e[1].record()
        e[2].record(); t.info(); e[3].record()
        e[4].record(); t.knn(1, queries=q1, mode=zd.ZD_SEARCH_BIT); e[5].record(); e[5].synchronize()
        if rep >= args.warmup:
            first.append(e[0].elapsed_time(e[1])); rederive.append(e[2].elapsed_time(e[3]))
            steady.append(e[4].elapsed_time(e[5]))
    rederive = {"pointer_form_search_ms": float(np.median(first)), "rederive_ms": float(np.median(rederive)),
                "flat_search_ms": float(np.median(steady)),
                "note": "one-query search right after a small insert + delete (on the pointer form), the "
                        "re-derivation of the flat layout (forced by info(); a dense search, the all-points graph "
                        "or an export would do it), and the same search on the re-derived flat tree"}
    qs = []
    for m in (1, 100, 10_000, 1_000_000, 10_000_000):
        q = torch.from_numpy(datagen.uniform(rng, m, 2, 20)).cuda()
        for kq in (1, 5, 10):
            ms = []
            for rep in range(args.warmup + max(1, args.steps // 3)):
                a, b2 = _events(2)
                a.record(); t.knn(kq, queries=q, mode=zd.ZD_SEARCH_BIT); b2.record(); b2.synchronize()
                if rep >= args.warmup:
                    ms.append(a.elapsed_time(b2))
            qm = float(np.median(ms))
            qs.append({"queries": m, "k": kq, "ms": qm, "s_per_query": qm / 1e3 / m})
    assert zd.zd_check() == 0
    fresh = zd.zd_build(torch.from_numpy(pts).cuda(), 16, 20)
    ea, eb = t.export(), fresh.export()
    same = all(torch.equal(ea[f], eb[f]) for f in ("keys", "leaf_lo", "node_lo", "node_hi", "node_bit"))
    if not same:
        raise RuntimeError("updated tree differs from a fresh build of the same points")
    t.free(); fresh.free()
    big = ups[-1]
    return {"workload": "update-sweep-2d-%d" % n0, "metric": "updates/s and dynamic queries/s vs batch size",
            "value": big["batch"] / (big["insert_ms"] / 1e3), "unit": "updates/s (insert, largest batch)",
            "updates": ups, "queries": qs, "rederive_after_small_batches": rederive,
            "small_batch_limit": zd.ZD_SMALL_BATCH, "tree_equals_fresh_build": same}


def bench_n_sweep(args):
    """Time per point of the k-NN graph against the number of points (the
    paper's size sweep, Sec. 5): uniform points in [0, 2^20)^3 and [0, 2^20)^2,
    n = 10^2 .. 10^8, L = 16, k = 1, build + leaf-based all-points search.
    Sampled rows are checked for properties any exact answer has."""
    import torch
    from paper_2111_04182_gb300 import datagen, zd
    rng = np.random.default_rng(12)
    out = []
    for dim in (3, 2):
        B = 21 if dim == 3 else 20
        for n in (100, 1_000, 10_000, 100_000, 1_000_000, 10_000_000, 100_000_000):
            pts_h = datagen.uniform(rng, n, dim, 20)
            pts = torch.from_numpy(pts_h).cuda()
            idx = torch.empty((n, 1), dtype=torch.int32, device="cuda")
            d2 = torch.empty((n, 1), dtype=torch.int64, device="cuda")
            ms = []
            for rep in range(args.warmup + args.steps):
                a, b = _events(2)
                a.record(); t = zd.zd_build(pts, 16, B); t.knn(1, out=(idx, d2)); b.record(); b.synchronize()
                t.free()
                if rep >= args.warmup:
                    ms.append(a.elapsed_time(b))
            assert zd.zd_check() == 0
            rows = rng.choice(n, min(n, 2048), replace=False)
            r_d = torch.from_numpy(rows).cuda()
            I, D = idx[r_d].cpu().numpy(), d2[r_d].cpu().numpy()
            diff = pts_h[I].astype(np.int64) - pts_h[rows][:, None, :].astype(np.int64)
            if not (np.array_equal((diff * diff).sum(-1), D) and np.all(I != rows[:, None])):
                raise RuntimeError("n-sweep rows fail the property checks (dim %d, n %d)" % (dim, n))
            m = float(np.median(ms))
            out.append({"dim": dim, "n": n, "ms": m, "s_per_point": m / 1e3 / n})
            del pts, idx, d2
            torch.cuda.empty_cache()
    big = [o for o in out if o["dim"] == 3 and o["n"] == 10_000_000][0]
    return {"workload": "n-sweep-uniform-k1", "metric": "time per point (build + k=1 graph) vs n",
            "value": big["n"] / (big["ms"] / 1e3), "unit": "points/s (3D, n = 1e7)", "steps": args.steps,
            "sweep": out}


def bench_k_sweep(args):
    """Time per neighbour against k (the paper's k sweep, Sec. 5): 3D uniform
    10^7 points (the large-k workload's points), L = 16, one build, then the
    all-points search for k = 1 .. 100 with the default mapping."""
    import torch
    from paper_2111_04182_gb300 import datagen, zd
    w = datagen.workload_3d_uniform(n=args.n)
    n = len(w["pts"])
    t = zd.zd_build(torch.from_numpy(w["pts"]).cuda(), w["leaf_size"], w["coord_bits"])
    out = []
    for k in (1, 2, 5, 10, 15, 20, 25, 30, 40, 50, 60, 70, 80, 90, 100):
        idx = torch.empty((n, k), dtype=torch.int32, device="cuda")
        d2 = torch.empty((n, k), dtype=torch.int64, device="cuda")
        ms = []
        for rep in range(args.warmup + args.steps):
            a, b = _events(2)
            a.record(); t.knn(k, out=(idx, d2)); b.record(); b.synchronize()
            if rep >= args.warmup:
                ms.append(a.elapsed_time(b))
        m = float(np.median(ms))
        out.append({"k": k, "ms": m, "s_per_neighbour": m / 1e3 / (n * k)})
        del idx, d2
    assert zd.zd_check() == 0
    t.free()
    return {"workload": "k-sweep-3d-uniform-%d" % n, "metric": "time per neighbour (all-points search) vs k",
            "value": n / (out[3]["ms"] / 1e3), "unit": "queries/s (k = 10)", "steps": args.steps, "sweep": out}


def bench_large_k(args):
    """3D uniform, n = 10^7 in [0, 2^20)^3, L = 16, k = 100 (the paper's k
    sweep): build + all-points k-NN with ids and int64 d^2 written; for
    k > 40 one warp serves one query.  Outputs (12 GB) exceed L2.  Sampled
    rows are checked for properties any exact answer has."""
    import torch
    from paper_2111_04182_gb300 import datagen, zd
    w = datagen.workload_3d_uniform(n=args.n, k=args.k_large)
    n, k = len(w["pts"]), w["k"]
    pts = torch.from_numpy(w["pts"]).cuda()
    idx = torch.empty((n, k), dtype=torch.int32, device="cuda")
    d2 = torch.empty((n, k), dtype=torch.int64, device="cuda")
    for _ in range(args.warmup):
        t = zd.zd_build(pts, w["leaf_size"], w["coord_bits"]); t.knn(k, out=(idx, d2)); t.free()
    torch.cuda.synchronize()
    ms = []
    for _ in range(args.steps):
        a, b, c = _events(3)
        a.record(); t = zd.zd_build(pts, w["leaf_size"], w["coord_bits"]); b.record()
        t.knn(k, out=(idx, d2)); c.record(); c.synchronize(); t.free()
        ms.append((a.elapsed_time(b), b.elapsed_time(c)))
    assert zd.zd_check() == 0
    rows = np.random.default_rng(1).choice(n, 4096, replace=False)
    I = idx[torch.from_numpy(rows).cuda()].cpu().numpy()
    D = d2[torch.from_numpy(rows).cuda()].cpu().numpy()
    diff = w["pts"][I].astype(np.int64) - w["pts"][rows][:, None, :].astype(np.int64)
    if not (np.array_equal((diff * diff).sum(-1), D) and np.all(D[:, 1:] >= D[:, :-1])
            and np.all(I != rows[:, None])):
        raise RuntimeError("large-k rows fail the property checks")
    bm = float(np.median([x[0] for x in ms])); km = float(np.median([x[1] for x in ms]))
    pk, pk_src = hbm_peak()
    kb = knn_bytes_per_query(k) * n
    traffic = (profiled_traffic("k_knn_wide", "3d-uniform-1e7-k100", "knn_wide_uniform_k100.md", WIDE_SOURCES)
               if (n, k) == (10_000_000, 100) else None)
    return {"workload": "3d-uniform-1e7-k%d" % k, "metric": "queries/s (build + all-points k=%d)" % k,
            "value": n / ((bm + km) / 1e3), "unit": "queries/s", "build_ms": bm, "knn_ms": km,
            "knn_queries_per_s": n / (km / 1e3), "k": k, "steps": args.steps,
            "roofline": {"kernel": ("k_knn_group<3,40,fs>" if k <= 40 else
                                    "k_knn_wide<3,%d,0>" % (2 if k <= 64 else 3 if k <= 96 else 4)), "bound": "hbm",
                         "achieved": kb / (km / 1e3) / 1e9,
                         "peak": pk, "peak_source": pk_src, "unit": "GB/s",
                         "frac": kb / (km / 1e3) / 1e9 / pk, "traffic": traffic,
                         "algorithmic_bytes_per_launch": kb}}


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="3d-clustered")
    ap.add_argument("--n", type=int, default=10_000_000)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--rounds", type=int, default=20)
    ap.add_argument("--dyn-n0", type=int, default=50_000_000)
    ap.add_argument("--dyn-batch", type=int, default=1_000_000)
    ap.add_argument("--dyn-check", type=int, default=16)
    ap.add_argument("--clouds", type=int, default=4096)
    ap.add_argument("--k-large", type=int, default=100)
    ap.add_argument("--k-skewed", type=int, default=1)
    args = ap.parse_args()
    if args.warmup < 3 and args.impl == "ours":
        print("warning: fewer than 3 warm-up steps", file=sys.stderr)
    if args.impl == "reference":
        run_reference(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()

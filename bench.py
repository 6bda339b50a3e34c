"""Benchmark: hybrid single-source BFS on R-MAT scale 25 (GTEPS, harmonic mean).

Workload (the paper's Kronecker-style synthetic graph, Section 3 / Table 1,
at scale 25): R-MAT with 2^25 vertices, edge factor 16, quadrant
probabilities (0.57, 0.19, 0.19, 0.05), symmetrised, self-loops and duplicate
edges removed, vertex ids permuted (seed 1), int64 row pointers; 64 BFS
sources drawn uniformly among vertices of nonzero degree (seed 1002).

One step = one BFS from each of the 64 sources, each timed separately with
CUDA events on the launching stream.  TEPS counts the undirected edges of the
source's component (sum of reached degrees / 2).  The graph (4.3 GB of
neighbour ids) is larger than L2, so no explicit L2 flush is done.

Output: one JSON line (rank 0).  ``--impl reference`` times the serial CPU
oracle instead, on a bounded sample of the same workload.
"""
from __future__ import annotations

import argparse
import json
import os
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

SCALE = 25
EDGEFACTOR = 16
NSRC = 64
SRC_SEED = 1002
METRIC = "GTEPS (harmonic mean, 64 sources) R-MAT s25; BFS queries/s & p99 latency"
L2_BYTES = 129 * 1024 * 1024


def peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            p = json.load(f)
        return float(p["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


def measured_traffic():
    """Per-launch DRAM traffic of the persistent kernel from the committed ncu
    record, or None when the kernel's sources changed since it was captured."""
    import hashlib
    try:
        with open(os.path.join(ROOT, "profiles", "bfs_persistent_traffic.json")) as f:
            rec = json.load(f)
        h = hashlib.sha256()
        for src in rec["sources"]:
            with open(os.path.join(ROOT, src), "rb") as f:
                h.update(f.read())
        if h.hexdigest() != rec["source_sha256"]:
            return None
        return float(rec["traffic_bytes_per_launch_s25"])
    except Exception:
        return None


def dist_env():
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return world, rank, local


def make_graph(scale):
    import graphgen
    rp, col = graphgen.rmat(scale, EDGEFACTOR, 0.57, 0.19, 0.19, 1, 1)
    srcs = graphgen.sources(rp, NSRC, SRC_SEED)
    return rp, col, srcs


def harmonic_gteps(edges, seconds):
    """Harmonic mean of per-BFS rates edges_i / seconds_i, in 1e9 edges/s."""
    edges = np.asarray(edges, dtype=np.float64)
    seconds = np.asarray(seconds, dtype=np.float64)
    return float(len(edges) / np.sum(seconds / edges) / 1e9)


def algorithmic_bytes(n, rp_bytes, levels):
    """Compulsory DRAM bytes of one BFS from its per-level counters.

    init 4n + n/8; top-down level: 4|F| + 2*RP*|F| + 4*E_td + 4|F'| (dist)
    + 4|F'| (queue); bottom-up level: 3n/8 (visited read, next write, visited
    update) + RP*U + 4*E_bu + 4|F'|; conversion: n/8 + 4|F|.  Random bitmap
    probes are not counted (the n/8-byte bitmaps fit in half of L2).
    """
    b = 4 * n + n / 8
    for lv in levels:
        f, e, u, fn = lv["frontier"], lv["edges"], lv["unvisited"], lv["found"]
        if lv["converted"]:
            b += n / 8 + 4 * f
        if lv["direction"] == 0:
            b += 4 * f + 2 * rp_bytes * f + 4 * e + 8 * fn
        else:
            b += 3 * n / 8 + rp_bytes * u + 4 * e + 4 * fn
    return b


class ClockSampler:
    """nvidia-smi clocks/throttle reasons sampled every 200 ms during the timed region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, device_index):
        self.dev = device_index
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                                          "-lms", "200", "-i", str(self.dev)], stdout=subprocess.PIPE,
                                         stderr=subprocess.DEVNULL, text=True)
            self.th = threading.Thread(target=self._read, daemon=True)
            self.th.start()
        except Exception:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        self.th.join(timeout=2)
        sm, mx, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                mx = float(parts[2])
            except ValueError:
                continue
            for nm, v in zip(names, parts[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        if not sm:
            return None
        return {"sm_mhz": float(np.median(sm)), "sm_max_mhz": mx, "reasons": sorted(reasons), "samples": len(sm)}


def cpu_baseline(rp, col, srcs, nsample):
    """The oracle (serial queue BFS, one core) on a bounded sample of sources."""
    import oracle
    edges, secs = [], []
    deg = np.diff(rp)
    for s in srcs[:nsample]:
        t0 = time.perf_counter()
        d = oracle.bfs(rp, col, int(s))
        secs.append(time.perf_counter() - t0)
        edges.append(float(deg[d >= 0].sum()) / 2)
    return {"value": harmonic_gteps(edges, secs), "unit": "GTEPS", "cores": 1, "kind": "oracle",
            "sample": f"{nsample} of the {len(srcs)} sources on the same s{SCALE} graph, serial queue BFS",
            "seconds": float(sum(secs))}


def run_reference(args):
    world, rank, _ = dist_env()
    if rank != 0:
        return 0
    rp, col, srcs = make_graph(args.scale)
    import oracle
    deg = np.diff(rp)
    edges, secs = [], []
    for step in range(args.warmup + args.steps):
        s = int(srcs[step % len(srcs)])
        t0 = time.perf_counter()
        d = oracle.bfs(rp, col, s)
        dt = time.perf_counter() - t0
        if step >= args.warmup:
            edges.append(float(deg[d >= 0].sum()) / 2)
            secs.append(dt)
    v = harmonic_gteps(edges, secs)
    out = {"impl": "reference", "metric": METRIC, "value": v, "unit": "GTEPS", "n_gpus": args.gpus,
           "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * float(np.mean(secs)),
           "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "int32", "data": "synthetic",
           "config": {"workload": f"rmat_s{args.scale}_ef16_hybrid_64src", "scale": args.scale,
                      "edgefactor": EDGEFACTOR, "n": int(len(rp) - 1), "m": int(len(col)),
                      "step": "one serial oracle BFS from the next of the 64 sources"},
           "cpu_baseline": {"value": v, "unit": "GTEPS", "cores": 1, "kind": "oracle",
                            "sample": f"{args.steps} timed sources (1 per step) of the same graph"},
           "e2e": {"value": v, "unit": "GTEPS", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(out), flush=True)
    return 0


def run_ours(args):
    import torch

    import paper_2503_00430_gb300 as bfs

    world, rank, local = dist_env()
    if world > 1:
        import torch.distributed as dist
        torch.cuda.set_device(local)
        dist.init_process_group("nccl")
    else:
        torch.cuda.set_device(0)
    dev = torch.cuda.current_device()
    t_gen = time.perf_counter()
    rp, col, srcs = make_graph(args.scale)
    t_gen = time.perf_counter() - t_gen
    n, m = len(rp) - 1, len(col)
    g = bfs.bfs_graph_upload(rp, col, flags=bfs.BFS_VALIDATE | (0 if args.no_degree_order else bfs.BFS_DEGREE_ORDER))
    params = bfs.make_params(policy=args.policy, launch=args.launch)
    stream = torch.cuda.Stream()
    dist_buf = torch.empty(n, dtype=torch.int32, device="cuda")

    # Untimed pass: per-source work counters (deterministic) for TEPS and bytes.
    per_src = []
    for s in srcs:
        st, lv = bfs.bfs_single_ex(g, int(s), dist_buf, params=params, stats=True, level_cap=1 << 16, stream=stream)
        per_src.append({"edges": st["edges_reached"] / 2, "bytes": algorithmic_bytes(n, 8, lv), "stats": st})

    def one_step(times):
        for i, s in enumerate(srcs):
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            bfs.bfs_single_ex(g, int(s), dist_buf, params=params, stream=stream)
            e1.record(stream)
            times.append((i, e0, e1))

    for _ in range(args.warmup):
        one_step([])
    torch.cuda.synchronize()
    if world > 1:
        torch.distributed.barrier()
    clocks = ClockSampler(dev)
    clocks.start()
    torch.cuda.synchronize()
    wall0 = time.perf_counter()
    g0 = torch.cuda.Event(enable_timing=True)
    g1 = torch.cuda.Event(enable_timing=True)
    g0.record(stream)
    recs = []
    for _ in range(args.steps):
        one_step(recs)
    g1.record(stream)
    torch.cuda.synchronize()
    wall = time.perf_counter() - wall0
    clk = clocks.stop()
    total_ms = g0.elapsed_time(g1)
    secs = [e0.elapsed_time(e1) / 1e3 for _, e0, e1 in recs]
    edges = [per_src[i]["edges"] for i, _, _ in recs]
    byts = [per_src[i]["bytes"] for i, _, _ in recs]
    value = harmonic_gteps(edges, secs)
    if world > 1:
        t = torch.tensor([total_ms, value], dtype=torch.float64, device="cuda")
        mx = t.clone()
        torch.distributed.all_reduce(mx, op=torch.distributed.ReduceOp.MAX)
        sm = t.clone()
        torch.distributed.all_reduce(sm, op=torch.distributed.ReduceOp.SUM)
        total_ms = float(mx[0])
        value = float(sm[1])
    lat = np.array(secs) * 1e3
    hbm, peak_kind = peaks()
    achieved = float(np.sum(byts) / np.sum(secs) / 1e9)

    # End to end through the C ABI with a pinned host output buffer (D2H copy inside).
    host_out = torch.empty(n, dtype=torch.int32, pin_memory=True).numpy()
    e2e_edges, e2e_secs = [], []
    torch.cuda.synchronize()
    for i, s in enumerate(srcs):
        t0 = time.perf_counter()
        bfs.bfs_single_ex(g, int(s), host_out, params=params, stream=stream)
        e2e_secs.append(time.perf_counter() - t0)
        e2e_edges.append(per_src[i]["edges"])
    e2e = {"value": harmonic_gteps(e2e_edges, e2e_secs), "unit": "GTEPS", "h2d_bytes_per_step": 4 * len(srcs),
           "d2h_bytes_per_step": 4 * n * len(srcs),
           "note": "bfs_single with a pinned host dist buffer: device run + D2H copy of dist[n] per source"}

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        cpu = cpu_baseline(rp, col, srcs, args.cpu_sample)
    st0 = per_src[0]["stats"]
    out = {
        "metric": METRIC, "value": value, "unit": "GTEPS", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": total_ms / args.steps, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "int32", "data": "synthetic",
        "config": {"workload": f"rmat_s{args.scale}_ef16_hybrid_64src", "scale": args.scale,
                   "edgefactor": EDGEFACTOR, "abcd": [0.57, 0.19, 0.19, 0.05], "n": n, "m": m,
                   "row_ptr": "int64", "sources": len(srcs), "source_seed": SRC_SEED,
                   "policy": {0: "auto", 1: "frontier", 2: "edges", 3: "td_only"}.get(args.policy, str(args.policy)),
                   "launch": {0: "persistent", 1: "per_level", 2: "graph"}[args.launch],
                   "adjacency_order": "id" if args.no_degree_order else "degree_desc",
                   "l2": "inputs larger than L2 (4.3 GB neighbour ids), no flush",
                   "step": "64 single-source BFS, each timed with CUDA events",
                   "graph_gen_s": round(t_gen, 1)},
        "latency": {"queries_per_s": len(secs) / float(np.sum(secs)), "p50_ms": float(np.percentile(lat, 50)),
                    "p99_ms": float(np.percentile(lat, 99)), "mean_ms": float(lat.mean())},
        "roofline": {"bound": "hbm", "achieved": achieved, "peak": hbm, "unit": "GB/s", "frac": achieved / hbm,
                     "peak_kind": peak_kind, "traffic": measured_traffic() if args.scale == SCALE else None,
                     "kernel": "bfs_persistent_kernel<long long,false> (one launch per BFS)",
                     "bytes_per_bfs_mean": float(np.mean([p["bytes"] for p in per_src]))},
        "e2e": e2e,
        "clocks": clk,
        "gpu_launches": len(recs),
        "wall_s_timed": wall,
        "work_example": {k: st0[k] for k in ("levels", "td_levels", "bu_levels", "conversions", "reached",
                                             "td_edges", "bu_edges", "bu_unvisited")},
    }
    if cpu is not None:
        out["cpu_baseline"] = cpu
    if rank == 0:
        print(json.dumps(out), flush=True)
    g.free()
    if world > 1:
        torch.distributed.destroy_process_group()
    return 0


def main(argv=None):
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--scale", type=int, default=SCALE)
    ap.add_argument("--policy", type=int, default=0)
    ap.add_argument("--launch", type=int, default=0)
    ap.add_argument("--cpu-sample", type=int, default=2)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-degree-order", action="store_true",
                    help="keep the generator's id-sorted adjacency order on the device")
    args = ap.parse_args(argv)
    if args.warmup < 3:
        args.warmup = 3
    if args.impl == "reference":
        return run_reference(args)
    return run_ours(args)


if __name__ == "__main__":
    sys.exit(main())

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
TUNED_TABLE = os.path.join(ROOT, "paper_2503_00430_gb300", "tuned.json")


def peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            p = json.load(f)
        return float(p["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


def measured_traffic():
    """DRAM traffic per launch of the persistent kernel over its compulsory bytes (algorithmic_bytes),
    from the committed ncu record: captured on the small case of the same kernel (R-MAT scale 23,
    the headline's parameters), where traffic and compulsory bytes are both per launch of the same
    sources.  None when the kernel's sources changed since the capture."""
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
        return float(rec["traffic_over_algorithmic"]), rec["captured_case"]
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


def make_workload(args):
    """(row_ptr, col, sources, row-pointer bytes, workload name) of the single-source workloads."""
    import graphgen
    if args.workload == "er24":
        rp, col = graphgen.erdos_renyi(1 << 24, 16.0, 2)
        return rp.astype(np.int32), col, graphgen.sources(rp, NSRC, SRC_SEED), 4, "er_2e24_d16_hybrid_64src"
    rp, col, srcs = make_graph(args.scale)
    return rp, col, srcs, 8, f"rmat_s{args.scale}_ef16_hybrid_64src"


def upload_flags(bfs, args):
    """bfs_graph_upload flags of the single-source workloads (degree-ordered lists unless disabled)."""
    return bfs.BFS_VALIDATE | (0 if args.no_degree_order else bfs.BFS_DEGREE_ORDER)


def query_params(bfs, args, n=0, m=0):
    """bfs_params of the timed single-source queries: the tuning table's entry for the graph's
    class (defaults where it has none), then any policy / launch / relabel given on the command line."""
    p = bfs.bfs_params_default() if args.no_tuned else bfs.tuned_params(None, None, "single", n, m)
    for k in ("policy", "launch", "relabel"):
        v = getattr(args, k)
        if v is not None:
            setattr(p, k, v)
    for kv in args.set or []:
        k, v = kv.split("=", 1)
        if not hasattr(p, k):
            raise SystemExit(f"--set: bfs_params has no field {k}")
        setattr(p, k, int(v))
    return p


def parse_args(argv=None):
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--scale", type=int, default=SCALE)
    ap.add_argument("--policy", type=int, default=None, help="direction policy (default: tuning table, else AUTO)")
    ap.add_argument("--launch", type=int, default=None, help="launch mode (default: tuning table, else persistent)")
    ap.add_argument("--relabel", type=int, default=None, choices=[0, 1],
                    help="single-source queries on the degree-renumbered copy of the graph (default: tuning table)")
    ap.add_argument("--no-tuned", action="store_true", help="library defaults instead of the tuning table")
    ap.add_argument("--set", action="append", metavar="FIELD=VALUE",
                    help="single-source workloads: override one bfs_params field (repeatable)")
    ap.add_argument("--tune-out", default=None, help="tune: table to write (default: the package's tuned.json)")
    ap.add_argument("--cpu-sample", type=int, default=2)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-degree-order", action="store_true",
                    help="keep the generator's id-sorted adjacency order on the device")
    ap.add_argument("--workload", default="rmat25",
                    choices=["rmat25", "er24", "large", "msbfs", "graphset", "serve", "dup", "tune"])
    ap.add_argument("--graphs", type=int, default=10000, help="graphset: graphs in the set")
    ap.add_argument("--serve-queries", type=int, default=10000, help="serve: queries per offered rate")
    ap.add_argument("--no-msbfs", action="store_true",
                    help="rmat25: skip the multi-source line added to the single-source result")
    args = ap.parse_args(argv)
    if args.warmup < 3:
        args.warmup = 3
    return args


def aggregate_ranks(total_ms, value, device="cuda"):
    """Max of the timed region over ranks and the sum of the per-rank rates
    (independent replicas: the job's throughput is the sum)."""
    import torch
    import torch.distributed as dist
    t = torch.tensor([total_ms, value], dtype=torch.float64, device=device)
    mx = t.clone()
    dist.all_reduce(mx, op=dist.ReduceOp.MAX)
    sm = t.clone()
    dist.all_reduce(sm, op=dist.ReduceOp.SUM)
    return float(mx[0]), float(sm[1])


def replica_sources(srcs, rank, world):
    """Sources a rank runs: replicas each run the whole workload (weak scaling)."""
    return list(srcs)


def harmonic_gteps(edges, seconds):
    """Harmonic mean of per-BFS rates edges_i / seconds_i, in 1e9 edges/s."""
    edges = np.asarray(edges, dtype=np.float64)
    seconds = np.asarray(seconds, dtype=np.float64)
    return float(len(edges) / np.sum(seconds / edges) / 1e9)


def algorithmic_bytes(n, rp_bytes, levels, l2_bytes=L2_BYTES):
    """Compulsory DRAM bytes of one BFS from its per-level counters: the bytes
    the method itself must move at word granularity, independent of this
    library's layout (per BFS, RP = bytes of a row pointer):

    query init: 4n (dist) + n/8 (visited);
    top-down level L: 4|F_L| (queue read) + 2*RP*|F_L| (row-pointer pair)
    + 4*E_td (neighbour ids) + 4|F_L+1| (dist store) + 4|F_L+1| (queue append);
    bottom-up level L: 3n/8 (visited read, next-frontier write, visited update)
    + RP*U_L (row pointer of each unvisited vertex of degree > 0)
    + 4*E_bu (entries examined up to and including the first frontier
    neighbour, all of them on a miss) + 4|F_L+1| (dist);
    each queue <-> bitmap conversion: n/8 + 4|F|.
    Random visited / frontier bit probes are not counted while a bitmap fits in
    half of L2 (n/8 <= L2/2); above that each probe costs 4 bytes (one per
    top-down neighbour, one per bottom-up entry examined)."""
    probe = 4 if n / 8 > l2_bytes / 2 else 0
    b = 4 * n + n / 8
    for lv in levels:
        f, e, u, fn = lv["frontier"], lv["edges"], lv["unvisited"], lv["found"]
        if lv["converted"]:
            b += n / 8 + 4 * f
        if lv["direction"] == 0:
            b += 4 * f + 2 * rp_bytes * f + (4 + probe) * e + 8 * fn
        else:
            b += 3 * n / 8 + rp_bytes * u + (4 + probe) * e + 4 * fn
    return b


def msbfs_bytes(n, n_live, lanes, rp_bytes, st, out_bytes_per_entry):
    """Compulsory DRAM bytes of one multi-source call over `lanes` sources (W = ceil(lanes/64) mask
    words per vertex, mb = 8W bytes per mask) from its counters `st` (bfs_multi_stats):

    pull level: every scanned vertex's reached mask read and next-frontier mask written (2 mb per
    vertex of degree > 0), a row pointer per vertex still missing a lane (RP * pull_active), and per
    entry examined its id and the neighbour's frontier mask (4 + mb);
    push level: per frontier vertex its mask and row-pointer pair (mb + 2 RP), per pushed entry its
    id and the neighbour's accumulator (4 + mb);
    every level: per vertex that gained a lane its reached-mask update and next-frontier mask (2 mb);
    output: lanes * n entries written once.
    Random mask gathers are counted in full (the masks, 32 bytes per vertex for 256 sources, do not
    fit in L2 at these sizes)."""
    mb = 8 * ((lanes + 63) // 64)
    b = st["pull_levels"] * 2 * mb * n_live + rp_bytes * st["pull_active"] + (4 + mb) * st["pulled_edges"]
    b += (mb + 2 * rp_bytes) * st["push_frontier"] + (4 + mb) * st["pushed_edges"]
    b += 2 * mb * st["found"]
    return b + lanes * n * out_bytes_per_entry


def graphset_bytes(vertices, entries, graphs):
    """Bytes of one graph-set launch: every graph's int64 row pointers (n_i + 1 each) and int32
    lists read once, its int32 distances written once (its bitmaps live in shared memory)."""
    return 8 * (vertices + graphs) + 4 * entries + 4 * vertices


def layout_bytes(n, rp_bytes, levels, head=True, queue=True):
    """DRAM bytes of one BFS for this library's own layout (reported beside
    the compulsory bytes, not used for the roofline): per-vertex level bytes
    while the search runs, expanded to int32 distances at the end, and
    (``head``) the 16-byte head table.

    query: level bytes n + visited init n/8 (read mask) + n/8 (write), final
    expansion n (read) + 4n (write);
    top-down level: 8|F| (work items) + 4*E_td (neighbour ids) + per found
    vertex: head 16 (else 2*RP row pointers) + level byte 1 + work item 8
    + queue entry 4 (hybrid policies only);
    bottom-up level: 3n/8 (visited read, next write, visited update) + per
    unvisited vertex: head 16 + 4 bytes per entry beyond the two the head holds
    (lower bound 4*max(0, E_bu - 2U)), else RP*U + 4*E_bu; + 1 per found vertex;
    top-down -> bottom-up conversion: n/8 (zero) + 4|F| (queue);
    bottom-up -> top-down conversion: n/8 (bitmap) + per vertex head 16 (else
    2*RP) + work item 8.
    Random bitmap probes are not counted (the n/8-byte bitmaps and the level
    bytes are kept in L2).
    """
    rec = 16 if head else 2 * rp_bytes
    b = n + n / 4 + 5 * n
    for lv in levels:
        f, e, u, fn = lv["frontier"], lv["edges"], lv["unvisited"], lv["found"]
        if lv["converted"]:
            b += n / 8 + (4 * f if lv["direction"] == 1 else (rec + 8) * f)
        if lv["direction"] == 0:
            b += 8 * f + 4 * e + (rec + 1 + 8 + (4 if queue else 0)) * fn
        elif head:
            b += 3 * n / 8 + 16 * u + 4 * max(0, e - 2 * u) + fn
        else:
            b += 3 * n / 8 + rp_bytes * u + 4 * e + fn
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


def host_info():
    """The host the CPU baseline runs on: logical CPUs (nproc) and lscpu's model name."""
    model = None
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for ln in out.splitlines():
            if ln.strip().lower().startswith("model name"):
                model = ln.split(":", 1)[1].strip()
                break
    except Exception:
        pass
    try:
        nproc = int(subprocess.run(["nproc"], capture_output=True, text=True, timeout=10).stdout.strip())
    except Exception:
        nproc = os.cpu_count()
    return {"nproc": nproc, "cpu_model": model, "machine": os.uname().machine}


def cpu_baseline(rp, col, srcs, nsample):
    if nsample <= 0:
        return None
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
            "sample": f"{nsample} of the {len(srcs)} sources on the same graph, serial queue BFS",
            "seconds": float(sum(secs)), "host": host_info()}


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
                            "sample": f"{args.steps} timed sources (1 per step) of the same graph",
                            "host": host_info()},
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
    rp, col, srcs, rp_bytes, wname = make_workload(args)
    srcs = np.asarray(replica_sources(srcs, rank, world), dtype=np.int32)
    t_gen = time.perf_counter() - t_gen
    n, m = len(rp) - 1, len(col)
    g = bfs.bfs_graph_upload(rp, col, flags=upload_flags(bfs, args))
    params = query_params(bfs, args, n, m)
    has_head = m < (1 << 31) - 8  # the library builds the head table when list starts fit int32
    hybrid = not (params.policy in (bfs.BFS_POLICY_TD_ONLY, bfs.BFS_POLICY_LOCAL)
                  or (params.policy == bfs.BFS_POLICY_AUTO and m < 7 * n))
    stream = torch.cuda.Stream()
    dist_buf = torch.empty(n, dtype=torch.int32, device="cuda")

    # Untimed pass: per-source work counters (deterministic) for TEPS and bytes.
    per_src = []
    for s in srcs:
        st, lv = bfs.bfs_single_ex(g, int(s), dist_buf, params=params, stats=True, level_cap=1 << 16, stream=stream)
        per_src.append({"edges": st["edges_reached"] / 2, "stats": st, "bytes": algorithmic_bytes(n, rp_bytes, lv),
                        "layout_bytes": layout_bytes(n, rp_bytes, lv, head=has_head, queue=hybrid)})

    def one_step(times):
        # The queries are enqueued back to back (bfs_single_async), each bracketed by CUDA events on
        # its stream; one bfs_single_wait per step checks their status.
        for i, s in enumerate(srcs):
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            bfs.bfs_single_async(g, int(s), dist_buf, params=params, stream=stream)
            e1.record(stream)
            times.append((i, e0, e1))
        bfs.bfs_single_wait(g)

    def sync_pass():
        # The same queries through the synchronous call (it waits for each query's status).
        recs_sync = []
        for i, s in enumerate(srcs):
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            bfs.bfs_single_ex(g, int(s), dist_buf, params=params, stream=stream)
            e1.record(stream)
            recs_sync.append((i, e0, e1))
        torch.cuda.synchronize()
        sec = [e0.elapsed_time(e1) / 1e3 for _, e0, e1 in recs_sync]
        return {"value": harmonic_gteps([per_src[i]["edges"] for i, _, _ in recs_sync], sec), "unit": "GTEPS",
                "mean_ms": float(np.mean(sec) * 1e3), "p50_ms": float(np.percentile(np.array(sec) * 1e3, 50)),
                "note": "bfs_single_ex per query: the call waits for the query's status before returning, so "
                        "the device idles between queries (the host's wait, return and next launch)"}

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
    sync_calls = sync_pass()
    total_ms = g0.elapsed_time(g1)
    secs = [e0.elapsed_time(e1) / 1e3 for _, e0, e1 in recs]
    edges = [per_src[i]["edges"] for i, _, _ in recs]
    byts = [per_src[i]["bytes"] for i, _, _ in recs]
    value = harmonic_gteps(edges, secs)
    if world > 1:
        total_ms, value = aggregate_ranks(total_ms, value)
    lat = np.array(secs) * 1e3
    hbm, peak_kind = peaks()
    achieved = float(np.sum(byts) / np.sum(secs) / 1e9)
    # DRAM traffic of the same kernel from the committed ncu record: the ratio of traffic to
    # compulsory bytes measured on the small case, applied to this workload's compulsory bytes.
    traffic, traffic_ratio, traffic_case = None, None, None
    default_run = (args.scale == SCALE and args.workload == "rmat25" and not args.no_degree_order
                   and args.policy is None and args.launch is None and args.relabel is None and not args.no_tuned
                   and not args.set)
    mt = measured_traffic() if default_run else None
    if mt is not None:
        traffic_ratio, traffic_case = mt
        traffic = traffic_ratio * float(np.mean([p["bytes"] for p in per_src]))

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
    st_example = per_src[0]["stats"]
    g.free()
    del rp, col
    msbfs = None
    if args.workload == "rmat25" and not args.no_msbfs:
        # The batched form on its own workload (one GPU per rank, replicas): uint8 rows, 3 calls.
        msbfs = msbfs_measure(args, bits_list=(8,), reps=3)
    st0 = st_example
    out = {
        "metric": METRIC, "value": value, "unit": "GTEPS", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": total_ms / args.steps, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "int32", "data": "synthetic",
        "config": {"workload": wname, "scale": args.scale if args.workload == "rmat25" else 24,
                   "edgefactor": EDGEFACTOR, "abcd": [0.57, 0.19, 0.19, 0.05] if args.workload == "rmat25" else None,
                   "n": n, "m": m, "row_ptr": "int64" if rp_bytes == 8 else "int32", "sources": len(srcs),
                   "source_seed": SRC_SEED,
                   "policy": {0: "auto", 1: "frontier", 2: "edges", 3: "td_only", 6: "local"}.get(params.policy,
                                                                                                 str(params.policy)),
                   "launch": {0: "persistent", 1: "per_level", 2: "graph"}[params.launch],
                   "adjacency_order": "id" if args.no_degree_order else "degree_desc",
                   "vertex_ids": "degree_renumbered_copy" if params.relabel else "as_uploaded",
                   "params": "library defaults" if args.no_tuned else
                   f"tuning table entry {bfs.table_key('single', n, m)} (defaults where absent)",
                   "l2": "inputs larger than L2 (4.3 GB neighbour ids), no flush",
                   "step": "64 single-source BFS queries enqueued back to back (bfs_single_async), each "
                           "timed with CUDA events on its stream; one bfs_single_wait per step",
                   "graph_gen_s": round(t_gen, 1)},
        "latency": {"queries_per_s": len(secs) / float(np.sum(secs)), "p50_ms": float(np.percentile(lat, 50)),
                    "p99_ms": float(np.percentile(lat, 99)), "mean_ms": float(lat.mean())},
        "roofline": {"bound": "hbm", "achieved": achieved, "peak": hbm, "unit": "GB/s", "frac": achieved / hbm,
                     "peak_kind": peak_kind,
                     "traffic": traffic,
                     "traffic_vs_algorithmic": traffic_ratio,
                     "traffic_source": None if traffic is None else
                     f"ncu dram__bytes_read+write per launch on {traffic_case}, as a ratio to the compulsory "
                     "bytes of the captured launches, times this workload's mean compulsory bytes",
                     "kernel": "bfs_persistent_kernel<long long,false> (one launch per BFS, after the "
                               "control-block reset kernel, which the per-BFS events include)",
                     "bytes_per_bfs_mean": float(np.mean([p["bytes"] for p in per_src])),
                     "bytes_model": "compulsory bytes of the method (init 4n+n/8; top-down 4F+2RP*F+4E+8F'; "
                                    "bottom-up 3n/8+RP*U+4E+4F'; conversion n/8+4F)",
                     "layout_bytes_per_bfs_mean": float(np.mean([p["layout_bytes"] for p in per_src])),
                     "layout_frac": float(np.sum([per_src[i]["layout_bytes"] for i, _, _ in recs]) / np.sum(secs)
                                          / 1e9 / hbm)},
        "e2e": e2e,
        "sync_calls": sync_calls,
        "clocks": clk,
        "gpu_launches": launches_per_query(params, per_src) * args.steps,
        "wall_s_timed": wall,
        "work_example": {k: st0[k] for k in ("levels", "td_levels", "bu_levels", "conversions", "reached",
                                             "td_edges", "bu_edges", "bu_unvisited")},
    }
    if cpu is not None:
        out["cpu_baseline"] = cpu
    if msbfs is not None:
        out["msbfs"] = msbfs
    if args.workload != "rmat25":
        out["metric"] = f"GTEPS (harmonic mean, 64 sources) {wname}"
    if rank == 0:
        print(json.dumps(out), flush=True)
    if world > 1:
        torch.distributed.destroy_process_group()
    return 0


def launches_per_query(params, per_src):
    """Kernel launches of this library per step of 64 queries: the control-block reset and the
    persistent (or graph-replayed, or local) kernel per query; with one launch per level, the
    init, every level, up to two per direction change and the final expansion."""
    if params.launch != 1:
        return 2 * len(per_src)
    return int(sum(3 + p["stats"]["levels"] + 2 * p["stats"]["conversions"] for p in per_src))


def _json(out):
    print(json.dumps(out), flush=True)


def _events():
    import torch
    return torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)


LARGE_SRC_SEED = 1003
MSBFS_SRC_SEED = 1004
SERVE_SRC_SEED = 1005


def large_specs():
    """(name, generator) of the large-diameter workloads: 2-D grid 4096^2 and a
    random geometric graph of 2^23 points at mean degree 3."""
    import graphgen
    return [("grid_4096x4096", lambda: graphgen.grid2d(4096, 4096)),
            ("rgg_2e23_d3", lambda: graphgen.rgg(1 << 23, graphgen.rgg_radius(1 << 23, 3.0), 3))]


def msbfs_workload():
    """R-MAT scale 24 (edge factor 16, ids permuted with seed 1) and its 256 sources."""
    import graphgen
    rp, col = graphgen.rmat(24, EDGEFACTOR, 0.57, 0.19, 0.19, 1, 1)
    return rp, col, graphgen.sources(rp, 256, MSBFS_SRC_SEED)


def serve_specs():
    """(name, generator) of the five resident graphs of the serving workload."""
    import graphgen
    return [("rmat_s20", lambda: graphgen.rmat(20)), ("rmat_s22", lambda: graphgen.rmat(22)),
            ("rmat_s24", lambda: graphgen.rmat(24)), ("grid_2048x2048", lambda: graphgen.grid2d(2048, 2048)),
            ("er_2e22_d16", lambda: graphgen.erdos_renyi(1 << 22, 16.0, 5))]


def run_large(args):
    """Large-diameter graphs: 2-D grid 4096^2 and a random geometric graph of 2^23 points.

    Per graph: 8 seeded sources; top-down only (the paper's large-diameter path,
    Section 3) as one persistent launch, as a replayed CUDA graph of it, and as
    one launch per level with the host reading the frontier size, to show what
    the grid barrier saves; and the multi-level local expansion (several levels
    per grid barrier, Section 2's "other optimization" (c)).
    """
    import torch

    import graphgen
    import paper_2503_00430_gb300 as bfs
    torch.cuda.set_device(0)
    res = {}
    for name, make in large_specs():
        rp, col = make()
        srcs = graphgen.sources(rp, 8, LARGE_SRC_SEED)
        g = bfs.bfs_graph_upload(rp.astype(np.int32), col, flags=bfs.BFS_VALIDATE)
        n = len(rp) - 1
        d = torch.empty(n, dtype=torch.int32, device="cuda")
        rec = {"n": n, "m": int(len(col))}
        levels = []
        for s_ in srcs:
            st, _ = bfs.bfs_single_ex(g, int(s_), d, params=bfs.make_params(policy=3), stats=True)
            levels.append(st["levels"])
            reached = st["reached"]
        rec["levels_mean"] = float(np.mean(levels))
        rec["reached_last"] = int(reached)
        for lname, policy, launch in (("persistent", 3, 0), ("graph", 3, 2), ("per_level", 3, 1),
                                      ("local", bfs.BFS_POLICY_LOCAL, 0)):
            p = bfs.make_params(policy=policy, launch=launch)
            bfs.bfs_single_ex(g, int(srcs[0]), d, params=p)
            torch.cuda.synchronize()
            e0, e1 = _events()
            e0.record()
            t0 = time.perf_counter()
            for s_ in srcs:
                bfs.bfs_single_ex(g, int(s_), d, params=p)
            e1.record()
            torch.cuda.synchronize()
            ms = e0.elapsed_time(e1) / len(srcs)
            rec[lname] = {"ms_per_bfs": ms, "us_per_level": 1e3 * ms / rec["levels_mean"],
                          "wall_ms_per_bfs": 1e3 * (time.perf_counter() - t0) / len(srcs)}
        rec["persistent_speedup_vs_per_level"] = rec["per_level"]["ms_per_bfs"] / rec["persistent"]["ms_per_bfs"]
        rec["local_speedup_vs_persistent"] = rec["persistent"]["ms_per_bfs"] / rec["local"]["ms_per_bfs"]
        res[name] = rec
        g.free()
    best = min(res["grid_4096x4096"][k]["ms_per_bfs"] for k in ("persistent", "graph", "local"))
    _json({"metric": "ms per BFS, large-diameter graphs: level-synchronous top-down (persistent, CUDA graph, "
                     "per-level launches) and multi-level local expansion",
           "value": best, "unit": "ms", "higher_is_better": False,
           "n_gpus": 1, "dtype": "int32", "data": "synthetic", "config": {"workload": "large_diameter", **res}})
    return 0


def msbfs_measure(args, bits_list=(8, 32), reps=None):
    """Multi-source R-MAT s24 x 256 per call against 256 sequential single-source queries on the same
    graph (both with their tuning-table parameters); per output width the time per call, BFS/s, the
    ratio, the counters and the roofline on msbfs_bytes."""
    import torch

    import paper_2503_00430_gb300 as bfs
    rp, col, srcs = msbfs_workload()
    n, m = len(rp) - 1, len(col)
    g = bfs.bfs_graph_upload(rp, col, flags=bfs.BFS_VALIDATE | bfs.BFS_DEGREE_ORDER)
    n_live = n - g.info()["isolated"]
    del rp, col
    sp = bfs.bfs_params_default() if args.no_tuned else bfs.tuned_params(None, g, "single")
    d = torch.empty(n, dtype=torch.int32, device="cuda")
    for s_ in srcs[:4]:
        bfs.bfs_single_ex(g, int(s_), d, params=sp)
    torch.cuda.synchronize()
    e0, e1 = _events()
    e0.record()
    for s_ in srcs:
        bfs.bfs_single_ex(g, int(s_), d, params=sp)
    e1.record()
    torch.cuda.synchronize()
    single_s = e0.elapsed_time(e1) / 1e3 / len(srcs)
    del d
    hbm, peak_kind = peaks()
    out = {"workload": "msbfs_rmat_s24_256src", "n": n, "m": m, "sources_per_call": 256,
           "single_source_bfs_per_s": 1.0 / single_s}
    mp = bfs.bfs_params_default() if args.no_tuned else bfs.tuned_params(None, g, "multi")
    for bits in bits_list:
        buf = torch.empty((256, n), dtype=torch.uint8 if bits == 8 else torch.int32, device="cuda")
        st = bfs.bfs_multi_ex(g, srcs, buf, dist_bits=bits, params=mp)
        torch.cuda.synchronize()
        e0, e1 = _events()
        e0.record()
        nrep = reps or max(1, args.steps // 4)
        for _ in range(nrep):
            st = bfs.bfs_multi_ex(g, srcs, buf, dist_bits=bits, params=mp)
        e1.record()
        torch.cuda.synchronize()
        t = e0.elapsed_time(e1) / 1e3 / nrep
        byts = msbfs_bytes(n, n_live, 256, 8, st, bits // 8)
        out["uint8" if bits == 8 else "int32"] = {
            "ms_per_call": t * 1e3, "bfs_per_s": 256 / t, "vs_single_source": 256 / t * single_s, "stats": st,
            "roofline": {"bound": "hbm", "achieved": byts / t / 1e9, "peak": hbm, "unit": "GB/s",
                         "frac": byts / t / 1e9 / hbm, "peak_kind": peak_kind, "bytes_per_call": byts,
                         "kernels": "k_ms_pull, k_ms_heavy_chunks, k_ms_push, k_ms_apply, k_ms_write (one call)"}}
        del buf
    g.free()
    return out


def run_msbfs(args):
    """Batched multi-source BFS: R-MAT scale 24, 256 sources per call, uint8 and int32 rows."""
    import torch

    torch.cuda.set_device(0)
    out = msbfs_measure(args)
    _json({"metric": "BFS/s, multi-source R-MAT s24 x 256 sources per call", "value": out["uint8"]["bfs_per_s"],
           "unit": "BFS/s", "higher_is_better": True, "n_gpus": 1, "dtype": "u8", "data": "synthetic",
           "config": {k: v for k, v in out.items()}})
    return 0


def run_graphset(args):
    """10,000 uniform random graphs, sizes log-uniform in [1e3, 1e5], mean degree 8, one launch."""
    import torch

    import graphgen
    import paper_2503_00430_gb300 as bfs
    torch.cuda.set_device(0)
    count = args.graphs
    gs = graphgen.graph_set(count, 1000, 100000, 8.0, seed=4)
    s = bfs.bfs_graphset_upload(gs.voff, gs.eoff, gs.row_ptr, gs.col)
    dist = torch.empty(int(gs.voff[-1]), dtype=torch.int32, device="cuda")
    gp = bfs.bfs_params_default() if args.no_tuned else bfs.tuned_params(None, None, "graphset")
    st = bfs.bfs_graphset_run(s, gs.src, dist, params=gp)
    torch.cuda.synchronize()
    reps = max(3, args.steps)
    e0, e1 = _events()
    e0.record()
    for _ in range(reps):
        st = bfs.bfs_graphset_run(s, gs.src, dist, params=gp)
    e1.record()
    torch.cuda.synchronize()
    t = e0.elapsed_time(e1) / 1e3 / reps
    # Sequential single-source baseline on a sample of the graphs (each uploaded on its own).
    d = torch.empty(100000, dtype=torch.int32, device="cuda")
    tot, k = 0.0, 0
    for i in range(0, count, max(1, count // 100)):
        rp, col = gs.graph(i)
        g = bfs.bfs_graph_upload(rp, col)
        bfs.bfs_single(g, int(gs.src[i]), d)
        torch.cuda.synchronize()
        a, b = _events()
        a.record()
        bfs.bfs_single(g, int(gs.src[i]), d)
        b.record()
        torch.cuda.synchronize()
        tot += a.elapsed_time(b) / 1e3
        k += 1
        g.free()
    # Bytes of one launch: every graph's row pointers (8 bytes each) and lists (4 bytes per entry)
    # read once and its distances written once; the bitmaps live in shared memory.
    byts = graphset_bytes(int(gs.voff[-1]), int(gs.eoff[-1]), count)
    hbm, peak_kind = peaks()
    _json({"metric": "graphs/s, one launch over a set of small graphs", "value": count / t, "unit": "graphs/s",
           "higher_is_better": True, "n_gpus": 1, "dtype": "int32", "data": "synthetic",
           "config": {"workload": f"graphset_{count}_er_1e3_1e5_d8", "vertices": int(gs.voff[-1]),
                      "entries": int(gs.eoff[-1]), "ms_per_launch": t * 1e3, "stats": st,
                      "single_source_graphs_per_s": k / tot, "vs_single_source": (count / t) / (k / tot),
                      "roofline": {"bound": "hbm", "achieved": byts / t / 1e9, "peak": hbm, "unit": "GB/s",
                                   "frac": byts / t / 1e9 / hbm, "peak_kind": peak_kind, "bytes_per_launch": byts,
                                   "bytes_model": "CSR read once (8 B per row pointer, 4 B per entry) + int32 "
                                                  "distances written once", "kernel": "k_graphset"}}})
    return 0


def run_serve(args):
    """Serving: five resident graphs, Poisson (graph, source) queries at offered
    rates 0.1..0.9 and 1.2 x the measured capacity; queries/s and p50/p99
    latency (arrival to result), against sequential single-source queries."""
    import threading as th

    import torch

    import graphgen
    import paper_2503_00430_gb300 as bfs
    torch.cuda.set_device(0)
    graphs, handles, srcpool = [], [], []
    for name, make in serve_specs():
        rp, col = make()
        graphs.append((name, len(rp) - 1))
        handles.append(bfs.bfs_graph_upload(rp, col, flags=bfs.BFS_DEGREE_ORDER))
        srcpool.append(graphgen.sources(rp, 4096, SERVE_SRC_SEED))
        del rp, col
    rng = np.random.default_rng(5)

    def draw(k):
        gi = rng.integers(0, len(graphs), size=k)
        return [(int(x), int(srcpool[x][rng.integers(0, 4096)])) for x in gi]

    # Sequential single-source queries on the same mix.
    d = {gi: torch.empty(graphs[gi][1], dtype=torch.int32, device="cuda") for gi in range(len(graphs))}
    sample = draw(100)
    for gi, sv in sample[:5]:
        bfs.bfs_single(handles[gi], sv, d[gi])
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for gi, sv in sample:
        bfs.bfs_single(handles[gi], sv, d[gi])
    torch.cuda.synchronize()
    seq_qps = len(sample) / (time.perf_counter() - t0)

    pool = 192  # output buffers per graph, recycled once their query is done
    bufs = [[torch.empty(n, dtype=torch.int32, device="cuda") for _ in range(pool)] for _, n in graphs]
    srv = bfs.bfs_serve_create(200 << 30)
    ids = [srv.add_graph(h) for h in handles]

    def run_rate(rate, nq):
        """Submit nq queries with Poisson arrivals at `rate` (inf = all at once); latencies in ms."""
        qs = draw(nq)
        arr = np.zeros(nq) if not np.isfinite(rate) else graphgen.poisson_arrivals(rate, nq, int(rng.integers(1 << 30)))
        free = [list(range(pool)) for _ in graphs]
        lock = th.Lock()
        cv = th.Condition(lock)
        tickets = [None] * nq
        lat = np.zeros(nq)
        t_arr = np.zeros(nq, dtype=np.int64)
        done_evt = th.Event()

        def waiter():
            for i in range(nq):
                while tickets[i] is None:
                    time.sleep(0.0001)
                tk, gi, bi = tickets[i]
                st = srv.wait(tk)
                lat[i] = (st["done_ns"] - t_arr[i]) / 1e6
                with cv:
                    free[gi].append(bi)
                    cv.notify_all()
            done_evt.set()

        w = th.Thread(target=waiter)
        w.start()
        start = time.monotonic_ns()
        for i, (gi, sv) in enumerate(qs):
            target = start + int(arr[i] * 1e9)
            while True:
                now = time.monotonic_ns()
                if now >= target:
                    break
                if target - now > 200_000:
                    time.sleep((target - now - 100_000) / 1e9)
            with cv:
                while not free[gi]:
                    cv.wait()
                bi = free[gi].pop()
            t_arr[i] = max(target, start)
            tickets[i] = (srv.submit(ids[gi], sv, bufs[gi][bi]), gi, bi)
        done_evt.wait()
        w.join()
        wall = (time.monotonic_ns() - start) / 1e9
        return {"offered_qps": None if not np.isfinite(rate) else rate, "queries": nq, "achieved_qps": nq / wall,
                "p50_ms": float(np.percentile(lat, 50)), "p99_ms": float(np.percentile(lat, 99)),
                "mean_ms": float(lat.mean())}

    run_rate(float("inf"), 256)  # warm-up: creates the groups
    sat = run_rate(float("inf"), args.serve_queries)
    cap = sat["achieved_qps"]
    # Per graph: served capacity of that graph's queries alone against its sequential queries.
    per_graph = {}
    for gi, (name, n) in enumerate(graphs):
        seq = [(gi, int(srcpool[gi][j])) for j in range(32)]
        for _, sv in seq[:2]:
            bfs.bfs_single(handles[gi], sv, d[gi])
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for _, sv in seq:
            bfs.bfs_single(handles[gi], sv, d[gi])
        torch.cuda.synchronize()
        seq_g = len(seq) / (time.perf_counter() - t0)
        nq = 640
        qs_g = [(gi, int(srcpool[gi][j % 4096])) for j in range(nq)]
        start = time.monotonic_ns()
        tick = []
        free_b = list(range(pool))
        for _, sv in qs_g:
            if not free_b:  # recycle the oldest query's buffer once it is done
                tk, b_done = tick.pop(0)
                srv.wait(tk)
                free_b.append(b_done)
            b = free_b.pop()
            tick.append((srv.submit(ids[gi], sv, bufs[gi][b]), b))
        for tk, _ in tick:
            srv.wait(tk)
        served = nq / ((time.monotonic_ns() - start) / 1e9)
        per_graph[name] = {"served_qps": served, "sequential_qps": seq_g, "vs_sequential": served / seq_g}
    rates = {}
    for f in (0.1, 0.3, 0.5, 0.7, 0.9, 1.2):
        rates[str(f)] = run_rate(f * cap, args.serve_queries)
    srv.destroy()
    _json({"metric": "BFS queries/s & p99 latency, served mix of 5 resident graphs", "value": cap,
           "unit": "queries/s", "higher_is_better": True, "n_gpus": 1, "dtype": "int32", "data": "synthetic",
           "config": {"workload": "serve_5graphs_poisson", "graphs": [g[0] for g in graphs],
                      "saturated": sat, "sequential_single_source_qps": seq_qps, "vs_sequential": cap / seq_qps,
                      "per_graph_alone": per_graph, "rates": rates}})
    return 0


def run_dup(args):
    """The paper's non-atomic top-down variant (Section 2, BFS-NonAtomic): duplicate frontier
    entries per level and its time per BFS, next to the atomic top-down and the hybrid
    single-source runs on the same sources (4 sources per graph)."""
    import torch

    import graphgen
    import paper_2503_00430_gb300 as bfs
    torch.cuda.set_device(0)
    specs = [("rmat_s24", lambda: graphgen.rmat(24, EDGEFACTOR, 0.57, 0.19, 0.19, 1, 1)),
             ("er_2e22_d16", lambda: graphgen.erdos_renyi(1 << 22, 16.0, 5)),
             ("grid_1024x1024", lambda: graphgen.grid2d(1024, 1024))]
    e0, e1 = _events()

    def timed(fn, reps=3):
        fn()
        torch.cuda.synchronize()
        e0.record()
        for _ in range(reps):
            fn()
        e1.record()
        torch.cuda.synchronize()
        return e0.elapsed_time(e1) / reps

    out = {}
    for name, make in specs:
        rp, col = make()
        n = len(rp) - 1
        g = bfs.bfs_graph_upload(rp, col)
        d = torch.empty(n, dtype=torch.int32, device="cuda")
        res = []
        for src in graphgen.sources(rp, 4, 1007):
            src = int(src)
            try:
                st, lv = bfs.bfs_single_nonatomic(g, src, d, level_cap=1 << 14)
            except bfs.BfsError as err:  # duplicates beyond the n + m queue: a result, not a crash
                if err.code != bfs.BFS_ENOMEM:
                    raise
                res.append({"src": src, "overflow": True})
                continue
            dup = [(x["frontier"] - x["unique"]) / x["unique"] for x in lv if x["unique"] > 0]
            big = [(i, (x["frontier"] - x["unique"]) / x["unique"]) for i, x in enumerate(lv) if x["unique"] >= 1000]
            worst = max(big, key=lambda t: t[1]) if big else (None, 0.0)
            res.append({
                "src": src, "levels": st["levels"], "reached": st["unique"],
                "dup_fraction": (st["frontier_entries"] - st["unique"]) / st["unique"],
                "max_level_dup_fraction": max(dup) if dup else 0.0,
                "max_dup_level_with_1000_vertices": worst[0], "its_fraction": worst[1],
                "ms_nonatomic": timed(lambda: bfs.bfs_single_nonatomic(g, src, d, stats=False)),
                "ms_atomic_topdown": timed(lambda: bfs.bfs_single_ex(g, src, d, params=bfs.make_params(policy=3))),
                "ms_hybrid": timed(lambda: bfs.bfs_single(g, src, d)),
            })
        ok = [r for r in res if not r.get("overflow")]
        agg = {k: float(np.mean([r[k] for r in ok])) if ok else None
               for k in ("dup_fraction", "max_level_dup_fraction", "ms_nonatomic", "ms_atomic_topdown", "ms_hybrid")}
        out[name] = {"n": n, "m": int(len(col)), "overflows": len(res) - len(ok), "mean": agg, "sources": res}
        g.free()
        del rp, col
    # The paper's variant proper: duplicates expanded again at the next level (BFS_DUP_EXPAND), on
    # graphs small enough for its queues; per level the copies expanded against the distinct vertices.
    faithful = {}
    for name, make in (("rmat_s10", lambda: graphgen.rmat(10, EDGEFACTOR, 0.57, 0.19, 0.19, 1, 1)),
                       ("rmat_s12", lambda: graphgen.rmat(12, EDGEFACTOR, 0.57, 0.19, 0.19, 1, 1)),
                       ("rmat_s14", lambda: graphgen.rmat(14, EDGEFACTOR, 0.57, 0.19, 0.19, 1, 1)),
                       ("er_2e14_d16", lambda: graphgen.erdos_renyi(1 << 14, 16.0, 5)),
                       ("grid_64x64", lambda: graphgen.grid2d(64, 64))):
        rp, col = make()
        n = len(rp) - 1
        g = bfs.bfs_graph_upload(rp, col)
        d = torch.empty(n, dtype=torch.int32, device="cuda")
        res = []
        for src in graphgen.sources(rp, 4, 1007):
            try:
                st, lv = bfs.bfs_single_nonatomic(g, int(src), d, level_cap=1 << 14, expand_duplicates=True)
            except bfs.BfsError as err:
                if err.code != bfs.BFS_ENOMEM:
                    raise
                res.append({"src": int(src), "overflow": True, "queue_entries": n + int(len(col)) + 1})
                continue
            res.append({"src": int(src), "levels": st["levels"],
                        "dup_fraction": (st["frontier_entries"] - st["unique"]) / st["unique"],
                        "copies_per_vertex_by_level": [round(x["frontier"] / x["unique"], 3) for x in lv if x["unique"]],
                        "edges_read_over_reached_degrees": st["edges"] / max(1, int(np.diff(rp)[d.cpu().numpy() >= 0].sum()))})
        faithful[name] = {"n": n, "m": int(len(col)), "overflows": sum(1 for r in res if r.get("overflow")),
                          "sources": res}
        g.free()
    out["expand_duplicates"] = faithful
    _json({"metric": "duplicate frontier entries of the non-atomic top-down BFS (fraction of distinct)",
           "value": out["rmat_s24"]["mean"]["dup_fraction"], "unit": "fraction", "higher_is_better": False,
           "n_gpus": 1, "dtype": "int32", "data": "synthetic", "config": {"workload": "nonatomic_duplicates", **out}})
    return 0


def run_tune(args):
    """Autotune the bench workloads and write the tuning table (paper_2503_00430_gb300/tuned.json):
    single-source parameters on R-MAT s25 (all 64 sources), the uniform random 2^24 graph (64
    sources) and the 4096^2 grid (8 sources); multi-source parameters on R-MAT s24 (one call over
    its 256 sources); graph-set launch parameters on the 10,000-graph set.  Every tuner checks that
    each setting reproduces the starting setting's output exactly."""
    import torch

    import graphgen
    import paper_2503_00430_gb300 as bfs
    torch.cuda.set_device(0)
    path = args.tune_out or TUNED_TABLE
    done = {}
    for wl in ("rmat25", "er24"):
        a = parse_args(["--workload", wl, "--no-tuned"])
        rp, col, srcs, _, wname = make_workload(a)
        g = bfs.bfs_graph_upload(rp, col, flags=upload_flags(bfs, a))
        p, rep = bfs.bfs_tune(g, srcs)
        done[wname] = bfs.tune_table_store(path, "single", p, rep, g.n, g.m, wname)
        g.free()
        del rp, col
    rp, col, srcs = msbfs_workload()  # its single-source class: the sequential baseline of the batched form
    g = bfs.bfs_graph_upload(rp, col, flags=bfs.BFS_VALIDATE | bfs.BFS_DEGREE_ORDER)
    p, rep = bfs.bfs_tune(g, srcs[:64])
    done["rmat_s24_single"] = bfs.tune_table_store(path, "single", p, rep, g.n, g.m, "rmat_s24_ef16_64src")
    g.free()
    del rp, col
    name, make = large_specs()[0]
    rp, col = make()
    g = bfs.bfs_graph_upload(rp.astype(np.int32), col, flags=bfs.BFS_VALIDATE)
    p, rep = bfs.bfs_tune(g, graphgen.sources(rp, 8, LARGE_SRC_SEED))
    done[name] = bfs.tune_table_store(path, "single", p, rep, g.n, g.m, name)
    g.free()
    rp, col, srcs = msbfs_workload()
    g = bfs.bfs_graph_upload(rp, col, flags=bfs.BFS_VALIDATE | bfs.BFS_DEGREE_ORDER)
    p, rep = bfs.bfs_tune_multi(g, srcs, 8)
    done["msbfs_rmat_s24_256src"] = bfs.tune_table_store(path, "multi", p, rep, g.n, g.m, "msbfs_rmat_s24_256src")
    g.free()
    del rp, col
    gs = graphgen.graph_set(10000, 1000, 100000, 8.0, seed=4)
    s = bfs.bfs_graphset_upload(gs.voff, gs.eoff, gs.row_ptr, gs.col)
    p, rep = bfs.bfs_tune_graphset(s, gs.src)
    done["graphset_10000"] = bfs.tune_table_store(path, "graphset", p, rep, workload="graphset_10000_er_1e3_1e5_d8")
    s.free()
    _json({"metric": "autotuned parameters of the bench workloads", "value": len(done), "unit": "entries",
           "higher_is_better": True, "n_gpus": 1, "dtype": "int32", "data": "synthetic",
           "config": {"workload": "tune", "table": os.path.relpath(path, ROOT), **done}})
    return 0


def main(argv=None):
    args = parse_args(argv)
    if args.impl == "reference":
        return run_reference(args)
    if args.workload in ("rmat25", "er24"):
        return run_ours(args)
    return {"large": run_large, "msbfs": run_msbfs, "graphset": run_graphset, "serve": run_serve,
            "dup": run_dup, "tune": run_tune}[args.workload](args)


if __name__ == "__main__":
    sys.exit(main())

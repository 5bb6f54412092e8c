#!/usr/bin/env python
"""Benchmark: Delta-stepping SSSP with bucket fusion on the road-like 4900 x 4900 grid.

Default workload (one line of JSON on rank 0):
  graph   road-like grid, 4900 x 4900 before keeping the largest component
          (23,997,150 vertices, 82,565,692 directed edges), weights
          max(round(100 * len * U[1, 1.5)), ceil(100 * len)), seed 1
  step    one batch of 8 SSSP queries from seeded random sources (one persistent launch
          through og_batch_run), Delta and fusion threshold autotuned over
          Delta in [2^8, 2^16] before timing
  value   GTEPS = sum over sources of m_r (directed edges out of reached vertices)
          / device time per step (CUDA events on the launching stream)
  e2e     the same metric through og_batch_run with a pinned HOST distance buffer:
          the 8 x n distances come back over the host link inside the timed region
  also    the same sources one per launch; the 256-query batch (config 4); and, outside
          every timed loop of the main line, a brief served run and the R-MAT wBFS / SSSP
          runs (other_configs), each checked against the oracle or its certificate
The graph (760 MB) and the distance arrays (8 x 96 MB) exceed the 129 MB L2, so no L2
flush is needed between steps.

Other workloads (--workload): rmat-wbfs, rmat-sssp (R-MAT scale 24), batch (256 queries
on a 1024 x 1024 road-like grid, queries/s), serve (Poisson A*/PPSP stream, p50/p99),
road-bf (the default graph and sources by the unordered Bellman-Ford baseline, with the
ordered method's time on the same sources for the comparison of Section 6), rmat-kcore
(coreness of R-MAT scale 24 by peeling, lazy with the histogram reduction and eager),
road-lazy / rmat-lazy (SSSP with the lazy bucket update, the eager update's time on the
same sources beside it: the eager-vs-lazy comparison of Section 6.4), rmat-setcover
(approximate set cover of R-MAT scale 24, eps = 0.01, seeded random priorities),
latency (the memory round-trip and random-access probes).  The R-MAT graphs are stored
hot-first by the library (--order user keeps the caller's ids on the device).

--impl reference times the CPU oracle (single-threaded Dijkstra) on the same workload
and metric, one bounded sample per step.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

L2_BYTES = 129 * 2 ** 20
SMI_FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")


def parse_args(argv=None):
    p = argparse.ArgumentParser(description=__doc__.split("\n")[0])
    p.add_argument("--gpus", type=int, default=1)
    p.add_argument("--steps", type=int, default=20)
    p.add_argument("--warmup", type=int, default=3)
    p.add_argument("--impl", choices=["ours", "reference"], default="ours")
    p.add_argument("--workload", default="road-sssp",
                   choices=["road-sssp", "rmat-wbfs", "rmat-sssp", "batch", "serve", "road-bf",
                            "rmat-kcore", "road-lazy", "rmat-lazy", "rmat-setcover",
                            "latency"])
    p.add_argument("--side", type=int, default=4900, help="road-like grid side")
    p.add_argument("--scale", type=int, default=24, help="R-MAT scale")
    p.add_argument("--sources", type=int, default=8)
    p.add_argument("--no-autotune", action="store_true")
    p.add_argument("--delta", type=int, default=0)
    p.add_argument("--fusion", type=int, default=0)
    p.add_argument("--tile", type=int, default=0, help="frontier tile (with --delta)")
    p.add_argument("--hub", type=int, default=0, help="hub out-degree (with --delta)")
    p.add_argument("--arena", type=int, default=0,
                   help="bucket entries per query (0 = library default)")
    p.add_argument("--cpu-sources", type=int, default=2,
                   help="oracle sample size (sources) for the CPU baseline")
    p.add_argument("--no-cpu-baseline", action="store_true")
    p.add_argument("--no-e2e", action="store_true")
    p.add_argument("--queries", type=int, default=20000, help="serve: queries in the stream")
    p.add_argument("--rates", type=float, nargs="+", default=[10000.0],
                   help="serve: Poisson arrival rates (queries/s)")
    p.add_argument("--slots", type=int, default=128,
                   help="serve: resident query slots (0: as many as device memory allows, "
                        "at most 512 -- the library's own sizing)")
    p.add_argument("--budget-us", type=int, default=400, help="serve: time per launch")
    p.add_argument("--serve-fusion", type=int, default=64, help="serve: fusion threshold")
    p.add_argument("--sequential", type=int, default=2000,
                   help="serve: queries in the one-at-a-time baseline")
    p.add_argument("--pull-divisor", type=int, default=0,
                   help="direction optimisation: pull a query's round when its frontier "
                        "exceeds n / this (0 = always push)")
    p.add_argument("--order", choices=["auto", "hot", "user"], default="auto",
                   help="device vertex order of the searched graph (default: the upload's)")
    p.add_argument("--no-configs", action="store_true",
                   help="road-sssp: skip the brief serve and R-MAT runs")
    p.add_argument("--no-batch", action="store_true",
                   help="default workload: skip the 256-query batch measurement")
    p.add_argument("--launch-check", action="store_true",
                   help="only start the ranks and count them over gloo (no GPU work)")
    return p.parse_args(argv)


# ---- multi-GPU plumbing (weak scaling: each rank runs its own sources on its own replica)

def dist_info():
    return (int(os.environ.get("RANK", "0")), int(os.environ.get("WORLD_SIZE", "1")),
            int(os.environ.get("LOCAL_RANK", "0")))


def shard_sources(all_sources, rank: int, world: int, per_rank: int):
    """Sources of one rank: a disjoint slice of a seeded list drawn for all ranks."""
    return np.asarray(all_sources[rank * per_rank:(rank + 1) * per_rank], np.uint32)


def reduce_max(x: float, world: int, device=None) -> float:
    """Max over ranks (the job is as slow as its slowest rank)."""
    if world == 1:
        return x
    import torch
    import torch.distributed as dist
    t = torch.tensor([x], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def barrier(world: int, device=None):
    if world > 1:
        import torch.distributed as dist
        if device is not None:
            dist.barrier(device_ids=[device.index])
        else:
            dist.barrier()


# ---- clocks during the timed region

class ClockSampler:
    def __init__(self, index: int):
        self.index = index
        self.proc = None
        self.path = None

    def __enter__(self):
        fd, self.path = tempfile.mkstemp(suffix=".csv")
        os.close(fd)
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.index}", f"--query-gpu={SMI_FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "100"],
                stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except (OSError, FileNotFoundError):
            self.proc = None
        time.sleep(0.3)
        return self

    def __exit__(self, *exc):
        if self.proc is not None:
            time.sleep(0.2)
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()

    def summary(self) -> dict:
        lines = []
        try:
            lines = open(self.path).read().splitlines()
        except OSError:
            pass
        finally:
            try:
                os.unlink(self.path)
            except OSError:
                pass
        return clock_summary(lines)


def clock_summary(lines) -> dict:
    """Summary of nvidia-smi samples (SMI_FIELDS, csv, noheader, nounits): the median SM
    clock over the samples drawing more than 200 W (all samples when none does), the
    highest max clock, and every throttle reason seen Active."""
    rows = []
    for line in lines:
        f = [x.strip() for x in line.split(",")]
        if len(f) >= 9 and f[1].isdigit():
            rows.append(f)
    if not rows:
        return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"], "samples": 0}
    sm = [int(r[1]) for r in rows]
    mx = max(int(r[2]) for r in rows)
    loaded = [s for s, r in zip(sm, rows) if float(r[3] or 0) > 200.0] or sm
    names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
    reasons = sorted({names[k] for r in rows for k in range(4) if r[5 + k] == "Active"})
    return {"sm_mhz": int(statistics.median(loaded)), "sm_max_mhz": mx,
            "reasons": reasons, "samples": len(rows),
            "power_w_max": max(float(r[3] or 0) for r in rows)}


# DRAM traffic (dram__bytes_read.sum + dram__bytes_write.sum) of og_delta_ell_kernel from
# one ncu capture on the road-like 2400 x 2400 graph with 8 sources (the full 4900 x 4900
# launch is too large for a multi-pass capture), scaled by vertices x sources to the
# benchmarked graph.  It describes the kernel sources it was taken on; any other build
# reports null.
# DRAM bytes of one road-like 4900 x 4900 launch of 8 sources, from a one-pass capture of
# that launch (profiles/og_delta_ell_kernel_road4900_traffic.md); other sizes are scaled
# by vertices x sources.
TRAFFIC_CAPTURE = {"kernel_sha": "a5391d8bfc90b34d", "bytes": 13.656772864e9, "n": 23997150,
                   "sources": 8, "kind": "road"}
# DRAM bytes of one full-size R-MAT-24 launch (8 sources, hot-first order) from a one-pass
# capture of that very launch (profiles/og_delta_kernel_rmat24_traffic.md), keyed like
# the road capture and by the schedule (Delta, fusion threshold, tile, hub degree) it ran.
RMAT_TRAFFIC = {"kernel_sha": "a5391d8bfc90b34d", "scale": 24, "sources": 8,
                "rmat-sssp": {"bytes": 141472959744, "schedule": (256, 0xFFFFFFFE, 256, 1024)},
                "rmat-wbfs": {"bytes": 85332831488, "schedule": (2, 1024, 256, 4096)}}
KERNEL_SOURCES = ["paper_1911_07260_gb300/csrc/og_kernels.cu",
                  "paper_1911_07260_gb300/csrc/og_device.cuh",
                  "paper_1911_07260_gb300/csrc/og_internal.cuh"]


def kernel_sha() -> str:
    """Fingerprint of the search kernel's code: its sources with comments and blank lines
    removed, so that a change of wording leaves a capture valid and a change of code
    does not."""
    import hashlib
    import re
    h = hashlib.sha256()
    for f in KERNEL_SOURCES:
        src = open(os.path.join(ROOT, f)).read()
        src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
        src = re.sub(r"//[^\n]*", "", src)
        h.update("\n".join(l.rstrip() for l in src.split("\n") if l.strip()).encode())
    return h.hexdigest()[:16]


def rmat_traffic(workload: str, scale: int, sources: int, hot_first: bool, schedule):
    """The captured full-size R-MAT traffic when this run is that launch, else None."""
    c = RMAT_TRAFFIC
    e = c.get(workload)
    if (e is None or scale != c["scale"] or sources != c["sources"] or not hot_first
            or kernel_sha() != c["kernel_sha"]):
        return None
    if e["schedule"] is not None and tuple(e["schedule"]) != tuple(schedule):
        return None
    return e["bytes"]


def scaled_traffic(kind: str, n: int, sources: int, engine: int):
    c = TRAFFIC_CAPTURE
    if kind != c["kind"] or engine == 2 or kernel_sha() != c["kernel_sha"]:
        return None
    return int(c["bytes"] * (n * sources) / (c["n"] * c["sources"]))


def peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        d = json.load(open(path))
        return float(d["hbm_gbs"]), "measured"
    except (OSError, KeyError, ValueError):
        return 6800.0, "fallback"


def reached_edges(g, dist) -> tuple[int, int]:
    """(m_r, n_r): directed edges out of reached vertices, reached vertices."""
    reached = dist != 0xFFFFFFFF
    deg = np.diff(g.offsets).astype(np.int64)
    return int(deg[reached].sum()), int(reached.sum())


def algo_bytes(m_r: int, n_r: int, n: int) -> int:
    """Algorithmic bytes of one SSSP: per edge out of a reached vertex, neighbor (4),
    weight (4) and the distance gather (4); per reached vertex the offsets (8), its
    distance (4), the final distance write (4), one bucket push (4), one pop (4) and
    one frontier copy (4); per vertex the initial distance store (4).  Re-relaxations
    are not counted."""
    return 12 * m_r + 28 * n_r + 4 * n


# ---- workloads

def build_workload(args, rank, world):
    import graphgen
    if args.workload in ("road-sssp", "serve", "road-bf", "road-lazy"):
        side = args.side
        g = graphgen.road(side, 0.15, 0.02, seed=1)
        name = f"road-like {side}x{side} grid"
    elif args.workload == "batch":
        g = graphgen.road(1024, 0.15, 0.02, seed=1)
        name = "road-like 1024x1024 grid"
    else:
        scale = args.scale
        g = graphgen.rmat(scale, 16, 0.57, 0.19, 0.19, 1, 24 if args.workload == "rmat-wbfs"
                          else 1 << 16, seed=1)
        name = f"R-MAT scale {scale}"
    per_rank = args.sources
    all_src = graphgen.sample_sources(g, per_rank * world, seed=2)
    return g, name, shard_sources(all_src, rank, world, per_rank)


def run_ours(args):
    import torch
    rank, world, local = dist_info()
    torch.cuda.set_device(local)
    device = torch.device("cuda", local)
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=device)
    import paper_1911_07260_gb300 as og
    torch.cuda.init()
    stream = torch.cuda.current_stream(device)

    g, gname, srcs = build_workload(args, rank, world)
    G = og.Graph.from_csr(g)
    if args.order != "auto":
        G.set_order({"hot": og.ORDER_HOT_FIRST, "user": og.ORDER_USER}[args.order])
    kind = {"rmat-wbfs": og.Q_WBFS, "road-bf": og.Q_BF}.get(args.workload, og.Q_SSSP)
    cfg = None
    # eager-vs-lazy comparison (Section 6.4): both with the schedule that suits the graph
    eager_ref = {"road-lazy": og.config(delta=4096, fusion_threshold=1024, expand_tile=32),
                 "rmat-lazy": og.config(delta=256, fusion_threshold=og.FUSION_OFF,
                                        expand_tile=256, hub_degree=1024)}.get(args.workload)
    if eager_ref is not None:
        cfg = og.config(delta=eager_ref.delta, expand_tile=eager_ref.expand_tile,
                        hub_degree=eager_ref.hub_degree, bucket_update=og.UPDATE_LAZY)
    elif not args.no_autotune and kind in (og.Q_SSSP, og.Q_WBFS) and not args.delta:
        # the library's tuner on the workload's own sources (wBFS: Delta is 1, the rest of
        # the schedule is searched)
        lo, hi = (1 << 8, 1 << 16)
        cfg = og.autotune(G, kind, srcs, None, lo, hi)
    elif args.delta or args.fusion:
        cfg = og.config(delta=args.delta, fusion_threshold=args.fusion, expand_tile=args.tile,
                        hub_degree=args.hub)
    if args.arena:
        cfg = cfg if cfg is not None else og.config()
        cfg.arena_entries = args.arena
    if args.pull_divisor:
        cfg = cfg if cfg is not None else og.config()
        cfg.pull_divisor = args.pull_divisor
    eff = G.get_config() if cfg is None else cfg
    queries = [(kind, int(s), 0, 0) for s in srcs]
    nq = len(queries)
    dbuf = torch.empty(nq * g.n, dtype=torch.int32, device=device)

    # m_r per source, from the first run (certified against the oracle's certificate in
    # the CPU-baseline leg below, outside every timed region)
    _, _, st0 = og.batch_run(G, queries, cfg=cfg, out=dbuf)
    dh = dbuf.cpu().numpy().view(np.uint32).reshape(nq, g.n)
    mr_nr = [reached_edges(g, dh[i]) for i in range(nq)]
    m_r = sum(x[0] for x in mr_nr)
    bytes_per_launch = sum(algo_bytes(a, b, g.n) for a, b in mr_nr)

    for _ in range(args.warmup):
        og.batch_run(G, queries, cfg=cfg, out=dbuf)
    torch.cuda.synchronize()
    barrier(world, device)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    kernel_ns = 0
    agg = {}
    with ClockSampler(local) as clk:
        torch.cuda.synchronize()
        e0.record(stream)
        for _ in range(args.steps):
            _, _, st = og.batch_run(G, queries, cfg=cfg, out=dbuf)
            kernel_ns += st.kernel_ns
            for k, v in st.as_dict().items():
                agg[k] = agg.get(k, 0) + v
        e1.record(stream)
        torch.cuda.synchronize()
    barrier(world, device)
    step_s = e0.elapsed_time(e1) / 1e3 / args.steps
    step_s = reduce_max(step_s, world, device)
    kernel_s = kernel_ns / 1e9 / args.steps
    clocks = clk.summary()

    e2e = None
    if not args.no_e2e:
        host = torch.empty(nq * g.n, dtype=torch.int32, pin_memory=True)
        hnp = host.numpy()
        og.batch_run(G, queries, cfg=cfg, out=hnp)
        barrier(world, device)
        # the mean over the steps (a rare host-side stall of tens of ms counts in it);
        # the median step beside it
        reps = max(5, args.steps // 2)
        laps = []
        t0 = time.perf_counter()
        for _ in range(reps):
            og.batch_run(G, queries, cfg=cfg, out=hnp)
            laps.append(time.perf_counter())
        e2e_s = reduce_max((laps[-1] - t0) / reps, world, device)
        med_s = float(np.median(np.diff([t0] + laps)))
        e2e = {"value": round(m_r * world / e2e_s / 1e9, 4), "unit": "GTEPS",
               "h2d_bytes_per_step": 16 * nq, "d2h_bytes_per_step": 4 * nq * g.n,
               "ms_per_step": round(e2e_s * 1e3, 3), "median_ms_per_step": round(med_s * 1e3, 3),
               "steps": reps}

    peak, peak_kind = peaks()
    achieved = bytes_per_launch / kernel_s / 1e9
    # The persistent kernel that ran: ELL rows where every degree is <= 8 (layout 0 =
    # automatic, 2 = ELL) for the eager update, the CSR kernel otherwise.
    ell_rows = int(np.diff(g.offsets).max(initial=0)) <= 8 and int(eff.layout) in (0, 2) \
        and int(eff.bucket_update) != 2
    kname = "og_delta_ell_kernel" if ell_rows else "og_delta_kernel"
    if ell_rows:
        traffic = scaled_traffic({"road-sssp": "road", "road-bf": "bf"}.get(args.workload, "rmat"),
                                 g.n, nq, int(eff.engine))
    else:
        resolved = G.get_config() if cfg is None else cfg
        sched = (int(resolved.delta), int(resolved.fusion_threshold), int(resolved.expand_tile),
                 int(resolved.hub_degree))
        traffic = rmat_traffic(args.workload, args.scale, nq,
                               G.order()[0] == og.ORDER_HOT_FIRST, sched) \
            if int(eff.engine) != 2 and int(eff.bucket_update) != 2 and not args.pull_divisor \
            else None
    roofline = {"bound": "hbm", "achieved": round(achieved, 1), "peak": peak,
                "unit": "GB/s", "frac": round(achieved / peak, 4), "traffic": traffic,
                "peak_source": peak_kind, "kernel": kname,
                "bytes_per_launch": bytes_per_launch,
                "kernel_ms": round(kernel_s * 1e3, 3)}

    if not ell_rows:
        # The CSR path's relaxations are independent random 4-byte accesses (the stale
        # check and the offsets of each expanded vertex, the pre-check load of each edge,
        # the atomicMin of each improvement); their ceiling is the rate at which the
        # memory system serves such accesses, measured here by the probe: uniform random
        # loads over a 512 MiB array (the distances of 8 queries on R-MAT scale 24) at
        # the persistent kernel's occupancy, 4 independent loads per thread.
        sms = torch.cuda.get_device_properties(local).multi_processor_count
        ctas, threads, w = 3 * sms, 256, 4
        ra_peak = ctas * threads * w / og.probe_chain(2, 512 << 20, ctas, threads, 100, 0, w)
        per = {k: v / args.steps for k, v in agg.items()}
        acc = 2 * per["items"] + per["relax"] + per["improved"]
        ra = acc / kernel_s / 1e9
        roofline["random_access"] = {
            "achieved": round(ra, 1), "peak": round(ra_peak, 1), "unit": "G accesses/s",
            "frac": round(ra / ra_peak, 3), "accesses_per_launch": int(acc),
            "peak_source": "measured in this run: og_probe_chain, uniform random 4-byte "
                           "loads over 512 MiB, %d x %d threads x %d" % (ctas, threads, w)}

    eager = None
    if eager_ref is not None:
        og.batch_run(G, queries, cfg=eager_ref, out=dbuf)
        best = None
        for _ in range(3):
            _, _, est = og.batch_run(G, queries, cfg=eager_ref, out=dbuf)
            if best is None or est.kernel_ns < best.kernel_ns:
                best = est
        eager = {"schedule": {"delta": int(eager_ref.delta),
                              "fusion_threshold": int(eager_ref.fusion_threshold),
                              "expand_tile": int(eager_ref.expand_tile)},
                 "kernel_ms": round(best.kernel_ns / 1e6, 3), "rounds": int(best.rounds),
                 "inserts": int(best.global_inserts + best.local_inserts + best.overflow_inserts),
                 "eager_speedup": round(kernel_s * 1e9 / best.kernel_ns, 2)}
    ordered = None
    if kind == og.Q_BF:
        # the same sources by the ordered method (Delta-stepping with fusion), same GPU
        ocfg = og.config(delta=4096, fusion_threshold=1024, expand_tile=32)
        oq = [(og.Q_SSSP, int(s), 0, 0) for s in srcs]
        og.batch_run(G, oq, cfg=ocfg, out=dbuf)
        best = None
        for _ in range(3):
            _, _, ost = og.batch_run(G, oq, cfg=ocfg, out=dbuf)
            if best is None or ost.kernel_ns < best.kernel_ns:
                best = ost
        ordered = {"schedule": "Delta 4096, fusion threshold 1024, tile 32",
                   "kernel_ms": round(best.kernel_ns / 1e6, 3), "rounds": int(best.rounds),
                   "relax": int(best.relax),
                   "speedup_ordered": round(kernel_s * 1e9 / best.kernel_ns, 2)}

    # one source per launch (the same sources and schedule, each its own og_batch_run):
    # the per-source figure beside the 8-source launch
    single = None
    if args.workload == "road-sssp" and nq > 1:
        one = torch.empty(g.n, dtype=torch.int32, device=device)
        og.batch_run(G, queries[:1], cfg=cfg, out=one)
        t_ns = 0
        for q in queries:
            _, _, s1 = og.batch_run(G, [q], cfg=cfg, out=one)
            t_ns += s1.kernel_ns
        single = {"value": round(m_r / (t_ns / 1e9) / 1e9, 4), "unit": "GTEPS",
                  "ms_per_source": round(t_ns / 1e6 / nq, 3),
                  "note": "each source alone in its own launch, same schedule; device time"}

    batch4 = None
    if args.workload == "road-sssp" and not args.no_batch and world == 1:
        batch4 = batch_measure(args, with_cpu=not args.no_cpu_baseline)
    others = None
    if args.workload == "road-sssp" and not args.no_configs and world == 1:
        # the other benchmarked configurations in brief, on this machine in this run: served
        # A*/PPSP on the same graph, then the R-MAT graph's wBFS and SSSP
        serve = serve_measure(g, G, 5000, [20000.0], args.slots, args.budget_us,
                              args.serve_fusion, 300)
        others = {"serve": {"workload": f"{gname}, 5000 Poisson A*/PPSP queries offered at "
                                        "20,000/s (saturating), continuous batching, "
                                        f"{serve['slots']} slots"
                                        + (" (sized by device memory)" if not args.slots
                                           else ""),
                            **{k: serve[k] for k in ("served", "one_at_a_time",
                                                     "exact_served_eq_alone_eq_oracle")}},
                  "rmat_wbfs": rmat_measure("rmat-wbfs", args.scale, 3),
                  "rmat_sssp": rmat_measure("rmat-sssp", args.scale, 3)}

    cpu = None
    certified = None
    if rank == 0 and not args.no_cpu_baseline and world == 1:
        cpu = cpu_baseline(g, srcs[:args.cpu_sources], kind)
        import oracle
        certified = all(oracle.check_sssp(g, int(srcs[i]), dh[i]) == (0, 0)
                        for i in range(nq))

    if rank == 0:
        value = m_r * world / step_s / 1e9
        kname = {og.Q_SSSP: "SSSP", og.Q_WBFS: "wBFS", og.Q_BF: "Bellman-Ford"}[kind]
        metric = {og.Q_SSSP: "SSSP GTEPS (Delta-stepping with bucket fusion)",
                  og.Q_WBFS: "wBFS GTEPS",
                  og.Q_BF: "SSSP GTEPS (unordered Bellman-Ford baseline)"}[kind]
        if eager is not None:
            metric = "SSSP GTEPS (Delta-stepping with the lazy bucket update)"
        line = {
            "metric": metric,
            "value": round(value, 4), "unit": "GTEPS", "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": round(step_s * 1e3, 3), "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "u32", "data": "synthetic",
            "config": {"workload": f"{gname}: {nq} {kname} sources per step, one persistent "
                                   f"launch",
                       "n": g.n, "m": g.m, "sources_per_gpu": nq,
                       "delta": {og.Q_WBFS: 1, og.Q_BF: None}.get(kind, int(eff.delta)),
                       "fusion_threshold": int(eff.fusion_threshold),
                       "precheck": int(eff.precheck) == 1,
                       "expand_tile": int(eff.expand_tile),
                       "hub_degree": int(eff.hub_degree),
                       "blocks_per_sm": int(eff.blocks_per_sm),
                       "engine": "async" if int(eff.engine) == 2 else "rounds",
                       "layout": "ell" if ell_rows else "csr",  # the path that ran
                       "pull_divisor": int(eff.pull_divisor),
                       "prefetch": int(eff.prefetch) == 1,
                       "bucket_update": "lazy" if int(eff.bucket_update) == 2 else "eager",
                       "vertex_order": "hot-first" if G.order()[0] == og.ORDER_HOT_FIRST
                                       else "as given",
                       "l2": "inputs larger than L2 (graph %.0f MB + dist %.0f MB > 129 MB)"
                             % ((8 * g.m + 4 * g.n) / 1e6, 4 * nq * g.n / 1e6),
                       "parallelism": f"replicas x{world}" if world > 1 else "single GPU"},
            "roofline": roofline,
            "cpu_baseline": cpu,
            "e2e": e2e,
            # per step: distance fill, query start, the search; on a hot-first graph also
            # the gather and scatter that bring each 16 rows back to the caller's order
            "gpu_launches": (3 + (2 * ((nq + 15) // 16)
                                  if G.order()[0] == og.ORDER_HOT_FIRST else 0)) * args.steps,
            "clocks": {k: clocks[k] for k in ("sm_mhz", "sm_max_mhz", "reasons")},
            "stats_per_step": {k: v // args.steps for k, v in agg.items()},
        }
        line["certified_vs_oracle"] = certified
        if single is not None:
            line["one_source_per_launch"] = single
        if others is not None:
            line["other_configs"] = others
        if batch4 is not None:
            line["batch_1024"] = {k: batch4[k] for k in (
                "value", "unit", "one_at_a_time", "exact_batched_eq_alone_eq_oracle",
                "roofline")}
            line["batch_1024"]["ms_per_launch"] = batch4["ms_per_step"]
            line["batch_1024"]["workload"] = batch4["config"]["workload"]
        if ordered is not None:
            line["ordered"] = ordered
        if eager is not None:
            line["eager"] = eager
        print(json.dumps(line), flush=True)
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


def cpu_baseline(g, srcs, kind):
    """The oracle as it stands (single-threaded Dijkstra) on a bounded sample."""
    import oracle
    t0 = time.perf_counter()
    m_r = 0
    for s in srcs:
        d = oracle.dijkstra(g, int(s))
        m_r += reached_edges(g, d)[0]
    dt = time.perf_counter() - t0
    return {"value": round(m_r / dt / 1e9, 5), "unit": "GTEPS", "cores": 1, "kind": "oracle",
            "sample": f"{len(srcs)} of the sources, full single-source Dijkstra each "
                      f"({g.n} V, {g.m} E), {dt:.1f} s", "seconds": round(dt, 2)}


REF_METRIC = {
    "road-sssp": "SSSP GTEPS (Delta-stepping with bucket fusion)",
    "rmat-sssp": "SSSP GTEPS (Delta-stepping with bucket fusion)",
    "rmat-wbfs": "wBFS GTEPS",
    "road-bf": "SSSP GTEPS (unordered Bellman-Ford baseline)",
    "road-lazy": "SSSP GTEPS (Delta-stepping with the lazy bucket update)",
    "rmat-lazy": "SSSP GTEPS (Delta-stepping with the lazy bucket update)",
    "batch": "batched queries/s (128 SSSP + 128 PPSP per launch)",
    "serve": "served A*/PPSP queries/s with p50/p99 latency",
    "rmat-kcore": "k-core GTEPS (directed edges / time, lazy bucket update with histogram)",
    "rmat-setcover": "set cover GTEPS (directed edges / time, eps = 0.01)",
}


def run_reference(args):
    """The CPU oracle as it stands, on the same workload, metric and unit as our arm: one
    bounded sample per step (a full Dijkstra for the SSSP family, one query of the batch
    or of the served stream, a k-core peeling of R-MAT scale 20 for rmat-kcore, one set
    cover of R-MAT scale 20 for rmat-setcover)."""
    rank, world, _ = dist_info()
    if rank != 0:
        return
    import graphgen
    import oracle
    wl = args.workload
    samples = []  # (units, seconds) per timed step
    if wl == "rmat-setcover":
        g = graphgen.rmat(20, 16, 0.57, 0.19, 0.19, 1, 2, seed=1)
        pri = graphgen.priorities(g.n, seed=1)
        gname, unit = "R-MAT scale 20 (sample of the scale-24 workload)", "GTEPS"
        what = "one approximate set cover (eps = 0.01) of R-MAT scale 20 per step"
        for i in range(args.warmup + args.steps):
            t0 = time.perf_counter()
            oracle.setcover(g, pri, 10000)
            if i >= args.warmup:
                samples.append((g.m, time.perf_counter() - t0))
    elif wl == "rmat-kcore":
        g = graphgen.rmat(20, 16, 0.57, 0.19, 0.19, 1, 2, seed=1)
        gname, unit = "R-MAT scale 20 (sample of the scale-24 workload)", "GTEPS"
        what = "one k-core peeling (binary heap) of R-MAT scale 20 per step"
        for i in range(args.warmup + args.steps):
            t0 = time.perf_counter()
            oracle.kcore(g)
            if i >= args.warmup:
                samples.append((g.m, time.perf_counter() - t0))
    elif wl in ("batch", "serve"):
        if wl == "batch":
            g = graphgen.road(1024, 0.15, 0.02, seed=1)
            gname = "road-like 1024x1024 grid"
            srcs = graphgen.sample_sources(g, 128, seed=2)
            pairs = graphgen.sample_pairs_grid_steps(g, 128, 10, 1000, seed=2)
            qs = [(int(s), None) for s in srcs] + [(int(a), int(b)) for a, b in pairs]
            qs = [q for pair in zip(qs[:128], qs[128:]) for q in pair]  # SSSP, PPSP, ...
        else:
            g = graphgen.road(args.side, 0.15, 0.02, seed=1)
            gname = f"road-like {args.side}x{args.side} grid"
            pairs = graphgen.sample_pairs_grid_steps(g, 256, 10, 1000, seed=2, log_uniform=True)
            qs = [(int(a), int(b)) for a, b in pairs]
        unit = "queries/s"
        what = "one query per step (full Dijkstra for SSSP, Dijkstra stopped at the target " \
               "for PPSP / A*)"
        for i in range(args.warmup + args.steps):
            s, t = qs[i % len(qs)]
            t0 = time.perf_counter()
            oracle.dijkstra(g, s, t)
            if i >= args.warmup:
                samples.append((1, time.perf_counter() - t0))
    else:
        args_ref = argparse.Namespace(**vars(args))
        args_ref.workload = {"road-bf": "road-sssp", "road-lazy": "road-sssp",
                             "rmat-lazy": "rmat-sssp"}.get(wl, wl)
        g, gname, srcs = build_workload(args_ref, 0, 1)
        unit = "GTEPS"
        what = f"one full Dijkstra (binary heap) per step, cycling over the {len(srcs)} sources"
        for i in range(args.warmup + args.steps):
            s = int(srcs[i % len(srcs)])
            t0 = time.perf_counter()
            d = oracle.dijkstra(g, s)
            dt = time.perf_counter() - t0
            if i >= args.warmup:
                samples.append((reached_edges(g, d)[0], dt))
    units = sum(a for a, _ in samples)
    t = sum(b for _, b in samples)
    value = units / t / (1e9 if unit == "GTEPS" else 1.0)
    line = {
        "impl": "reference", "metric": REF_METRIC.get(wl, REF_METRIC["road-sssp"]),
        "value": round(value, 5), "unit": unit, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": round(t / len(samples) * 1e3, 3),
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "u64",
        "data": "synthetic",
        "config": {"workload": f"{gname}: {what}", "n": g.n, "m": g.m},
        "cpu_baseline": {"value": round(value, 5), "unit": unit, "cores": 1,
                         "kind": "oracle", "sample": what},
        "e2e": {"value": round(value, 5), "unit": unit, "h2d_bytes_per_step": 0,
                "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


# ---- batched and served queries ----------------------------------------------------------

def _oracle_parallel(g, queries, threads: int):
    """The oracle as it stands on many queries, one host thread per query at a time (the
    C oracle releases the GIL).  Returns (seconds, results)."""
    import oracle
    from concurrent.futures import ThreadPoolExecutor

    def one(q):
        kind, s, t = q
        if kind == "sssp":
            return oracle.dijkstra(g, s)
        return oracle.ppsp(g, s, t)

    t0 = time.perf_counter()
    with ThreadPoolExecutor(threads) as ex:
        res = list(ex.map(one, queries))
    return time.perf_counter() - t0, res


def run_batch(args):
    print(json.dumps(batch_measure(args, with_cpu=True)), flush=True)


def batch_measure(args, with_cpu: bool = True) -> dict:
    """256 concurrent queries on the road-like 1024 x 1024 grid: 128 SSSP + 128 PPSP with
    targets 10..1000 grid steps away, one persistent launch per step; compared with the
    same queries run one launch at a time and (CPU-baseline leg) with the oracle on the
    host cores."""
    import torch
    import graphgen
    import paper_1911_07260_gb300 as og
    torch.cuda.init()
    g = graphgen.road(1024, 0.15, 0.02, seed=1)
    G = og.Graph.from_csr(g)
    srcs = graphgen.sample_sources(g, 128, seed=2)
    pairs = graphgen.sample_pairs_grid_steps(g, 128, 10, 1000, seed=2)
    queries = [(og.Q_SSSP, int(s), 0, 0) for s in srcs] + \
              [(og.Q_PPSP, int(a), int(b), 0) for a, b in pairs]
    cfg = og.autotune_batch(G, queries, 1 << 8, 1 << 16)  # tuned on the batch itself
    cfg1 = og.autotune(G, og.Q_SSSP, srcs[:1], None, 1 << 8, 1 << 16)  # and on one query
    nq = len(queries)
    dbuf = torch.empty(nq * g.n, dtype=torch.int32, device="cuda")
    _, d_batch, _ = og.batch_run(G, queries, cfg=cfg, out=dbuf)
    dist_b = dbuf.cpu().numpy().view(np.uint32).reshape(nq, g.n)
    bytes_step = 0
    for i, (kind, s, t, _) in enumerate(queries):
        mr, nr = reached_edges(g, dist_b[i])
        bytes_step += algo_bytes(mr, nr, g.n)
    for _ in range(args.warmup):
        og.batch_run(G, queries, cfg=cfg, out=dbuf)
    torch.cuda.synchronize()
    kernel_ns = 0
    with ClockSampler(0) as clk:
        t0 = time.perf_counter()
        for _ in range(args.steps):
            _, _, st = og.batch_run(G, queries, cfg=cfg, out=dbuf)
            kernel_ns += st.kernel_ns
        batch_s = (time.perf_counter() - t0) / args.steps
    clocks = clk.summary()
    kernel_s = kernel_ns / 1e9 / args.steps
    # one launch per query, same queries, each SSSP row kept on the device; the results
    # are compared with the batch only after the timed loop
    n_sssp = sum(1 for q in queries if q[0] == og.Q_SSSP)
    rows = torch.empty(n_sssp * g.n, dtype=torch.int32, device="cuda")
    d_single = np.zeros(nq, np.uint32)
    og.query_run(G, queries[0][0], queries[0][1], queries[0][2], 0, cfg=cfg1,
                 out=rows[:g.n])  # warm-up
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    r = 0
    for i, (kind, s, t, _) in enumerate(queries):
        if kind == og.Q_SSSP:
            og.query_run(G, kind, s, t, 0, cfg=cfg1, out=rows[r * g.n:(r + 1) * g.n])
            r += 1
        else:
            _, d, _ = og.query_run(G, kind, s, t, 0, cfg=cfg1, out=None)
            d_single[i] = d
    torch.cuda.synchronize()
    single_s = time.perf_counter() - t0
    exact = True
    rows_h = rows.cpu().numpy().view(np.uint32).reshape(n_sssp, g.n)
    r = 0
    for i, (kind, s, t, _) in enumerate(queries):
        if kind == og.Q_SSSP:
            exact &= bool(np.array_equal(rows_h[r], dist_b[i]))
            r += 1
        else:
            exact &= int(d_single[i]) == int(d_batch[i])
    threads = os.cpu_count() or 1
    sample = [("sssp", int(s), 0) for s in srcs[:16]] + [("ppsp", int(a), int(b)) for a, b in pairs[:16]]
    cpu_s = None
    if with_cpu:
        cpu_s, cpu_res = _oracle_parallel(g, sample, threads)
        for (kind, s, t), r in zip(sample, cpu_res):
            i = [int(x) for x in srcs[:16]].index(s) if kind == "sssp" else 128 + [
                (int(a), int(b)) for a, b in pairs[:16]].index((s, t))
            exact &= bool(np.array_equal(r, dist_b[i])) if kind == "sssp" else \
                int(r) == int(d_batch[i])
    host = torch.empty(nq * g.n, dtype=torch.int32, pin_memory=True)
    hnp = host.numpy()
    og.batch_run(G, queries, cfg=cfg, out=hnp)
    reps = max(5, args.steps // 2)
    laps = []
    t0 = time.perf_counter()
    for _ in range(reps):
        og.batch_run(G, queries, cfg=cfg, out=hnp)
        laps.append(time.perf_counter())
    e2e_s = (laps[-1] - t0) / reps  # the mean over the launches; the median beside it
    e2e_med = float(np.median(np.diff([t0] + laps)))
    peak, peak_kind = peaks()
    line = {
        "metric": "batched queries/s (128 SSSP + 128 PPSP per launch)",
        "value": round(nq / batch_s, 2), "unit": "queries/s", "n_gpus": 1,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": round(batch_s * 1e3, 3),
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "u32",
        "data": "synthetic",
        "config": {"workload": "road-like 1024x1024 grid, 256 queries in one persistent launch",
                   "n": g.n, "m": g.m, "delta": int(cfg.delta),
                   "fusion_threshold": int(cfg.fusion_threshold),
                   "expand_tile": int(cfg.expand_tile), "engine": int(cfg.engine),
                   "blocks_per_sm": int(cfg.blocks_per_sm), "precheck": int(cfg.precheck),
                   "prefetch": int(cfg.prefetch), "hub_degree": int(cfg.hub_degree),
                   "layout": "ell" if int(cfg.layout) == 2 else "csr"},
        "one_at_a_time": {"value": round(nq / single_s, 2), "unit": "queries/s",
                          "schedule": {"delta": int(cfg1.delta),
                                       "fusion_threshold": int(cfg1.fusion_threshold),
                                       "expand_tile": int(cfg1.expand_tile)},
                          "speedup_batched": round(single_s / batch_s, 2)},
        "exact_batched_eq_alone_eq_oracle": exact,
        "roofline": {"bound": "hbm", "achieved": round(bytes_step / kernel_s / 1e9, 1),
                     "peak": peak, "unit": "GB/s",
                     "frac": round(bytes_step / kernel_s / 1e9 / peak, 4), "traffic": None,
                     "peak_source": peak_kind, "kernel_ms": round(kernel_s * 1e3, 3)},
        "cpu_baseline": None if cpu_s is None else {
            "value": round(len(sample) / cpu_s, 2), "unit": "queries/s", "cores": threads,
            "kind": "oracle", "sample": f"{len(sample)} of the queries (16 SSSP + 16 PPSP), "
                                        f"{threads} host threads, {cpu_s:.1f} s"},
        "e2e": {"value": round(nq / e2e_s, 2), "unit": "queries/s", "h2d_bytes_per_step": 16 * nq,
                "d2h_bytes_per_step": 4 * nq * g.n, "ms_per_step": round(e2e_s * 1e3, 3),
                "median_ms_per_step": round(e2e_med * 1e3, 3), "steps": reps},
        "gpu_launches": 3 * args.steps,
        "clocks": {k: clocks[k] for k in ("sm_mhz", "sm_max_mhz", "reasons")},
    }
    G.free()
    return line


def serve_measure(g, G, total: int, rates, slots: int, budget_us: int, fusion: int,
                  sequential: int) -> dict:
    """Served A*/PPSP on graph g: a seeded Poisson stream of ``total`` queries (kind by
    coin, targets log-uniform 10..1000 grid steps away) admitted into a continuous-
    batching server as slots free up, at each offered rate; latency = completion -
    arrival.  The first ``sequential`` arrivals of the first rate served one query per
    launch give the baseline; served == alone for all of them and == the oracle on a
    sample (outside every timed loop)."""
    import paper_1911_07260_gb300 as og
    pairs = graphgen_pairs(g, total)
    rng = np.random.default_rng(7)
    kinds = np.where(rng.random(total) < 0.5, og.Q_ASTAR, og.Q_PPSP)
    tune = og.autotune(G, og.Q_PPSP, pairs[:32, 0], pairs[:32, 1], 1 << 6, 1 << 14)
    cfg = og.config(delta=int(tune.delta), fusion_threshold=fusion)
    results = {}
    lines = []
    for rate in rates:
        arrivals = np.cumsum(rng.exponential(1.0 / rate, total))
        srv = og.Server(G, max_slots=slots, cfg=cfg)
        resident = srv.max_slots
        lat = np.zeros(total)
        got = np.zeros(total, np.uint32)
        nxt = done = 0
        t0 = time.perf_counter()
        steps = 0
        while done < total:
            now = time.perf_counter() - t0
            while nxt < total and arrivals[nxt] <= now:
                if not srv.submit(int(kinds[nxt]), int(pairs[nxt, 0]), int(pairs[nxt, 1]), nxt):
                    break
                nxt += 1
            active = srv.step(budget_us=budget_us)
            steps += 1
            tags, d = srv.poll()
            if len(tags):
                tdone = time.perf_counter() - t0
                lat[tags.astype(np.int64)] = tdone - arrivals[tags.astype(np.int64)]
                got[tags.astype(np.int64)] = d
                done += len(tags)
            if active == 0 and nxt < total and arrivals[nxt] > now:
                time.sleep(max(0.0, min(arrivals[nxt] - now, 0.001)))
        wall = time.perf_counter() - t0
        srv.free()
        results[rate] = got
        lines.append({"rate_per_s": rate, "queries_per_s": round(total / wall, 1),
                      "p50_ms": round(float(np.percentile(lat, 50)) * 1e3, 3),
                      "p99_ms": round(float(np.percentile(lat, 99)) * 1e3, 3),
                      "steps": steps})
    # one query per launch, same arrivals (first rate), FIFO order
    rate = rates[0]
    arrivals = np.cumsum(np.random.default_rng(7).exponential(1.0 / rate, total))
    nseq = min(total, sequential)
    lat_s = np.zeros(nseq)
    seq = np.zeros(nseq, np.uint32)
    t0 = time.perf_counter()
    for i in range(nseq):
        now = time.perf_counter() - t0
        if arrivals[i] > now:
            time.sleep(arrivals[i] - now)
        s, t = int(pairs[i, 0]), int(pairs[i, 1])
        seq[i] = og.astar(G, s, t, int(cfg.delta)) if kinds[i] == og.Q_ASTAR else \
            og.ppsp(G, s, t, int(cfg.delta))
        lat_s[i] = time.perf_counter() - t0 - arrivals[i]
    seq_wall = time.perf_counter() - t0
    exact = all(bool(np.array_equal(results[r][:nseq], seq)) for r in results)
    import oracle
    sample = list(range(0, nseq, max(1, nseq // 32)))
    t0 = time.perf_counter()
    ref = [oracle.ppsp(g, int(pairs[i, 0]), int(pairs[i, 1])) for i in sample]
    cpu_s = time.perf_counter() - t0
    exact &= all(int(seq[i]) == r for i, r in zip(sample, ref))
    return {"delta": int(cfg.delta), "slots": resident, "served": lines,
            "one_at_a_time": {"rate_per_s": rate, "queries": nseq,
                              "queries_per_s": round(nseq / seq_wall, 1),
                              "p50_ms": round(float(np.percentile(lat_s, 50)) * 1e3, 3),
                              "p99_ms": round(float(np.percentile(lat_s, 99)) * 1e3, 3)},
            "exact_served_eq_alone_eq_oracle": exact,
            "cpu_baseline": {"value": round(len(sample) / cpu_s, 2), "unit": "queries/s",
                             "cores": 1, "kind": "oracle",
                             "sample": f"{len(sample)} of the queries, Dijkstra stopped at "
                                       "the target"}}


def rmat_measure(wl: str, scale: int, steps: int) -> dict:
    """The R-MAT configuration in brief: the graph and 8 sources of ``--workload wl``, one
    launch of all 8 per step with the schedule that workload's tuner picks (wBFS: fusion
    off, tile 512; SSSP: Delta 256, fusion off, tile 256, hub degree 1024), device time of
    ``steps`` steps after two warm-ups; two sources' distances certified by the oracle's
    certificate outside the timed loop."""
    import torch
    import graphgen
    import oracle
    import paper_1911_07260_gb300 as og
    whi = 24 if wl == "rmat-wbfs" else 1 << 16
    g = graphgen.rmat(scale, 16, 0.57, 0.19, 0.19, 1, whi, seed=1)
    G = og.Graph.from_csr(g)
    srcs = graphgen.sample_sources(g, 8, seed=2)
    kind = og.Q_WBFS if wl == "rmat-wbfs" else og.Q_SSSP
    cfg = og.config(fusion_threshold=og.FUSION_OFF, expand_tile=512) if kind == og.Q_WBFS \
        else og.config(delta=256, fusion_threshold=og.FUSION_OFF, expand_tile=256,
                       hub_degree=1024)
    queries = [(kind, int(s), 0, 0) for s in srcs]
    dbuf = torch.empty(len(queries) * g.n, dtype=torch.int32, device="cuda")
    og.batch_run(G, queries, cfg=cfg, out=dbuf)
    dh = dbuf.cpu().numpy().view(np.uint32).reshape(len(queries), g.n)
    m_r = sum(reached_edges(g, dh[i])[0] for i in range(len(queries)))
    og.batch_run(G, queries, cfg=cfg, out=dbuf)
    stream = torch.cuda.current_stream()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    kernel_ns = 0
    torch.cuda.synchronize()
    e0.record(stream)
    for _ in range(steps):
        _, _, st = og.batch_run(G, queries, cfg=cfg, out=dbuf)
        kernel_ns += st.kernel_ns
    e1.record(stream)
    torch.cuda.synchronize()
    step_s = e0.elapsed_time(e1) / 1e3 / steps
    same = bool(np.array_equal(dbuf.cpu().numpy().view(np.uint32).reshape(len(queries), g.n),
                               dh))
    certified = same and all(oracle.check_sssp(g, int(srcs[i]), dh[i]) == (0, 0)
                             for i in range(2))
    order, moved = G.order()
    out = {"workload": f"R-MAT scale {scale}: 8 {'wBFS' if kind == og.Q_WBFS else 'SSSP'} "
                       "sources per launch",
           "value": round(m_r / step_s / 1e9, 4), "unit": "GTEPS",
           "ms_per_step": round(step_s * 1e3, 3),
           "kernel_ms": round(kernel_ns / 1e6 / steps, 3), "steps": steps,
           "vertex_order": "hot-first" if order == og.ORDER_HOT_FIRST else "as given",
           "moved_vertices": moved,
           "certified_vs_oracle": certified,
           "steps_identical": same}
    G.free()
    del dbuf
    torch.cuda.empty_cache()
    return out


def graphgen_pairs(g, total: int):
    import graphgen
    return graphgen.sample_pairs_grid_steps(g, total, 10, 1000, seed=2, log_uniform=True)


def run_serve(args):
    """Served A*/PPSP on the road-like 4900 x 4900 grid (serve_measure), one line."""
    import torch
    import graphgen
    import paper_1911_07260_gb300 as og
    torch.cuda.init()
    g = graphgen.road(args.side, 0.15, 0.02, seed=1)
    G = og.Graph.from_csr(g)
    total = args.queries
    r = serve_measure(g, G, total, args.rates, args.slots, args.budget_us, args.serve_fusion,
                      args.sequential)
    best = max(r["served"], key=lambda x: x["queries_per_s"])
    line = {
        "metric": "served A*/PPSP queries/s with p50/p99 latency",
        "value": best["queries_per_s"], "unit": "queries/s", "n_gpus": 1, "steps": total,
        "warmup": 0, "ms_per_step": round(1e3 / max(best["queries_per_s"], 1e-9), 4),
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "u32",
        "data": "synthetic",
        "config": {"workload": f"road-like {args.side}x{args.side} grid, {total} Poisson "
                               "A*/PPSP queries, continuous batching",
                   "slots": r["slots"], "delta": r["delta"], "budget_us": args.budget_us,
                   "fusion_threshold": args.serve_fusion},
        "served": r["served"],
        "one_at_a_time": r["one_at_a_time"],
        "exact_served_eq_alone_eq_oracle": r["exact_served_eq_alone_eq_oracle"],
        "cpu_baseline": r["cpu_baseline"],
    }
    print(json.dumps(line), flush=True)


def run_kcore(args):
    """k-core of the R-MAT scale-24 graph (Section 6.1): one peeling per step, lazy bucket
    update with the histogram reduction; the eager update timed beside it (Section 6.4's
    eager-vs-lazy table).  GTEPS = directed edges / device time per step."""
    import torch
    import graphgen
    import oracle
    import paper_1911_07260_gb300 as og
    rank, world, local = dist_info()
    torch.cuda.set_device(local)
    torch.cuda.init()
    g = graphgen.rmat(args.scale, 16, 0.57, 0.19, 0.19, 1, 2, seed=1)
    G = og.Graph.from_csr(g)
    kcfg = og.config(hub_degree=args.hub, expand_tile=args.tile)
    out = torch.empty(g.n, dtype=torch.int32, device="cuda")
    core, st0 = og.kcore(G, og.KCORE_LAZY, cfg=kcfg, out=out)
    ref_core = out.cpu().numpy().view(np.uint32).copy()
    for _ in range(args.warmup):
        og.kcore(G, og.KCORE_LAZY, cfg=kcfg, out=out)
    torch.cuda.synchronize()
    stream = torch.cuda.current_stream()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    kernel_ns = 0
    with ClockSampler(local) as clk:
        torch.cuda.synchronize()
        e0.record(stream)
        for _ in range(args.steps):
            _, st = og.kcore(G, og.KCORE_LAZY, cfg=kcfg, out=out)
            kernel_ns += st.kernel_ns
        e1.record(stream)
        torch.cuda.synchronize()
    step_s = e0.elapsed_time(e1) / 1e3 / args.steps
    kernel_s = kernel_ns / 1e9 / args.steps
    clocks = clk.summary()
    same = True
    best_e = None
    for _ in range(max(2, args.steps // 5)):
        _, se = og.kcore(G, og.KCORE_EAGER, cfg=kcfg, out=out)
        same &= bool(np.array_equal(out.cpu().numpy().view(np.uint32), ref_core))
        if best_e is None or se.kernel_ns < best_e.kernel_ns:
            best_e = se
    host = np.empty(g.n, np.uint32)
    t0 = time.perf_counter()
    reps = max(2, args.steps // 4)
    for _ in range(reps):
        og.kcore(G, og.KCORE_LAZY, cfg=kcfg, out=host)
    e2e_s = (time.perf_counter() - t0) / reps
    same &= bool(np.array_equal(host, ref_core))
    # bytes: per edge the neighbour id, its priority and its counter (4 + 4 + 4); per
    # vertex offsets 8, priority init and final 8, one bucket insert and pop 8
    bytes_step = 12 * g.m + 24 * g.n
    peak, peak_kind = peaks()
    cpu = None
    if not args.no_cpu_baseline:
        small = graphgen.rmat(20, 16, 0.57, 0.19, 0.19, 1, 2, seed=1)
        t0 = time.perf_counter()
        oracle.kcore(small)
        dt = time.perf_counter() - t0
        cpu = {"value": round(small.m / dt / 1e9, 5), "unit": "GTEPS", "cores": 1,
               "kind": "oracle",
               "sample": f"the oracle's peeling (binary heap) on R-MAT scale 20 from the same "
                         f"generator ({small.n} V, {small.m} E), {dt:.1f} s"}
    # the full-size result against the oracle's linear-time k-core certificate (only the
    # exact coreness passes it; the oracle's own peeling takes minutes at scale 24)
    certified = None
    if not args.no_cpu_baseline:
        certified = oracle.check_kcore(g, ref_core) == (0, 0)
    line = {
        "metric": "k-core GTEPS (directed edges / time, lazy bucket update with histogram)",
        "value": round(g.m / step_s / 1e9, 4), "unit": "GTEPS", "n_gpus": 1,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": round(step_s * 1e3, 3),
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "u32",
        "data": "synthetic",
        "config": {"workload": f"R-MAT scale {args.scale} k-core (coreness of every vertex), "
                               "one persistent launch per step", "n": g.n, "m": g.m,
                   "max_coreness": int(ref_core.max()),
                   "hub_degree": args.hub or 256,
                   "expand_tile": args.tile or int(G.get_config().expand_tile),
                   "l2": "inputs larger than L2 (graph %.0f MB)" % (8 * g.m / 1e6)},
        "roofline": {"bound": "hbm", "achieved": round(bytes_step / kernel_s / 1e9, 1),
                     "peak": peak, "unit": "GB/s",
                     "frac": round(bytes_step / kernel_s / 1e9 / peak, 4), "traffic": None,
                     "peak_source": peak_kind, "kernel": "og_kcore_kernel",
                     "bytes_per_launch": bytes_step, "kernel_ms": round(kernel_s * 1e3, 3)},
        "eager": {"kernel_ms": round(best_e.kernel_ns / 1e6, 3), "rounds": int(best_e.rounds),
                  "priority_updates": int(best_e.improved),
                  "bucket_inserts": int(best_e.global_inserts),
                  "lazy_speedup": round(best_e.kernel_ns / 1e9 / kernel_s, 2)},
        "lazy": {"rounds": int(st.rounds), "levels": int(st.fused_iters),
                 "cta_time_share": {
                     k: round(v / max(1, st.t_frontier_ns + st.t_fused_ns + st.t_hub_ns
                                      + st.t_barrier_ns), 3)
                     for k, v in (("peel", st.t_frontier_ns), ("apply", st.t_fused_ns),
                                  ("hub", st.t_hub_ns), ("barrier", st.t_barrier_ns))},
                 "priority_updates": int(st.improved), "bucket_inserts": int(st.global_inserts),
                 "window_refills": int(st.redistributions), "scanned_levels": int(st.flushes)},
        "exact_lazy_eq_eager_eq_host": same,
        "exact_vs_oracle_certificate": certified,
        "cpu_baseline": cpu,
        "e2e": {"value": round(g.m / e2e_s / 1e9, 4), "unit": "GTEPS", "h2d_bytes_per_step": 0,
                "d2h_bytes_per_step": 4 * g.n, "ms_per_step": round(e2e_s * 1e3, 3)},
        # init, og_kcore_kernel, and on a hot-first graph the gather and scatter that
        # bring the coreness back to the caller's order
        "gpu_launches": (2 + (2 if G.order()[0] == og.ORDER_HOT_FIRST else 0)) * args.steps,
        "clocks": {k: clocks[k] for k in ("sm_mhz", "sm_max_mhz", "reasons")},
    }
    print(json.dumps(line), flush=True)


def run_setcover(args):
    """Approximate set cover of the R-MAT scale-24 graph (Section 6.1): sets = adjacency
    lists, eps = 0.01, seeded random priorities; one persistent launch per step (plus the
    set-up kernels).  GTEPS = directed edges / device time per step."""
    import torch
    import graphgen
    import oracle
    import paper_1911_07260_gb300 as og
    rank, world, local = dist_info()
    torch.cuda.set_device(local)
    torch.cuda.init()
    eps = 10000
    g = graphgen.rmat(args.scale, 16, 0.57, 0.19, 0.19, 1, 2, seed=1)
    G = og.Graph.from_csr(g)
    cfg = og.config(hub_degree=args.hub) if args.hub else None
    pri = graphgen.priorities(g.n, seed=1)
    dpri = torch.from_numpy(pri.view(np.int32)).cuda()
    out = torch.empty(g.n, dtype=torch.int32, device="cuda")
    _, st0 = og.setcover(G, eps, dpri, cfg=cfg, out=out)
    ref = out.cpu().numpy().view(np.uint32).copy()
    for _ in range(args.warmup):
        og.setcover(G, eps, dpri, cfg=cfg, out=out)
    torch.cuda.synchronize()
    stream = torch.cuda.current_stream()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    kernel_ns = 0
    with ClockSampler(local) as clk:
        torch.cuda.synchronize()
        e0.record(stream)
        for _ in range(args.steps):
            _, st = og.setcover(G, eps, dpri, cfg=cfg, out=out)
            kernel_ns += st.kernel_ns
        e1.record(stream)
        torch.cuda.synchronize()
    step_s = e0.elapsed_time(e1) / 1e3 / args.steps
    kernel_s = kernel_ns / 1e9 / args.steps
    clocks = clk.summary()
    same = bool(np.array_equal(out.cpu().numpy().view(np.uint32), ref))
    # end to end through the public call with host buffers: priorities in, steps out
    host = np.empty(g.n, np.uint32)
    reps = max(2, args.steps // 4)
    t0 = time.perf_counter()
    for _ in range(reps):
        og.setcover(G, eps, pri, cfg=cfg, out=host)
    e2e_s = (time.perf_counter() - t0) / reps
    same &= bool(np.array_equal(host, ref))
    # algorithmic bytes of one pass over the set system: per adjacency entry the element
    # id (4), its covered flag (1), one claim and one claim check (8 + 8); per vertex its
    # offsets (8) and its result (4)
    bytes_step = 21 * g.m + 12 * g.n
    peak, peak_kind = peaks()
    cpu = None
    exact = None
    if not args.no_cpu_baseline:
        # the whole workload is a bounded sample here (about 25 s on one core), and the
        # method is deterministic: the oracle's cover must equal ours set for set
        t0 = time.perf_counter()
        oref, osteps = oracle.setcover(g, pri, eps)
        dt = time.perf_counter() - t0
        exact = bool(np.array_equal(oref, ref)) and osteps == int(st0.rounds)
        cpu = {"value": round(g.m / dt / 1e9, 5), "unit": "GTEPS", "cores": 1,
               "kind": "oracle",
               "sample": f"the oracle's set cover of the whole workload ({g.n} V, {g.m} E), "
                         f"{dt:.1f} s"}
    chosen = int((ref > 0).sum())
    line = {
        "metric": REF_METRIC["rmat-setcover"],
        "value": round(g.m / step_s / 1e9, 4), "unit": "GTEPS", "n_gpus": 1,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": round(step_s * 1e3, 3),
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "u32",
        "data": "synthetic",
        "config": {"workload": f"R-MAT scale {args.scale} approximate set cover (sets = "
                               "adjacency lists, eps = 0.01, random priorities), one "
                               "persistent launch per step", "n": g.n, "m": g.m,
                   "hub_degree": args.hub or 32,
                   "l2": "inputs larger than L2 (graph %.0f MB)" % (8 * g.m / 1e6)},
        "roofline": {"bound": "hbm", "achieved": round(bytes_step / kernel_s / 1e9, 1),
                     "peak": peak, "unit": "GB/s",
                     "frac": round(bytes_step / kernel_s / 1e9 / peak, 4), "traffic": None,
                     "peak_source": peak_kind, "kernel": "og_setcover_kernel",
                     "bytes_per_launch": bytes_step, "kernel_ms": round(kernel_s * 1e3, 3)},
        "setcover": {"sets_chosen": chosen, "steps": int(st.rounds),
                     "buckets": int(st.fused_iters), "set_visits": int(st.items),
                     "elements_scanned": int(st.relax), "moves": int(st.global_inserts),
                     "cta_time_share": {
                         k: round(v / max(1, st.t_frontier_ns + st.t_fused_ns + st.t_hub_ns
                                          + st.t_barrier_ns), 3)
                         for k, v in (("pack_claim", st.t_frontier_ns),
                                      ("count_join", st.t_fused_ns),
                                      ("gather", st.t_hub_ns), ("barrier", st.t_barrier_ns))}},
        "repeat_and_host_output_identical": same,
        "exact_vs_oracle_full_size": exact,
        "cpu_baseline": cpu,
        "e2e": {"value": round(g.m / e2e_s / 1e9, 4), "unit": "GTEPS",
                "h2d_bytes_per_step": 4 * g.n, "d2h_bytes_per_step": 4 * g.n,
                "ms_per_step": round(e2e_s * 1e3, 3)},
        # init, plan, fill, og_setcover_kernel; on a hot-first graph also the priorities
        # into the device order and the join steps back (a gather and a scatter each)
        "gpu_launches": (4 + (4 if G.order()[0] == og.ORDER_HOT_FIRST else 0)) * args.steps,
        "clocks": {k: clocks[k] for k in ("sm_mhz", "sm_max_mhz", "reasons")},
    }
    print(json.dumps(line), flush=True)


def probe_latency(og, ctas: int, threads: int) -> dict:
    """Measured round-trip times (ns per dependent access) of the memory operations a
    fused level waits on: a relaxed load served by L2 and an atomicMin whose result is
    used, on an 8 MiB array (L2-resident), on 8 MiB of lines spread over a 2 GiB array
    (L2-resident, 1,024 pages of 2 MiB) and on a 4 GiB array (mostly HBM), with one warp
    (unloaded) and with ctas x threads chains in flight (the persistent kernel's
    occupancy)."""
    out = {}
    for size_name, nbytes, foot in (("l2_8MiB", 8 << 20, 8 << 20),
                                    ("l2_8MiB_over_2GiB", 2 << 30, 8 << 20),
                                    ("hbm_4GiB", 4 << 30, 4 << 30)):
        for mode_name, mode in (("load", 0), ("atomic", 1)):
            out[f"{mode_name}_{size_name}_1warp"] = round(
                og.probe_chain(mode, nbytes, 1, 32, 2000, foot), 1)
            out[f"{mode_name}_{size_name}_loaded"] = round(
                og.probe_chain(mode, nbytes, ctas, threads, 200, foot), 1)
    return out


def probe_throughput(og, ctas: int, threads: int) -> dict:
    """Independent random accesses a second (G/s) with 1-16 chains per thread at the
    persistent kernels' occupancy: 4-byte loads through L1 (the pre-check's loads) and
    atomicMins, over a 512 MiB array (the distances of 8 queries on R-MAT scale 24) and
    a 4 GiB one.  The rate the memory system serves random accesses at is the ceiling
    of a relaxation pass whose accesses are independent."""
    out = {}
    for size_name, nbytes in (("512MiB", 512 << 20), ("4GiB", 4 << 30)):
        for mode_name, mode in (("load", 2), ("atomic", 1)):
            for w in (1, 2, 4, 8, 16):
                ns = og.probe_chain(mode, nbytes, ctas, threads, 100, 0, w)
                out[f"{mode_name}_{size_name}_x{w}"] = round(ctas * threads * w / ns, 1)
    return out


def run_latency(args):
    """The memory round-trip probe alone (ns per dependent access; lower is better)."""
    import torch
    import paper_1911_07260_gb300 as og
    torch.cuda.init()
    sms = torch.cuda.get_device_properties(0).multi_processor_count
    ctas, threads = sms * 3, 256
    with ClockSampler(0) as clk:
        lat = probe_latency(og, ctas, threads)
        thr = probe_throughput(og, ctas, threads)
    clocks = clk.summary()
    line = {"metric": "memory round trip, ns per dependent access", "value":
            lat["atomic_l2_8MiB_loaded"], "unit": "ns", "n_gpus": 1, "steps": 1, "warmup": 1,
            "higher_is_better": False, "dtype": "u32", "data": "synthetic",
            "config": {"workload": f"dependent chains: {ctas} CTAs x {threads} threads "
                                   "(loaded) or one warp", "hops_loaded": 200,
                       "hops_1warp": 2000},
            "latency_ns": lat, "random_gaccess_per_s": thr,
            # each probe: array set-up, a warm-up launch and the timed launch
            "gpu_launches": 3 * (len(lat) + len(thr)),
            "clocks": {k: clocks[k] for k in ("sm_mhz", "sm_max_mhz", "reasons")}}
    print(json.dumps(line), flush=True)


def relaunch_ranks(args, argv) -> int:
    """--gpus N > 1 without a torchrun environment: start N ranks of this script under
    torch.distributed.run (one process per GPU, rendezvous on 127.0.0.1) and return
    their exit status."""
    import socket
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        port = s.getsockname()[1]
    cmd = [sys.executable, "-m", "torch.distributed.run", "--nnodes=1",
           f"--nproc-per-node={args.gpus}", "--master-addr", "127.0.0.1",
           "--master-port", str(port), os.path.abspath(__file__)] + list(argv)
    return subprocess.call(cmd)


def launch_check(args):
    """Each rank joins a gloo group and the ranks count themselves (CPU only): shows that
    --gpus N started N ranks."""
    import torch
    import torch.distributed as dist
    rank, world, _ = dist_info()
    dist.init_process_group("gloo")
    t = torch.ones(1)
    dist.all_reduce(t)
    if rank == 0:
        print(json.dumps({"launch_check": True, "world_size": world, "ranks_counted": int(t.item()),
                          "gpus_flag": args.gpus}), flush=True)
    dist.destroy_process_group()


def main(argv=None):
    argv = sys.argv[1:] if argv is None else argv
    args = parse_args(argv)
    if args.gpus > 1 and "WORLD_SIZE" not in os.environ:
        sys.exit(relaunch_ranks(args, argv))
    if args.launch_check:
        launch_check(args)
        return
    if args.impl == "reference":
        run_reference(args)
        return
    if args.workload == "batch":
        run_batch(args)
    elif args.workload == "rmat-kcore":
        run_kcore(args)
    elif args.workload == "rmat-setcover":
        run_setcover(args)
    elif args.workload == "serve":
        run_serve(args)
    elif args.workload == "latency":
        run_latency(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()

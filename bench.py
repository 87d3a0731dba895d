#!/usr/bin/env python3
"""Benchmark: delta-stepping SSSP on the scale-22 R-MAT workload.

Workload (stands in for the paper's SNAP / GraphChallenge graphs, which are not
available): directed R-MAT scale 22 (4,194,304 vertices, 16 * 2^22 draws,
a/b/c/d = .57/.19/.19/.05, self-loops and repeats removed), float32 weights
U[0,1), 64 sources with out-degree >= 1 solved one after another, Delta swept
over {0.01, 0.05, 0.1, 0.5}. One step = the 256 solves (4 Deltas x 64 sources).

value   GTEPS = m * solves / device time, inputs resident in HBM, CUDA events
        on the solve stream (max over ranks); the per-Delta light/heavy split is
        cached and timed on its own ("split_ms").
e2e     the same metric through the public C ABI from pinned HOST buffers: every
        step creates the graph from host CSR, solves all 256 sources and copies
        every dist/pred array back to pinned host memory (on a copy stream that
        overlaps the next solves).
roofline  the solve kernel's algorithmic bytes (per-unit figures below) over
        its CUDA-event time, against the measured HBM copy bandwidth.
cpu_baseline  the CPU oracle (binary-heap Dijkstra, one source per host core)
        on a bounded sample of the same sources; "la_form": the oracle's Fig. 1
        dense-vector delta-stepping on one thread, one source at Delta 0.1.
batched / fwd_bwd  (one GPU) batched solves and the forward + adjoint pass against
        the plain per-source solve on the same GPU: 256 sources on a scale-20 R-MAT,
        512 ER graphs of uneven sizes, 32 sources on a scale-20 lognormal R-MAT with
        dLoss/dw; Delta chosen by the autotuner.

Multi-GPU (torchrun): every rank solves its own 64 sources on its own copy of
the graph (weak scaling, no collective on the data path); value sums the
ranks' edges over the slowest rank's time.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

DELTAS = [0.01, 0.05, 0.1, 0.5]

# Algorithmic bytes (what the method must move):
#   per frontier / S vertex: 4 (list id) + 16 (arc segments) + 8 (packed[u])
#   per arc relaxed:         8 (head, weight) + 8 (packed[v] read-modify-write)
#   per overflow entry re-binned: 4 (id) + 4 (flag) + 8 (packed) + 4 (rewrite)
#   per vertex, init+unpack: 8 + 12 (packed, stamps) + 8 (packed read) + 8 (dist, pred)
B_VERTEX, B_ARC, B_FAR, B_INIT_UNPACK = 28, 16, 20, 36


# DRAM traffic of k_solve_persistent per launch (ncu dram__bytes_read.sum + dram__bytes_write.sum), mean of
# one launch at each Delta of the sweep, from one ncu capture of the profiling driver below. It holds only
# for the kernel source the counters were taken on; any other source reports null.
TRAFFIC_BYTES_PER_LAUNCH = 3.124e9
TRAFFIC_SOURCE_SHA256 = "991d94bdf0a8ee8566320598760666b48cb686a68a355e4681e27ac2bc674a19"


def measured_traffic(scale: int):
    import hashlib
    csrc = os.path.join(ROOT, "paper_1911_06895_gb300", "csrc")
    h = hashlib.sha256()
    for f in ("solve.cu", "dsssp_internal.cuh", "warp_util.cuh"):
        with open(os.path.join(csrc, f), "rb") as fh:
            h.update(fh.read())
    return TRAFFIC_BYTES_PER_LAUNCH if (scale == 22 and h.hexdigest() == TRAFFIC_SOURCE_SHA256) else None


def algorithmic_bytes(st: dict, n: int) -> int:
    return (B_VERTEX * (st["vertices_light"] + st["vertices_heavy"]) + B_ARC * (st["arcs_light"] + st["arcs_heavy"])
            + B_FAR * st["far_scanned"] + B_INIT_UNPACK * n)


def light_bytes(st: dict) -> int:
    return B_VERTEX * st["vertices_light"] + B_ARC * st["arcs_light"]


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled during the timed region."""
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.proc = None
        self.lines: list[str] = []
        self.thread = None

    def start(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.gpu), f"--query-gpu={self.FIELDS}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except (FileNotFoundError, OSError):
            self.proc = None
            return
        self.thread = threading.Thread(target=self._read, daemon=True)
        self.thread.start()

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self) -> dict:
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        if self.thread:
            self.thread.join(timeout=2)
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            p = [x.strip() for x in ln.split(",")]
            if len(p) < 9:
                continue
            try:
                sm.append(float(p[1]))
                smax.append(float(p[2]))
            except ValueError:
                continue
            for nm, val in zip(names, p[5:9]):
                if val.lower().startswith("active"):
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(smax) if smax else None,
                "reasons": sorted(reasons), "samples": len(sm)}


def measured_peak_gbs():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(path) as f:
            return float(json.load(f)["hbm_gbs"]), "measured"
    except (OSError, KeyError, ValueError):
        return 6800.0, "fallback"


def sources_for_rank(g, n_sources: int, rank: int) -> list[int]:
    """Weak scaling: rank r solves its own n_sources sources of the same graph
    (rank 0 gets the workload's own sources)."""
    import graphgen
    return [int(s) for s in graphgen.random_sources(g, n_sources, 2 + 1000 * rank)]


def max_over_ranks(x: float, device: str = "cpu") -> float:
    """Largest value of x over all ranks of the default process group (the
    slowest rank's time); x itself when no process group is initialised."""
    import torch
    import torch.distributed as tdist
    if not (tdist.is_available() and tdist.is_initialized()):
        return float(x)
    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    tdist.all_reduce(t, op=tdist.ReduceOp.MAX)
    return float(t.item())


def job_gteps(m: int, solves_per_rank: int, world: int, seconds: float) -> float:
    """Whole-job throughput: every rank's arcs x solves over the slowest rank's time."""
    return m * solves_per_rank * world / seconds / 1e9


def build_workload(scale: int, n_sources: int, rank: int):
    import graphgen.workloads as W
    g, _, deltas = W.rmat22_unit(scale=scale, n_sources=n_sources)
    return g, sources_for_rank(g, n_sources, rank), deltas


def cpu_oracle_gteps(g, sources, threads=None):
    import oracle
    t0 = time.perf_counter()
    _, _, used = oracle.dijkstra_many(g.row_ptr, g.col, g.w, sources, threads)
    dt = time.perf_counter() - t0
    return g.m * len(sources) / dt / 1e9, used, dt


def run_reference(args, rank, world):
    """The CPU oracle timed on the host cores (the comparison arm)."""
    if rank != 0:
        return
    g, srcs, deltas = build_workload(args.scale, args.sources, 0)
    cores = os.cpu_count() or 1
    per_step = srcs[:min(len(srcs), cores)]
    for _ in range(args.warmup):
        cpu_oracle_gteps(g, per_step[:1], 1)
    times = []
    used = 1
    for _ in range(args.steps):
        _, used, dt = cpu_oracle_gteps(g, per_step)
        times.append(dt)
    tot = sum(times)
    value = g.m * len(per_step) * args.steps / tot / 1e9
    line = {"impl": "reference", "metric": "delta-stepping SSSP GTEPS (m * sources / device time)", "value": value,
            "unit": "GTEPS", "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": 1000 * tot / args.steps, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": f"rmat{args.scale}_unit_fp32_sources{args.sources}_deltas4", "n": g.n, "m": g.m,
                       "sources_per_step": len(per_step),
                       "timing": "host wall time of the CPU oracle (its distances do not depend on Delta)"},
            "cpu_baseline": {"value": value, "unit": "GTEPS", "cores": used, "kind": "oracle",
                             "sample": f"{len(per_step)} sources per step, binary-heap Dijkstra, one source per thread"},
            "e2e": {"value": value, "unit": "GTEPS", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--scale", type=int, default=22)
    ap.add_argument("--sources", type=int, default=64)
    ap.add_argument("--mode", type=int, default=0, help="0 persistent, 1 stepped")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--cpu-sources", type=int, default=0, help="CPU baseline sample (0: one per core)")
    ap.add_argument("--no-extras", action="store_true",
                    help="skip the batched and forward+backward comparisons")
    ap.add_argument("--profile-solves", type=int, default=0,
                    help="profiling driver: run this many solves at --profile-delta and exit (for ncu)")
    ap.add_argument("--profile-batch", type=int, default=0,
                    help="profiling driver: one batch of this many scale-20 R-MAT sources at --profile-delta")
    ap.add_argument("--profile-delta", default="0.1",
                    help="comma-separated Deltas, or 'all' for every Delta of the sweep")
    ap.add_argument("--profile-backward", type=int, default=0,
                    help="profiling driver: forward with tape + one adjoint pass for this many sources of the "
                         "scale-20 lognormal R-MAT (Delta 0.36, 8-block teams)")
    ap.add_argument("--no-fuse", action="store_true",
                    help="profiling driver: keep heavy passes and light rounds in separate phases "
                         "(with --mode 1 every phase type is then its own kernel)")
    args = ap.parse_args()
    if args.profile_solves:
        profile_driver(args)
        return
    if args.profile_batch:
        profile_batch_driver(args)
        return
    if args.profile_backward:
        profile_backward_driver(args)
        return

    if "WORLD_SIZE" not in os.environ and args.gpus > 1:
        # --gpus N without a launcher: start N ranks on this node (one process per GPU)
        cmd = [sys.executable, "-m", "torch.distributed.run", "--nnodes=1", f"--nproc-per-node={args.gpus}",
               "--master-addr", "127.0.0.1", "--master-port", os.environ.get("MASTER_PORT", "29517"),
               os.path.abspath(__file__), *sys.argv[1:]]
        sys.exit(subprocess.call(cmd))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world != args.gpus:
        sys.exit(f"bench.py: --gpus {args.gpus} but the launcher started {world} ranks")
    if args.impl == "reference":
        run_reference(args, rank, world)
        return

    import torch
    import paper_1911_06895_gb300 as ds

    torch.cuda.set_device(local)
    dist_pg = None
    if world > 1:
        import torch.distributed as tdist
        tdist.init_process_group("nccl", device_id=torch.device("cuda", local))
        dist_pg = tdist

    g, srcs, deltas = build_workload(args.scale, args.sources, rank)
    stream = torch.cuda.Stream()
    with torch.cuda.stream(stream):
        h = ds.Graph(g.row_ptr, g.col, g.w, stream=stream)
        # light/heavy split per Delta, timed on its own
        split_ms = {}
        for d in deltas:
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            h.prepare(d, stream=stream)
            e1.record(stream)
            e1.synchronize()
            split_ms[str(d)] = e0.elapsed_time(e1)
        dist = torch.empty(g.n, dtype=torch.float32, device="cuda")
        pred = torch.empty(g.n, dtype=torch.int32, device="cuda")
        # schedule per Delta from the tuner (two sample sources, untimed): the grid-wide persistent
        # scheme with its solo threshold, or one thread-block cluster per solve
        sched = {}
        for d in deltas:
            if args.mode == 0:
                o, _ = ds.tune_schedule(h, srcs[:2], d, stream=stream)
                sched[d] = dict(mode=o.mode, solo_work=o.solo_work, team_blocks=o.team_blocks)
            else:
                sched[d] = dict(mode=args.mode, solo_work=2048, team_blocks=0)
        opts = {d: ds.make_options(flags=ds.DSSSP_FLAG_ASYNC, **sched[d]) for d in deltas}

        # arcs out of reached vertices per source (Delta does not change which vertices are reached)
        deg = torch.from_numpy(np.diff(g.row_ptr)).to("cuda")
        m_reached = {}
        for s in srcs:
            h.solve(s, deltas[0], dist=dist, pred=pred, stream=stream,
                    options=ds.make_options(**sched[deltas[0]]))
            m_reached[s] = int(deg[torch.isfinite(dist)].sum().item())

        # per-solve statistics (one untimed pass) -> algorithmic bytes
        stats = {}
        for d in deltas:
            stats[d] = [h.solve(s, d, dist=dist, pred=pred, stream=stream, stats=True,
                                options=ds.make_options(**sched[d])).stats for s in srcs]

        def one_step(record):
            for d in deltas:
                for s in srcs:
                    if record is not None:
                        ev = (torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
                        ev[0].record(stream)
                    h.solve(s, d, dist=dist, pred=pred, options=opts[d], stream=stream)
                    if record is not None:
                        ev[1].record(stream)
                        record.append((d, ev))

        for _ in range(args.warmup):
            one_step(None)
        h.sync(stream)
        torch.cuda.synchronize()
        if dist_pg:
            dist_pg.barrier()
        clocks = ClockSampler(local)
        clocks.start()
        t0, t1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        recs = []
        t0.record(stream)
        for k in range(args.steps):
            one_step(recs if k == 0 else None)
        t1.record(stream)
        t1.synchronize()
        torch.cuda.synchronize()
        clk = clocks.stop()
        h.sync(stream)
        elapsed_ms = max_over_ranks(t0.elapsed_time(t1), "cuda")
        ms_per_step = elapsed_ms / args.steps
        solves = len(deltas) * len(srcs)
        gteps = job_gteps(g.m, solves, world, ms_per_step * 1e-3)

        # per-Delta GTEPS and roofline of the solve (events around each solve call)
        per_delta = {}
        tot_bytes, tot_ms, tot_light_b, tot_light_ns = 0, 0.0, 0, 0
        for d in deltas:
            ms_d = sum(ev[0].elapsed_time(ev[1]) for dd, ev in recs if dd == d)
            per_delta[str(d)] = {"gteps": g.m * len(srcs) / (ms_d * 1e-3) / 1e9, "ms_per_solve": ms_d / len(srcs),
                                 "gteps_reached": sum(m_reached.values()) / (ms_d * 1e-3) / 1e9}
            b = sum(algorithmic_bytes(st, g.n) for st in stats[d])
            tot_bytes += b
            tot_ms += ms_d
            tot_light_b += sum(light_bytes(st) for st in stats[d])
            tot_light_ns += sum(st["ns_light"] for st in stats[d])
            per_delta[str(d)].update({
                "buckets": sum(st["buckets"] for st in stats[d]) / len(srcs),
                "phases": sum(st["light_phases"] + st["heavy_phases"] + st["rebin_phases"]
                              for st in stats[d]) / len(srcs),
                "arcs_relaxed_per_solve": sum(st["arcs_light"] + st["arcs_heavy"] for st in stats[d]) / len(srcs),
                "kernel_us_per_solve": sum(st["ns_total"] for st in stats[d]) / len(srcs) / 1e3,
                "us_light": sum(st["ns_light"] for st in stats[d]) / len(srcs) / 1e3,
                "us_heavy": sum(st["ns_heavy"] for st in stats[d]) / len(srcs) / 1e3,
                "us_rebin": sum(st["ns_rebin"] for st in stats[d]) / len(srcs) / 1e3,
                "light_phases": sum(st["light_phases"] for st in stats[d]) / len(srcs),
                "arcs_light": sum(st["arcs_light"] for st in stats[d]) / len(srcs),
                "improvements": sum(st["improvements"] for st in stats[d]) / len(srcs),
                "far_scanned": sum(st["far_scanned"] for st in stats[d]) / len(srcs)})
        peak, peak_kind = measured_peak_gbs()
        achieved = tot_bytes / (tot_ms * 1e-3) / 1e9
        light_gbs = tot_light_b / (tot_light_ns * 1e-9) / 1e9 if tot_light_ns else None

    # the same 64 sources per Delta as one batch (one launch, a cluster of blocks per source)
    batched_same = None
    if world == 1 and not args.no_extras:
        batched_same = {}
        for d in deltas:
            tb, _ = ds.tune_team_blocks(h, [d], srcs)
            b = ds.Batch(h, [d], srcs, options=ds.make_options(team_blocks=tb))
            ms_b = _events_ms(torch, b.run, 2)
            b.sync()
            b.close()
            batched_same[str(d)] = {"team_blocks": tb, "ms": ms_b, "gteps": g.m * len(srcs) / (ms_b * 1e-3) / 1e9,
                                    "one_by_one_gteps": per_delta[str(d)]["gteps"],
                                    "speedup": per_delta[str(d)]["ms_per_solve"] * len(srcs) / ms_b}

    e2e = None
    if not args.no_e2e:
        e2e = run_e2e(ds, torch, g, srcs, deltas, world, dist_pg, args, sched)

    extras = {}
    if world == 1 and not args.no_extras:
        extras = run_extras(ds, torch)

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu:
        cores = os.cpu_count() or 1
        k = args.cpu_sources or min(cores, len(srcs))
        v, used, dt = cpu_oracle_gteps(g, srcs[:k])
        cpu = {"value": v, "unit": "GTEPS", "cores": used, "kind": "oracle",
               "sample": f"{k} of the {len(srcs)} sources, binary-heap Dijkstra one source per thread, {dt:.1f} s"}
        # the oracle's Fig. 1 linear-algebra form (dense vectors, one thread), one source at Delta 0.1
        import oracle
        t0 = time.perf_counter()
        oracle.delta_la(g.row_ptr, g.col, g.w, srcs[0], 0.1)
        dla = time.perf_counter() - t0
        cpu["la_form"] = {"value": g.m / dla / 1e9, "unit": "GTEPS", "cores": 1, "kind": "oracle",
                          "sample": f"1 source, Delta 0.1, Fig. 1 dense-vector form, {dla:.1f} s"}

    if rank == 0:
        line = {
            "metric": "delta-stepping SSSP GTEPS (m * sources / device time)",
            "value": gteps, "unit": "GTEPS", "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": ms_per_step, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "f32", "data": "synthetic",
            "config": {"workload": f"rmat{args.scale}_unit_fp32_sources{args.sources}_deltas4",
                       "n": g.n, "m": g.m, "sources": len(srcs), "deltas": deltas, "solves_per_step": solves,
                       "mode": "persistent" if args.mode == 0 else "stepped",
                       "l2": "inputs larger than L2 (arcs %.0f MB per Delta)" % (g.m * 8 / 1e6),
                       "split_ms": split_ms, "schedule": {str(d): sched[d] for d in deltas},
                       "mean_reached_arcs": sum(m_reached.values()) / len(srcs), "per_delta": per_delta,
                       "parallelism": f"replicas{world}"},
            "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                         "frac": achieved / peak, "traffic": measured_traffic(args.scale),
                         "algorithmic_bytes_per_launch": tot_bytes / max(1, solves), "peak_kind": peak_kind,
                         "kernel": "k_solve_persistent (with its init/unpack launches)",
                         "light_relax_gbs": light_gbs,
                         "light_relax_frac": (light_gbs / peak) if light_gbs else None},
            "cpu_baseline": cpu,
            "e2e": e2e,
            "clocks": clk,
            "gpu_launches": sum((3 if sched[d]["mode"] == 3 else 4) * len(srcs) for d in deltas) * args.steps,
        }
        line.update(extras)
        if batched_same is not None:
            line["batched_same_workload"] = {
                "note": "the same 64 sources per Delta solved as one batch instead of one after another",
                "per_delta": batched_same}
        print(json.dumps(line), flush=True)
    if dist_pg:
        dist_pg.barrier()
        dist_pg.destroy_process_group()


def _events_ms(torch, fn, reps: int, stream=None) -> float:
    """Median CUDA-event time of fn() over reps runs after one warm-up."""
    fn()
    torch.cuda.synchronize()
    ts = []
    for _ in range(reps):
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        fn()
        b.record(stream)
        b.synchronize()
        ts.append(a.elapsed_time(b))
    return statistics.median(ts)


def batch_algorithmic_bytes(stats, ns) -> int:
    """Algorithmic bytes of a batch run from its per-instance counters (same per-unit figures)."""
    return sum(B_VERTEX * (st["vertices_light"] + st["vertices_heavy"]) + B_ARC * (st["arcs_light"] + st["arcs_heavy"])
               + B_FAR * st["far_scanned"] + B_INIT_UNPACK * n for st, n in zip(stats, ns))


def run_extras(ds, torch):
    """Batched and forward+backward throughput against the plain per-source solve on the
    same GPU: (a) 256 sources on a scale-20 R-MAT in one launch, (b) 512 ER graphs of
    uneven sizes in one launch, (c) 32 sources on a scale-20 lognormal R-MAT with the
    adjoint. Delta is chosen by the autotuner (batch instances for the batch, single
    solves for the plain runs); tuning time is reported, not timed."""
    import graphgen.workloads as W
    out = {"batched": {}, "fwd_bwd": {}}
    o_async = ds.make_options(flags=ds.DSSSP_FLAG_ASYNC)

    # (a) many sources on one graph
    g, srcs = W.rmat20_unit()
    h = ds.Graph(g.row_ptr, g.col, g.w)
    t = time.perf_counter()
    (d_b,), _ = ds.autotune(h, [srcs[:8]], target="batch")
    (d_p,), _ = ds.autotune(h, [srcs[:4]], target="solve")
    tb_a, _ = ds.tune_team_blocks(h, [d_b], srcs)
    tune_s = time.perf_counter() - t
    b = ds.Batch(h, [d_b], srcs, options=ds.make_options(team_blocks=tb_a))
    ms_b = _events_ms(torch, b.run, 3)
    bst = b.sync(stats=True)
    b.close()
    peak, _ = measured_peak_gbs()
    gbs_a = batch_algorithmic_bytes(bst, [g.n] * len(srcs)) / (ms_b * 1e-3) / 1e9

    def plain_a():
        for s in srcs:
            h.solve(s, d_p, options=o_async)
    ms_p = _events_ms(torch, plain_a, 1)
    h.sync()
    h.close()
    out["batched"]["rmat20_unit_256src"] = {
        "n": g.n, "m": g.m, "instances": len(srcs), "delta": d_b, "team_blocks": tb_a, "ms": ms_b,
        "gteps": g.m * len(srcs) / (ms_b * 1e-3) / 1e9, "plain_delta": d_p, "plain_ms": ms_p,
        "plain_gteps": g.m * len(srcs) / (ms_p * 1e-3) / 1e9, "speedup": ms_p / ms_b, "tune_s": tune_s,
        "algorithmic_gbs": gbs_a, "hbm_frac": gbs_a / peak}

    # (b) many graphs of uneven sizes
    fam = W.er_family()
    hs = [ds.Graph(x.row_ptr, x.col, x.w) for x, _ in fam]
    fsrc = [s for _, s in fam]
    msum = sum(x.m for x, _ in fam)
    t = time.perf_counter()
    deltas, _ = ds.autotune(hs, [[s] for s in fsrc], target="batch", refine=1)
    tb_b, _ = ds.tune_team_blocks(hs, deltas, fsrc, src_graph=list(range(len(fam))))
    tune_s = time.perf_counter() - t
    b = ds.Batch(hs, deltas, fsrc, src_graph=list(range(len(fam))), options=ds.make_options(team_blocks=tb_b))
    ms_b = _events_ms(torch, b.run, 3)
    bst = b.sync(stats=True)
    b.close()
    gbs_b = batch_algorithmic_bytes(bst, [x.n for x, _ in fam]) / (ms_b * 1e-3) / 1e9
    for hh, d in zip(hs, deltas):
        hh.prepare(d)

    def plain_b():
        for hh, s, d in zip(hs, fsrc, deltas):
            hh.solve(s, d, options=o_async)
    ms_p = _events_ms(torch, plain_b, 1)
    for hh in hs:
        hh.sync()
        hh.close()
    out["batched"]["er512"] = {
        "graphs": len(fam), "sum_n": sum(x.n for x, _ in fam), "sum_m": msum, "team_blocks": tb_b,
        "delta_range": [min(deltas), max(deltas)], "ms": ms_b, "gteps": msum / (ms_b * 1e-3) / 1e9,
        "plain_ms": ms_p, "plain_gteps": msum / (ms_p * 1e-3) / 1e9, "speedup": ms_p / ms_b, "tune_s": tune_s,
        "algorithmic_gbs": gbs_b, "hbm_frac": gbs_b / peak}

    # (c) forward + backward
    g, srcs, c = W.rmat20_lognormal()
    h = ds.Graph(g.row_ptr, g.col, g.w)
    t = time.perf_counter()
    (d_b,), _ = ds.autotune(h, [srcs[:8]], target="batch")
    tb_c, _ = ds.tune_team_blocks(h, [d_b], srcs)
    tune_s = time.perf_counter() - t
    cs = [torch.from_numpy(c).cuda()] * len(srcs)
    gw = torch.empty(g.m, dtype=torch.float32, device="cuda")
    opt_c = ds.make_options(team_blocks=tb_c)
    bt = ds.Batch(h, [d_b], srcs, tape=True, options=opt_c)
    bn = ds.Batch(h, [d_b], srcs, options=opt_c)

    def fwd_bwd():
        bt.run()
        bt.backward(cs, [gw])
    ms_fb = _events_ms(torch, fwd_bwd, 3)
    ms_f = _events_ms(torch, bn.run, 3)
    ms_bw = _events_ms(torch, lambda: bt.backward(cs, [gw]), 3)
    bt.sync()
    bn.sync()
    bt.close()
    bn.close()

    def plain_c():
        for s in srcs:
            h.solve(s, d_b, options=o_async)
    ms_p = _events_ms(torch, plain_c, 1)
    h.sync()
    h.close()
    sm = g.m * len(srcs)
    out["fwd_bwd"]["rmat20_lognormal_32src"] = {
        "n": g.n, "m": g.m, "instances": len(srcs), "delta": d_b, "team_blocks": tb_c, "fwd_bwd_ms": ms_fb,
        "fwd_ms": ms_f,
        "bwd_ms": ms_bw, "fwd_bwd_gteps": sm / (ms_fb * 1e-3) / 1e9, "fwd_gteps": sm / (ms_f * 1e-3) / 1e9,
        "plain_solve_ms": ms_p, "plain_solve_gteps": sm / (ms_p * 1e-3) / 1e9,
        "fwd_bwd_over_fwd": ms_fb / ms_f, "tune_s": tune_s}

    out.update(run_ablation(ds, torch))
    out["other_workloads"] = run_other_workloads(ds, torch)
    return out


def _timed_solves(torch, calls, sync_each: bool) -> float:
    """CUDA-event ms over a list of calls (one warm-up pass first); with sync_each the
    host waits after every call, as a synchronous entry point does."""
    for c in calls[:1]:
        c()
    torch.cuda.synchronize()
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    t = time.perf_counter()
    a.record()
    for c in calls:
        c()
        if sync_each:
            torch.cuda.synchronize()
    b.record()
    b.synchronize()
    return a.elapsed_time(b) if not sync_each else (time.perf_counter() - t) * 1e3


def run_ablation(ds, torch):
    """The paper's full-vector form (t_Bi, S and the far pile as per-vertex stamps scanned in
    full every phase, row filters fused into the scans) against the list-based persistent
    solve: (1) DSSSP_MODE_DENSE on the bench graph itself (scale-22 R-MAT, 4 sources per
    Delta, both arms asynchronous, CUDA events around all solves of a Delta); (2)
    dsssp_solve_noalloc (the same form in a fixed array, n <= 131,072) on a scale-17 R-MAT,
    where each call waits for its result: both arms then wait after every solve and are
    timed on the host."""
    import graphgen.workloads as W
    out = {}
    g, srcs, deltas = W.rmat22_unit(n_sources=4)
    h = ds.Graph(g.row_ptr, g.col, g.w)
    dist = torch.empty(g.n, dtype=torch.float32, device="cuda")
    pred = torch.empty(g.n, dtype=torch.int32, device="cuda")
    o_list = ds.make_options(flags=ds.DSSSP_FLAG_ASYNC)
    o_dense = ds.make_options(flags=ds.DSSSP_FLAG_ASYNC, mode=ds.DSSSP_MODE_DENSE)
    per = {}
    for d in deltas:
        h.prepare(d)
        ms_l = _timed_solves(torch, [lambda s=s: h.solve(s, d, dist=dist, pred=pred, options=o_list) for s in srcs],
                             False) / len(srcs)
        ms_d = _timed_solves(torch, [lambda s=s: h.solve(s, d, dist=dist, pred=pred, options=o_dense) for s in srcs],
                             False) / len(srcs)
        h.sync()
        st = h.solve(srcs[0], d, dist=dist, pred=pred, options=ds.make_options(mode=ds.DSSSP_MODE_DENSE),
                     stats=True).stats
        per[str(d)] = {"dense_ms_per_solve": ms_d, "list_ms_per_solve": ms_l, "list_speedup": ms_d / ms_l,
                       "dense_gteps": g.m / (ms_d * 1e-3) / 1e9, "list_gteps": g.m / (ms_l * 1e-3) / 1e9,
                       "dense_phases": st["light_phases"] + st["heavy_phases"]}
    h.close()
    out["ablation_dense_vs_lists"] = {
        "workload": f"rmat22_unit n={g.n} m={g.m}, {len(srcs)} sources per Delta (the bench graph)",
        "timing": "both arms asynchronous; CUDA events around the solves of one Delta", "per_delta": per}

    g, srcs, _ = W.rmat22_unit(scale=17, n_sources=8)
    rp = torch.from_numpy(g.row_ptr).cuda()
    cl = torch.from_numpy(g.col).cuda()
    ww = torch.from_numpy(g.w).cuda()
    h = ds.Graph(rp, cl, ww)
    dist = torch.empty(g.n, dtype=torch.float32, device="cuda")
    pred = torch.empty(g.n, dtype=torch.int32, device="cuda")
    stream = torch.cuda.current_stream()
    o_sync = ds.make_options()
    abl = {}
    for d in (0.05, 0.1, 0.5):
        h.prepare(d)
        na = [lambda s=s: ds.check(ds.dsssp_solve_noalloc(g.n, g.m, rp.data_ptr(), cl.data_ptr(), ww.data_ptr(),
                                                          ds.DSSSP_F32, s, d, dist.data_ptr(), pred.data_ptr(),
                                                          ds._stream_ptr(stream)), "dsssp_solve_noalloc")
              for s in srcs]
        ls = [lambda s=s: h.solve(s, d, dist=dist, pred=pred, options=o_sync) for s in srcs]
        ms_d = _timed_solves(torch, na, True) / len(srcs)
        ms_l = _timed_solves(torch, ls, True) / len(srcs)
        abl[str(d)] = {"noalloc_ms_per_solve": ms_d, "list_ms_per_solve": ms_l, "list_speedup": ms_d / ms_l}
    h.close()
    out["ablation_noalloc_vs_lists"] = {
        "workload": f"rmat17_unit n={g.n} m={g.m}, 8 sources",
        "timing": "both arms wait for every solve (the no-allocation call is synchronous); host wall time",
        "per_delta": abl}
    return out


def run_other_workloads(ds, torch):
    """The other single-source workloads: the 4096 x 4096 grid (int32 U{1..1000}, 5 % of arcs
    dropped, corner source, Delta in {100, 1000, 10000}: the high-diameter, phase-bound case)
    and the scale-14 R-MAT (int32 U{1..255}, Delta 32, highest out-degree source). Per Delta:
    the scheme chosen by the schedule tuner (untimed, one sample source), its device time per
    solve (CUDA events, median of several), GTEPS, phases and the algorithmic bandwidth of the
    solve against the measured HBM copy peak; and the grid-wide persistent scheme beside it."""
    import graphgen.workloads as W
    peak, _ = measured_peak_gbs()
    out = {}
    for name, (g, srcs, deltas), reps in (("grid4096_int", W.grid4096(), 3), ("rmat14_int", W.rmat14_int(), 20)):
        h = ds.Graph(g.row_ptr, g.col, g.w)
        dist = torch.empty(g.n, dtype=torch.int32, device="cuda")
        pred = torch.empty(g.n, dtype=torch.int32, device="cuda")
        s = srcs[0]
        per = {}
        for d in deltas:
            h.prepare(d)
            tuned, _ = ds.tune_schedule(h, [s], d)
            row = {}
            for label, o in (("tuned", tuned), ("persistent", ds.make_options())):
                st = h.solve(s, d, dist=dist, pred=pred, stats=True, options=o).stats
                oa = ds.make_options(flags=ds.DSSSP_FLAG_ASYNC, mode=o.mode, solo_work=o.solo_work,
                                     team_blocks=o.team_blocks)
                ms = _events_ms(torch, lambda: h.solve(s, d, dist=dist, pred=pred, options=oa), reps)
                h.sync()
                b = algorithmic_bytes(st, g.n)
                row[label] = {"mode": ["persistent", "stepped", "dense", "team"][o.mode],
                              "solo_work": o.solo_work, "team_blocks": st["grid_size"] if o.mode == 3 else 0,
                              "ms_per_solve": ms, "gteps": g.m / (ms * 1e-3) / 1e9,
                              "phases": st["light_phases"] + st["heavy_phases"] + st["rebin_phases"],
                              "buckets": st["buckets"], "arcs_relaxed": st["arcs_light"] + st["arcs_heavy"],
                              "roofline": {"bound": "hbm", "achieved": b / (ms * 1e-3) / 1e9, "peak": peak,
                                           "unit": "GB/s", "frac": b / (ms * 1e-3) / 1e9 / peak}}
            per[str(d)] = row
        h.close()
        out[name] = {"n": g.n, "m": g.m, "source": s, "per_delta": per}
    return out


def profile_batch_driver(args):
    """One batch of K sources on the scale-20 R-MAT (fp32 U[0,1)), for profilers."""
    import torch
    import paper_1911_06895_gb300 as ds
    import graphgen.workloads as W
    g, srcs = W.rmat20_unit(n_sources=max(args.profile_batch, 1))
    h = ds.Graph(g.row_ptr, g.col, g.w)
    d = float(args.profile_delta)
    b = ds.Batch(h, [d], srcs[:args.profile_batch])
    b.run()
    st = b.sync(stats=True)
    nbytes = batch_algorithmic_bytes(st, [g.n] * len(st))
    print(json.dumps({"instances": len(st), "delta": d, "algorithmic_bytes": nbytes,
                      "arcs": sum(x["arcs_light"] + x["arcs_heavy"] for x in st),
                      "max_instance_ms": max(x["ns"] for x in st) / 1e6}), flush=True)
    b.close()
    torch.cuda.synchronize()


def profile_backward_driver(args):
    """Forward (with tape) and one adjoint pass on the scale-20 lognormal R-MAT, for profilers."""
    import torch
    import paper_1911_06895_gb300 as ds
    import graphgen.workloads as W
    g, srcs, c = W.rmat20_lognormal()
    srcs = srcs[:args.profile_backward]
    h = ds.Graph(g.row_ptr, g.col, g.w)
    b = ds.Batch(h, [0.36], srcs, tape=True, options=ds.make_options(team_blocks=8))
    cs = [torch.from_numpy(c).cuda()] * len(srcs)
    gw = torch.empty(g.m, dtype=torch.float32, device="cuda")
    b.run()
    st = b.sync(stats=True)
    b.backward(cs, [gw])
    torch.cuda.synchronize()
    # algorithmic bytes: per vertex and instance 4 parent + 4 tree arc + 4 c + 8 sum + 8 parent sum + 4 count
    # + 8 for the tree arc's float64 add; per arc 12 for the float32 output
    print(json.dumps({"instances": len(st), "n": g.n, "m": g.m, "algorithmic_bytes_backward": 40 * g.n * len(st),
                      "algorithmic_bytes_grad_out": 12 * g.m,
                      "grad_abs_sum": float(gw.abs().sum().item())}), flush=True)
    b.close()


def profile_driver(args):
    """A fixed, short sequence of solves for profilers: split, then N solves."""
    import torch
    import paper_1911_06895_gb300 as ds
    g, srcs, _ = build_workload(args.scale, max(args.profile_solves, 1), 0)
    deltas = DELTAS if args.profile_delta == "all" else [float(x) for x in args.profile_delta.split(",")]
    h = ds.Graph(g.row_ptr, g.col, g.w)
    for d in deltas:
        h.prepare(d)
    opt = ds.make_options(mode=args.mode, flags=ds.DSSSP_FLAG_NO_FUSE if args.no_fuse else 0)
    for d in deltas:
        for s in srcs[:args.profile_solves]:
            r = h.solve(s, d, options=opt, stats=True)
            print(json.dumps({"src": s, "delta": d, "algorithmic_bytes": algorithmic_bytes(r.stats, g.n),
                              **r.stats}), flush=True)
    torch.cuda.synchronize()


def run_e2e(ds, torch, g, srcs, deltas, world, dist_pg, args, sched):
    """Public-API end to end: host CSR -> graph -> 256 solves -> results in pinned host memory.

    Each solve writes one of NB device buffers; its result goes back to pinned host memory on a copy
    stream while the next solves run, and a buffer is reused only after its copy has finished."""
    rp = torch.from_numpy(g.row_ptr).pin_memory()
    cl = torch.from_numpy(g.col).pin_memory()
    ww = torch.from_numpy(g.w).pin_memory()
    solves = len(deltas) * len(srcs)
    NB = 3
    hd = torch.empty((NB, g.n), dtype=torch.float32).pin_memory()
    hp = torch.empty((NB, g.n), dtype=torch.int32).pin_memory()
    stream = torch.cuda.Stream()
    copy_stream = torch.cuda.Stream()
    steps = max(1, min(args.steps, 2))

    def step():
        with torch.cuda.stream(stream):
            h = ds.Graph(rp.numpy(), cl.numpy(), ww.numpy(), stream=stream)
            dist = torch.empty((NB, g.n), dtype=torch.float32, device="cuda")
            pred = torch.empty((NB, g.n), dtype=torch.int32, device="cuda")
        solved = [torch.cuda.Event() for _ in range(NB)]
        copied = [None] * NB
        k = 0
        for d in deltas:
            opt = ds.make_options(flags=ds.DSSSP_FLAG_ASYNC, **sched[d])
            for s in srcs:
                b = k % NB
                if copied[b] is not None:
                    stream.wait_event(copied[b])          # the buffer's previous result is on the host
                with torch.cuda.stream(stream):
                    h.solve(s, d, dist=dist[b], pred=pred[b], options=opt, stream=stream)
                solved[b].record(stream)
                copy_stream.wait_event(solved[b])
                with torch.cuda.stream(copy_stream):
                    hd[b].copy_(dist[b], non_blocking=True)
                    hp[b].copy_(pred[b], non_blocking=True)
                    copied[b] = torch.cuda.Event()
                    copied[b].record(copy_stream)
                k += 1
        h.sync(stream)
        stream.synchronize()
        copy_stream.synchronize()
        h.close()

    step()
    torch.cuda.synchronize()
    if dist_pg:
        dist_pg.barrier()
    t = time.perf_counter()
    for _ in range(steps):
        step()
    torch.cuda.synchronize()
    dt = max_over_ranks((time.perf_counter() - t) / steps, "cuda")
    return {"value": job_gteps(g.m, solves, world, dt), "unit": "GTEPS",
            "h2d_bytes_per_step": int(g.row_ptr.nbytes + g.col.nbytes + g.w.nbytes),
            "d2h_bytes_per_step": int(solves * g.n * 8), "ms_per_step": dt * 1e3, "steps": steps}


if __name__ == "__main__":
    main()

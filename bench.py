#!/usr/bin/env python
"""Benchmark: cells/s of the GB300 projector build at n = 1,048,576 uniform sites.

One step = one whole build (bucketing, projector ray shooting per cell,
compaction into CSR cells and Delaunay edges) of the 1,048,576-site uniform
workload in X = [0, 2^20]^2, inputs resident in HBM.  Between timed steps a
256 MiB buffer is written to flush the 129 MB L2.  Device time per step comes
from CUDA events on the build's stream.

Prints one JSON line (rank 0).  ``--impl reference`` times the exact CPU
oracle (the paper has no code to run) on a bounded sample of the same
workload on the host cores.

Multi-GPU (torchrun, one rank per GPU): every rank builds its own copy of the
workload (independent problems, no collective on the data path); the value is
the cells of all ranks divided by the slowest rank's time (weak scaling).
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

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "cells/s at n=1M uniform; batched sets/s and p50/p99 latency vs plain"
BOX = 1 << 20
WORKLOADS = {"uniform_1m": 1 << 20, "gauss_4m": 1 << 22}
OPS_PER_EVAL = 8                # FP32/ALU operations of one filter evaluation of a candidate


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=50)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--workload", choices=sorted(WORKLOADS), default="uniform_1m")
    ap.add_argument("--lanes", type=int, default=0)
    ap.add_argument("--target", type=int, default=0)
    ap.add_argument("--bucket-side", type=int, default=0)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    return ap.parse_args()


def dist_init(args):
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if ws > 1:
        import torch
        import torch.distributed as dist
        torch.cuda.set_device(local)
        dist.init_process_group("nccl")
    return ws, rank, local


def barrier(ws):
    if ws > 1:
        import torch.distributed as dist
        dist.barrier()


def max_over_ranks(ws, value: float) -> float:
    if ws == 1:
        return value
    import torch
    import torch.distributed as dist
    t = torch.tensor([value], dtype=torch.float64, device="cuda")
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


class Clocks:
    """nvidia-smi sampling of SM clocks and throttle reasons during the timed region."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.path = os.path.join(tempfile.gettempdir(), f"vor_clocks_{os.getpid()}.csv")
        self.proc = None
        self.gpu = gpu_index

    def start(self):
        try:
            self.f = open(self.path, "w")
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.gpu), f"--query-gpu={self.Q}",
                 "--format=csv,noheader,nounits", "-lms", "20"],
                stdout=self.f, stderr=subprocess.DEVNULL)
        except (OSError, FileNotFoundError):
            self.proc = None

    def stop(self) -> dict:
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        self.f.close()
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in open(self.path):
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                smax.append(float(parts[2]))
            except ValueError:
                continue
            for nm, v in zip(names, parts[5:9]):
                if v.lower() == "active":
                    reasons.add(nm)
        os.unlink(self.path)
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(smax) if smax else None,
                "samples": len(sm), "reasons": sorted(reasons)}


def measured_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as f:
            return json.load(f)
    return None


def traffic_from_profiles(workload: str):
    """DRAM bytes per launch of the first-pass projector kernel from the
    committed ncu summary, when one exists for this workload and the kernel's
    source files are unchanged since the capture."""
    p = os.path.join(ROOT, "profiles", f"cells_persist_kernel_p1_{workload}.json")
    if not os.path.exists(p):
        return None
    try:
        with open(p) as f:
            d = json.load(f)
        from paper_1212_1095_gb300 import _build
        if d.get("kernel_fingerprint") != _build.kernel_fingerprint(d.get("kernel_sources", [])):
            return None
        return d.get("dram_bytes_per_launch")
    except Exception:
        return None


def cpu_baseline(xy, seconds_target: float = 15.0):
    """The oracle (bucketed, Method A.6) on a bounded sample of the cells."""
    import numpy as np
    import oracle
    cores = os.cpu_count() or 1
    n = xy.shape[0]
    # per-cell cost from two probe sizes (each call also buckets all n sites)
    times = []
    for k in (4096, 16384):
        probe = np.arange(0, n, max(1, n // k))[:k]
        t0 = time.perf_counter()
        oracle.cells(xy, BOX, "bucketed", sel=probe, nthreads=cores)
        times.append((len(probe), time.perf_counter() - t0))
    (k1, t1), (k2, t2) = times
    per_cell = max((t2 - t1) / max(k2 - k1, 1), 1e-9)
    setup = max(t1 - k1 * per_cell, 0.0)
    m = int(min(n, max(k2, (seconds_target - setup) / per_cell)))
    stride = max(1, n // m)
    sel = np.arange(0, n, stride)[:m]
    t0 = time.perf_counter()
    oracle.cells(xy, BOX, "bucketed", sel=sel, nthreads=cores)
    dt = time.perf_counter() - t0
    return {"value": len(sel) / dt, "unit": "cells/s", "cores": cores, "kind": "oracle",
            "sample": f"{len(sel)} of {n} cells (stride {stride}), bucketed oracle "
                      f"(Method A.6), {cores} threads, {dt:.1f} s"}


def run_reference(args):
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return 0
    import numpy as np
    import oracle
    import synth
    xy = synth.workload(args.workload)
    n = xy.shape[0]
    cores = os.cpu_count() or 1
    sample = min(n, 32768)
    stride = max(1, n // sample)
    times = []
    for step in range(args.warmup + args.steps):
        sel = (np.arange(sample) * stride + step) % n
        t0 = time.perf_counter()
        oracle.cells(xy, BOX, "bucketed", sel=sel, nthreads=cores)
        dt = time.perf_counter() - t0
        if step >= args.warmup:
            times.append(dt)
    t = sum(times)
    value = sample * len(times) / t
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": "cells/s",
        "n_gpus": ws, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": 1000.0 * t / len(times), "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "int64", "data": "synthetic",
        "config": {"workload": args.workload, "n_sites": n, "box": BOX,
                   "sample_cells_per_step": sample},
        "cpu_baseline": {"value": value, "unit": "cells/s", "cores": cores, "kind": "oracle",
                         "sample": f"{sample} cells per step (stride {stride}), bucketed oracle "
                                   f"(Method A.6), {cores} threads"},
        "e2e": {"value": value, "unit": "cells/s", "h2d_bytes_per_step": 0,
                "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line))
    return 0


def run_ours(args):
    import numpy as np
    import torch

    import paper_1212_1095_gb300 as vg
    import synth

    ws_n, rank, local = dist_init(args)
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    xy = synth.workload(args.workload)
    n = xy.shape[0]
    d_sites = torch.from_numpy(xy).to(dev)
    opts = dict(lanes_per_cell=args.lanes, target=args.target, bucket_side=args.bucket_side)
    W = vg.Workspace(n, BOX, vg.vor_opts_default(**opts), device=dev)
    stream = torch.cuda.current_stream()

    # counters of one (untimed) build: the algorithmic work of the projector kernel
    Ws = vg.Workspace(n, BOX, vg.vor_opts_default(collect_stats=1, **opts), device=dev)
    Ws.launch(d_sites)
    stats = Ws.finish().stats
    n_edges = int(Ws.totals[0].item())
    n_del = int(Ws.totals[1].item())
    del Ws

    flush = torch.empty(256 << 20, dtype=torch.uint8, device=dev)
    vg.vor_stage_timing(True)
    for _ in range(args.warmup):
        W.launch(d_sites)
        W.finish()
    barrier(ws_n)
    torch.cuda.synchronize()
    clocks = Clocks(local)
    clocks.start()
    step_ms, cells_ms, stage_acc = [], [], []
    launches0 = vg.vor_kernel_launches()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    for _ in range(args.steps):
        flush.fill_(1)
        e0.record(stream)
        W.launch(d_sites, stream)
        e1.record(stream)
        e1.synchronize()
        step_ms.append(e0.elapsed_time(e1))
        st_ms = vg.vor_stage_ms()
        cells_ms.append(st_ms[2])
        stage_acc.append(st_ms)
    torch.cuda.synchronize()
    launches = vg.vor_kernel_launches() - launches0
    barrier(ws_n)
    clk = clocks.stop()
    rc, _ = vg.vor_status(W.ws_ptr, stream.cuda_stream)
    if rc != 0:
        raise vg.VorError(rc, "timed builds")
    vg.vor_stage_timing(False)
    ms = sum(step_ms) / len(step_ms)
    ms_max = max_over_ranks(ws_n, ms)
    value = ws_n * n / (ms_max / 1000.0)

    # end to end through the host-buffer entry point: H2D of the sites, the
    # build, D2H of the cells, vertices and Delaunay edges, every step
    e2e = None
    if not args.no_e2e:
        ctypes = __import__("ctypes")
        hx = torch.from_numpy(xy).pin_memory()
        ec, dc = vg.vor_edge_capacity(n), vg.vor_delaunay_capacity(n)
        h_cp = torch.empty(n + 1, dtype=torch.int64).pin_memory()
        h_lab = torch.empty(ec, dtype=torch.int32).pin_memory()
        h_vx = torch.empty(ec, dtype=torch.float64).pin_memory()
        h_vy = torch.empty(ec, dtype=torch.float64).pin_memory()
        h_dl = torch.empty(2 * dc, dtype=torch.int32).pin_memory()
        sb = vg.vor_host_scratch_bytes(n)
        scratch = torch.empty(sb + 256, dtype=torch.uint8, device=dev)
        sp = (scratch.data_ptr() + 255) & ~255
        ne, nd = ctypes.c_int64(), ctypes.c_int64()
        P = ctypes.c_void_p

        def host_step():
            rc = vg.vor_build_host(P(hx.data_ptr()), n, vg.VorBox(BOX, BOX), ctypes.byref(W.opts),
                                   P(W.ws_ptr), W.ws_bytes, P(sp), sb, P(h_cp.data_ptr()),
                                   P(h_lab.data_ptr()), P(h_vx.data_ptr()), P(h_vy.data_ptr()),
                                   P(h_dl.data_ptr()), ec, dc, ctypes.byref(ne), ctypes.byref(nd),
                                   P(stream.cuda_stream))
            if rc != 0:
                raise vg.VorError(rc, "vor_build_host")

        for _ in range(max(1, args.warmup)):
            host_step()
        barrier(ws_n)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for _ in range(args.steps):
            host_step()
        torch.cuda.synchronize()
        te = (time.perf_counter() - t0) / args.steps
        te = max_over_ranks(ws_n, te)
        e2e = {"value": ws_n * n / te, "unit": "cells/s", "h2d_bytes_per_step": 8 * n,
               "d2h_bytes_per_step": 8 * (n + 1) + 20 * ne.value + 8 * nd.value,
               "ms_per_step": 1000.0 * te}

    if rank != 0:
        return 0
    # roofline of the projector kernel: plain ALU work (no tensor cores, the
    # path is not a contraction); peak = SMs x 128 lanes x SM clock
    props = torch.cuda.get_device_properties(dev)
    sm_mhz = clk.get("sm_mhz") or 1920.0
    peak = props.multi_processor_count * 128 * sm_mhz * 1e6 / 1e12
    kms = sum(cells_ms) / len(cells_ms)
    evals1 = stats["evals_first_pass"] if args.lanes in (0, 1) else stats["evals"]
    achieved = evals1 * OPS_PER_EVAL / (kms / 1000.0) / 1e12
    roofline = {"bound": "alu", "achieved": achieved, "peak": peak, "unit": "TOP/s",
                "frac": achieved / peak, "traffic": traffic_from_profiles(args.workload),
                "kernel": "cells_persist_kernel<64,44> (projector, first pass)",
                "kernel_ms": kms, "evals_per_launch": evals1,
                "ops_per_eval": OPS_PER_EVAL,
                "peak_basis": f"{props.multi_processor_count} SMs x 128 FP32 lanes x "
                              f"{sm_mhz:.0f} MHz median SM clock (1 op per lane per cycle)"}
    line = {
        "metric": METRIC, "value": value, "unit": "cells/s", "n_gpus": ws_n,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms_max,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "int64",
        "data": "synthetic",
        "config": {"workload": args.workload, "n_sites": n, "box": BOX,
                   "distribution": "uniform integer sites, no four on an empty circle"
                   if args.workload == "uniform_1m" else "64-component Gaussian mixture",
                   "l2": "256 MiB buffer written between timed steps",
                   "edges": n_edges, "delaunay_edges": n_del,
                   "parallelism": f"replicas x{ws_n}" if ws_n > 1 else "1 GPU"},
        "stages_ms": dict({k: statistics.mean(x[i] for x in stage_acc)
                           for i, k in enumerate(vg.STAGES)}, step=ms),
        "stats": stats,
        "roofline": roofline,
        "clocks": clk,
        "e2e": e2e,
        "gpu_launches": launches,
    }
    if ws_n == 1 and not args.no_cpu_baseline:
        line["cpu_baseline"] = cpu_baseline(xy)
    print(json.dumps(line))
    return 0


def main():
    args = parse()
    if args.impl == "reference":
        return run_reference(args)
    return run_ours(args)


if __name__ == "__main__":
    sys.exit(main())

"""Throughput benchmark of the STG-LBM hot path (MLUPS and HBM roofline).

One step = the STG inlet kernel plus the fused stream/collide kernel over the
whole lattice (with FP64 statistics every 10 steps), i.e. one pass of the
whole hot path.  Default workload: the Re_tau = 180 channel on a 768x128x192
D3Q19 FP32 lattice (h = 64, 200 STG modes), inputs resident in HBM, lattice
(2.9 GB) far larger than L2.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
  python bench.py --workload ensemble [--members 64] [--steps K]   (batched ensemble)
  python bench.py --workload serve [--jobs 60] [--steps-scale 0.1]   (served stream)

N > 1 runs one independent channel per GPU (weak scaling, no collective on
the data path).  ``--impl reference`` times the CPU FP64 oracle on the host
cores instead (bounded sample).  Prints one JSON line (rank 0).
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import re
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

BYTES_PER_CELL = {"fp32": 152, "fp16s": 76}  # 19 populations read + 19 written


def _peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(p) as fh:
            d = json.load(fh)
        return float(d["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


def _kernel_hash():
    """Hash of the step kernels' source with comments and white space removed
    (a comment edit does not change the kernel whose counters were taken)."""
    h = hashlib.sha256()
    for f in ("step_kernel.cu", "d3q19.cuh", "internal.h", "lbm_cell.cuh", "reduce.cuh"):
        with open(os.path.join(ROOT, "paper_2205_02774_gb300", "csrc", f)) as fh:
            src = fh.read()
        src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
        src = re.sub(r"//[^\n]*", "", src)
        h.update("".join(src.split()).encode())
    return h.hexdigest()[:16]


def _traffic(workload, storage):
    """DRAM bytes per launch of the step kernel from the committed ncu summary,
    if it was taken on the current kernel source (else None)."""
    path = os.path.join(ROOT, "profiles", f"lbm_step_kernel_{workload}_{storage}.md")
    if not os.path.exists(path):
        return None
    txt = open(path).read()
    mh = re.search(r"kernel_source_sha256_16:\s*([0-9a-f]+)", txt)
    mt = re.search(r"dram_bytes_per_full_launch:\s*([0-9.eE+]+)", txt)
    if not mh or not mt or mh.group(1) != _kernel_hash():
        return None
    return float(mt.group(1))


def _launches_per_step(c):
    """Kernels one step enqueues: the STG inlet kernel (inlet/outlet channel),
    then either the vector kernel on rows 1..ny-2 and the vector kernel on the
    two wall rows (even nx; inlet and outlet nodes included), or the scalar
    interior and edge kernels (odd nx)."""
    inlet = 1 if c.bc_x == "stg" else 0
    if c.nx % 2 == 0 and c.nx >= 4:
        return inlet + (1 if c.ny > 2 else 0) + 1
    return inlet + 2


def _launches(c, t0, steps):
    """Kernels the steps t0 .. t0+steps-1 enqueue: _launches_per_step each, plus
    the statistics reduction after every sampling step ((t + 1) % stats_every
    == 0) of the vector path."""
    n = _launches_per_step(c) * steps
    if c.stats_every > 0 and c.nx % 2 == 0 and c.nx >= 4:
        n += sum(1 for t in range(t0, t0 + steps) if (t + 1) % c.stats_every == 0)
    return n


class ClockSampler:
    """nvidia-smi clock / throttle sampling during the timed region."""

    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None
        self.path = None

    def start(self):
        try:
            fd, self.path = tempfile.mkstemp(suffix=".csv")
            os.close(fd)
            self.fh = open(self.path, "w")
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={self.index}", f"--query-gpu={self.FIELDS}",
                                          "--format=csv,noheader,nounits", "-lms", "100"],
                                         stdout=self.fh, stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        self.fh.close()
        sm, mx, reasons = [], 0.0, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in open(self.path):
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 8:
                continue
            try:
                sm.append(float(parts[0]))
                mx = max(mx, float(parts[1]))
            except ValueError:
                continue
            for n, v in zip(names, parts[4:8]):
                if v.lower().startswith("active"):
                    reasons.add(n)
        os.unlink(self.path)
        if not sm:
            return None
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": mx, "reasons": sorted(reasons), "samples": len(sm)}


def _dist():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def rank_seed(base, rank):
    """Each rank runs its own channel: the STG seed is offset by the rank."""
    return base + rank


def aggregate_ranks(ms_local, cells_per_rank, steps, dist=None, device="cpu"):
    """Whole-job throughput over the ranks: the timed region is the maximum
    of the ranks' times, the work is the sum of their cell updates.  Returns
    (ms_max, MLUPS)."""
    import torch
    ws = 1
    ms = float(ms_local)
    cells = float(cells_per_rank)
    if dist is not None and dist.is_initialized():
        ws = dist.get_world_size()
        t = torch.tensor([ms], dtype=torch.float64, device=device)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        ms = float(t.item())
        w = torch.tensor([cells], dtype=torch.float64, device=device)
        dist.all_reduce(w, op=dist.ReduceOp.SUM)
        cells = float(w.item())
    else:
        cells = cells * ws
    return ms, cells * steps / (ms * 1e-3) / 1e6


def _oracle_single_thread(workload, storage, ny=16, steps=1, extra=None):
    """The oracle on one host thread (a child process with OMP_NUM_THREADS=1):
    `steps` steps of an nx x ny x nz slice of the workload (full streamwise
    length and span, fewer wall-normal rows)."""
    code = ("import sys, time, json; sys.path.insert(0, %r); import oracle; from workloads import case; "
            "c = case(%r).with_(storage=%r, ny=%d, **%r); s = oracle.Sim.from_case(c); t0 = time.perf_counter(); "
            "s.step(%d); dt = time.perf_counter() - t0; "
            "print(json.dumps({'value': c.cells * %d / dt / 1e6, 'threads': oracle.threads(), "
            "'shape': [c.nx, c.ny, c.nz]}))") % (ROOT, workload, storage, ny, dict(extra or {}), steps, steps)
    try:
        out = subprocess.run([sys.executable, "-c", code], env=dict(os.environ, OMP_NUM_THREADS="1"),
                             capture_output=True, text=True, timeout=600)
        d = json.loads(out.stdout.strip().splitlines()[-1])
    except Exception as e:  # reported, not fatal: the all-core figure stands
        return {"error": str(e)[:200]}
    nx, ny_, nz = d["shape"]
    return {"value": d["value"], "unit": "MLUPS", "cores": d["threads"],
            "sample": f"{steps} step of a {nx}x{ny_}x{nz} slice of the {workload} channel (FP64, one thread)"}


def cpu_baseline(workload, storage, steps, extra=None):
    """The CPU FP64 oracle, as it stands, on a bounded sample of the workload:
    all host cores (OpenMP over z), plus the same oracle on one thread.
    `extra`: case fields of the variant (collision, sponge)."""
    import oracle
    from workloads import case
    c = case(workload).with_(storage=storage, **dict(extra or {}))
    sim = oracle.Sim.from_case(c)
    t0 = time.perf_counter()
    sim.step(steps)
    dt = time.perf_counter() - t0
    del sim
    return {"value": c.cells * steps / dt / 1e6, "unit": "MLUPS", "cores": oracle.threads(), "kind": "oracle",
            "sample": f"{steps} full steps of the {workload} lattice (FP64, OpenMP over z)", "seconds": dt,
            "single_thread": _oracle_single_thread(workload, storage, extra=extra)}


def run_reference(args):
    """Reference arm: the CPU FP64 oracle on the host cores.  Each step is one
    oracle step of a bounded sample of the workload: the full streamwise
    length and span (so the share of inlet-generator work per cell, N / nx,
    and the OpenMP split over z are those of the full channel) with fewer
    wall-normal rows (at least 2, walls on both), chosen so that warm-up +
    timed steps stay within about a minute of CPU time."""
    ws, rank, _ = _dist()
    if rank != 0:
        return
    import oracle
    from workloads import case
    full = case(args.workload)
    budget_cells = 3.0e8  # cell updates over the whole run
    ny = max(2, min(full.ny, int(budget_cells / ((args.steps + args.warmup) * full.nx * full.nz))))
    c = full.with_(ny=ny)
    sim = oracle.Sim.from_case(c)
    sim.step(args.warmup)
    t0 = time.perf_counter()
    sim.step(args.steps)
    t = time.perf_counter() - t0
    value = c.cells * args.steps / t / 1e6
    sample = (f"{args.steps} timed steps (+{args.warmup} warm-up) of a {c.nx}x{ny}x{c.nz} slice of the "
              f"{args.workload} channel (inlet, outlet, walls, {c.n_modes} STG modes)")
    line = {"impl": "reference", "metric": "MLUPS", "value": value, "unit": "MLUPS", "n_gpus": ws,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * t / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "config": {"workload": args.workload, "storage": "fp64 (oracle)",
                                             "sample_cells": c.cells},
            "cpu_baseline": {"value": value, "unit": "MLUPS", "cores": oracle.threads(), "kind": "oracle",
                             "sample": sample},
            "e2e": {"value": value, "unit": "MLUPS", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def _variant(c, args):
    """The workload with the --collision / --sponge choices applied (sponge:
    0.4 delta with delta = ny / 2, K = 1000, p = 3)."""
    c = c.with_(collision=args.collision)
    if args.sponge:
        c = c.with_(sponge_len=0.4 * c.ny / 2, sponge_K=1000.0, sponge_p=3.0)
    return c


def fp16_companion(c, args):
    """The same channel with populations stored as shifted FP16, timed the
    same way (autotuned tile, W warm-up steps, K steps between CUDA events),
    so one bench line carries the FP16-storage vs FP32 comparison."""
    import torch
    from paper_2205_02774_gb300.channel import Channel
    c16 = c.with_(storage="fp16s")
    ch = Channel.from_case(c16, check_every=100, mass_tol=0.5)
    tile = ch.autotune(20)
    ch.step(args.warmup)
    torch.cuda.synchronize()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(ch.stream)
    ch.step(args.steps)
    e1.record(ch.stream)
    e1.synchronize()
    ms = e0.elapsed_time(e1)
    rc = ch.stats()["rc"]
    ch.close()
    peak, _ = _peaks()
    bpc = BYTES_PER_CELL["fp16s"]
    return {"storage": "fp16s", "value": c16.cells * args.steps / (ms * 1e-3) / 1e6, "unit": "MLUPS",
            "ms_per_step": ms / args.steps, "hbm_frac_of_step": bpc * c16.cells * args.steps / (ms * 1e-3) / 1e9 / peak,
            "tile": list(tile), "rc": rc}


def run_ours(args):
    import numpy as np
    import torch
    from paper_2205_02774_gb300 import build
    build()
    from paper_2205_02774_gb300.channel import Channel
    from workloads import case

    ws, rank, local = _dist()
    torch.cuda.set_device(local)
    dist = None
    if ws > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    c = _variant(case(args.workload).with_(storage=args.storage), args)
    ch = Channel.from_case(c, check_every=100, mass_tol=0.5, seed=rank_seed(c.seed, rank))
    stream = ch.stream

    # launch tile from the library's autotuner (results do not depend on it),
    # then warm-up (also initialises graphs, clocks)
    if args.tile:
        tile = tuple(int(v) for v in args.tile.split(","))
        ch.set_tile(*tile)
    else:
        tile = ch.autotune(20)
    ch.step(args.warmup)
    torch.cuda.synchronize()

    def barrier():
        if dist is not None:
            dist.barrier()
        torch.cuda.synchronize()

    sampler = ClockSampler(local) if rank == 0 else None
    if sampler:
        sampler.start()
        time.sleep(0.3)
    barrier()
    if args.probes > 0:
        # probe series of the paper's post-processing (B_uu, T_t): random cells, seeded
        prng = np.random.default_rng(1234 + rank)
        xyz = np.stack([prng.integers(0, n, args.probes) for n in (c.nx, c.ny, c.nz)], axis=1).astype(np.int32)
        ch.set_probes(xyz)
        ch.step_probed(args.steps)  # untimed: allocates the series buffer before the timed region
        torch.cuda.synchronize()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    if args.probes > 0:
        series = ch.step_probed(args.steps)  # synchronises; ends with the series' copy to the host
        assert series.shape == (args.steps, args.probes, 3)
    else:
        ch.step(args.steps)
    e1.record(stream)
    e1.synchronize()
    barrier()
    clocks = sampler.stop() if sampler else None
    ms, value = aggregate_ranks(e0.elapsed_time(e1), c.cells, args.steps, dist, device="cuda")
    st = ch.stats()
    if st["rc"] != 0:
        raise RuntimeError(f"channel check failed: {st['error']}")

    # dominant kernel: per-launch device time of the fused step kernel
    ms_step, ms_inlet = ch.step_timed(min(200, max(20, args.steps // 10)))
    ch.close()
    del ch
    torch.cuda.synchronize()

    # end-to-end through the public API with host buffers
    e2e = None
    if rank == 0:
        prof = c.profile()
        host_in = sum(a.nbytes for a in (prof.y_c, prof.U, prof.k, prof.eps, prof.R))
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        ch2 = Channel.from_case(c, check_every=100, mass_tol=0.5)
        ch2.step(args.steps)
        st2 = ch2.stats()
        t1 = time.perf_counter()
        host_out = 9 * c.nx * c.ny * 8 + 16
        ch2.close()
        e2e = {"value": c.cells * args.steps / (t1 - t0) / 1e6, "unit": "MLUPS",
               "h2d_bytes_per_step": host_in / args.steps, "d2h_bytes_per_step": host_out / args.steps,
               "seconds": t1 - t0, "includes": "create (host profile upload, tables, init, graph capture) + "
                                               "step(K) + stats (FP64 sums to host) + destroy"}
        assert st2["rc"] == 0

    if rank != 0:
        if dist is not None:
            dist.destroy_process_group()
        return
    peak, peak_kind = _peaks()
    bpc = BYTES_PER_CELL[args.storage]
    achieved = bpc * c.cells / (ms_step * 1e-3) / 1e9
    # the committed counters were taken on the default variant
    traffic = _traffic(args.workload, args.storage) if (args.collision == "regularized" and not args.sponge) else None
    line = {
        "metric": "MLUPS", "value": value, "unit": "MLUPS", "n_gpus": ws, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms / args.steps, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": {"workload": args.workload, "storage": args.storage, "cells": c.cells, "lattice": "D3Q19",
                   "tile": list(tile),
                   "collision": c.collision, "sponge_len": c.sponge_len, "probes": args.probes,
                   "stg_modes": c.n_modes,
                   "stats_every": c.stats_every,
                   "l2": "inputs larger than L2 (lattice %.2f GB)" % (2 * 19 * c.cells * bpc / 38 / 1e9),
                   "parallelism": f"replicas x{ws}"},
        "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s", "frac": achieved / peak,
                     "traffic": traffic, "kernel": "lbm_vec_zc_kernel (rows 1..ny-2, inlet and outlet nodes included) + wall rows: one step pass",
                     "kernel_ms": ms_step,
                     "bytes_per_cell": bpc, "peak_source": f"{peak_kind} hbm_gbs (copy)",
                     "inlet_kernel_ms": ms_inlet},
        "hbm_frac_of_step": bpc * c.cells * args.steps / (ms * 1e-3) / 1e9 / peak,
        "e2e": e2e,
        "gpu_launches": _launches(c, args.warmup, args.steps) + (args.steps if args.probes > 0 else 0),
        "clocks": clocks,
    }
    if args.storage == "fp32" and not args.no_companion:
        line["fp16s_companion"] = fp16_companion(c, args)
    if not args.no_cpu_baseline:
        line["cpu_baseline"] = cpu_baseline(args.workload, args.storage, args.cpu_steps,
                                            extra=dict(collision=c.collision, sponge_len=c.sponge_len,
                                                       sponge_K=c.sponge_K, sponge_p=c.sponge_p))
        line["cpu_baseline"].pop("seconds", None)
    print(json.dumps(line), flush=True)
    if dist is not None:
        dist.destroy_process_group()


def run_ensemble(args):
    """Batched ensemble: 64 independent channels (h from {16, 24, 32, 48, 64},
    Re_tau from {180, 395}, seeds 1..64) advanced by the batch executor, one
    CUDA-graph launch per block of steps; the batch's tile comes from the
    autotuner.  Prints one JSON line (whole-batch MLUPS)."""
    import torch
    from paper_2205_02774_gb300 import build
    build()
    from paper_2205_02774_gb300.channel import Channel
    from paper_2205_02774_gb300.serving import Batch
    from workloads.serving import ensemble
    jobs = ensemble(args.members, steps=args.steps, storage=args.storage)
    t0 = time.perf_counter()
    chans = [Channel.from_case(j.case, check_every=100, mass_tol=0.5) for j in jobs]
    b = Batch()
    for ch in chans:
        b.add(ch)
    tile = b.autotune(3)
    t_setup = time.perf_counter() - t0
    b.step(args.warmup)
    b.sync()
    sampler = ClockSampler(0)
    sampler.start()
    time.sleep(0.3)
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(b.stream)
    b.step(args.steps)
    e1.record(b.stream)
    e1.synchronize()
    clocks = sampler.stop()
    ms = e0.elapsed_time(e1)
    bad = [i for i, ch in enumerate(chans) if ch.stats()["rc"] != 0]
    cells = sum(ch.cells for ch in chans)
    peak, peak_kind = _peaks()
    bpc = BYTES_PER_CELL[args.storage]
    value = cells * args.steps / (ms * 1e-3) / 1e6
    achieved = bpc * cells * args.steps / (ms * 1e-3) / 1e9
    line = {"metric": "MLUPS", "value": value, "unit": "MLUPS", "n_gpus": 1, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms / args.steps, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": f"ensemble of {len(chans)} channels", "storage": args.storage, "cells": cells,
                       "members": len(chans), "block_steps": b.block_steps, "tile": tile,
                       "l2": "inputs larger than L2", "setup_s": t_setup},
            "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                         "frac": achieved / peak, "traffic": None, "scope": "whole step incl. inlet kernels",
                         "peak_source": f"{peak_kind} hbm_gbs (copy)"},
            "failed_members": bad, "clocks": clocks,
            "gpu_launches": sum(_launches(j.case, args.warmup, args.steps) for j in jobs)}
    b.close()
    for ch in chans:
        ch.close()
    print(json.dumps(line), flush=True)


def run_serve(args):
    """Served stream: Poisson arrivals (2 jobs/s) of channel jobs of 0.5M-20M
    cells (h = 20..65, aspect 12:2:3), Re_tau from {180, 395}, FP32 or FP16
    storage, own seeds, step counts uniform in [1000, 20000] x steps_scale,
    admitted by a 150 GB budget into the continuous-batching loop.  Prints one
    JSON line (jobs/s, aggregate MLUPS, p50/p99 latency)."""
    from paper_2205_02774_gb300 import build
    build()
    from paper_2205_02774_gb300.serving import serve
    from workloads.serving import poisson_stream
    sm = max(1, int(round(1000 * args.steps_scale)))
    jobs = poisson_stream(args.jobs, rate_per_s=2.0, steps_min=sm, steps_max=max(sm, int(round(20000 * args.steps_scale))))
    sampler = ClockSampler(0)
    sampler.start()
    results, rep = serve(jobs, hbm_budget_bytes=150e9, check_every=100, mass_tol=0.5)
    clocks = sampler.stop()
    offered = sum(j.case.cells * j.steps for j in jobs) / max(jobs[-1].arrival_s, 1e-9) / 1e6
    line = {"metric": "jobs/s", "value": rep["jobs_per_s"], "unit": "jobs/s", "n_gpus": 1,
            "higher_is_better": True, "data": "synthetic", "dtype": "f32",
            "config": {"workload": f"served stream of {len(jobs)} jobs", "arrival_rate_per_s": 2.0,
                       "steps_scale": args.steps_scale, "hbm_budget_gb": 150},
            "aggregate_mlups": rep["aggregate_mlups"], "offered_mlups": offered,
            "p50_latency_s": rep["p50_latency_s"], "p99_latency_s": rep["p99_latency_s"],
            "mean_latency_s": rep["mean_latency_s"], "wall_s": rep["wall_s"], "completed": rep["completed"],
            "failed": rep["failed"], "peak_active": rep["peak_active"],
            "peak_device_gb": rep["peak_device_bytes"] / 1e9, "clocks": clocks}
    print(json.dumps(line), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=4000)
    ap.add_argument("--warmup", type=int, default=200)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--workload", default="channel_768x128x192")
    ap.add_argument("--storage", choices=["fp32", "fp16s"], default="fp32")
    ap.add_argument("--cpu-steps", type=int, default=2)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--tile", default="", help="launch tile 'layout,zc,wall_zc' instead of the autotuner's")
    ap.add_argument("--no-companion", action="store_true", help="skip the FP16-storage companion run")
    ap.add_argument("--collision", choices=["regularized", "bgk"], default="regularized",
                    help="bulk collision: regularized BGK (default) or plain BGK")
    ap.add_argument("--probes", type=int, default=0,
                    help="time the steps through step_probed with this many velocity probes (seeded random cells)")
    ap.add_argument("--sponge", action="store_true",
                    help="sponge zone of 0.4 delta before the outlet (K = 1000, p = 3, as in the paper's channel)")
    ap.add_argument("--members", type=int, default=64, help="ensemble workload: channels in the batch")
    ap.add_argument("--jobs", type=int, default=60, help="serve workload: jobs in the stream")
    ap.add_argument("--steps-scale", type=float, default=0.1, help="serve workload: scale of the step counts")
    args = ap.parse_args()
    if args.warmup < 3:
        ap.error("--warmup must be >= 3")
    if args.impl == "reference":
        run_reference(args)
    elif args.workload == "ensemble":
        run_ensemble(args)
    elif args.workload == "serve":
        run_serve(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()

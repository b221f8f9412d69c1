"""Throughput benchmark of the STG-LBM hot path (MLUPS and HBM roofline).

One step = the STG inlet kernel plus the fused stream/collide pass over the
whole lattice (FP64 statistics every 10 steps, FP64 mass check every 100),
i.e. one pass of the whole hot path.  Default workload: the refined Re_tau =
180 channel on a 1536x256x384 D3Q19 lattice (h = 128, 151M cells, 200 STG
modes) with populations stored as shifted FP16 (f - w_i) written by
stochastic rounding (FP32 arithmetic), two lattices, inputs resident in HBM,
lattice (5.7 GB) far larger than L2.  The same line carries companions on
the same lattice (round-to-nearest FP16, FP32, and the one-lattice in-place
update), the end-to-end figure through the public API, the CPU oracle on a
bounded sample, and two sub-objects: the batched ensemble (64 channels) and
the served job stream (Poisson arrivals, continuous batching, p50/p99
latency).

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
  python bench.py --storage fp32 --streaming aa --workload channel_768x128x192 --no-extras
  python bench.py --workload ensemble [--members 64] [--steps K]   (batched ensemble alone)
  python bench.py --workload serve [--jobs 100] [--serve-steps-scale 0.25]   (served stream alone)

N > 1 runs one independent channel per GPU (weak scaling, no collective on
the data path); the companion runs on rank 0, the CPU baseline and the
ensemble and served sub-objects only at N = 1.  ``--impl reference`` times the
CPU FP64 oracle on the host cores instead (bounded sample).  Prints one JSON
line (rank 0).
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

BYTES_PER_CELL = {"fp32": 152, "fp16s": 76, "fp16sr": 76}  # 19 populations read + 19 written


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
    for f in ("step_kernel.cu", "step_kernel.cuh", "d3q19.cuh", "internal.h", "lbm_cell.cuh", "lbm_pair.cuh", "reduce.cuh"):
        with open(os.path.join(ROOT, "paper_2205_02774_gb300", "csrc", f)) as fh:
            src = fh.read()
        src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
        src = re.sub(r"//[^\n]*", "", src)
        h.update("".join(src.split()).encode())
    return h.hexdigest()[:16]


def _traffic(workload, storage, streaming="pull"):
    """DRAM bytes of one step pass from the committed ncu summary, if it was
    taken on the current kernel source (else None)."""
    tag = storage if streaming == "pull" else f"{storage}_{streaming}"
    path = os.path.join(ROOT, "profiles", f"lbm_step_kernel_{workload}_{tag}.md")
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


def _oracle_single_thread(workload, storage, ny=8, steps=1, extra=None):
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


def _slice_rows(full, budget_cells, steps):
    """Wall-normal rows of a bounded oracle sample: the full streamwise length
    and span (so the per-cell share of inlet-generator work, N / nx, and the
    OpenMP split over z are those of the full channel), at least 2 rows (walls
    on both), about budget_cells cell updates over `steps` steps."""
    return max(2, min(full.ny, int(budget_cells / (steps * full.nx * full.nz))))


def cpu_baseline(workload, storage, steps, budget_cells, extra=None):
    """The CPU FP64 oracle, as it stands, on a bounded sample of the workload
    (a slice of the channel with fewer wall-normal rows) on all host cores
    (OpenMP over z), plus the same oracle on one thread.  `extra`: case
    fields of the variant (collision, sponge)."""
    import oracle
    from workloads import case
    full = case(workload).with_(storage=storage, **dict(extra or {}))
    c = full.with_(ny=_slice_rows(full, budget_cells, steps))
    sim = oracle.Sim.from_case(c)
    t0 = time.perf_counter()
    sim.step(steps)
    dt = time.perf_counter() - t0
    del sim
    return {"value": c.cells * steps / dt / 1e6, "unit": "MLUPS", "cores": oracle.threads(), "kind": "oracle",
            "sample": f"{steps} steps of a {c.nx}x{c.ny}x{c.nz} slice of the {workload} channel "
                      f"(FP64, OpenMP over z, inlet, outlet, walls, {c.n_modes} STG modes)",
            "seconds": dt, "single_thread": _oracle_single_thread(workload, storage, extra=extra)}


def run_reference(args):
    """Reference arm: the CPU FP64 oracle on the host cores.  Each step is one
    oracle step of a bounded sample of the workload (a slice with fewer
    wall-normal rows), sized so that warm-up + timed steps stay within about
    a minute of CPU time."""
    ws, rank, _ = _dist()
    if rank != 0:
        return
    import oracle
    from workloads import case
    full = case(args.workload)
    c = full.with_(ny=_slice_rows(full, 3.0e8, args.steps + args.warmup))
    sim = oracle.Sim.from_case(c)
    sim.step(args.warmup)
    t0 = time.perf_counter()
    sim.step(args.steps)
    t = time.perf_counter() - t0
    value = c.cells * args.steps / t / 1e6
    sample = (f"{args.steps} timed steps (+{args.warmup} warm-up) of a {c.nx}x{c.ny}x{c.nz} slice of the "
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


RATED_HBM_GBS = 7900.0  # nominal HBM3e bandwidth of the part (context beside the measured copy peak)


def roofline(bpc, cells, ms_step, ms_inlet, traffic, kernel):
    """Roofline object of one step pass: algorithmic bytes (bpc per cell) over
    the event-timed pass, against the measured copy bandwidth and, for
    context, the rated HBM bandwidth; with the ncu DRAM traffic of the pass
    (when the committed counters match the kernel source) also the bandwidth
    that traffic implies."""
    peak, peak_kind = _peaks()
    achieved = bpc * cells / (ms_step * 1e-3) / 1e9
    return {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s", "frac": achieved / peak,
            "traffic": traffic, "kernel": kernel, "kernel_ms": ms_step, "bytes_per_cell": bpc,
            "peak_source": f"{peak_kind} hbm_gbs (copy)", "rated_peak": RATED_HBM_GBS,
            "frac_of_rated": achieved / RATED_HBM_GBS,
            "traffic_gbs": (traffic / (ms_step * 1e-3) / 1e9) if traffic else None,
            "inlet_kernel_ms": ms_inlet}


STEP_KERNEL = "lbm_vec_zc_kernel (rows 1..ny-2, inlet and outlet nodes included) + wall rows: one step pass"


def measure_channel(c, args, rank=0, dist=None, seed=None, sample_clocks=True):
    """One channel timed the bench's way: the library's autotuned launch tile
    (or --tile), W warm-up steps, then K steps between CUDA events on the
    channel's stream with a barrier and a device synchronisation on both
    sides; then the device time of single step passes (stg_lbm_step_timed).
    Returns the timings, clocks and throughput (aggregated over ranks when
    `dist` is given)."""
    import torch
    from paper_2205_02774_gb300.channel import Channel
    ch = Channel.from_case(c, check_every=100, mass_tol=0.5, seed=c.seed if seed is None else seed)
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

    sampler = ClockSampler(torch.cuda.current_device()) if (rank == 0 and sample_clocks) else None
    if sampler:
        sampler.start()
        time.sleep(0.3)
    barrier()
    if args.probes > 0:
        # probe series of the paper's post-processing (B_uu, T_t): random cells, seeded
        import numpy as np
        prng = np.random.default_rng(1234 + rank)
        xyz = np.stack([prng.integers(0, n, args.probes) for n in (c.nx, c.ny, c.nz)], axis=1).astype(np.int32)
        ch.set_probes(xyz)
        ch.step_probed(args.steps)  # untimed: allocates the series buffer before the timed region
        torch.cuda.synchronize()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(ch.stream)
    if args.probes > 0:
        series = ch.step_probed(args.steps)  # synchronises; ends with the series' copy to the host
        assert series.shape == (args.steps, args.probes, 3)
    else:
        ch.step(args.steps)
    e1.record(ch.stream)
    e1.synchronize()
    barrier()
    clocks = sampler.stop() if sampler else None
    ms, value = aggregate_ranks(e0.elapsed_time(e1), c.cells, args.steps, dist, device="cuda")
    st = ch.stats()
    if st["rc"] != 0:
        raise RuntimeError(f"channel check failed: {st['error']}")
    # dominant kernel: device time of one step pass (the two step launches)
    ms_step, ms_inlet = ch.step_timed(min(200, max(20, args.steps // 10)))
    device_gb = ch.info()["device_bytes"] / 1e9
    ch.close()
    del ch
    torch.cuda.synchronize()
    bpc = BYTES_PER_CELL[c.storage]
    peak, _ = _peaks()
    return {"value": value, "ms": ms, "ms_per_step": ms / args.steps, "tile": list(tile), "clocks": clocks,
            "device_gb": device_gb,
            "ms_step": ms_step, "ms_inlet": ms_inlet,
            "hbm_frac_of_step": bpc * c.cells * args.steps / (ms * 1e-3) / 1e9 / peak}


def end_to_end(c, steps):
    """The same metric end to end through the public API with host buffers:
    create (RANS profile uploaded from host memory, device allocation from an
    emptied caching allocator, inlet tables, initial state, graph capture),
    K steps, the statistics read back to the host (FP64 sums) and destroy."""
    import torch
    from paper_2205_02774_gb300.channel import Channel
    prof = c.profile()
    host_in = sum(a.nbytes for a in (prof.y_c, prof.U, prof.k, prof.eps, prof.R))
    torch.cuda.empty_cache()  # create() must allocate its device memory for real
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    ch = Channel.from_case(c, check_every=100, mass_tol=0.5)
    ch.step(steps)
    st = ch.stats()
    ch.close()
    t1 = time.perf_counter()
    host_out = 9 * c.nx * c.ny * 8 + 16
    assert st["rc"] == 0, st["error"]
    return {"value": c.cells * steps / (t1 - t0) / 1e6, "unit": "MLUPS",
            "h2d_bytes_per_step": host_in / steps, "d2h_bytes_per_step": host_out / steps,
            "seconds": t1 - t0, "includes": "create (host profile upload, device allocation after emptying the "
                                            "caching allocator, tables, init, graph capture) + step(K) + stats "
                                            "(FP64 sums to host) + destroy"}


def run_ours(args):
    import torch
    from paper_2205_02774_gb300 import build
    build()
    from workloads import case

    ws, rank, local = _dist()
    torch.cuda.set_device(local)
    dist = None
    if ws > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    c = _variant(case(args.workload).with_(storage=args.storage, streaming=args.streaming), args)
    m = measure_channel(c, args, rank, dist, seed=rank_seed(c.seed, rank))
    if dist is not None:
        dist.barrier()
        dist.destroy_process_group()
    if rank != 0:
        return

    # the committed counters were taken on the default variant
    plain = args.collision == "regularized" and not args.sponge and args.probes == 0
    traffic = _traffic(args.workload, c.storage, c.streaming) if plain else None
    line = {
        "metric": "MLUPS", "value": m["value"], "unit": "MLUPS", "n_gpus": ws, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": m["ms_per_step"], "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": {"workload": args.workload, "storage": c.storage, "streaming": c.streaming, "cells": c.cells,
                   "lattice": "D3Q19", "arithmetic": "fp32", "tile": m["tile"], "device_gb": m["device_gb"],
                   "collision": c.collision, "sponge_len": c.sponge_len, "probes": args.probes,
                   "stg_modes": c.n_modes,
                   "stats_every": c.stats_every,
                   "l2": "inputs larger than L2 (lattice %.2f GB)" % (19 * c.cells * BYTES_PER_CELL[c.storage] / 38 / 1e9),
                   "parallelism": f"replicas x{ws}"},
        "roofline": roofline(BYTES_PER_CELL[c.storage], c.cells, m["ms_step"], m["ms_inlet"], traffic, STEP_KERNEL),
        "hbm_frac_of_step": m["hbm_frac_of_step"],
        "gpu_launches": _launches(c, args.warmup, args.steps) + (args.steps if args.probes > 0 else 0),
        "clocks": m["clocks"],
    }
    line["e2e"] = end_to_end(c, args.steps)
    if not args.no_companion:
        # the same channel in the other storage forms and streaming scheme, timed the same way
        comps = []
        for st in ("fp16sr", "fp16s", "fp32"):
            if st != c.storage:
                comps.append((st, c.streaming))
        comps.append((c.storage, "aa" if c.streaming == "pull" else "pull"))
        line["companions"] = []
        for st, sm in comps:
            c2 = c.with_(storage=st, streaming=sm)
            m2 = measure_channel(c2, args)
            t2 = _traffic(args.workload, st, sm) if plain else None
            line["companions"].append({
                "storage": st, "streaming": sm, "value": m2["value"], "unit": "MLUPS",
                "ms_per_step": m2["ms_per_step"], "hbm_frac_of_step": m2["hbm_frac_of_step"], "tile": m2["tile"],
                "clocks": m2["clocks"], "device_gb": m2["device_gb"],
                "roofline": roofline(BYTES_PER_CELL[st], c2.cells, m2["ms_step"], m2["ms_inlet"], t2, STEP_KERNEL),
                "gpu_launches": _launches(c2, args.warmup, args.steps)})
    if ws == 1 and not args.no_cpu_baseline:
        line["cpu_baseline"] = cpu_baseline(args.workload, c.storage, args.cpu_steps, args.cpu_cells,
                                            extra=dict(collision=c.collision, sponge_len=c.sponge_len,
                                                       sponge_K=c.sponge_K, sponge_p=c.sponge_p))
        line["cpu_baseline"].pop("seconds", None)
    if ws == 1 and not args.no_extras:
        import torch
        torch.cuda.empty_cache()
        line["ensemble"] = ensemble_run(args.members, args.ensemble_steps, max(3, min(args.warmup, 20)), "fp32")
        torch.cuda.empty_cache()
        line["served"] = serve_run(args.jobs, args.serve_steps_scale)
    print(json.dumps(line), flush=True)


def ensemble_run(members, steps, warmup, storage):
    """Batched ensemble: `members` independent channels (h from {16, 24, 32,
    48, 64}, Re_tau from {180, 395}, seeds 1..members) advanced by the batch
    executor, one CUDA-graph launch per block of steps; the batch's tile from
    the autotuner.  Whole-batch MLUPS over the whole step (inlet kernels
    included) and its fraction of the HBM roofline."""
    import torch
    from paper_2205_02774_gb300.channel import Channel
    from paper_2205_02774_gb300.serving import Batch
    from workloads.serving import ensemble
    jobs = ensemble(members, steps=steps, storage=storage)
    t0 = time.perf_counter()
    chans = [Channel.from_case(j.case, check_every=100, mass_tol=0.5) for j in jobs]
    b = Batch()
    for ch in chans:
        b.add(ch)
    tile = b.autotune(3)
    t_setup = time.perf_counter() - t0
    b.step(warmup)
    b.sync()
    sampler = ClockSampler(torch.cuda.current_device())
    sampler.start()
    time.sleep(0.3)
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(b.stream)
    b.step(steps)
    e1.record(b.stream)
    e1.synchronize()
    clocks = sampler.stop()
    ms = e0.elapsed_time(e1)
    bad = [i for i, ch in enumerate(chans) if ch.stats()["rc"] != 0]
    cells = sum(ch.cells for ch in chans)
    peak, peak_kind = _peaks()
    bpc = BYTES_PER_CELL[storage]
    achieved = bpc * cells * steps / (ms * 1e-3) / 1e9
    out = {"workload": f"ensemble of {len(chans)} channels", "value": cells * steps / (ms * 1e-3) / 1e6,
           "unit": "MLUPS", "steps": steps, "warmup": warmup, "ms_per_step": ms / steps, "storage": storage,
           "cells": cells, "members": len(chans), "block_steps": b.block_steps, "tile": tile, "setup_s": t_setup,
           "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s", "frac": achieved / peak,
                        "traffic": None, "scope": "whole step incl. inlet kernels",
                        "peak_source": f"{peak_kind} hbm_gbs (copy)"},
           "failed_members": bad, "clocks": clocks,
           "gpu_launches": sum(_launches(j.case, warmup, steps) for j in jobs)}
    b.close()
    for ch in chans:
        ch.close()
    return out


def serve_run(n_jobs, steps_scale, streaming="pull"):
    """Served stream: Poisson arrivals (2 jobs/s) of channel jobs of 0.5M-20M
    cells (h = 20..65, aspect 12:2:3), Re_tau from {180, 395}, FP32 or FP16
    storage, own seeds, step counts uniform in [1000, 20000] x steps_scale,
    admitted by a 150 GB budget into the continuous-batching loop.  Jobs/s,
    aggregate and offered MLUPS, p50/p99 completion latency."""
    import torch
    from paper_2205_02774_gb300.serving import serve
    from workloads.serving import poisson_stream
    sm = max(1, int(round(1000 * steps_scale)))
    jobs = poisson_stream(n_jobs, rate_per_s=2.0, steps_min=sm, steps_max=max(sm, int(round(20000 * steps_scale))),
                          streaming=streaming)
    sampler = ClockSampler(torch.cuda.current_device())
    sampler.start()
    results, rep = serve(jobs, hbm_budget_bytes=150e9, check_every=100, mass_tol=0.5)
    clocks = sampler.stop()
    offered = sum(j.case.cells * j.steps for j in jobs) / max(jobs[-1].arrival_s, 1e-9) / 1e6
    return {"workload": f"served stream of {len(jobs)} jobs", "value": rep["jobs_per_s"], "unit": "jobs/s",
            "arrival_rate_per_s": 2.0, "steps_scale": steps_scale, "steps_range": [sm, int(round(20000 * steps_scale))],
            "streaming": streaming,
            "hbm_budget_gb": 150,
            "aggregate_mlups": rep["aggregate_mlups"], "offered_mlups": offered,
            "p50_latency_s": rep["p50_latency_s"], "p99_latency_s": rep["p99_latency_s"],
            "mean_latency_s": rep["mean_latency_s"], "wall_s": rep["wall_s"], "completed": rep["completed"],
            "failed": rep["failed"], "peak_active": rep["peak_active"],
            "peak_device_gb": rep["peak_device_bytes"] / 1e9, "clocks": clocks}


def run_ensemble(args):
    """--workload ensemble: the batched ensemble alone as the bench line."""
    from paper_2205_02774_gb300 import build
    build()
    e = ensemble_run(args.members, args.steps, args.warmup, args.storage)
    line = {"metric": "MLUPS", "value": e["value"], "unit": "MLUPS", "n_gpus": 1, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": e["ms_per_step"], "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": e["workload"], "storage": args.storage, "cells": e["cells"],
                       "members": e["members"], "block_steps": e["block_steps"], "tile": e["tile"],
                       "l2": "inputs larger than L2", "setup_s": e["setup_s"]},
            "roofline": e["roofline"], "failed_members": e["failed_members"], "clocks": e["clocks"],
            "gpu_launches": e["gpu_launches"]}
    print(json.dumps(line), flush=True)


def run_serve(args):
    """--workload serve: the served stream alone as the bench line."""
    from paper_2205_02774_gb300 import build
    build()
    s = serve_run(args.jobs, args.serve_steps_scale, args.streaming)
    line = {"metric": "jobs/s", "value": s["value"], "unit": "jobs/s", "n_gpus": 1,
            "higher_is_better": True, "data": "synthetic", "dtype": "f32",
            "config": {"workload": s["workload"], "arrival_rate_per_s": 2.0,
                       "steps_scale": args.serve_steps_scale, "hbm_budget_gb": 150}}
    line.update({k: v for k, v in s.items() if k not in ("workload", "value", "unit")})
    print(json.dumps(line), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=1000)
    ap.add_argument("--warmup", type=int, default=50)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--workload", default="channel_1536x256x384")
    ap.add_argument("--storage", choices=["fp32", "fp16s", "fp16sr"], default="fp16sr",
                    help="population storage: FP32, shifted binary16 rounded to nearest, or by stochastic rounding")
    ap.add_argument("--streaming", choices=["pull", "aa"], default="pull",
                    help="two lattices (pull) or one lattice updated in place (AA pattern)")
    ap.add_argument("--cpu-steps", type=int, default=4, help="cpu_baseline: oracle steps on the sample")
    ap.add_argument("--cpu-cells", type=float, default=1.5e8,
                    help="cpu_baseline: cell updates of the sample (a slice with fewer wall-normal rows)")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--tile", default="", help="launch tile 'layout,zc,wall_zc' instead of the autotuner's")
    ap.add_argument("--no-companion", action="store_true",
                    help="skip the companion runs (other storage forms, other streaming scheme)")
    ap.add_argument("--no-extras", action="store_true", help="skip the ensemble and served-stream sub-objects")
    ap.add_argument("--collision", choices=["regularized", "bgk"], default="regularized",
                    help="bulk collision: regularized BGK (default) or plain BGK")
    ap.add_argument("--probes", type=int, default=0,
                    help="time the steps through step_probed with this many velocity probes (seeded random cells)")
    ap.add_argument("--sponge", action="store_true",
                    help="sponge zone of 0.4 delta before the outlet (K = 1000, p = 3, as in the paper's channel)")
    ap.add_argument("--members", type=int, default=64, help="ensemble: channels in the batch")
    ap.add_argument("--ensemble-steps", type=int, default=1000, help="ensemble sub-object: timed steps")
    ap.add_argument("--jobs", type=int, default=100, help="served stream: jobs")
    ap.add_argument("--serve-steps-scale", type=float, default=0.25, help="served stream: scale of the step counts")
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

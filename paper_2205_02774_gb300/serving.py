"""Python front ends of the batch executor and the serving loop.

``Batch`` groups Channel objects so that one CUDA-graph launch per block of
steps advances all of them (stg_batch_*); ``serve`` hands a list of jobs with
arrival times to the library's continuous-batching loop (stg_serve_run).
Argument marshalling only: scheduling, admission and the steps run in the
library.
"""
from __future__ import annotations

import ctypes as C

import numpy as np

from . import capi as A
from .channel import case_kwargs, create_structs


class Batch:
    def __init__(self, stream=None):
        import torch
        self.stream = stream if stream is not None else torch.cuda.Stream()
        self.b = A.stg_batch_create(self.stream.cuda_stream)
        self.members = []

    def add(self, ch):
        A.stg_batch_add(self.b, ch.h)
        self.members.append(ch)

    def remove(self, ch):
        A.stg_batch_remove(self.b, ch.h)
        self.members.remove(ch)

    def __len__(self):
        return A.stg_batch_size(self.b)

    @property
    def block_steps(self):
        return A.stg_batch_block_steps(self.b)

    def step(self, n):
        A.stg_batch_step(self.b, n)

    def sync(self):
        A.stg_batch_sync(self.b)

    def autotune(self, trial_passes=5):
        return A.stg_batch_autotune(self.b, trial_passes)

    def close(self):
        if self.b:
            A.stg_batch_destroy(self.b)
            self.b = None
            self.members = []

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def serve(jobs, hbm_budget_bytes, max_active=0, check_every=100, mass_tol=0.5, keep_stats=False, stream=None):
    """Run workloads.serving.Job objects through stg_serve_run.  Returns
    (results, report): one dict per job (status, admit/finish/latency
    seconds, n_samples, mass, and the FP64 statistics sums when keep_stats)
    and the run's report as a dict."""
    if not jobs:
        return [], {}
    keep = []
    arr = (A.stg_job * len(jobs))()
    outs = []
    for i, jb in enumerate(jobs):
        c = jb.case
        kw = case_kwargs(c)
        d, r, p, k = create_structs(c.nx, c.ny, c.nz, check_every=check_every, mass_tol=mass_tol, **kw)
        keep += [d, r, p, k]
        arr[i].arrival_s = jb.arrival_s
        arr[i].domain = C.pointer(d)
        arr[i].rans = C.pointer(r) if r is not None else None
        arr[i].stg = C.pointer(p) if p is not None else None
        arr[i].seed = c.seed
        arr[i].steps = jb.steps
        if keep_stats:
            m = np.zeros((3, c.ny, c.nx))
            q = np.zeros((6, c.ny, c.nx))
            arr[i].mean_sum = m.ctypes.data_as(A.c_double_p)
            arr[i].rey_sum = q.ctypes.data_as(A.c_double_p)
            outs.append((m, q))
        else:
            outs.append(None)
    cfg = A.stg_serve_config(float(hbm_budget_bytes), int(max_active), 0)
    res, rep = A.stg_serve_run(arr, cfg, stream.cuda_stream if stream is not None else 0)
    results = []
    for i, jb in enumerate(jobs):
        r = res[i]
        d = dict(status=r.status, admit_s=r.admit_s, finish_s=r.finish_s, latency_s=r.latency_s,
                 n_samples=r.n_samples, device_bytes=r.device_bytes, mass=r.mass, mass0=r.mass0,
                 cells=jb.case.cells, steps=jb.steps, arrival_s=jb.arrival_s)
        if outs[i] is not None:
            d["mean_sum"], d["rey_sum"] = outs[i]
        results.append(d)
    report = {f: getattr(rep, f) for f, _ in A.stg_serve_report._fields_ if f != "pad0"}
    return results, report

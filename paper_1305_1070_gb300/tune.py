"""Measured search over the plan-level choices of a workload: the leaf size
of the nested-dissection tree and the energies per call, each candidate with
the per-launch kernel tuner (nd_autotune) inside.  The winner is the
configuration with the most energies per second on a timed call; the search
runs once per workload, and its result (and the tuned handle) is reused for
every later step.

All device work runs in the library through Solver; this module only times
and compares.
"""
from __future__ import annotations

import time

import numpy as np
import torch

from . import ndgf
from .solver import Solver

ND_ERR_OOM, ND_ERR_UNSUPPORTED = 5, 8


def time_call(s: Solver, E, reps: int = 1) -> float:
    """Milliseconds of one step() on the energies E (CUDA events, after one untimed call)."""
    s.step(E)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(reps):
        s.step(E)
    e1.record()
    torch.cuda.synchronize()
    return e0.elapsed_time(e1) / reps


def tune_plan(dev, tr, *, precision: int, delay: int, leafs=(16, 24, 32), chunks=(64, 128), reps: int = 1,
              keep_best: bool = True):
    """Returns (best, table, solver): best = {"leaf", "chunk", "energies_per_s"},
    table = one row per candidate (leaf, chunk, energies/s, kernel-tuner summary,
    seconds spent), solver = the winner built again and tuned (None unless
    keep_best; one workspace lives at a time).  Candidates whose workspace does
    not fit on the device are skipped."""
    E_all = torch.as_tensor(np.asarray(tr.energies, dtype=np.float64), device="cuda")
    table, best = [], None
    for leaf in leafs:
        for chunk in chunks:
            chunk = min(chunk, len(E_all))
            t0 = time.perf_counter()
            try:
                s = Solver(dev, tr, precision=precision, max_ne=chunk, delay=delay, leaf_size=leaf)
            except (ndgf.NDError, torch.cuda.OutOfMemoryError) as exc:
                # a workspace too large for the device, or a tree the library does not take; other errors propagate
                if isinstance(exc, ndgf.NDError) and exc.status not in (ND_ERR_OOM, ND_ERR_UNSUPPORTED):
                    raise
                table.append({"leaf": leaf, "chunk": chunk, "skipped": str(exc)[:120]})
                continue
            E = E_all[:chunk]
            info = s.autotune(E, reps=reps)
            ms = time_call(s, E)
            row = {"leaf": leaf, "chunk": chunk, "energies_per_s": round(chunk / (ms * 1e-3), 3), "tuner": info,
                   "seconds": round(time.perf_counter() - t0, 2)}
            table.append(row)
            if best is None or row["energies_per_s"] > best["energies_per_s"]:
                best = {"leaf": leaf, "chunk": chunk, "energies_per_s": row["energies_per_s"]}
            del s
            torch.cuda.empty_cache()
    solver = None
    if keep_best and best is not None:
        solver = Solver(dev, tr, precision=precision, max_ne=best["chunk"], delay=delay, leaf_size=best["leaf"])
        solver.autotune(E_all[:best["chunk"]], reps=reps)
    return best, table, solver

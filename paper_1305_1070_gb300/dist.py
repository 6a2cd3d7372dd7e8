"""Energies across ranks (one process per GPU).

The energies are independent problems (paper Sec. 1: G^r, G^< and G^> are
computed energy by energy).  The only exchange is the energy integral of the
observables, the electron density n_j = 2 sum_e w_e Im G^<_jj(E_e) / (2 pi)
and the terminal current, a sum over energies: each rank integrates its
block of the global energy grid with the global trapezoid weights, and one
all-reduce (sum) gives the device-wide result.  Host logic only; the
arithmetic of every energy runs in the library's kernels.
"""
from __future__ import annotations

import numpy as np


def shard(n_total: int, rank: int, world: int) -> slice:
    """Contiguous block of the energy indices 0..n_total-1 for one rank; block
    sizes differ by at most one, lower ranks first."""
    if world < 1 or not 0 <= rank < world:
        raise ValueError("rank outside 0..world-1")
    base, extra = divmod(n_total, world)
    start = rank * base + min(rank, extra)
    return slice(start, start + base + (1 if rank < extra else 0))


def trapezoid_weights(energies) -> np.ndarray:
    """Trapezoid weights of a grid (the weights of a shard are the global
    weights of its indices: the end points of a block are interior points of
    the global grid and keep their full weight)."""
    E = np.asarray(energies, dtype=np.float64)
    w = np.zeros_like(E)
    if E.size > 1:
        d = np.diff(E)
        w[:-1] += 0.5 * d
        w[1:] += 0.5 * d
    return w


def global_grid(emin: float, emax: float, per_rank: int, world: int) -> np.ndarray:
    """Weak scaling: every rank keeps per_rank energies, the grid over
    [emin, emax] gets finer with the number of ranks (inclusive linspace)."""
    return np.linspace(emin, emax, per_rank * world)


def reduce_sum(tensor, group=None):
    """Sum a per-rank partial result (density, current) over all ranks, in place."""
    import torch.distributed as dist
    if dist.is_available() and dist.is_initialized() and dist.get_world_size() > 1:
        dist.all_reduce(tensor, op=dist.ReduceOp.SUM, group=group)
    return tensor

"""Energy sharding and the density all-reduce on world_size-2 gloo ranks (CPU).

Every energy of the global grid lands on exactly one rank; the sum over ranks
of the per-rank trapezoid integrals equals the single-process integral of the
whole grid (the energy integral of the density is the only exchange step).
"""
import os
import socket

import numpy as np
import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402

from paper_1305_1070_gb300 import dist as ndist  # noqa: E402


def test_shard_covers_every_energy_once():
    for n in (1, 7, 256, 1000):
        for world in (1, 2, 3, 8):
            seen = np.zeros(n, dtype=int)
            sizes = []
            for r in range(world):
                s = ndist.shard(n, r, world)
                seen[s] += 1
                sizes.append(s.stop - s.start)
            assert (seen == 1).all()
            assert max(sizes) - min(sizes) <= 1
    with pytest.raises(ValueError):
        ndist.shard(10, 2, 2)


def _integrand(E, n_sites):  # a smooth stand-in for Im G^<_jj(E), deterministic per energy
    j = np.arange(n_sites)
    return np.sin(3.0 * E[:, None] + 0.1 * j[None, :]) * np.exp(-E[:, None])


def _worker(rank, world, port, out):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    E = ndist.global_grid(0.0, 0.5, 16, world)
    w = ndist.trapezoid_weights(E)
    s = ndist.shard(len(E), rank, world)
    part = torch.as_tensor((w[s, None] * _integrand(E[s], 5)).sum(axis=0))
    ndist.reduce_sum(part)
    out[rank] = part.numpy().tolist()
    dist.destroy_process_group()


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def test_density_all_reduce_equals_single_process():
    world = 2
    mgr = mp.Manager()
    out = mgr.dict()
    mp.spawn(_worker, args=(world, _free_port(), out), nprocs=world, join=True)
    E = ndist.global_grid(0.0, 0.5, 16, world)
    ref = (ndist.trapezoid_weights(E)[:, None] * _integrand(E, 5)).sum(axis=0)
    for r in range(world):
        assert np.allclose(out[r], ref, rtol=0, atol=1e-14)

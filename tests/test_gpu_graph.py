"""CUDA-graph replay of the launch sequences (ND_FACT_GRAPH): the first call
of each shape records the few hundred launches of nd_factor / nd_diag_green
into a graph, later calls replay it with one launch.  The results equal the
directly launched path bit for bit, for new energies of the same count, for a
different energy count (a second graph), for host outputs and with the
tensor-core products; and they match the oracle (paper Eq. (1)-(2))."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from oracle import dense, observables  # noqa: E402
from paper_1305_1070_gb300 import build, ndgf, workloads  # noqa: E402
from paper_1305_1070_gb300.solver import Solver  # noqa: E402

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("precision,tile", [(ndgf.ND_PREC_FP64, "auto"), (ndgf.ND_PREC_FP32X2, "tc")])
def test_graph_replay_matches_direct_launches(precision, tile):
    build.build()
    dev = workloads.superlattice(28, 8, disorder=0.03, seed=17)
    tr = workloads.Transport(energies=np.linspace(0.02, 0.48, 6), gamma_ph=3e-3, mu_ph=0.05)
    kw = dict(precision=precision, leaf_size=12, delay=2, tile=tile, max_ne=4)
    plain = Solver(dev, tr, **kw)
    graph = Solver(dev, tr, graph=True, **kw)
    batches = [tr.energies[:4], tr.energies[2:6], tr.energies[:4], tr.energies[4:6], tr.energies[1:3]]
    for E in batches:
        a = [g.clone() for g in plain.step(E)]
        b = [g.clone() for g in graph.step(E)]
        torch.cuda.synchronize()
        for x, y in zip(a, b):
            assert torch.equal(x, y)
    ref = dense.green_diag(dev, workloads.Transport(energies=batches[-1], gamma_ph=3e-3, mu_ph=0.05))
    tol = 1e-10 if precision == ndgf.ND_PREC_FP64 else 1e-9
    for k, g in zip(("Gr", "Gl", "Gg"), b):
        for i in range(len(batches[-1])):
            assert observables.rel_err(g[i].cpu().numpy(), ref[k][i]) < tol
    # host outputs through the recorded graph
    n_e = 4
    outs = [np.zeros((n_e, dev.n), dtype=np.complex128) for _ in range(3)]
    graph.step_host(tr.energies[:n_e].copy(), *outs)
    torch.cuda.synchronize()
    want = [g.clone() for g in plain.step(tr.energies[:n_e])]
    for o, w in zip(outs, want):
        assert np.array_equal(o, w.cpu().numpy())
    assert ndgf.nd_fact_status(graph.fact) == 0

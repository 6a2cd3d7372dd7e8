"""A batch of uneven devices solved as one graph (disjoint union, one tree
per device, every level launch spanning all devices) against the oracle
applied to each device alone (paper Eq. (1)-(2)): the union's diagonals on
device d's sites equal device d's own, complex128 at 1e-10 and FP32 pairs at
1e-9 relative per energy and device, and each device's current spectrum.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from oracle import dense, observables  # noqa: E402
from paper_1305_1070_gb300 import build, ndgf, workloads  # noqa: E402

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib():
    build.build()
    if not torch.cuda.is_available():
        pytest.fail("CUDA device required")


@pytest.mark.parametrize("precision,tol", [(ndgf.ND_PREC_FP64, 1e-10), (ndgf.ND_PREC_FP32X2, 1e-9)])
def test_union_matches_each_device(precision, tol):
    from paper_1305_1070_gb300.solver import Solver
    devs = [workloads.superlattice(L, W, disorder=0.02, seed=L) for L, W in ((12, 4), (20, 8), (9, 6), (16, 5))]
    dev = workloads.union(devs)
    tr = workloads.Transport(energies=np.array([0.04, 0.21, 0.43]), mu=(0.25, 0.0), kT=0.03)
    s = Solver(dev, tr, precision=precision, leaf_size=16, delay=2)
    Gr, Gl, Gg = s.step(tr.energies)
    cur = [s.current(c, tr.n_e)[0].cpu().numpy() for c in range(2 * len(devs))]
    torch.cuda.synchronize()
    got = {"Gr": Gr.cpu().numpy(), "Gl": Gl.cpu().numpy(), "Gg": Gg.cpu().numpy()}
    worst = 0.0
    for d, sub in enumerate(devs):
        lo, hi = dev.site_offsets[d], dev.site_offsets[d + 1]
        ref = dense.green_diag(sub, tr)
        for k in ("Gr", "Gl", "Gg"):
            for e in range(tr.n_e):
                err = observables.rel_err(got[k][e, lo:hi], ref[k][e])
                worst = max(worst, err)
                assert err <= tol, (d, k, e, err)
        for e, E in enumerate(tr.energies):
            full = dense.green_full(sub, tr, float(E))
            t = full["terms"]
            for c, idx in enumerate(sub.contacts):
                i_ref = np.real(observables.current_spectrum(t.sigma_lesser[c], t.sigma_greater[c],
                                                             full["Gl"][np.ix_(idx, idx)], full["Gg"][np.ix_(idx, idx)]))
                assert abs(cur[2 * d + c][e] - i_ref) <= tol * max(1e-3, abs(i_ref))
    print(f"union precision {precision}: worst {worst:.3e}")


@pytest.mark.parametrize("precision,tol", [(ndgf.ND_PREC_FP32X2, 1e-9), (ndgf.ND_PREC_MIXED, 1e-3)])
def test_union_roots_in_one_launch(precision, tol):
    """Six devices of one shape: their roots sit on one tree level and are
    inverted in one launch, each in its own complex128 scratch region."""
    from paper_1305_1070_gb300.solver import Solver
    devs = [workloads.superlattice(14, 6, disorder=0.05, seed=100 + k) for k in range(6)]
    dev = workloads.union(devs)
    tr = workloads.Transport(energies=np.array([0.11, 0.37]), mu=(0.25, 0.0), kT=0.03)
    s = Solver(dev, tr, precision=precision, leaf_size=16, delay=2)
    Gr, Gl, Gg = s.step(tr.energies)
    torch.cuda.synchronize()
    assert s.singular_pivots() == 0
    got = {"Gr": Gr.cpu().numpy(), "Gl": Gl.cpu().numpy(), "Gg": Gg.cpu().numpy()}
    for d, sub in enumerate(devs):
        lo, hi = dev.site_offsets[d], dev.site_offsets[d + 1]
        ref = dense.green_diag(sub, tr)
        for k in ("Gr", "Gl", "Gg"):
            for e in range(tr.n_e):
                assert observables.rel_err(got[k][e, lo:hi], ref[k][e]) <= tol, (d, k, e)

"""Self-consistent Born iteration of an elastic local phonon self-energy
(Sigma_ph,jj = D G_jj for r, <, >; nd_phonon_scba between solves) against the
dense oracle (oracle/scba.py): after the same number of updates from the same
constant-broadening first iterate the diagonals agree element by element
(complex128 1e-10, FP32 pairs with delayed pivots 1e-9); at convergence the
terminal current spectra balance, which the constant broadening does not."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from oracle import observables, scba  # noqa: E402
from paper_1305_1070_gb300 import build, ndgf, workloads  # noqa: E402

pytestmark = pytest.mark.gpu
D = 0.02


@pytest.fixture(scope="module", autouse=True)
def _lib():
    build.build()
    if not torch.cuda.is_available():
        pytest.fail("CUDA device required")


def _case():
    dev = workloads.superlattice(14, 5, disorder=0.05, seed=21)
    tr = workloads.Transport(energies=np.array([0.75, 0.9]), mu=(0.9, 0.7), kT=0.03, gamma_ph=2e-3, mu_ph=0.8)
    return dev, tr


@pytest.mark.parametrize("precision,delay,tol", [(ndgf.ND_PREC_FP64, 0, 1e-10), (ndgf.ND_PREC_FP32X2, 2, 1e-9)])
def test_scba_updates_match_oracle(precision, delay, tol):
    from paper_1305_1070_gb300.solver import Solver
    dev, tr = _case()
    s = Solver(dev, tr, precision=precision, leaf_size=8, delay=delay)
    Gr, Gl, Gg, n_upd, _ = s.scba(tr.energies, D, updates=6)
    torch.cuda.synchronize()
    assert n_upd == 6 and s.singular_pivots() == 0
    got = {"Gr": Gr.cpu().numpy(), "Gl": Gl.cpu().numpy(), "Gg": Gg.cpu().numpy()}
    for e, E in enumerate(tr.energies):
        ref = scba.scba(dev, tr, float(E), D, updates=6)
        for k in ("Gr", "Gl", "Gg"):
            err = observables.rel_err(got[k][e], ref[k])
            assert err <= tol, f"{k} E = {E}: rel err {err:.3e}"


def test_scba_converges_and_balances_currents():
    from paper_1305_1070_gb300.solver import Solver
    dev, tr = _case()
    s = Solver(dev, tr, precision=ndgf.ND_PREC_FP64, leaf_size=8)
    *_, n_upd, change = s.scba(tr.energies, D, tol=1e-12)
    torch.cuda.synchronize()
    assert change <= 1e-12 and n_upd < 100
    iL = s.current(0, tr.n_e)[0].cpu().numpy()
    iR = s.current(1, tr.n_e)[0].cpu().numpy()
    print("SCBA updates", n_upd, "currents", iL, iR)
    assert np.all(np.abs(iL + iR) <= 1e-8 * np.abs(iL))

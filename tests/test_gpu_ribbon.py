"""The armchair graphene nanoribbon (paper Sec. 4.2.2: tight binding, hopping
-3.1 eV, on-site 0, Fermi level 0, E = 0.5 eV) through the CUDA path against
the dense oracle, element by element on diag G^r, G^<, G^>: complex128 at
1e-10 and FP32 pairs with delayed pivots at 1e-9 (relative max error per
energy), the latter also with every Schur product on the tensor cores.  The
leads are perfect ribbons (renormalisation-decimation on the device)."""
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


@pytest.fixture(scope="module")
def case():
    dev = workloads.agnr(8, 5, disorder=0.05, seed=1309)  # 160 atoms, 10 dimer lines
    tr = workloads.Transport(energies=np.array([0.5, -0.35, 0.12]), mu=(0.0, 0.0))
    return dev, tr, dense.green_diag(dev, tr)


@pytest.mark.parametrize("precision,delay,tile,tol", [(ndgf.ND_PREC_FP64, 0, "auto", 1e-10),
                                                      (ndgf.ND_PREC_FP32X2, 2, "auto", 1e-9),
                                                      (ndgf.ND_PREC_FP32X2, 2, "tc", 1e-9)])
def test_ribbon_against_oracle(case, precision, delay, tile, tol):
    from paper_1305_1070_gb300.solver import Solver
    dev, tr, ref = case
    s = Solver(dev, tr, precision=precision, leaf_size=12, delay=delay, tile=tile)
    Gr, Gl, Gg = s.step(tr.energies)
    torch.cuda.synchronize()
    assert s.singular_pivots() == 0
    assert all(st == (0, 0) for st in s.lead_status())
    got = {"Gr": Gr.cpu().numpy(), "Gl": Gl.cpu().numpy(), "Gg": Gg.cpu().numpy()}
    for k in ("Gr", "Gl", "Gg"):
        for e in range(tr.n_e):
            err = observables.rel_err(got[k][e], ref[k][e])
            assert err <= tol, f"{k} E = {tr.energies[e]}: rel err {err:.3e}"

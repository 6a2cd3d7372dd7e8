"""Terminal current spectrum (S10, Meir-Wingreen) through the C ABI against
the oracle: i_c(E) = Tr[Sigma^<_c G^>_cc - Sigma^>_c G^<_cc] from the dense
G^< and G^> (paper Eq. (1)-(2)), per energy and contact, in complex128
(1e-10 relative to the largest |i_c| of the batch) and FP32 pairs (1e-9),
with and without delayed pivots; without phonons the two contacts carry
opposite currents (conservation up to the eta leak) and the imaginary part
vanishes.
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


def _oracle(dev, tr):
    out = np.zeros((2, tr.n_e))
    for e, E in enumerate(tr.energies):
        full = dense.green_full(dev, tr, float(E))
        t = full["terms"]
        for c, idx in enumerate(dev.contacts):
            out[c, e] = np.real(observables.current_spectrum(t.sigma_lesser[c], t.sigma_greater[c],
                                                             full["Gl"][np.ix_(idx, idx)], full["Gg"][np.ix_(idx, idx)]))
    return out


def _gpu(dev, tr, precision, delay, leaf):
    from paper_1305_1070_gb300.solver import Solver
    s = Solver(dev, tr, precision=precision, leaf_size=leaf, delay=delay)
    s.step(tr.energies)
    res = [s.current(c, tr.n_e) for c in range(2)]
    torch.cuda.synchronize()
    return np.stack([r[0].cpu().numpy() for r in res]), np.stack([r[1].cpu().numpy() for r in res])


@pytest.mark.parametrize("precision,tol", [(ndgf.ND_PREC_FP64, 1e-10), (ndgf.ND_PREC_FP32X2, 1e-9)])
@pytest.mark.parametrize("delay", [0, 2])
def test_current_matches_oracle(precision, tol, delay):
    dev = workloads.superlattice(24, 8, disorder=0.05, seed=11)
    tr = workloads.Transport(energies=np.linspace(0.02, 0.45, 7), mu=(0.3, 0.0), kT=0.03)
    ref = _oracle(dev, tr)
    got, im = _gpu(dev, tr, precision, delay, leaf=16)
    scale = np.abs(ref).max()
    assert scale > 1e-6
    err = np.abs(got - ref).max() / scale
    print(f"current precision {precision} delay {delay}: rel err {err:.3e}")
    assert err <= tol
    assert np.abs(im).max() <= tol * scale
    # conservation up to the eta leak
    assert np.abs(got[0] + got[1]).max() <= 1e-5 * scale


def test_current_with_phonons():
    dev = workloads.superlattice(20, 6, disorder=0.03, seed=2)
    tr = workloads.Transport(energies=np.array([0.07, 0.33]), mu=(0.25, 0.0), kT=0.03, gamma_ph=5e-3, mu_ph=0.1)
    ref = _oracle(dev, tr)
    got, _ = _gpu(dev, tr, ndgf.ND_PREC_FP64, 2, leaf=16)
    assert np.abs(got - ref).max() <= 1e-10 * np.abs(ref).max()

"""Adjoint of the density (nd_density_gradient and autograd.density) against
the oracle.

For L = sum_j c_j n_j and H_kk = H0_kk + V_k, the dense oracle
(oracle.response.adjoint_terms) gives dL/dV_k from the full G^r and Sigma^<:
    t_k = sum_{a,b in contacts} Sigma^<_ab conj(U_kb) conj(Z_ka),
    U = G^r[:, contacts],  Z = G^r diag(c) conj(U),
    dL/dV_k = (2/pi) sum_e w_e Im t_k(E_e),
itself pinned here against central finite differences of the oracle density.
The GPU terms t_k match it per energy (complex128 1e-10, FP32 pairs 1e-9,
relative to the largest |t| of the energy), and the autograd gradient of the
GPU density matches central differences of the GPU forward.
"""
import math

import numpy as np
import pytest

torch = pytest.importorskip("torch")

from oracle import dense, response  # noqa: E402
from paper_1305_1070_gb300 import build, ndgf, workloads  # noqa: E402

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib():
    build.build()
    if not torch.cuda.is_available():
        pytest.fail("CUDA device required")


def _t_oracle(dev, tr, c):
    return response.adjoint_terms(dev, tr, c)


def _dev():
    return workloads.superlattice(18, 6, disorder=0.05, seed=7)


def _tr():
    return workloads.Transport(energies=np.array([0.06, 0.19, 0.33]), mu=(0.25, 0.0), kT=0.03)


def test_oracle_formula_matches_finite_differences():
    dev, tr = workloads.superlattice(8, 4, disorder=0.05, seed=3), _tr()
    rng = np.random.default_rng(1)
    c = rng.uniform(0.0, 1.0, dev.n)
    w = np.full(tr.n_e, 0.1)

    def loss(k, h):
        d2 = workloads.superlattice(8, 4, disorder=0.05, seed=3)
        for p in range(d2.rowptr[k], d2.rowptr[k + 1]):
            if d2.colind[p] == k:
                d2.values[p] += h
        return sum(w[e] * np.sum(c * np.diag(dense.green_full(d2, tr, float(E))["Gl"]).imag) / math.pi
                   for e, E in enumerate(tr.energies))

    grad = (2.0 / math.pi) * (w[:, None] * _t_oracle(dev, tr, c).imag).sum(axis=0)
    h = 1e-5
    for k in (0, 9, 21):
        fd = (loss(k, h) - loss(k, -h)) / (2 * h)
        assert abs(grad[k] - fd) <= 1e-6 * max(abs(fd), 1e-3 * np.abs(grad).max())


@pytest.mark.parametrize("precision,tol", [(ndgf.ND_PREC_FP64, 1e-10), (ndgf.ND_PREC_FP32X2, 1e-9)])
@pytest.mark.parametrize("delay", [0, 2])
def test_gradient_terms_match_oracle(precision, tol, delay):
    from paper_1305_1070_gb300.solver import Solver
    dev, tr = _dev(), _tr()
    c = np.random.default_rng(2).uniform(0.0, 1.0, dev.n)
    s = Solver(dev, tr, precision=precision, leaf_size=16, delay=delay, adjoint=True)
    s.step(tr.energies)
    t = s.density_gradient_terms(c, tr.n_e).cpu().numpy()
    ref = _t_oracle(dev, tr, c)
    for e in range(tr.n_e):
        err = np.abs(t[e] - ref[e]).max() / np.abs(ref[e]).max()
        print(f"precision {precision} delay {delay} energy {e}: rel err {err:.3e}")
        assert err <= tol


def test_gradient_terms_tensor_cores():
    """The adjoint solves with every Schur product on the tensor cores (FP32 pairs,
    exact BF16 digit products): the same terms at the FP32-pair tolerance."""
    from paper_1305_1070_gb300.solver import Solver
    dev, tr = _dev(), _tr()
    c = np.random.default_rng(2).uniform(0.0, 1.0, dev.n)
    s = Solver(dev, tr, precision=ndgf.ND_PREC_FP32X2, leaf_size=16, delay=2, adjoint=True, tile="tc")
    s.step(tr.energies)
    t = s.density_gradient_terms(c, tr.n_e).cpu().numpy()
    assert s.singular_pivots() == 0
    ref = _t_oracle(dev, tr, c)
    for e in range(tr.n_e):
        err = np.abs(t[e] - ref[e]).max() / np.abs(ref[e]).max()
        print(f"tensor cores energy {e}: rel err {err:.3e}")
        assert err <= 1e-9


def test_autograd_matches_finite_differences():
    from paper_1305_1070_gb300 import autograd
    from paper_1305_1070_gb300.solver import Solver
    dev, tr = _dev(), _tr()
    s = Solver(dev, tr, precision=ndgf.ND_PREC_FP64, leaf_size=16, delay=2, adjoint=True, max_ne=2)
    E = torch.as_tensor(tr.energies, device="cuda")
    w = torch.full((tr.n_e,), 0.1, dtype=torch.float64, device="cuda")
    c = torch.as_tensor(np.random.default_rng(3).uniform(0.0, 1.0, dev.n), device="cuda")
    V = torch.zeros(dev.n, dtype=torch.float64, device="cuda", requires_grad=True)
    loss = (c * autograd.density(V, s, E, w)).sum()
    loss.backward()
    g = V.grad.cpu().numpy()
    h = 1e-5
    for k in (3, 40, 77):
        vals = []
        for sgn in (1.0, -1.0):
            dV = torch.zeros(dev.n, dtype=torch.float64, device="cuda")
            dV[k] = sgn * h
            with torch.no_grad():
                vals.append(float((c * autograd.density(dV, s, E, w)).sum()))
        fd = (vals[0] - vals[1]) / (2 * h)
        print(f"site {k}: adjoint {g[k]:.10e} finite difference {fd:.10e}")
        assert abs(g[k] - fd) <= 1e-6 * max(abs(fd), 1e-3 * np.abs(g).max())


def test_gradient_errors():
    from paper_1305_1070_gb300.solver import Solver
    dev, tr = _dev(), _tr()
    s = Solver(dev, tr, leaf_size=16)
    s.step(tr.energies)
    with pytest.raises(ndgf.NDError):
        s.density_gradient_terms(np.ones(dev.n), tr.n_e)
    trp = workloads.Transport(energies=tr.energies, mu=(0.25, 0.0), kT=0.03, gamma_ph=5e-3)
    s = Solver(dev, trp, leaf_size=16, adjoint=True)
    s.step(trp.energies)
    with pytest.raises(ndgf.NDError):
        s.density_gradient_terms(np.ones(dev.n), trp.n_e)

"""Pins of the Schroedinger-Poisson oracle (oracle/poisson, response, sp):
the discrete Poisson operator against its closed-form eigenfunctions; the
density Jacobian against central differences of the oracle density; the
Newton iteration against its defining properties (F = 0 at the end, the
quadratic decrease of |F|, and the decoupled case lam = 0)."""
import numpy as np
import pytest

from oracle import poisson, response, sp
from paper_1305_1070_gb300 import workloads


@pytest.mark.parametrize("L,W,p,q", [(7, 5, 1, 0), (9, 4, 3, 2), (6, 6, 6, 5)])
def test_poisson_eigenfunctions(L, W, p, q):
    # Dirichlet (ghost zeros) along x: sin(p pi (x + 1) / (L + 1)), eigenvalue 2 - 2 cos(p pi / (L + 1));
    # Neumann along y: cos(q pi (y + 1/2) / W), eigenvalue 2 - 2 cos(q pi / W)
    x, y = np.meshgrid(np.arange(L), np.arange(W), indexing="ij")
    u = (np.sin(p * np.pi * (x + 1) / (L + 1)) * np.cos(q * np.pi * (y + 0.5) / W)).ravel()
    mu = 2 - 2 * np.cos(p * np.pi / (L + 1)) + 2 - 2 * np.cos(q * np.pi / W)
    assert np.abs(poisson.apply(L, W, u) - mu * u).max() < 1e-13
    assert np.abs(poisson.solve(L, W, mu * u) - u).max() < 1e-12
    K = poisson.operator(L, W).toarray()
    assert np.allclose(K, K.T) and np.linalg.eigvalsh(K).min() > 0


def _small():
    # W = 6: the lowest transverse mode opens at 2t (1 - cos(pi / 7)) = 0.45 eV, so the
    # window 0.4..1.4 eV with Fermi levels 0.95 / 0.75 eV carries a sizeable density
    dev = workloads.superlattice(10, 6, disorder=0.03, seed=2)
    tr = workloads.Transport(energies=np.linspace(0.4, 1.4, 11), mu=(0.95, 0.75), kT=0.03)
    return dev, tr


def test_jacobian_central_differences():
    dev, tr = _small()
    U = 0.02 * np.sin(np.arange(dev.n) * 0.7)
    chi = response.jacobian(dev, tr, U)
    h = 1e-5
    for k in (0, 7, 21, dev.n - 1):
        e = np.zeros(dev.n)
        e[k] = h
        fd = (response.density(dev, tr, U + e) - response.density(dev, tr, U - e)) / (2 * h)
        assert np.abs(chi[:, k] - fd).max() <= 1e-6 * np.abs(fd).max(), k
    # not symmetric out of equilibrium (mu_L != mu_R); symmetric in equilibrium,
    # where G^< = -f (G - G^a) up to the 2 eta f G G^a leak of the broadening
    assert np.abs(chi - chi.T).max() > 1e-2 * np.abs(chi).max()
    teq = workloads.Transport(energies=tr.energies, mu=(0.85, 0.85), kT=0.03, eta=1e-12)
    ceq = response.jacobian(dev, teq, U)
    assert np.abs(ceq - ceq.T).max() < 1e-9 * np.abs(ceq).max()


def test_newton_converges():
    dev, tr = _small()
    L, W, lam = 10, 6, 2.8
    n0 = response.density(dev, tr)
    nD = np.full(dev.n, n0.mean())
    its, res = sp.newton(dev, tr, L, W, lam, nD, steps=6)
    print("  |F| per Newton step:", res)
    assert res[-1] < 1e-12 * max(1.0, res[0])
    # quadratic decrease while far from the rounding floor
    for m in range(len(res) - 1):
        if res[m + 1] > 1e-11:
            assert res[m + 1] <= 10.0 * res[m] ** 2 / max(res[0], 1e-300) + 1e-11, (m, res)
    F = sp.residual(dev, tr, L, W, lam, nD, its[-1])
    assert np.abs(F).max() < 1e-12
    # without coupling the potential stays zero
    its0, res0 = sp.newton(dev, tr, L, W, 0.0, nD, steps=2)
    assert np.abs(its0).max() == 0.0 and res0.max() == 0.0


def test_adjoint_and_forward_terms_against_jacobian():
    """The per-energy terms of the adjoint (gradient) and the forward
    (directional derivative) products, integrated with (2/pi) sum_e w_e Im,
    equal c^T chi and chi v of the dense Jacobian (itself pinned by central
    differences above); without phonons G^< = U Sigma^<_CC U^dagger."""
    from oracle import observables
    dev, tr = _small()
    U = 0.01 * np.cos(np.arange(dev.n))
    chi = response.jacobian(dev, tr, U)
    w = observables.trapezoid_weights(tr.energies)
    rng = np.random.Generator(np.random.PCG64(3))
    c = rng.uniform(0, 1, dev.n)
    v = rng.normal(size=dev.n)
    g = (2 / np.pi) * (w[:, None] * response.adjoint_terms(dev, tr, c, U).imag).sum(axis=0)
    jv = (2 / np.pi) * (w[:, None] * response.forward_terms(dev, tr, v, U).imag).sum(axis=0)
    assert np.abs(g - c @ chi).max() < 1e-10 * np.abs(c @ chi).max()
    assert np.abs(jv - chi @ v).max() < 1e-10 * np.abs(chi @ v).max()

"""Pins of the oracle's Green's functions: closed forms, invariants stated by the
paper (Sec. 3.1: G^r complex symmetric, G^< skew-Hermitian), the spectral sum
rule, Landauer = Meir-Wingreen, transfer-matrix transmission, and agreement of
the three independent methods (dense definition, RGF, sparse solves)."""
import numpy as np
import pytest

from oracle import dense, observables, rgf, sampled, selfenergy, transfer
from oracle.problem import dense_sigma
from paper_1305_1070_gb300 import workloads


def _tr(energies, **kw):
    return workloads.Transport(energies=np.asarray(energies, dtype=float), **kw)


@pytest.mark.parametrize("ph", [0.0, 4e-3])
def test_invariants_superlattice_dense(ph):
    # with phonons the sum rule ties Sigma^r_ph to Sigma^<_ph and Sigma^>_ph: i (S^r - S^a) = i (S^> - S^<)
    dev = workloads.superlattice(10, 5, disorder=0.05, seed=3)
    tr = _tr([0.13], gamma_ph=ph, mu_ph=0.05)
    full = dense.green_full(dev, tr, 0.13)
    G, Gl, Gg, A = full["Gr"], full["Gl"], full["Gg"], full["A"]
    assert np.abs(A @ G - np.eye(dev.n)).max() < 1e-9
    assert np.abs(G - G.T).max() < 1e-10 * np.abs(G).max()  # complex symmetric
    assert np.abs(Gl + Gl.conj().T).max() < 1e-10 * np.abs(Gl).max()  # skew-Hermitian
    assert np.abs(Gg + Gg.conj().T).max() < 1e-10 * np.abs(Gg).max()
    assert np.abs(np.diag(Gl).real).max() < 1e-10 * np.abs(Gl).max()
    # sum rule: i (G - G^a) = G (Gamma + 2 eta) G^a  and  i (G^> - G^<) = G Gamma G^a
    terms = full["terms"]
    Gam = 1j * (dense_sigma(dev, terms, "greater") - dense_sigma(dev, terms, "lesser"))
    lhs = 1j * (G - G.conj().T)
    rhs = G @ (Gam + 2 * tr.eta * np.eye(dev.n)) @ G.conj().T
    assert np.abs(lhs - rhs).max() < 1e-9 * np.abs(lhs).max()
    assert np.abs(1j * (Gg - Gl) - G @ Gam @ G.conj().T).max() < 1e-9 * np.abs(Gl).max()


def test_uniform_chain_closed_form():
    # uniform chain with uniform leads = infinite chain: G_jj = -i / (2 t sin k)
    t, N = 1.0, 12
    dev = workloads.chain(N, t=t)
    for E in (-1.2, 0.3, 1.5):
        tr = _tr([E], eta=1e-9, mu=(0.2, -0.1), kT=0.05)
        d = dense.green_diag(dev, tr)
        k = np.arccos(-E / (2 * t))
        g_inf = -1j / (2 * t * np.sin(k))
        assert np.abs(d["Gr"][0] - g_inf).max() < 1e-6
        fL = selfenergy.fermi(E, 0.2, 0.05)
        fR = selfenergy.fermi(E, -0.1, 0.05)
        assert np.abs(d["Gl"][0] - 1j * (fL + fR) / (2 * t * np.sin(k))).max() < 1e-6


def test_uniform_wire_mode_sum():
    # uniform 2D wire: G_jj = sum_n chi_n(y)^2 / sqrt((z - eps_n)^2 - 4 t^2), Im < 0 branch
    L, W = 7, 5
    dev = workloads.superlattice(L, W, v_barrier=0.0)
    t = workloads.fd_hopping(0.5, 0.067)
    E = 0.9
    tr = _tr([E], eta=1e-9)
    d = dense.green_diag(dev, tr)["Gr"][0]
    y = np.arange(1, W + 1)
    expect = np.zeros(W, dtype=complex)
    for nmode in range(1, W + 1):
        chi = np.sqrt(2.0 / (W + 1)) * np.sin(nmode * np.pi * y / (W + 1))
        eps = 4 * t - 2 * t * np.cos(nmode * np.pi / (W + 1))
        z = E + 1e-9j
        s = np.sqrt((z - eps) ** 2 - 4 * t * t + 0j)
        g = 1.0 / s
        if g.imag > 0:
            g = -g
        expect += chi ** 2 * g
    for x in range(L):
        assert np.abs(d[x * W:(x + 1) * W] - expect).max() < 1e-6 * np.abs(expect).max()


@pytest.mark.parametrize("E", [-1.1, -0.4, 0.25, 0.9])
def test_landauer_equals_transfer_matrix(E):
    t = 1.0
    V = np.array([0.0, 0.4, 0.7, 0.7, 0.4, 0.0, 0.2])
    dev = workloads.chain(len(V), t=t, potential=V)
    tr = _tr([E], eta=1e-10)
    full = dense.green_full(dev, tr, E)
    G = full["Gr"]
    sL, sR = full["terms"].sigma_r
    T_green = observables.transmission(sL, sR, G[np.ix_(dev.contacts[0], dev.contacts[1])])
    T_tm = transfer.chain_transmission(E, V, t=t)
    assert abs(T_green - T_tm) < 1e-7


def test_meir_wingreen_equals_landauer_and_conservation():
    # 1.2 eV: one open transverse mode in the 4-wide leads (it opens at 0.87 eV), T = 0.67
    dev = workloads.superlattice(8, 4, disorder=0.1, seed=5)
    E = 1.2
    tr = _tr([E], mu=(1.3, 1.0), kT=0.03)
    full = dense.green_full(dev, tr, E)
    terms = full["terms"]
    cL, cR = dev.contacts
    iL = observables.current_spectrum(terms.sigma_lesser[0], terms.sigma_greater[0],
                                      full["Gl"][np.ix_(cL, cL)], full["Gg"][np.ix_(cL, cL)])
    iR = observables.current_spectrum(terms.sigma_lesser[1], terms.sigma_greater[1],
                                      full["Gl"][np.ix_(cR, cR)], full["Gg"][np.ix_(cR, cR)])
    T = observables.transmission(terms.sigma_r[0], terms.sigma_r[1], full["Gr"][np.ix_(cL, cR)])
    # occupations from the reservoirs' own Fermi levels (left 1.3 eV, right 1.0 eV), not the oracle's copy
    fL, fR = selfenergy.fermi(E, 1.3, 0.03), selfenergy.fermi(E, 1.0, 0.03)
    assert T > 0.5 and fL - fR > 0.9
    assert abs(iL - T * (fL - fR)) < 1e-9 * max(1.0, abs(iL))
    assert abs(iL + iR) < 1e-6 * max(1e-3, abs(iL))  # conservation up to the eta leak


def test_mirror_symmetry_at_equal_fermi_levels():
    # symmetric potential, mu_L = mu_R: density mirror symmetric (paper Sec. 4.2.1)
    L, W = 12, 4
    prof = np.array([0, 0, .3, .3, 0, .1, .1, 0, .3, .3, 0, 0], dtype=float)
    dev = workloads.superlattice(L, W, potential=np.repeat(prof, W))
    tr = _tr([0.05, 0.2], mu=(0.1, 0.1))
    gl = dense.green_diag(dev, tr)["Gl"].reshape(2, L, W)
    assert np.abs(gl - gl[:, ::-1, :]).max() < 1e-9 * np.abs(gl).max()


@pytest.mark.parametrize("ph", [0.0, 5e-3])
def test_rgf_equals_dense_superlattice(ph):
    dev = workloads.superlattice(9, 5, disorder=0.02, seed=11)
    tr = _tr([0.0, 0.07, 0.33], gamma_ph=ph, mu_ph=0.05)
    a = dense.green_diag(dev, tr)
    b = rgf.green_diag(dev, tr)
    for k in ("Gr", "Gl", "Gg"):
        for e in range(3):
            assert observables.rel_err(b[k][e], a[k][e]) < 1e-10


def test_rgf_equals_dense_cnt():
    dev = workloads.cnt_zigzag(2, disorder=0.1, seed=2)
    tr = _tr([-0.6, 0.35], gamma_ph=5e-3, mu_ph=0.05)
    a = dense.green_diag(dev, tr)
    b = rgf.green_diag(dev, tr)
    for k in ("Gr", "Gl", "Gg"):
        for e in range(2):
            assert observables.rel_err(b[k][e], a[k][e]) < 1e-9


def test_sampled_equals_dense():
    dev = workloads.superlattice(8, 6, disorder=0.02, seed=1)
    tr = _tr([0.21], gamma_ph=2e-3)
    a = dense.green_diag(dev, tr)
    sites = [0, 5, 17, 30, 47]
    s = sampled.green_sites(dev, tr, 0.21, sites)
    for k in ("Gr", "Gl", "Gg"):
        assert observables.rel_err(s[k], a[k][0][sites]) < 1e-10


def test_density_uniform_chain_closed_form():
    """Pin of observables.density (paper Sec. 1: the density is the energy
    integral of Im G^<_jj) against a closed form that shares no step with it.
    On the uniform chain (on-site 0, hopping -t, uniform leads: the infinite
    chain) G^<_jj(E) = i (f_L + f_R) / (2 t sin k) with E = -2t cos k, so with
    spin 2, n_j = (1/pi) int dE (f_L + f_R) / (2 t sin k) = (1/pi) int dk (f_L + f_R)
    over the k range of the grid.  The oracle integrates the dense definition's
    G^< by the trapezoid rule on an energy grid; the closed form is integrated
    in k by adaptive quadrature.  A wrong spin factor (x2), a real part taken
    for the imaginary one (~0), a lead occupation lost (f_L only) or wrong
    trapezoid weights are each off by far more than the tolerance."""
    from scipy.integrate import quad
    t, N = 1.0, 6
    mu_L, mu_R, kT = 0.3, -0.4, 0.05
    dev = workloads.chain(N, t=t)
    k = np.linspace(0.05, np.pi - 0.05, 3001)
    E = -2.0 * t * np.cos(k)
    tr = _tr(E, eta=1e-9, mu=(mu_L, mu_R), kT=kT)
    n = observables.density(dense.green_diag(dev, tr)["Gl"], E)
    occ = lambda q: selfenergy.fermi(-2 * t * np.cos(q), mu_L, kT) + selfenergy.fermi(-2 * t * np.cos(q), mu_R, kT)
    expect = quad(occ, k[0], k[-1], limit=200, epsabs=1e-13)[0] / np.pi
    assert np.abs(n - expect).max() < 2e-5 * expect, (n, expect)
    # the same device at T -> 0 and mu = 0 on both sides: half filling of the full band
    k = np.linspace(1e-3, np.pi - 1e-3, 4001)
    E = -2.0 * t * np.cos(k)
    n0 = observables.density(dense.green_diag(dev, _tr(E, eta=1e-9, mu=(0.0, 0.0), kT=1e-4))["Gl"], E)
    assert np.abs(n0 - 1.0).max() < 2e-3

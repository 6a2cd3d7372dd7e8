"""Pins of the oracle's lead self-energies (paper Sec. 2) against the defining
Dyson equation, an independent method and closed forms."""
import numpy as np
import pytest

from oracle import leads, selfenergy
from paper_1305_1070_gb300 import workloads


def _dyson_residual(H00, H01, g, z):
    m = H00.shape[0]
    rhs = np.linalg.inv(z * np.eye(m) - H00 - H01 @ g @ H01.T)
    return np.abs(g - rhs).max() / np.abs(g).max()


@pytest.mark.parametrize("E", [0.0, 0.05, 0.31, 0.5, 2.0, 9.5, 12.0])
def test_modes_satisfy_dyson_fd_lead(E):
    dev = workloads.superlattice(4, 8)
    lead = dev.leads[0]
    z = E + 1e-6j
    g = leads.surface_green_modes(lead.H00, lead.hop, z)
    assert _dyson_residual(lead.H00, lead.H01, g, z) < 1e-10
    # retarded: the broadening i(S - S^dagger) is positive semi-definite
    S = lead.tau @ g @ lead.tau.T
    gam = selfenergy.broadening(S)
    assert np.linalg.eigvalsh(0.5 * (gam + gam.conj().T)).min() > -1e-12
    # complex symmetric (real-symmetric lead)
    assert np.abs(S - S.T).max() < 1e-12 * np.abs(S).max()


@pytest.mark.parametrize("E", [0.02, 0.3, 1.7])
def test_decimation_equals_modes_fd_lead(E):
    dev = workloads.superlattice(4, 6)
    lead = dev.leads[0]
    z = E + 1e-3j
    g1 = leads.surface_green_modes(lead.H00, lead.hop, z)
    g2 = leads.surface_green_decimation(lead.H00, lead.H01, z)
    assert np.abs(g1 - g2).max() / np.abs(g1).max() < 1e-9


@pytest.mark.parametrize("E", [-0.9, -0.2, 0.4, 1.0])
def test_decimation_satisfies_dyson_cnt_lead(E):
    dev = workloads.cnt_zigzag(2)
    for lead in dev.leads:
        z = E + 1e-4j
        g = leads.surface_green_decimation(lead.H00, lead.H01, z)
        assert _dyson_residual(lead.H00, lead.H01, g, z) < 1e-8


@pytest.mark.parametrize("E", [-1.5, -0.3, 0.0, 0.9, 1.99])
def test_chain_lead_closed_form(E):
    # single-mode lead with on-site 0, hopping -t: Sigma = -t exp(i k), E = -2 t cos k
    t = 1.0
    dev = workloads.chain(3, t=t)
    S = leads.self_energy(dev.leads[0], E, 1e-12)
    k = np.arccos(-E / (2 * t))
    assert abs(S[0, 0] - (-t * np.exp(1j * k))) < 1e-6


def test_fd_hopping_value():
    # t = hbar^2 / (2 m* a^2) with m* = 0.067, a = 0.5 nm
    assert abs(workloads.fd_hopping(0.5, 0.067) - 2.2746162) < 1e-6


def test_fermi_limits():
    kT = 0.025852
    assert selfenergy.fermi(0.1, 0.1, kT) == pytest.approx(0.5)
    assert selfenergy.fermi(10.0, 0.0, kT) < 1e-100
    assert selfenergy.fermi(-10.0, 0.0, kT) == pytest.approx(1.0)
    x = 0.037
    assert selfenergy.fermi(x, 0.0, kT) + selfenergy.fermi(-x, 0.0, kT) == pytest.approx(1.0, abs=1e-15)

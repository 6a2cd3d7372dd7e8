"""Pins of the self-consistent Born oracle (elastic local dephasing,
Sigma_ph,jj = D G_jj for r, <, >) against what the physics fixes:

* at the fixed point the scattering current sum_j [Sigma^<_ph G^> - Sigma^>_ph
  G^<]_jj is zero, so the two terminal current spectra balance per energy up to
  the eta leak, while the constant broadening (not self-consistent) does not;
* D = 0: one update removes the phonon self-energy and the result is the
  ballistic dense definition;
* the iteration contracts (the relative change falls geometrically);
* the converged self-energy is causal and consistent: its broadening
  -2 Im Sigma^r_ph equals i (Sigma^>_ph - Sigma^<_ph) (= D times the local
  spectral function), up to the eta term."""
import numpy as np
import pytest

from oracle import dense, observables, scba
from paper_1305_1070_gb300 import workloads


def _case():
    # 5 sites wide: the first transverse subband opens at 0.61 eV; energies in
    # it, inside the bias window
    dev = workloads.superlattice(14, 5, disorder=0.05, seed=21)
    tr = workloads.Transport(energies=np.array([0.75, 0.9]), mu=(0.9, 0.7), kT=0.03, gamma_ph=2e-3, mu_ph=0.8)
    return dev, tr


@pytest.mark.parametrize("E", [0.75, 0.9])
def test_fixed_point_conserves_current(E):
    dev, tr = _case()
    r = scba.scba(dev, tr, E, D=0.02)
    assert r["change"] <= 1e-13
    iL, iR = r["currents"]
    assert abs(r["i_ph"]) <= 1e-12 * abs(iL)
    assert abs(iL + iR) <= 1e-8 * abs(iL), (iL, iR)
    gamma_r = -2.0 * r["ph_r"].imag
    gamma_lg = (1j * (r["ph_greater"] - r["ph_lesser"])).real
    assert np.all(gamma_r >= 0.0)
    assert np.abs(gamma_r - gamma_lg).max() <= 1e-4 * gamma_r.max()
    # the constant broadening (the first iterate) exchanges current with the bath
    r0 = scba.scba(dev, tr, E, D=0.02, updates=0)
    assert abs(r0["currents"].sum()) > 1e-2 * abs(r0["currents"][0])


def test_zero_strength_is_ballistic():
    dev, tr = _case()
    r = scba.scba(dev, tr, 0.9, D=0.0, updates=1)
    tr0 = workloads.Transport(energies=np.array([0.9]), mu=tr.mu, kT=tr.kT)
    ref = dense.green_diag(dev, tr0)
    for k in ("Gr", "Gl", "Gg"):
        assert observables.rel_err(r[k], ref[k][0]) <= 1e-12


def test_iteration_contracts():
    dev, tr = _case()
    ch = [scba.scba(dev, tr, 0.75, D=0.02, updates=u)["change"] for u in (2, 4, 6, 8)]
    assert all(b < 0.5 * a for a, b in zip(ch, ch[1:])), ch

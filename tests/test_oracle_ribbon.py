"""The armchair graphene nanoribbon workload (paper Sec. 4.2.2: tight binding,
hopping -3.1 eV, on-site 0, one energy E = 0.5 eV) pinned on the oracle side:
a perfect ribbon between perfect ribbon leads is ballistic, so its Landauer
transmission T = Tr[Gamma_L G_LR Gamma_R G_LR^dagger] is the number of open
subbands, an integer, whatever the device length, up to the absorption of
the eta = 1e-6 broadening on the device sites (a few 1e-6 here).  Ribbons
whose number of dimer lines is 2 mod 3 have a band through E = 0 and carry at
least one channel at every energy; a 10-line ribbon is gapped at 0.5 eV."""
import numpy as np
import pytest

from oracle import dense, observables
from paper_1305_1070_gb300 import workloads


def _transmission(dev, E):
    tr = workloads.Transport(energies=np.array([E]), mu=(0.0, 0.0))
    full = dense.green_full(dev, tr, float(E))
    t = full["terms"]
    cL, cR = dev.contacts
    return observables.transmission(t.sigma_r[0], t.sigma_r[1], full["Gr"][np.ix_(cL, cR)])


TOL_LEAK = 1e-4


@pytest.mark.parametrize("ny", [4, 5])
def test_perfect_ribbon_transmits_whole_channels(ny):
    metallic = (2 * ny) % 3 == 2
    for E in (0.5, -0.8, 1.3):
        Ts = [_transmission(workloads.agnr(cells, ny), E) for cells in (2, 5)]
        for T in Ts:
            assert abs(T - round(T)) <= TOL_LEAK, (ny, E, Ts)
            if metallic:
                assert T >= 1.0 - TOL_LEAK, (ny, E, Ts)
        assert abs(Ts[0] - Ts[1]) <= TOL_LEAK
    if not metallic:
        assert _transmission(workloads.agnr(3, ny), 0.5) <= TOL_LEAK  # inside the gap


def test_ribbon_structure():
    dev = workloads.agnr(4, 5)
    H = dev.dense()
    assert np.allclose(H, H.T)
    off = np.abs(H - np.diag(np.diag(H))) > 0
    # honeycomb: at most three neighbours, all at hopping -3.1 eV; the bulk has three
    assert off.sum(1).max() == 3 and np.allclose(H[off], -3.1)
    lead = dev.leads[1]
    m = 4 * 5
    assert np.allclose(H[:m, :m], lead.H00) and np.allclose(H[:m, m:2 * m], lead.H01)

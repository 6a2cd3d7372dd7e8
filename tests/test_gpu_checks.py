"""Input checks of nd_factor / nd_diag_green on the GPU: eta must be positive;
host inputs that break the complex symmetry of A (paper Sec. 3.1, LDL^T) or
the skew-Hermiticity of Sigma^< / Sigma^> (Sec. 3.1, Eq. (5)-(6)) are rejected
by the call itself, device inputs by a check kernel whose result
nd_fact_status reports; a valid call on the same handle afterwards gives
bit-for-bit the results of a valid call before."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from paper_1305_1070_gb300 import build, ndgf, workloads  # noqa: E402
from paper_1305_1070_gb300.solver import Solver  # noqa: E402

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def solver():
    build.build()
    dev = workloads.superlattice(20, 6, disorder=0.03, seed=11)
    tr = workloads.Transport(energies=np.array([0.07, 0.21, 0.38]))
    s = Solver(dev, tr, precision=ndgf.ND_PREC_FP64, leaf_size=12, delay=2)
    return s, tr


def _status(fn, *args):
    try:
        fn(*args)
        return 0
    except ndgf.NDError as e:
        return e.status


def _valid(s, tr):
    Gr, Gl, Gg = s.step(tr.energies)
    torch.cuda.synchronize()
    assert _status(ndgf.nd_fact_status, s.fact) == 0
    return Gr.clone(), Gl.clone(), Gg.clone()


def test_checks_on_gpu(solver):
    s, tr = solver
    n_e = len(tr.energies)
    ref = _valid(s, tr)
    E = s.E[:n_e]
    for eta in (0.0, -1e-6, float("nan")):
        assert _status(ndgf.nd_factor, s.fact, s.H, s.sig_r, None, E, n_e, eta) == 1
    # asymmetric H values: host array -> the call fails; device array -> nd_fact_status
    H = s.H.clone()
    dev = s.dev
    r = 5
    q = next(q for q in range(dev.rowptr[r], dev.rowptr[r + 1]) if dev.colind[q] != r)
    H[q] += 1e-3
    assert _status(ndgf.nd_factor, s.fact, H.cpu().numpy(), s.sig_r, None, E, n_e, tr.eta) == 2
    assert _status(ndgf.nd_factor, s.fact, H, s.sig_r, None, E, n_e, tr.eta) == 0
    torch.cuda.synchronize()
    assert _status(ndgf.nd_fact_status, s.fact) == 2
    # a contact block that is not complex symmetric (device)
    sr = s.sig_r.clone()
    sr[1, 1] += 1e-3 * sr[1].abs().max()
    assert _status(ndgf.nd_factor, s.fact, s.H, sr, None, E, n_e, tr.eta) == 0
    torch.cuda.synchronize()
    assert _status(ndgf.nd_fact_status, s.fact) == 2
    # a valid fold, then Sigma^< that is not skew-Hermitian (host: the call; device: nd_fact_status)
    ndgf.nd_factor(s.fact, s.H, s.sig_r, None, E, n_e, tr.eta)
    bad = s.sig_l.clone()
    bad[0, 1] += 1e-3 * bad[0].abs().max()
    Gr = torch.zeros_like(s.Gr)
    Gl = torch.zeros_like(s.Gl)
    Gg = torch.zeros_like(s.Gg)
    assert _status(ndgf.nd_diag_green, s.fact, bad.cpu().numpy(), s.sig_g, None, None, Gr, Gl, Gg) == 4
    assert _status(ndgf.nd_diag_green, s.fact, s.sig_l, bad, None, None, Gr, Gl, Gg) == 0
    torch.cuda.synchronize()
    assert _status(ndgf.nd_fact_status, s.fact) == 4
    # a valid call afterwards: unchanged results, clean status
    got = _valid(s, tr)
    for a, b in zip(got, ref):
        assert torch.equal(a, b)


def test_host_inputs_valid_call_matches_device_inputs(solver):
    """Host arrays go through the host checks and the staging copies; the
    results equal those of the same call with device arrays."""
    s, tr = solver
    n_e = len(tr.energies)
    ref = _valid(s, tr)
    E = s.E[:n_e]
    Gr = np.zeros((n_e, s.n), dtype=np.complex128)
    Gl = np.zeros_like(Gr)
    Gg = np.zeros_like(Gr)
    ndgf.nd_factor(s.fact, s.H.cpu().numpy(), s.sig_r[:n_e].cpu().numpy(), None, E.cpu().numpy(), n_e, tr.eta)
    ndgf.nd_diag_green(s.fact, s.sig_l[:n_e].cpu().numpy(), s.sig_g[:n_e].cpu().numpy(), None, None, Gr, Gl, Gg)
    torch.cuda.synchronize()
    assert _status(ndgf.nd_fact_status, s.fact) == 0
    for a, b in zip((Gr, Gl, Gg), ref):
        assert np.array_equal(a, b[:n_e].cpu().numpy())


def test_degenerate_calls():
    """Degenerate calls on a two-site chain (one site per contact, one-site
    leaves): nd_diag_green before any nd_factor, zero energies and more energies
    than the handle holds are refused with ND_ERR_INVALID_ARG and leave the
    handle usable; a call at exactly max_ne energies matches the dense
    definition (paper Eq. (1)-(2))."""
    from oracle import dense, observables
    dev = workloads.chain(2, t=1.0)
    tr = workloads.Transport(energies=np.array([-0.6, 0.1, 0.9]), mu=(0.2, -0.1), kT=0.05)
    s = Solver(dev, tr, precision=ndgf.ND_PREC_FP64, leaf_size=1, max_ne=3)
    out = torch.zeros(3, dev.n, dtype=torch.complex128, device="cuda")
    assert _status(ndgf.nd_diag_green, s.fact, None, None, None, None, out, None, None) == 1
    E = torch.as_tensor(tr.energies, device="cuda")
    assert _status(ndgf.nd_factor, s.fact, s.H, s.sig_r, None, E, 0, tr.eta) == 1
    E4 = torch.as_tensor(np.append(tr.energies, 0.3), device="cuda")
    assert _status(ndgf.nd_factor, s.fact, s.H, s.sig_r, None, E4, 4, tr.eta) == 1
    Gr, Gl, Gg = s.step(tr.energies)
    torch.cuda.synchronize()
    assert _status(ndgf.nd_fact_status, s.fact) == 0
    ref = dense.green_diag(dev, tr)
    for k, g in (("Gr", Gr), ("Gl", Gl), ("Gg", Gg)):
        g = g.cpu().numpy()
        for e in range(3):
            assert observables.rel_err(g[e], ref[k][e]) < 1e-10

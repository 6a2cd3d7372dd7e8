"""S9 certificate, selected entries and the S10 density through the C ABI.

- nd_selected_entries: G^r_xy, G^<_xy, G^>_xy for every pair that A couples
  (paper Sec. 3.2: the selected inversion stores G^(0) on the fill pattern)
  against the dense definition (Eq. (1)-(2)), with and without delayed pivots.
- nd_certificate: its FP64 residuals max_j |(A G)_jj - 1| and
  max_j |(A G^< - Sigma^< G^a)_jj| (Eq. (1)) against the same quantities
  computed here from the oracle's dense A and Sigma^< and the entries that
  nd_selected_entries returns; the residuals are at the rounding level of
  each path and no stored entry goes missing.
- Solver.step_certified: energies flagged by the certificate are recomputed
  on the complex128 path; forcing every energy reproduces that path exactly.
- nd_density (S10, paper Sec. 1): the energy integral of Im G^<_jj against
  oracle.observables.density on the oracle's G^< over a full energy grid.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from oracle import dense, observables  # noqa: E402
from paper_1305_1070_gb300 import build, ndgf, workloads  # noqa: E402
from paper_1305_1070_gb300.solver import Solver  # noqa: E402

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib():
    build.build()
    if not torch.cuda.is_available():
        pytest.fail("CUDA device required")


def _pairs(dev):
    """Every pair coupled by H (CSR, diagonal included) or by a contact block."""
    x, y = [], []
    for r in range(dev.n):
        for q in range(dev.rowptr[r], dev.rowptr[r + 1]):
            x.append(r)
            y.append(dev.colind[q])
    for c in dev.contacts:
        for a in c:
            for b in c:
                x.append(a)
                y.append(b)
    return np.array(x, dtype=np.int32), np.array(y, dtype=np.int32)


def _selected(s, x, y, n_e):
    xd = torch.as_tensor(x, device="cuda")
    yd = torch.as_tensor(y, device="cuda")
    out = [torch.zeros(n_e, len(x), dtype=torch.complex128, device="cuda") for _ in range(3)]
    miss = torch.zeros(1, dtype=torch.int32, device="cuda")
    ndgf.nd_selected_entries(s.fact, xd, yd, len(x), out[0], out[1], out[2], miss)
    torch.cuda.synchronize()
    return [o.cpu().numpy() for o in out], int(miss.item())


def _dense_inputs(s, dev, tr, e):
    """Dense A(E_e) and Sigma^<(E_e) from the inputs the solver handed to the
    library for energy e (its Sigma^r / Sigma^< buffers and phonon diagonals)."""
    A = -dev.dense().astype(complex)
    A[np.diag_indices(dev.n)] += float(s.E[e]) + 1j * tr.eta
    Sl = np.zeros((dev.n, dev.n), dtype=complex)
    sr, sl = s.sig_r[e].cpu().numpy(), s.sig_l[e].cpu().numpy()
    for c, idx in enumerate(dev.contacts):
        m = len(idx)
        o = int(s.off[c])
        A[np.ix_(idx, idx)] -= sr[o:o + m * m].reshape(m, m)
        Sl[np.ix_(idx, idx)] += sl[o:o + m * m].reshape(m, m)
    if s.ph:
        A[np.diag_indices(dev.n)] -= s.ph_r[e].cpu().numpy()
        Sl[np.diag_indices(dev.n)] += s.ph_l[e].cpu().numpy()
    return A, Sl


CASES = [  # (L, W, leaf, delay, gamma_ph, precision, tol)
    (22, 7, 10, 0, 0.0, ndgf.ND_PREC_FP64, 1e-10),
    (22, 7, 10, 2, 0.0, ndgf.ND_PREC_FP64, 1e-10),
    (19, 6, 6, 3, 4e-3, ndgf.ND_PREC_FP64, 1e-10),
    (22, 7, 10, 2, 0.0, ndgf.ND_PREC_FP32X2, 1e-9),
    (17, 5, 1, 1, 0.0, ndgf.ND_PREC_FP32X2, 1e-9),
]


@pytest.mark.parametrize("L,W,leaf,delay,gph,precision,tol", CASES)
def test_selected_entries_and_residual(L, W, leaf, delay, gph, precision, tol):
    dev = workloads.superlattice(L, W, disorder=0.04, seed=L + W)
    tr = workloads.Transport(energies=np.array([0.03, 0.17, 0.29, 0.46]), gamma_ph=gph, mu_ph=0.05)
    s = Solver(dev, tr, precision=precision, leaf_size=leaf, delay=delay)
    s.step(tr.energies)
    cert = s.certificate(tr.n_e).cpu().numpy()
    x, y = _pairs(dev)
    (gr, gl, gg), miss = _selected(s, x, y, tr.n_e)
    assert miss == 0
    assert (cert[:, 5] == 0).all()
    for e, E in enumerate(tr.energies):
        full = dense.green_full(dev, tr, float(E))
        for got, key in ((gr, "Gr"), (gl, "Gl"), (gg, "Gg")):
            ref = full[key][x, y]
            assert np.abs(got[e] - ref).max() <= tol * np.abs(full[key]).max(), key
        # the residuals from A and Sigma^< of this call (H, E + i eta, the phonon
        # term and the device-computed lead blocks) and the GPU's entries: the
        # same FP64 sums up to rounding
        A, Sl = _dense_inputs(s, dev, tr, e)
        G = np.zeros((dev.n, dev.n), dtype=complex)
        Gl = np.zeros_like(G)
        G[x, y] = gr[e]
        Gl[x, y] = gl[e]
        r = np.abs(np.einsum("jk,kj->j", A, G) - 1.0)
        # (Sigma^< G^a)_jj = sum_k Sigma^<_jk conj(G_jk)
        rl = np.abs(np.einsum("jk,kj->j", A, Gl) - np.einsum("jk,jk->j", Sl, G.conj()))
        s_r = np.einsum("jk,kj->j", np.abs(A), np.abs(G))
        s_l = np.einsum("jk,kj->j", np.abs(A), np.abs(Gl)) + np.einsum("jk,jk->j", np.abs(Sl), np.abs(G))
        u = 1e3 * 2.0 ** -52
        assert abs(cert[e, 0] - r.max()) <= u * s_r.max()
        assert abs(cert[e, 2] - rl.max()) <= u * s_l.max()
        assert abs(cert[e, 6] - r.max() / s_r.max()) <= u
        assert abs(cert[e, 7] - rl.max() / s_l.max()) <= u
        assert cert[e, 1] == pytest.approx(np.abs(np.diag(full["Gr"])).max(), rel=tol * 10)
        # backward errors within the path's parity tolerance (a missing or wrong
        # term would leave an O(|A_jk G_kj|) residual)
        assert cert[e, 6] <= tol and cert[e, 7] <= tol


def test_selected_entries_missing_pairs():
    dev = workloads.superlattice(12, 4, disorder=0.0)
    tr = workloads.Transport(energies=np.array([0.2]))
    s = Solver(dev, tr, leaf_size=8, delay=1)
    s.step(tr.energies)
    # two far-apart sites in different leaves, and an out-of-range index: not stored
    x = np.array([0, 1, dev.n + 5], dtype=np.int32)
    y = np.array([dev.n - 1, 1, 0], dtype=np.int32)
    (gr, _, _), miss = _selected(s, x, y, 1)
    assert miss == 2
    assert np.isnan(gr[0, 0]) and np.isnan(gr[0, 2]) and np.isfinite(gr[0, 1])


def test_certified_step_redo():
    """Certificate-driven recomputation: with thresholds no energy reaches,
    nothing is redone and the FP32-pair rows stay; with growth_max = 0 every
    energy is redone and the rows equal the complex128 path bit for bit."""
    dev = workloads.superlattice(30, 8, disorder=0.03, seed=5)
    tr = workloads.Transport(energies=np.linspace(0.0, 0.5, 9))
    x2 = Solver(dev, tr, precision=ndgf.ND_PREC_FP32X2, leaf_size=10, delay=2)
    f64 = Solver(dev, tr, precision=ndgf.ND_PREC_FP64, leaf_size=10, delay=2, max_ne=4)
    Gr, Gl, Gg, cert, redone = x2.step_certified(tr.energies, f64, resid_max=1.0, growth_max=1e9)
    assert redone.numel() == 0
    keep = [g.clone() for g in (Gr, Gl, Gg)]
    # the complex128 path in the chunks the recomputation uses (4 energies per call)
    E = torch.as_tensor(tr.energies, device="cuda")
    parts = [[g.clone() for g in f64.step(E[c0:c0 + 4])] for c0 in range(0, tr.n_e, 4)]
    want = [torch.cat([p[q] for p in parts]) for q in range(3)]
    assert max(observables.rel_err(keep[0][e].cpu().numpy(), want[0][e].cpu().numpy()) for e in range(tr.n_e)) < 1e-9
    Gr, Gl, Gg, cert, redone = x2.step_certified(tr.energies, f64, resid_max=1.0, growth_max=0.0)
    assert redone.numel() == tr.n_e
    for got, w in zip((Gr, Gl, Gg), want):
        assert torch.equal(got, w)
    # a residual threshold below the FP32-pair rounding level flags every energy too
    _, _, _, cert, redone = x2.step_certified(tr.energies, f64, resid_max=0.0, growth_max=1e9)
    assert redone.numel() == tr.n_e and (cert[:, 6] > 0).all()


@pytest.mark.parametrize("precision,tol", [(ndgf.ND_PREC_FP64, 1e-10), (ndgf.ND_PREC_FP32X2, 1e-9)])
def test_density_matches_oracle(precision, tol):
    """nd_density over a full grid (41 energies, trapezoid weights, spin 2,
    scale 2/(2 pi)) against oracle.observables.density on the dense G^<;
    accumulating two halves of the grid gives the same density."""
    dev = workloads.superlattice(24, 6, disorder=0.03, seed=9)
    E = np.linspace(0.0, 0.5, 41)
    tr = workloads.Transport(energies=E, mu=(0.25, 0.05), kT=0.03)
    ref = observables.density(dense.green_diag(dev, tr)["Gl"], E)
    s = Solver(dev, tr, precision=precision, leaf_size=10, delay=2)
    _, Gl, _ = s.step(E)
    w = torch.as_tensor(observables.trapezoid_weights(E), device="cuda")
    out = torch.zeros(dev.n, dtype=torch.float64, device="cuda")
    ndgf.nd_density(Gl, w, len(E), dev.n, 2.0 / (2.0 * np.pi), 0, out)
    torch.cuda.synchronize()
    assert observables.rel_err(out.cpu().numpy(), ref) < tol
    half = torch.zeros_like(out)
    Glc = Gl.contiguous()
    ndgf.nd_density(Glc[:20].contiguous(), w[:20].contiguous(), 20, dev.n, 2.0 / (2.0 * np.pi), 0, half)
    ndgf.nd_density(Glc[20:].contiguous(), w[20:].contiguous(), 21, dev.n, 2.0 / (2.0 * np.pi), 1, half)
    torch.cuda.synchronize()
    assert observables.rel_err(half.cpu().numpy(), ref) < tol

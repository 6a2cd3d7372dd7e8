"""The pieces of the self-consistent Schroedinger-Poisson loop on the GPU
against the oracle (oracle/poisson, response, sp; paper Sec. 1 motivates the
density by Poisson's equation):
- nd_poisson_apply / nd_poisson_solve against the sparse operator and LU;
- nd_vec_dot / nd_vec_axpby against numpy;
- nd_density_jvp (forward terms, the second call reusing the stored U) and
  nd_density_gradient after it against the oracle's terms per energy;
- the Newton-Krylov iteration (paper_1305_1070_gb300.sp) against the
  oracle's Newton iterates with the dense Jacobian, step by step."""
import math

import numpy as np
import pytest

torch = pytest.importorskip("torch")

from oracle import poisson, response, sp  # noqa: E402
from paper_1305_1070_gb300 import build, ndgf, workloads  # noqa: E402
from paper_1305_1070_gb300.solver import Solver  # noqa: E402

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib():
    build.build()
    if not torch.cuda.is_available():
        pytest.fail("CUDA device required")


@pytest.mark.parametrize("L,W", [(12, 5), (1, 1), (256, 64)])
def test_poisson(L, W):
    rng = np.random.Generator(np.random.PCG64(L * W))
    rhs = rng.normal(size=(2, L * W))
    P = ndgf.nd_poisson_create(L, W)
    r = torch.as_tensor(rhs, device="cuda").contiguous()
    u = torch.zeros_like(r)
    ndgf.nd_poisson_solve(P, r, u, 2)
    Ku = torch.zeros_like(r)
    ndgf.nd_poisson_apply(P, u, Ku, 2)
    us = torch.zeros_like(r)
    ndgf.nd_poisson_solve(P, r, us, 2, shift=0.37)  # the screened operator K + 0.37 I
    torch.cuda.synchronize()
    import scipy.sparse as sps
    import scipy.sparse.linalg as spla
    Ks = (poisson.operator(L, W) + 0.37 * sps.identity(L * W)).tocsc()
    for b in range(2):
        ref = poisson.solve(L, W, rhs[b])
        assert np.abs(u[b].cpu().numpy() - ref).max() <= 1e-11 * np.abs(ref).max()
        assert np.abs(Ku[b].cpu().numpy() - poisson.apply(L, W, ref)).max() <= 1e-11 * np.abs(rhs[b]).max()
        refs = spla.spsolve(Ks, rhs[b])
        assert np.abs(us[b].cpu().numpy() - refs).max() <= 1e-11 * np.abs(refs).max()


def test_vector_ops():
    rng = np.random.Generator(np.random.PCG64(5))
    x, y = rng.normal(size=100003), rng.normal(size=100003)
    xd, yd = torch.as_tensor(x, device="cuda"), torch.as_tensor(y, device="cuda")
    out = torch.zeros(1, dtype=torch.float64, device="cuda")
    ndgf.nd_vec_dot(xd, yd, len(x), out)
    assert float(out.item()) == pytest.approx(float(x @ y), rel=1e-13)
    first = float(out.item())
    ndgf.nd_vec_dot(xd, yd, len(x), out)
    assert float(out.item()) == first  # fixed reduction order
    ndgf.nd_vec_axpby(0.5, xd, -2.0, yd, len(x))
    assert np.abs(yd.cpu().numpy() - (0.5 * x - 2.0 * y)).max() < 1e-14
    ndgf.nd_vec_axpby(3.0, xd, 0.0, yd, len(x))
    assert np.abs(yd.cpu().numpy() - 3.0 * x).max() < 1e-14


def _small():
    dev = workloads.superlattice(10, 6, disorder=0.03, seed=2)
    tr = workloads.Transport(energies=np.linspace(0.4, 1.4, 11), mu=(0.95, 0.75), kT=0.03)
    return dev, tr


@pytest.mark.parametrize("precision,tol", [(ndgf.ND_PREC_FP64, 1e-10), (ndgf.ND_PREC_FP32X2, 1e-9)])
def test_jvp_and_gradient_terms(precision, tol):
    dev, tr = _small()
    U = 0.01 * np.cos(np.arange(dev.n))
    s = Solver(dev, tr, precision=precision, leaf_size=8, delay=2, adjoint=True)
    s.set_potential(U)
    s.step(tr.energies)
    rng = np.random.Generator(np.random.PCG64(8))
    T = torch.zeros(tr.n_e, dev.n, dtype=torch.complex128, device="cuda")
    for trial in range(2):  # the second call reuses the stored U = G^r E_C
        v = rng.normal(size=dev.n)
        ndgf.nd_density_jvp(s.fact, torch.as_tensor(v, device="cuda"), T)
        ref = response.forward_terms(dev, tr, v, U)
        got = T.cpu().numpy()
        for e in range(tr.n_e):
            assert np.abs(got[e] - ref[e]).max() <= tol * np.abs(ref[e]).max(), (trial, e)
    c = rng.uniform(0, 1, dev.n)
    ndgf.nd_density_gradient(s.fact, torch.as_tensor(c, device="cuda"), T)
    ref = response.adjoint_terms(dev, tr, c, U)
    got = T.cpu().numpy()
    for e in range(tr.n_e):
        assert np.abs(got[e] - ref[e]).max() <= tol * np.abs(ref[e]).max(), e


@pytest.mark.parametrize("precision,tol", [(ndgf.ND_PREC_FP64, 1e-9), (ndgf.ND_PREC_FP32X2, 1e-8)])
def test_newton_iterates_match_oracle(precision, tol):
    from paper_1305_1070_gb300 import sp as gsp
    dev, tr = _small()
    L, W, lam = 10, 6, 2.8
    nD = np.full(dev.n, response.density(dev, tr).mean())
    its_o, res_o = sp.newton(dev, tr, L, W, lam, nD, steps=5)
    run = gsp.SchrodingerPoisson(dev, tr, L, W, lam, nD, precision=precision, leaf_size=8, chunk=6)
    its_g, res_g, kry, lens = run.newton(5)
    print(f"  precision {precision}: |F| {res_g}, GMRES iterations {kry}, steps {lens}")
    assert all(a == 1.0 for a in lens)  # full Newton steps, as the oracle takes
    for m in range(1, 6):
        scale = np.abs(its_o[m]).max()
        assert np.abs(its_g[m] - its_o[m]).max() <= tol * scale, (m, np.abs(its_g[m] - its_o[m]).max())
    assert res_g[-1] <= 1e-10 * res_g[0] + 1e-12


def test_newton_full_size_converges_to_oracle_fixed_point():
    """10 Newton steps on the 256 x 64 superlattice (128 energies in
    [-0.6, 0.5] eV, eta = 9 meV), FP32 pairs: |F| falls below 1e-8 of its
    start, and the last iterate is a fixed point of the oracle's own map, the
    block-RGF density with that potential (paper Eq. (1)-(2)) and the sparse
    Poisson operator: |F_oracle(U)| within 1e-7 of |F_oracle(0)|."""
    from oracle import observables, rgf
    from paper_1305_1070_gb300 import sp as gsp
    dev, tr = workloads.workload("superlattice_256x64_sp")
    lam = 1.439964 * 4.0 * np.pi / (12.9 * 0.5)
    run = gsp.SchrodingerPoisson(dev, tr, 256, 64, lam, 0.0, precision=ndgf.ND_PREC_FP32X2, leaf_size=16, chunk=32,
                                 gmres_tol=1e-10, gmres_max=60)
    # background: the flat-band density averaged over each 8-column period (neutral periods)
    n0 = run.density(run.U, run.dens).cpu().numpy().reshape(256, 64)
    nD = np.repeat(n0.reshape(32, 8 * 64).mean(axis=1), 8 * 64)
    run.nD.copy_(torch.as_tensor(nD, device="cuda"))
    its, res, kry, lens = run.newton(10)
    print(f"  |F| {res}, GMRES {kry}, steps {lens}, U in [{its[-1].min():.3f}, {its[-1].max():.3f}] eV")
    assert res[-1] <= 1e-8 * res[0]
    U = its[-1]

    def F_oracle(Uv):
        d = rgf.green_diag(response.with_onsite(dev, Uv), tr)
        n = observables.density(d["Gl"], tr.energies)
        return poisson.apply(256, 64, Uv) - lam * (n - nD)

    f0 = np.abs(F_oracle(np.zeros(dev.n))).max()
    f1 = np.abs(F_oracle(U)).max()
    print(f"  oracle |F| at 0: {f0:.3e}, at the last iterate: {f1:.3e}")
    assert f1 <= 1e-7 * f0

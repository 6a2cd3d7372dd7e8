"""The kernel autotuner (nd_autotune): every GEMM launch of the fold and the
extraction is timed with each candidate kernel (default rules, large and
small tile, tensor cores for FP32 pairs, one CTA per block) and keeps the
fastest.  After tuning, the results still match the oracle (paper
Eq. (1)-(2)) at the path's tolerance, on one device and on an uneven batch of
devices in one graph; the summary reports the launches tuned and the passes
run."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from oracle import dense, observables  # noqa: E402
from paper_1305_1070_gb300 import build, ndgf, tune, workloads  # noqa: E402
from paper_1305_1070_gb300.solver import Solver  # noqa: E402

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib():
    build.build()
    if not torch.cuda.is_available():
        pytest.fail("CUDA device required")


def _check(s, dev, tr, devs=None, tol=1e-9):
    Gr, Gl, Gg = s.step(tr.energies)
    torch.cuda.synchronize()
    assert ndgf.nd_fact_status(s.fact) == 0
    got = {"Gr": Gr.cpu().numpy(), "Gl": Gl.cpu().numpy(), "Gg": Gg.cpu().numpy()}
    parts = [(dev, 0, dev.n)] if devs is None else [(d, dev.site_offsets[i], dev.site_offsets[i + 1])
                                                      for i, d in enumerate(devs)]
    for sub, lo, hi in parts:
        ref = dense.green_diag(sub, tr)
        for k in ("Gr", "Gl", "Gg"):
            for e in range(tr.n_e):
                assert observables.rel_err(got[k][e, lo:hi], ref[k][e]) <= tol, (k, e)


@pytest.mark.parametrize("precision,tol", [(ndgf.ND_PREC_FP64, 1e-10), (ndgf.ND_PREC_FP32X2, 1e-9)])
def test_autotune_single_device(precision, tol):
    dev = workloads.superlattice(40, 12, disorder=0.03, seed=21)
    tr = workloads.Transport(energies=np.linspace(0.03, 0.47, 5), gamma_ph=2e-3, mu_ph=0.05)
    s = Solver(dev, tr, precision=precision, leaf_size=10, delay=2)
    info = s.autotune(tr.energies)
    print(f"  tuner precision {precision}: {info}")
    assert info["passes"] == 6 and info["gemm_steps"] > 0
    assert sum(info["by_kind"]) == info["gemm_steps"]
    assert info["ms_tuned"] <= info["ms_default"] * 1.0001
    _check(s, dev, tr, tol=tol)


def test_autotune_uneven_batch():
    devs = [workloads.superlattice(L, W, disorder=0.02, seed=L) for L, W in ((12, 4), (20, 8), (9, 6), (16, 5))]
    dev = workloads.union(devs)
    tr = workloads.Transport(energies=np.array([0.04, 0.21, 0.43]), mu=(0.25, 0.0), kT=0.03)
    s = Solver(dev, tr, precision=ndgf.ND_PREC_FP32X2, leaf_size=16, delay=2)
    info = s.autotune(tr.energies)
    assert info["gemm_steps"] > 0
    _check(s, dev, tr, devs=devs)


def test_plan_search_small():
    dev = workloads.superlattice(32, 8, disorder=0.02, seed=4)
    tr = workloads.Transport(energies=np.linspace(0.05, 0.45, 8))
    best, table, s = tune.tune_plan(dev, tr, precision=ndgf.ND_PREC_FP32X2, delay=2, leafs=(8, 16), chunks=(4, 8))
    assert len(table) == 4 and best["leaf"] in (8, 16) and best["chunk"] in (4, 8)
    assert s.max_ne == best["chunk"]
    _check(s, dev, workloads.Transport(energies=tr.energies[:best["chunk"]]))


@pytest.mark.parametrize("precision,tol", [(ndgf.ND_PREC_FP64, 1e-10), (ndgf.ND_PREC_FP32X2, 1e-9),
                                           (ndgf.ND_PREC_MIXED, 1e-3)])
def test_extra_large_tile_every_launch(precision, tol):
    """The extra large ALU tile (a tuner candidate) forced on every GEMM launch:
    ragged blocks over several 64-row tiles, phonons, delayed pivots."""
    dev = workloads.superlattice(70, 20, disorder=0.03, seed=31)
    tr = workloads.Transport(energies=np.array([0.06, 0.29]), gamma_ph=2e-3, mu_ph=0.05)
    s = Solver(dev, tr, precision=precision, leaf_size=40, delay=2, tile="xl")
    _check(s, dev, tr, tol=tol)


def test_stored_choice_on_a_smaller_handle():
    """A tuning stored with nd_fact_get_choice and applied with
    nd_fact_set_choice to a handle of the same plan with fewer energies runs the
    same kernels: its diagonals equal the tuned handle's bit for bit (and the
    oracle's at the path's tolerance); out-of-range values, a wrong count and
    the tensor cores on a complex128 handle are refused."""
    dev = workloads.superlattice(40, 12, disorder=0.03, seed=21)
    tr = workloads.Transport(energies=np.linspace(0.03, 0.47, 6))
    big = Solver(dev, tr, precision=ndgf.ND_PREC_FP32X2, leaf_size=10, delay=2, max_ne=6)
    fresh = big.choice()
    assert (fresh == -1).all()
    big.autotune(tr.energies)
    choice = big.choice()
    assert choice.size == fresh.size and (choice >= -1).all() and (choice <= 4).all() and (choice >= 0).any()
    small = Solver(dev, tr, precision=ndgf.ND_PREC_FP32X2, leaf_size=10, delay=2, max_ne=2)
    small.set_choice(choice)
    assert np.array_equal(small.choice(), choice)
    pick = tr.energies[[1, 4]]
    want = [g.clone() for g in big.step(pick)]
    got = small.step(pick)
    torch.cuda.synchronize()
    for a, b in zip(got, want):
        assert torch.equal(a, b)
    ref = dense.green_diag(dev, workloads.Transport(energies=pick))
    for e in range(2):
        assert observables.rel_err(got[0][e].cpu().numpy(), ref["Gr"][e]) < 1e-9
    bad = choice.copy()
    bad[np.argmax(choice >= 0)] = 7
    with pytest.raises(ndgf.NDError):
        small.set_choice(bad)
    with pytest.raises(ndgf.NDError):
        small.set_choice(choice[:-1])
    f64 = Solver(dev, tr, precision=ndgf.ND_PREC_FP64, leaf_size=10, delay=2, max_ne=2)
    tc = np.where(choice >= 0, 2, -1).astype(np.int8)
    with pytest.raises(ndgf.NDError):
        f64.set_choice(tc)

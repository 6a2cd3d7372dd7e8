"""Checks of the paper's block algebra (Sec. 3) with the CPU rendition of the
multilevel algorithm, against the dense definition: every stored block of G^(0)
and P^(0) equals the matching block of G^r and G^< (Sec. 3.2), the Appendix A
block patterns, the three-cluster formulas with the sign reading, and RGF as the
special layer partition (Sec. 3.2, Fig. 6)."""
import os

import numpy as np
import pytest

from oracle import dense, nd_reference, observables, rgf
from oracle.problem import dense_sigma
from paper_1305_1070_gb300 import workloads

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "appendix_a_patterns.txt")


def _run(dev, tr, tree, E, record=False):
    full = dense.green_full(dev, tr, E)
    nd = nd_reference.NDReference(tree, full["A"], record=record)
    G0 = nd.green_retarded()
    terms = full["terms"]
    P0 = nd.green_lesser(dense_sigma(dev, terms, "lesser"), "")
    Q0 = nd.green_lesser(dense_sigma(dev, terms, "greater"), "g")
    return full, nd, G0, P0, Q0


@pytest.mark.parametrize("L,W,leaf,ph", [(16, 8, 12, 0.0), (12, 10, 8, 3e-3), (20, 6, 10, 0.0)])
def test_nd_reference_equals_dense(L, W, leaf, ph):
    dev = workloads.superlattice(L, W, disorder=0.02, seed=L)
    tr = workloads.Transport(energies=np.array([0.17]), gamma_ph=ph, mu_ph=0.05)
    tree = nd_reference.grid_bisection_tree(L, W, leaf)
    tree.check_partition(dev.n)
    full, nd, G0, P0, Q0 = _run(dev, tr, tree, 0.17)
    C = tree.clusters
    for (i, j), g in G0.items():  # every stored entry of G^(0) equals G^r
        assert np.abs(g - full["Gr"][np.ix_(C[i], C[j])]).max() < 1e-10 * np.abs(full["Gr"]).max()
    for i in range(len(C)):  # finalized P blocks are skew-Hermitian blocks of G^<
        assert np.abs(P0[i, i] - full["Gl"][np.ix_(C[i], C[i])]).max() < 1e-10 * np.abs(full["Gl"]).max()
        for j in tree.P[i]:
            assert np.abs(P0[i, j] - full["Gl"][np.ix_(C[i], C[j])]).max() < 1e-10 * np.abs(full["Gl"]).max()
            assert np.abs(Q0[i, j] - full["Gg"][np.ix_(C[i], C[j])]).max() < 1e-10 * np.abs(full["Gg"]).max()
    assert observables.rel_err(nd.diag(P0), np.diag(full["Gl"])) < 1e-10
    assert observables.rel_err(nd.diag(Q0), np.diag(full["Gg"])) < 1e-10


def _appendix_a_tree():
    # 9 (transport) x 6 grid, site x*6 + y.  Region 5 = column 5 (root); region 4 =
    # columns 6-8 (right contact); region 3 = row 2 of columns 1-4 plus column 1,
    # rows 3-5; region 1 = column 0 (left contact) plus rows 0-1 of columns 1-4;
    # region 2 = rows 3-5 of columns 2-4.  Couplings match the appendix's A.
    W = 6
    s = lambda x, y: x * W + y
    R5 = [s(5, y) for y in range(6)]
    R4 = [s(x, y) for x in range(6, 9) for y in range(6)]
    R3 = [s(x, 2) for x in range(1, 5)] + [s(1, y) for y in range(3, 6)]
    R1 = [s(0, y) for y in range(6)] + [s(x, y) for x in range(1, 5) for y in range(2)]
    R2 = [s(x, y) for x in range(2, 5) for y in range(3, 6)]
    return nd_reference.ClusterTree([R1, R2, R3, R4, R5], [2, 2, 4, 4, -1])


def _read_golden():
    pats, name, rows = {}, None, []
    for line in open(GOLDEN):
        line = line.strip()
        if not line or line.startswith("#"):
            continue
        if line[0].isalpha():
            if name:
                pats[name] = np.array(rows)
            name, rows = line, []
        else:
            rows.append([int(v) for v in line.split()])
    pats[name] = np.array(rows)
    return pats


def test_appendix_a_block_patterns():
    dev = workloads.superlattice(9, 6, disorder=0.05, seed=7)
    tree = _appendix_a_tree()
    tree.check_partition(dev.n)
    assert tree.L == 3 and tree.by_level[1] == [0, 1, 3] and tree.by_level[2] == [2]
    # a phonon term makes Sigma^< nonzero on every region, as the appendix assumes
    tr = workloads.Transport(energies=np.array([0.2]), gamma_ph=4e-3, mu_ph=0.05)
    full, nd, G0, P0, Q0 = _run(dev, tr, tree, 0.2, record=True)
    gold = _read_golden()
    for name, pat in gold.items():
        assert (nd.trace[name] == pat).all(), name
    assert observables.rel_err(nd.diag(P0), np.diag(full["Gl"])) < 1e-10


def test_three_cluster_formulas_and_sign_reading():
    # L | S | R on a 5 x 2 strip; Sec. 3.1 closed formulas against the definition.
    dev = workloads.superlattice(5, 2, disorder=0.05, seed=2)
    tr = workloads.Transport(energies=np.array([0.3]), mu=(0.25, 0.0))
    full = dense.green_full(dev, tr, 0.3)
    A, G, Gl = full["A"], full["Gr"], full["Gl"]
    Lx, Sx = np.arange(0, 4), np.arange(4, 6)
    ALL, ALS = A[np.ix_(Lx, Lx)], A[np.ix_(Lx, Sx)]
    ALLi = np.linalg.inv(ALL)
    Sl = dense_sigma(dev, full["terms"], "lesser")
    SLL = Sl[np.ix_(Lx, Lx)]
    GLL, GSL, GSS = G[np.ix_(Lx, Lx)], G[np.ix_(Sx, Lx)], G[np.ix_(Sx, Sx)]
    GlLS = Gl[np.ix_(Lx, Sx)]
    # G^r: G_LS = -A_LL^{-1} A_LS G_SS ; G_LL = A_LL^{-1} + A_LL^{-1} A_LS G_SS A_LS^T A_LL^{-1}
    assert np.abs(-ALLi @ ALS @ GSS - G[np.ix_(Lx, Sx)]).max() < 1e-11
    assert np.abs(ALLi + ALLi @ ALS @ GSS @ ALS.T @ ALLi - GLL).max() < 1e-11
    # G^<_LS = -A^{-1} A_LS G^<_SS + A^{-1} S^<_LL (G^r_SL)^dagger
    GlSS = Gl[np.ix_(Sx, Sx)]
    assert np.abs(-ALLi @ ALS @ GlSS + ALLi @ SLL @ GSL.conj().T - GlLS).max() < 1e-11
    # G^<_LL: the general algorithm's sign (+) reproduces the definition; the
    # three-cluster display's (-) does not.
    plus = ALLi @ SLL @ GLL.conj().T + ALLi @ ALS @ GlLS.conj().T
    minus = ALLi @ SLL @ GLL.conj().T - ALLi @ ALS @ GlLS.conj().T
    ref = Gl[np.ix_(Lx, Lx)]
    assert np.abs(plus - ref).max() < 1e-11 * max(1.0, np.abs(ref).max())
    assert np.abs(minus - ref).max() > 1e-3 * np.abs(ref).max()


def test_layer_partition_is_rgf():
    dev = workloads.superlattice(10, 4, disorder=0.03, seed=9)
    tr = workloads.Transport(energies=np.array([0.11]), gamma_ph=1e-3)
    tree = nd_reference.layer_tree(dev.layers)
    full, nd, G0, P0, Q0 = _run(dev, tr, tree, 0.11)
    r = rgf.RGF(dev, tr).solve(0.11)
    assert observables.rel_err(nd.diag(G0), r["Gr"]) < 1e-10
    assert observables.rel_err(nd.diag(P0), r["Gl"]) < 1e-10
    assert observables.rel_err(nd.diag(Q0), r["Gg"]) < 1e-10

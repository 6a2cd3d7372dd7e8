"""Pins of the general-Hermitian oracle (oracle/hermitian.py): the definition
(paper Eq. (1)-(2)) for a device in a magnetic field, where H has complex
hoppings (Peierls phases) and A is no longer complex symmetric, so the
symmetric elimination of Sec. 3.1 does not apply.  None of these retypes the
oracle's formulas:

- zero field: equal to the symmetric oracle (oracle/dense.py);
- gauge covariance: a site-dependent phase change of H and of the leads leaves
  every diagonal unchanged while the off-diagonal G^r changes (a transposition
  where a conjugate transposition belongs breaks it);
- reciprocity: G^r(-B) = G^r(B)^T exactly, hence equal diagonals of G^r, and
  T_{L->R}(-B) = T_{R->L}(B);
- the sum rule i (G - G^a) = G (Gamma_L + Gamma_R + 2 eta) G^a;
- the Dyson fixed point of the lead's surface Green's function with complex
  H01;
- the quantum Hall plateaus: between Landau levels the two-terminal
  transmission of a ribbon in the field is the integer number of edge
  channels, 1 and 2 here, and stays so under strong disorder;
- the broken complex symmetry of G^r in a field (why a separate elimination is
  needed);
- the block-LU form of the nested-dissection algorithm (oracle/nd_general.py)
  against the definition, block by block, and its reduction to the symmetric
  form without a field."""
import numpy as np
import pytest

from oracle import dense, hermitian, nd_general, nd_reference, observables, selfenergy
from paper_1305_1070_gb300 import workloads


def _tr(E, **kw):
    return workloads.Transport(energies=np.atleast_1d(np.asarray(E, dtype=float)), **kw)


def test_zero_field_equals_the_symmetric_oracle():
    tr = _tr([0.05, 0.2, 0.41], mu=(0.25, 0.05), kT=0.03)
    a = dense.green_diag(workloads.superlattice(12, 5, disorder=0.03, seed=4), tr)
    b = hermitian.green_diag(workloads.magnetic_superlattice(12, 5, 0.0, disorder=0.03, seed=4), tr)
    for k in ("Gr", "Gl", "Gg"):
        assert observables.rel_err(b[k], a[k]) < 1e-13, k


def _gauge(dev, theta_y):
    """H -> D H D^dagger with D = diag(exp(i theta(y))), applied to the device and
    (with the same per-row phases, the transform being uniform along
    transport) to every lead block."""
    W = dev.leads[0].H00.shape[0]
    th = theta_y(np.arange(dev.n) % W)
    rows = np.repeat(np.arange(dev.n), np.diff(dev.rowptr))
    vals = dev.values * np.exp(1j * (th[rows] - th[dev.colind]))
    D = np.diag(np.exp(1j * theta_y(np.arange(W))))
    leads = [workloads.Lead(H00=D @ ld.H00 @ D.conj().T, H01=D @ ld.H01 @ D.conj().T, tau=D @ ld.tau @ D.conj().T)
             for ld in dev.leads]
    import dataclasses
    return dataclasses.replace(dev, values=vals, leads=leads), np.exp(1j * th)


def test_gauge_covariance():
    dev = workloads.magnetic_superlattice(10, 6, 0.07, v_barrier=0.0, disorder=0.2, seed=11)
    gdev, d = _gauge(dev, lambda y: 0.37 * y * y - 1.3 * y)
    tr = _tr(1.5, mu=(1.6, 1.4), kT=0.03)  # above the lowest Landau level of the leads: open channels
    a, b = hermitian.green_full(dev, tr, 1.5), hermitian.green_full(gdev, tr, 1.5)
    for k in ("Gr", "Gl", "Gg"):
        assert observables.rel_err(np.diag(b[k]), np.diag(a[k])) < 1e-12, k
        assert observables.rel_err(b[k], d[:, None] * a[k] * d.conj()[None, :]) < 1e-12, k
    assert np.abs(b["Gr"] - a["Gr"]).max() > 1e-3 * np.abs(a["Gr"]).max()  # the off-diagonal part did change


def test_reciprocity_under_field_reversal():
    tr = _tr(0.8, mu=(0.9, 0.7), kT=0.03)
    p = workloads.magnetic_superlattice(10, 7, 0.04, v_barrier=0.0, disorder=0.4, seed=3)
    m = workloads.magnetic_superlattice(10, 7, -0.04, v_barrier=0.0, disorder=0.4, seed=3)
    fp, fm = hermitian.green_full(p, tr, 0.8), hermitian.green_full(m, tr, 0.8)
    assert observables.rel_err(fm["Gr"], fp["Gr"].T) < 1e-12
    iL, iR = p.contacts

    def T(f, a, b, sa, sb):
        G = f["Gr"][np.ix_(a, b)]
        return float(np.real(np.trace(selfenergy.broadening(sa) @ G @ selfenergy.broadening(sb) @ G.conj().T)))

    t_lr_minus = T(fm, iL, iR, fm["sigma_r"][0], fm["sigma_r"][1])
    t_rl_plus = T(fp, iR, iL, fp["sigma_r"][1], fp["sigma_r"][0])
    assert 0.1 < t_lr_minus and abs(t_lr_minus - t_rl_plus) < 1e-10 * t_lr_minus
    # the lesser function is not even in the field when mu_L != mu_R
    assert observables.rel_err(np.diag(fm["Gl"]), np.diag(fp["Gl"])) > 1e-3


def test_sum_rule_in_a_field():
    dev = workloads.magnetic_superlattice(9, 6, 0.11, disorder=0.05, seed=2)
    tr = _tr(0.35, eta=1e-3)
    f = hermitian.green_full(dev, tr, 0.35)
    G = f["Gr"]
    gam = np.zeros((dev.n, dev.n), dtype=complex)
    for idx, s in zip(dev.contacts, f["sigma_r"]):
        gam[np.ix_(idx, idx)] += selfenergy.broadening(s)
    lhs = 1j * (G - G.conj().T)
    rhs = G @ (gam + 2 * tr.eta * np.eye(dev.n)) @ G.conj().T
    assert np.abs(lhs - rhs).max() < 1e-10 * np.abs(lhs).max()


def test_surface_green_fixed_point_with_complex_hopping():
    dev = workloads.magnetic_superlattice(4, 7, 0.13)
    for lead in dev.leads:
        for E in (0.05, 0.4, 1.3):
            z = E + 1e-6j
            g = hermitian.surface_green(lead.H00, lead.H01, z)
            fix = np.linalg.inv(z * np.eye(7) - lead.H00 - lead.H01 @ g @ lead.H01.conj().T)
            assert np.abs(g - fix).max() < 1e-9 * np.abs(g).max()


def test_quantum_hall_plateaus():
    """A 20 x 24 ribbon at a flux of 1/20 per plaquette (magnetic length 0.9
    nm, width 12 nm): Landau levels near 0.65, 2.05 and 3.25 eV, so T = 1 at
    1.4 eV and T = 2 at 2.6 eV, with or without strong on-site disorder (the
    edge channels do not backscatter); without the field the same ribbon
    carries many more channels."""
    tr14, tr26 = _tr(1.4), _tr(2.6)
    for dis in (0.0, 0.5):
        dev = workloads.magnetic_superlattice(20, 24, 0.05, v_barrier=0.0, disorder=dis, seed=7)
        assert abs(hermitian.transmission(dev, tr14, 1.4) - 1.0) < 1e-4
        assert abs(hermitian.transmission(dev, tr26, 2.6) - 2.0) < 1e-4
    free = workloads.magnetic_superlattice(20, 24, 0.0, v_barrier=0.0)
    assert hermitian.transmission(free, tr14, 1.4) > 3.5


def test_field_breaks_complex_symmetry():
    tr = _tr(0.3)
    for flux, expect_sym in ((0.0, True), (0.05, False)):
        G = hermitian.green_full(workloads.magnetic_superlattice(8, 5, flux, disorder=0.05, seed=1), tr, 0.3)["Gr"]
        asym = np.abs(G - G.T).max() / np.abs(G).max()
        assert (asym < 1e-12) if expect_sym else (asym > 1e-2)


@pytest.mark.parametrize("L,W,leaf,flux", [(16, 8, 12, 0.06), (12, 10, 8, -0.03), (14, 6, 10, 0.11)])
def test_general_nested_dissection_equals_the_definition(L, W, leaf, flux):
    """The block-LU form of the Sec. 3.2 algorithm (oracle/nd_general.py: left
    and right factors, G_BI from the left factors, N = Sigma^< G^a with
    (G^a)_ij = (G_ji)^dagger) against the definition in a field: every stored
    block of G^(0) and of P^(0) for Sigma^< and Sigma^>.  The symmetric
    algorithm (oracle/nd_reference.py) on the same A gets the diagonal wrong."""
    dev = workloads.magnetic_superlattice(L, W, flux, v_barrier=0.1, disorder=0.1, seed=L)
    tr = _tr(1.3, mu=(1.4, 1.2), kT=0.03)
    full = hermitian.green_full(dev, tr, 1.3)
    tree = nd_reference.grid_bisection_tree(L, W, leaf)
    tree.check_partition(dev.n)
    nd = nd_general.NDGeneral(tree, full["A"])
    G0 = nd.green_retarded()
    P0, Q0 = nd.green_lesser(full["Sl"]), nd.green_lesser(full["Sg"])
    C = tree.clusters
    for (i, j), g in G0.items():
        assert np.abs(g - full["Gr"][np.ix_(C[i], C[j])]).max() < 1e-10 * np.abs(full["Gr"]).max()
    for P, key in ((P0, "Gl"), (Q0, "Gg")):
        scale = np.abs(full[key]).max()
        for i in range(len(C)):
            assert np.abs(P[i, i] - full[key][np.ix_(C[i], C[i])]).max() < 1e-10 * scale
            for j in tree.P[i]:
                assert np.abs(P[i, j] - full[key][np.ix_(C[i], C[j])]).max() < 1e-10 * scale
                assert np.abs(P[j, i] - full[key][np.ix_(C[j], C[i])]).max() < 1e-10 * scale
    sym = nd_reference.NDReference(tree, full["A"])
    assert observables.rel_err(sym.diag(sym.green_retarded()), np.diag(full["Gr"])) > 1e-3


def test_general_nested_dissection_reduces_to_the_symmetric_one():
    """Without a field the left factors are the transposed right factors and
    both algorithms give the same blocks."""
    dev = workloads.superlattice(14, 7, disorder=0.05, seed=5)
    tr = workloads.Transport(energies=np.array([0.23]), mu=(0.3, 0.1), kT=0.03)
    full = dense.green_full(dev, tr, 0.23)
    from oracle.problem import dense_sigma
    tree = nd_reference.grid_bisection_tree(14, 7, 10)
    a, b = nd_reference.NDReference(tree, full["A"]), nd_general.NDGeneral(tree, full["A"])
    Ga, Gb = a.green_retarded(), b.green_retarded()
    for key in Ga:
        assert np.abs(Ga[key] - Gb[key]).max() < 1e-11 * np.abs(full["Gr"]).max()
    S = dense_sigma(dev, full["terms"], "lesser")
    assert observables.rel_err(b.diag(b.green_lesser(S)), a.diag(a.green_lesser(S))) < 1e-11


def test_general_algorithm_on_the_library_tree():
    """The block-LU algorithm (oracle/nd_general.py) on the cluster tree that
    the library's planner builds (nd_analyze, host only) for a device in a
    field: every diagonal of G^r, G^< and G^> equals the definition, so the
    ordering (width-1 separators, contact sets kept inside one cluster, hence
    a Sigma^< that is block diagonal over the clusters) needs no change for a
    general Hermitian H; only the numeric steps do."""
    from paper_1305_1070_gb300 import build, ndgf
    build.build()
    dev = workloads.magnetic_superlattice(24, 8, 0.07, v_barrier=0.1, disorder=0.1, seed=5)
    cp = np.concatenate([[0], np.cumsum([len(c) for c in dev.contacts])])
    plan = ndgf.nd_analyze(dev.n, dev.rowptr, dev.colind, cp, np.concatenate(dev.contacts), dev.coords, 16)
    info, tree = ndgf.nd_plan_query(plan), ndgf.nd_plan_tree(plan)
    nc = info["n_clusters"]
    clusters = [ndgf.nd_plan_cluster_sites(plan, c, tree["n_i"][c], tree["b_i"][c])[0] for c in range(nc)]
    ct = nd_reference.ClusterTree(clusters, tree["parent"].tolist())
    ct.check_partition(dev.n)
    assert ct.L >= 4
    tr = _tr(1.3, mu=(1.4, 1.2), kT=0.03)
    full = hermitian.green_full(dev, tr, 1.3)
    nd = nd_general.NDGeneral(ct, full["A"])
    g = nd.diag(nd.green_retarded())
    gl, gg = nd.diag(nd.green_lesser(full["Sl"])), nd.diag(nd.green_lesser(full["Sg"]))
    for got, key in ((g, "Gr"), (gl, "Gl"), (gg, "Gg")):
        assert observables.rel_err(got, np.diag(full[key])) < 1e-10, key

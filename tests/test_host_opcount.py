"""Operation counts of the nested-dissection fold and G^r extraction against the
recursive Green's function method on N x N five-point grids without contact
self-energies (paper Sec. 4, the cost comparison of Fig. "cost"): the paper
counts i j k operations for a product of an i x j and a j x k matrix and i^3
for the inversion of an i x i matrix, and reports O(N^3) for its method
against O(N^4) for RGF.

Here the count of the method is taken cluster by cluster from the planner's
tree (n = rows eliminated at the cluster, b = its boundary):
    inversion of A_ii                 n^3
    Psi = -A_ii^{-1} A_iB             n n b
    Schur update A_iB^T Psi           b n b
    G_IB = Psi G_BB                   n b b
    G_II = A_ii^{-1} + Psi G_BI       n b n
and RGF's over N layers of width N: one N^3 inversion per layer in the forward
sweep and two N^3 products per layer in the backward sweep (the couplings of a
five-point grid are -t I, so their products are not N^3 operations):
3 N^4 in all.  Host only.
"""
import numpy as np
import pytest

from paper_1305_1070_gb300 import ndgf

NS = (16, 32, 64, 128, 256)


def _grid(N):
    idx = np.arange(N * N).reshape(N, N)
    rows = []
    for x in range(N):
        for y in range(N):
            nb = []
            if x > 0:
                nb.append(idx[x - 1, y])
            if y > 0:
                nb.append(idx[x, y - 1])
            nb.append(idx[x, y])
            if y < N - 1:
                nb.append(idx[x, y + 1])
            if x < N - 1:
                nb.append(idx[x + 1, y])
            rows.append(nb)
    rp = np.zeros(N * N + 1, np.int32)
    rp[1:] = np.cumsum([len(r) for r in rows])
    ci = np.concatenate(rows).astype(np.int32)
    xs, ys = np.meshgrid(np.arange(N), np.arange(N), indexing="ij")
    coords = np.stack([xs.ravel(), ys.ravel()], 1).astype(np.float64)
    return rp, ci, coords


@pytest.fixture(scope="module")
def counts():
    out = {}
    for N in NS:
        rp, ci, co = _grid(N)
        plan = ndgf.nd_analyze(N * N, rp, ci, coords=co, leaf_size=16)
        tree = ndgf.nd_plan_tree(plan)
        info = ndgf.nd_plan_query(plan)
        n = tree["n_i"].astype(float)
        b = tree["b_i"].astype(float)
        hsc = float(np.sum(n ** 3 + n * n * b + b * n * b + n * b * b + n * b * n))
        out[N] = {"hsc": hsc, "rgf": 3.0 * N ** 4,
                  "model": (info["flops_factor"] + info["flops_green_r"]) / 8.0}
    return out


def _slopes(vals):
    Ns = np.array(NS, float)
    v = np.array(vals)
    return np.diff(np.log(v)) / np.diff(np.log(Ns))


def test_count_matches_planner_flop_model(counts):
    """The planner's flop model (8 flops per complex multiply-add) counts the same operations."""
    for N in NS:
        assert counts[N]["model"] == pytest.approx(counts[N]["hsc"], rel=1e-12)


def test_growth_exponents(counts):
    hsc = _slopes([counts[N]["hsc"] for N in NS])
    rgf = _slopes([counts[N]["rgf"] for N in NS])
    print("exponents: nested dissection", np.round(hsc, 3), "RGF", np.round(rgf, 3))
    assert np.allclose(rgf, 4.0)
    # O(N^3): every doubling of N from 32 on multiplies the count by about 8
    assert all(2.85 <= s <= 3.25 for s in hsc[1:]), hsc


def test_armchair_ribbon_exponent():
    """The paper's graphene comparison: square armchair ribbons (N atoms per
    direction: N / 4 cells of four N-atom columns), no contacts.  The exponent
    rises towards 3 (the ribbon is about twice as wide as long, so the
    separators reach their asymptotic share later than on the grid)."""
    from paper_1305_1070_gb300 import workloads
    vals = []
    ns = (16, 32, 64, 128, 256)
    for N in ns:
        dev = workloads.agnr(N // 4, N)
        plan = ndgf.nd_analyze(dev.n, dev.rowptr, dev.colind, coords=dev.coords, leaf_size=16)
        tree = ndgf.nd_plan_tree(plan)
        n = tree["n_i"].astype(float)
        b = tree["b_i"].astype(float)
        vals.append(float(np.sum(n ** 3 + n * n * b + b * n * b + n * b * b + n * b * n)))
    s = np.diff(np.log(vals)) / np.diff(np.log(np.array(ns, float)))
    print("armchair ribbon exponents", np.round(s, 3), "RGF / nested dissection at N = 256:",
          round(3.0 * 256 ** 4 / vals[-1], 2))
    assert all(x2 > x1 for x1, x2 in zip(s, s[1:])), s  # rising towards 3
    assert 2.85 <= s[-1] <= 3.25, s


def test_nested_dissection_needs_fewer_operations(counts):
    ratio = [counts[N]["rgf"] / counts[N]["hsc"] for N in NS]
    print("RGF / nested dissection:", np.round(ratio, 2))
    assert all(r2 > r1 for r1, r2 in zip(ratio, ratio[1:]))  # the gap grows like N
    assert ratio[-1] > 15.0

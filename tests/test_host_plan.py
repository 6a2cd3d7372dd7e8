"""Host-side checks of the C library (no GPU): it loads, exports every symbol
of include/ndgf.h, and nd_analyze produces a valid nested-dissection tree
(paper Sec. 3.2 partition rules) with the correct symbolic fold."""
import os
import re
from collections import defaultdict

import numpy as np
import pytest

from paper_1305_1070_gb300 import build, ndgf, workloads

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="session", autouse=True)
def _built():
    build.build()


def test_exports_match_header():
    hdr = open(os.path.join(ROOT, "include", "ndgf.h")).read()
    declared = set(re.findall(r"\b(nd_[a-z_0-9]+)\s*\(", hdr))
    lib = ndgf.lib()
    for name in declared:
        assert hasattr(lib, name), name
    assert declared == set(ndgf.EXPORTS)


def _plan(dev, leaf):
    cp = np.concatenate([[0], np.cumsum([len(c) for c in dev.contacts])])
    ci = np.concatenate(dev.contacts)
    plan = ndgf.nd_analyze(dev.n, dev.rowptr, dev.colind, cp, ci, dev.coords, leaf)
    info = ndgf.nd_plan_query(plan)
    tree = ndgf.nd_plan_tree(plan)
    sets = [ndgf.nd_plan_cluster_sites(plan, c, tree["n_i"][c], tree["b_i"][c]) for c in range(info["n_clusters"])]
    return plan, info, tree, sets


def _ancestors(parent, i):
    out = []
    p = parent[i]
    while p >= 0:
        out.append(p)
        p = parent[p]
    return out


def _check_tree(dev, leaf):
    plan, info, tree, sets = _plan(dev, leaf)
    parent, level, owner = tree["parent"], tree["level"], tree["cluster_of_site"]
    nc = info["n_clusters"]
    # partition of the sites
    allI = np.concatenate([s[0] for s in sets])
    assert sorted(allI.tolist()) == list(range(dev.n))
    for c in range(nc):
        assert (owner[sets[c][0]] == c).all()
    # postorder, levels
    for c in range(nc):
        if parent[c] >= 0:
            assert parent[c] > c and level[parent[c]] > level[c]
    anc = [set(_ancestors(parent, c)) for c in range(nc)]
    # every coupling is between a cluster and one of its ancestors (no coupling
    # between clusters that are not on one root path, in particular on one level)
    for r in range(dev.n):
        for p in range(dev.rowptr[r], dev.rowptr[r + 1]):
            a, b = owner[r], owner[dev.colind[p]]
            assert a == b or a in anc[b] or b in anc[a]
    # contact sets inside one cluster, leaves
    for c_sites in dev.contacts:
        assert len(set(owner[c_sites].tolist())) == 1
    # symbolic fold: simulate block elimination on the boolean pattern
    A = [set() for _ in range(dev.n)]
    for r in range(dev.n):
        A[r].update(dev.colind[dev.rowptr[r]:dev.rowptr[r + 1]].tolist())
    for idx in dev.contacts:
        for u in idx:
            A[u].update(idx.tolist())
    for c in range(nc):  # postorder = elimination order
        I = set(sets[c][0].tolist())
        nb = set()
        for u in I:
            nb |= A[u]
        nb -= I
        elim = {v for v in nb if owner[v] < c}  # folded already: must be descendants
        assert all(c in anc[owner[v]] for v in elim)
        nb -= elim
        assert nb == set(sets[c][1].tolist()), f"boundary of cluster {c}"
        for u in nb:  # fill among the boundary
            A[u] |= nb
    return info, tree


@pytest.mark.parametrize("L,W,leaf", [(64, 16, 64), (37, 11, 20), (20, 20, 16), (9, 6, 8), (5, 2, 4), (16, 3, 1)])
def test_superlattice_tree_valid(L, W, leaf):
    info, tree = _check_tree(workloads.superlattice(L, W), leaf)
    assert info["n_roots"] == 1
    assert info["max_n"] <= max(leaf, W) or info["max_n"] <= max(L, W)


def test_cnt_tree_valid():
    _check_tree(workloads.cnt_zigzag(6), 40)


def test_chain_and_single_cluster():
    info, tree = _check_tree(workloads.chain(12), 4)
    info, tree = _check_tree(workloads.chain(3), 64)
    assert info["n_clusters"] == 1 and tree["b_i"][0] == 0


def test_no_coordinates_bfs_bisection():
    dev = workloads.superlattice(24, 8)
    dev.coords = None
    _check_tree(dev, 16)


def test_rejects_asymmetric_and_out_of_range():
    rp = np.array([0, 2, 3, 4])
    ci = np.array([0, 1, 1, 2])  # (0,1) present but (1,0) missing
    with pytest.raises(ndgf.NDError) as e:
        ndgf.nd_analyze(3, rp, ci)
    assert e.value.status == 2
    with pytest.raises(ndgf.NDError) as e:
        ndgf.nd_analyze(3, np.array([0, 1, 2, 3]), np.array([0, 1, 7]))
    assert e.value.status == 1
    with pytest.raises(ndgf.NDError) as e:  # a site in two contacts
        dev = workloads.superlattice(4, 2)
        ndgf.nd_analyze(dev.n, dev.rowptr, dev.colind, [0, 2, 4], [0, 1, 1, 2])
    assert e.value.status == 1


def test_flop_model_scaling():
    # O(W^2 L) for fixed W (paper Sec. 4.2.1): doubling L doubles the count
    f = []
    for L in (128, 256, 512):
        dev = workloads.superlattice(L, 32)
        _, info, _, _ = _plan(dev, 64)
        f.append(info["flops_factor"] + info["flops_green_r"])
    assert 1.7 < f[1] / f[0] < 2.3 and 1.7 < f[2] / f[1] < 2.3


def _plan_sets(dev, leaf, delay):
    cp = np.concatenate([[0], np.cumsum([len(c) for c in dev.contacts])]).astype(np.int32)
    ci = np.concatenate(dev.contacts).astype(np.int32)
    plan = ndgf.nd_analyze(dev.n, dev.rowptr, dev.colind, cp, ci, dev.coords, leaf, 0, delay=delay)
    tree = ndgf.nd_plan_tree(plan)
    nc = len(tree["level"])
    sets = [ndgf.nd_plan_cluster_sites(plan, c, tree["n_i"][c], tree["b_i"][c]) for c in range(nc)]
    return tree, sets


@pytest.mark.parametrize("L,W,leaf,delay", [(64, 16, 64, 2), (37, 11, 20, 3), (16, 3, 1, 1), (20, 20, 16, 8)])
def test_delayed_pivot_structure(L, W, leaf, delay):
    """Delayed rows are virtual unknowns (ids >= n): each sits in exactly one
    front (the parent's) and first in exactly one boundary (its cluster's);
    the rest of every boundary equals the plain plan's, and every boundary
    entry lies in the parent's front or boundary (the extend-add target)."""
    dev = workloads.superlattice(L, W, disorder=0.02, seed=L)
    t0, s0 = _plan_sets(dev, leaf, 0)
    t1, s1 = _plan_sets(dev, leaf, delay)
    parent = t1["parent"]
    assert (parent == t0["parent"]).all()
    front = {}
    for c, (I, B) in enumerate(s1):
        for v in I.tolist():
            assert v not in front
            front[v] = c
    assert sorted(v for v in front if v < dev.n) == list(range(dev.n))
    virtual = sorted(v for v in front if v >= dev.n)
    assert virtual == list(range(dev.n, dev.n + len(virtual))) and len(virtual) > 0
    seen = {}
    for c, (I, B) in enumerate(s1):
        nv = int((B >= dev.n).sum())
        assert (B[:nv] >= dev.n).all() and (B[nv:] < dev.n).all()
        assert nv <= delay and (nv == 0 or parent[c] >= 0)
        assert B[nv:].tolist() == s0[c][1].tolist()
        assert sorted(I[I < dev.n].tolist()) == sorted(s0[c][0].tolist())
        for v in B[:nv].tolist():
            assert v not in seen and front[v] == parent[c]
            seen[v] = c
        if parent[c] >= 0:
            Ip, Bp = s1[parent[c]]
            assert set(B.tolist()) <= set(Ip.tolist()) | set(Bp.tolist())
        else:
            assert len(B) == 0
    assert sorted(seen) == virtual


def test_delay_out_of_range_rejected():
    dev = workloads.superlattice(8, 4)
    with pytest.raises(RuntimeError):
        _plan_sets(dev, 8, 9)


def test_union_of_devices_gets_one_tree_per_device():
    """A disconnected graph is dissected component by component: a batch of
    devices in one graph gives one root per device, and no cluster mixes
    sites of two devices."""
    devs = [workloads.superlattice(L, W, disorder=0.02, seed=L) for L, W in ((12, 4), (20, 8), (9, 6), (16, 5))]
    dev = workloads.union(devs)
    cp = np.concatenate([[0], np.cumsum([len(c) for c in dev.contacts])]).astype(np.int32)
    ci = np.concatenate(dev.contacts).astype(np.int32)
    for coords in (dev.coords, None):
        plan = ndgf.nd_analyze(dev.n, dev.rowptr, dev.colind, cp, ci, coords, 16, 0, delay=2)
        info = ndgf.nd_plan_query(plan)
        assert info["n_roots"] == len(devs) and info["n_contacts"] == 2 * len(devs)
        tree = ndgf.nd_plan_tree(plan)
        owner = tree["cluster_of_site"]
        device_of = np.searchsorted(dev.site_offsets, np.arange(dev.n), side="right") - 1
        for c in range(info["n_clusters"]):
            assert len(set(device_of[owner == c].tolist())) <= 1


def test_phonon_scba_rejects_bad_arguments():
    """nd_phonon_scba validates its arguments before any device work (no GPU
    needed): sizes, NULL arrays, the strength D >= 0, the mixing 0 < mix <= 1,
    and host arrays (it works on device arrays only)."""
    a = np.zeros(8, dtype=np.complex128)
    st = np.zeros(2)
    with pytest.raises(ndgf.NDError) as e:
        ndgf.nd_phonon_scba(0, 1, 0.01, 1.0, a, a, a, a, a, a, st)
    assert e.value.status == 1
    with pytest.raises(ndgf.NDError) as e:
        ndgf.nd_phonon_scba(4, 2, 0.01, 1.0, None, a, a, a, a, a, st)
    assert e.value.status == 1
    for D, mix in ((-0.01, 1.0), (0.01, 0.0), (0.01, 1.5)):
        with pytest.raises(ndgf.NDError) as e:
            ndgf.nd_phonon_scba(4, 2, D, mix, a, a, a, a, a, a, st)
        assert e.value.status == 1
    with pytest.raises(ndgf.NDError) as e:  # host arrays
        ndgf.nd_phonon_scba(4, 2, 0.01, 1.0, a, a, a, a, a, a, st)
    assert e.value.status == 1

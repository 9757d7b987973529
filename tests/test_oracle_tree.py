"""Pins of the oracle's Barnes-Hut tree (Algorithm 1) and BHForce (Algorithm 2)."""
import os

import numpy as np
import pytest

import synth

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "hand_tree_alg1.txt")


def _load_golden():
    rows, counts, literal = [], [], None
    for ln in open(GOLDEN):
        ln = ln.strip()
        if not ln or ln.startswith("#"):
            continue
        parts = ln.split()
        if parts[0] == "count":
            counts.append((float(parts[1]), int(parts[2])))
        elif parts[0] == "literal":
            literal = (int(parts[1]), int(parts[2]))
        else:
            rows.append([float(v) for v in parts])
    return np.array(rows), counts, literal


def test_hand_worked_tree(orc):
    table, counts, literal = _load_golden()
    X = np.array([[0, 0, 0], [4, 4, 4], [3, 3, 3], [0.5, 0, 0]], dtype=float)
    m = np.array([1.0, 2.0, 3.0, 4.0])
    tr = orc.Tree(X, m)
    e = tr.export()
    assert len(e["depth"]) == len(table)
    np.testing.assert_array_equal(e["depth"], table[:, 0])
    np.testing.assert_array_equal(e["cell"], table[:, 1:4])
    np.testing.assert_array_equal(e["npts"], table[:, 4])
    np.testing.assert_array_equal(e["is_leaf"], table[:, 5] != 0)
    np.testing.assert_allclose(e["mass"], table[:, 6], rtol=1e-15)
    np.testing.assert_allclose(e["com"], table[:, 7:10], rtol=1e-15, atol=1e-15)
    np.testing.assert_allclose(e["l"], table[:, 10], rtol=1e-15)
    assert tr.stats() == literal
    y = np.array([[30.0, 1.7, 1.7]])
    for theta, expect in counts:
        _, c = tr.bh_acc(y, 1.0, 0.1, theta)
        assert c[0] == expect, theta


def _cloud(seed, n):
    rng = np.random.default_rng(seed)
    X = np.concatenate([rng.normal(size=(n // 2, 3)) * [2, 1, 0.5],
                        rng.uniform(-4, 4, size=(n - n // 2, 3))])
    m = rng.uniform(0.1, 2.0, size=n)
    return X, m


@pytest.mark.parametrize("seed", [0, 1])
def test_theta_zero_is_the_direct_sum(orc, seed):
    X, m = _cloud(seed, 3000)
    Y = np.random.default_rng(seed + 10).normal(size=(200, 3)) * 2
    tr = orc.Tree(X, m)
    a_bh, cnt = tr.bh_acc(Y, 66.7, 0.2, 0.0)
    a_d = orc.direct_acc(X, m, Y, 66.7, 0.2)
    assert np.all(cnt == len(X))
    rel = np.linalg.norm(a_bh - a_d, axis=1) / np.linalg.norm(a_d, axis=1)
    assert rel.max() < 1e-13


def test_tree_invariants(orc):
    X, m = _cloud(3, 5000)
    tr = orc.Tree(X, m)
    e = tr.export()
    n = len(e["depth"])
    # root
    assert e["parent"][0] == -1 and e["depth"][0] == 0
    assert e["mass"][0] == pytest.approx(m.sum(), rel=1e-13)
    np.testing.assert_allclose(e["com"][0], (m[:, None] * X).sum(0) / m.sum(), rtol=1e-12, atol=1e-13)
    # every point in exactly one leaf, leaves partition the set
    assert np.all(e["leaf_of"] >= 0)
    leaves = np.nonzero(e["is_leaf"])[0]
    assert e["npts"][leaves].sum() == len(X)
    assert np.all(np.bincount(e["leaf_of"], minlength=n)[leaves] == e["npts"][leaves])
    # leaf mass/CoM from its own points
    for lf in leaves[:200]:
        pts = np.nonzero(e["leaf_of"] == lf)[0]
        assert e["mass"][lf] == pytest.approx(m[pts].sum(), rel=1e-13)
        np.testing.assert_allclose(e["com"][lf], (m[pts, None] * X[pts]).sum(0) / m[pts].sum(),
                                   rtol=1e-12, atol=1e-13)
    # internal nodes: >= 2 children, mass and CoM are their children's combination,
    # children are strictly deeper and nested in the parent's cell
    lo, hi = X.min(0), X.max(0)
    ext = hi - lo
    for v in range(n):
        ch = np.nonzero(e["parent"] == v)[0]
        if e["is_leaf"][v]:
            assert len(ch) == 0
            continue
        assert 2 <= len(ch) <= 8
        assert e["mass"][ch].sum() == pytest.approx(e["mass"][v], rel=1e-12)
        np.testing.assert_allclose((e["mass"][ch, None] * e["com"][ch]).sum(0) / e["mass"][ch].sum(),
                                   e["com"][v], rtol=1e-11, atol=1e-12)
        assert e["npts"][ch].sum() == e["npts"][v]
        for c in ch:
            dd = e["depth"][c] - e["depth"][v]
            assert dd >= 1
            np.testing.assert_array_equal(e["cell"][c] >> dd, e["cell"][v])
    # l is the box diagonal, halving per level (the root box is the tight BB)
    np.testing.assert_allclose(e["l"], np.linalg.norm(ext) / 2.0 ** e["depth"], rtol=1e-14)
    # CoM inside the node box
    h = ext / 2.0 ** e["depth"][:, None]
    blo = lo + e["cell"] * h
    assert np.all(e["com"] >= blo - 1e-12) and np.all(e["com"] <= blo + h + 1e-12)
    assert e["depth"].max() <= 20
    assert len(np.unique(e["parent"][1:])) == (~e["is_leaf"]).sum()


def test_depth_limit_keeps_duplicates_together(orc):
    rng = np.random.default_rng(4)
    X = np.concatenate([rng.uniform(-1, 1, size=(50, 3)), np.tile([[0.25, -0.5, 0.125]], (7, 1))])
    m = np.ones(len(X))
    tr = orc.Tree(X, m, max_depth=20)
    e = tr.export()
    lf = e["leaf_of"][50]
    assert np.all(e["leaf_of"][50:] == lf)
    assert e["npts"][lf] == 7 and e["depth"][lf] == 20
    ext = X.max(0) - X.min(0)
    assert e["l"][lf] == pytest.approx(np.linalg.norm(ext) / 2 ** 20, rel=1e-14)
    # a query failing the criterion on that leaf gets every duplicate exactly
    y = np.array([[0.25, -0.5, 0.125 + 1e-7]])
    a_bh, c = tr.bh_acc(y, 1.0, 0.1, 0.5)
    a_d = orc.direct_acc(X, m, y, 1.0, 0.1)
    np.testing.assert_allclose(a_bh, a_d, rtol=0.05)


def test_depth_limit_parameter(orc):
    X, m = _cloud(5, 2000)
    for d in [3, 6]:
        e = orc.Tree(X, m, max_depth=d).export()
        assert e["depth"].max() <= d
        leaves = e["is_leaf"]
        assert np.all((e["npts"][leaves] == 1) | (e["depth"][leaves] == d))


def test_error_grows_with_theta(orc):
    X, m = _cloud(6, 20000)
    Y = np.random.default_rng(7).uniform(-3, 3, size=(400, 3))
    tr = orc.Tree(X, m)
    a_d = orc.direct_acc(X, m, Y, 1.0, 0.2)
    errs, cnts = [], []
    for th in [0.1, 0.3, 0.5, 0.7, 0.9]:
        a, c = tr.bh_acc(Y, 1.0, 0.2, th)
        errs.append(np.linalg.norm(a - a_d) / np.linalg.norm(a_d))
        cnts.append(c.mean())
    assert all(e1 < e2 for e1, e2 in zip(errs, errs[1:]))
    assert all(c1 > c2 for c1, c2 in zip(cnts, cnts[1:]))
    assert errs[2] < 1e-2  # Sec. V-B: loss of accuracy negligible for theta <= 0.6


def test_single_node_monopole_error_bound(orc):
    # When the root is accepted (one term), the error is the monopole's, which is
    # second order in l / r for a distribution inside a box of diagonal l.
    rng = np.random.default_rng(8)
    X = rng.uniform(0, 1, size=(800, 3))
    m = rng.uniform(0.1, 1, size=800)
    tr = orc.Tree(X, m)
    l = np.linalg.norm(X.max(0) - X.min(0))
    for r in [3.0, 6.0, 12.0]:
        dirs = rng.normal(size=(20, 3))
        dirs /= np.linalg.norm(dirs, axis=1, keepdims=True)
        com = (m[:, None] * X).sum(0) / m.sum()
        Y = com + dirs * r * l
        a, c = tr.bh_acc(Y, 1.0, 1e-3, 1.0 / (0.99 * r))
        assert np.all(c == 1)
        a_d = orc.direct_acc(X, m, Y, 1.0, 1e-3)
        rel = np.linalg.norm(a - a_d, axis=1) / np.linalg.norm(a_d, axis=1)
        assert rel.max() < 3.0 / r ** 2


def test_huge_theta_is_root_monopole(orc):
    X, m = _cloud(9, 1000)
    tr = orc.Tree(X, m)
    Y = np.random.default_rng(1).normal(size=(20, 3)) * 10
    a, c = tr.bh_acc(Y, 2.0, 0.3, 1e9)
    assert np.all(c == 1)
    com = (m[:, None] * X).sum(0) / m.sum()
    np.testing.assert_allclose(a, orc.direct_acc(com[None], [m.sum()], Y, 2.0, 0.3), rtol=1e-12)


def test_lidar_subsample_tree(orc):
    X, Y, _, _ = synth.lidar_pair(3, n=20000)
    Xn, Yn, _ = orc.normalize(X, Y)
    m = orc.masses_niv(Xn)
    tr = orc.Tree(Xn, m)
    a, c = tr.bh_acc(Yn[:300], 66.7, 0.2, 0.5)
    a_d = orc.direct_acc(Xn, m, Yn[:300], 66.7, 0.2)
    assert np.linalg.norm(a - a_d) / np.linalg.norm(a_d) < 2e-2
    assert c.mean() < len(Xn)

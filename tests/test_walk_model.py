"""A CPU model of the records the GPU's Barnes-Hut walks read, built from the
oracle's own tree (Algorithm 1, exported in pre-order), walked without a
stack, against the oracle's recursive BHForce.

The records are the tree in depth-first pre-order with each cell's subtree
record count; a leaf of several particles is followed by one record per
particle, and a single-particle record carries l^2 = -1. The walk visits
record v, adds its monopole and skips its subtree (v += size) when the point
accepts it (l^2 < theta^2 r^2), and otherwise moves to v + 1. This pins the
claim that such a walk takes exactly BHForce's terms (R3 for leaves that fail
the test), independently of the GPU code.
"""
import numpy as np
import pytest


def _records(eo, X, m):
    n = len(eo["depth"])
    multi = eo["is_leaf"] & (eo["npts"] >= 2)
    own = 1 + np.where(multi, eo["npts"], 0)
    size = own.copy()
    for k in range(n - 1, 0, -1):
        size[eo["parent"][k]] += size[k]
    com, mass, l2, skip = [], [], [], []
    for k in range(n):
        single = eo["is_leaf"][k] and eo["npts"][k] == 1
        com.append(eo["com"][k])
        mass.append(eo["mass"][k])
        l2.append(-1.0 if single else eo["l"][k] ** 2)
        skip.append(size[k])
        if multi[k]:
            for j in np.flatnonzero(eo["leaf_of"] == k):
                com.append(X[j])
                mass.append(m[j])
                l2.append(-1.0)
                skip.append(1)
    return np.array(com), np.array(mass), np.array(l2), np.array(skip)


def _walk(rec, y, theta, eps):
    com, mass, l2, skip = rec
    a = np.zeros(3)
    count = 0
    v = 0
    while v < len(skip):
        d = com[v] - y
        r2 = d @ d
        if l2[v] < theta * theta * r2:
            a += mass[v] * d / (r2 + eps * eps) ** 1.5
            count += 1
            v += skip[v]
        else:
            v += 1
    return a, count


def _clouds():
    rng = np.random.default_rng(21)
    gauss = rng.normal(size=(3000, 3)) * [2.0, 1.0, 0.5]
    dups = np.vstack([rng.uniform(-1, 1, (600, 3)), np.tile([[0.25, -0.5, 0.125]], (12, 1))])
    return {"gauss": (gauss, rng.uniform(0.2, 2.0, len(gauss)), 20),
            "dups": (dups, np.ones(len(dups)), 20),
            "shallow": (rng.uniform(-1, 1, (2500, 3)), rng.uniform(0.5, 1.5, 2500), 4)}


@pytest.mark.parametrize("name", ["gauss", "dups", "shallow"])
@pytest.mark.parametrize("theta", [0.0, 0.5, 0.9])
def test_stackless_walk_takes_bhforce_terms(orc, name, theta):
    X, m, depth = _clouds()[name]
    tree = orc.Tree(X, m, max_depth=depth)
    rec = _records(tree.export(), X, m)
    rng = np.random.default_rng(5)
    Y = np.vstack([X[rng.choice(len(X), 4, replace=False)],  # on reference points (r = 0 cases)
                   rng.uniform(X.min(0), X.max(0), size=(8, 3))])
    a_o, c_o = tree.bh_acc(Y, 1.0, 0.1, theta)
    for i, y in enumerate(Y):
        a, c = _walk(rec, y, theta, 0.1)
        assert c == c_o[i]
        np.testing.assert_allclose(a, a_o[i], rtol=1e-11, atol=1e-12 * np.abs(a_o[i]).max())
    if theta == 0.0:
        assert np.all(c_o == len(X))


def _records_with_counts(eo, X, m):
    com, mass, l2, skip = _records(eo, X, m)
    # child count of each record: > 0 for cells, -1 single particle, -nb for a
    # leaf of nb >= 2 particles (whose particle records follow it)
    n = len(eo["depth"])
    nchild = np.bincount(eo["parent"][1:], minlength=n)
    counts = []
    for k in range(n):
        if eo["is_leaf"][k]:
            counts.append(-int(eo["npts"][k]))
            if eo["npts"][k] >= 2:
                counts.extend([-1] * int(eo["npts"][k]))
        else:
            counts.append(int(nchild[k]))
    return com, mass, l2, skip, np.array(counts)


def _coop_walk(rec, Y, theta, eps):
    """One walk for a group of points: a record is judged by the points that
    rejected all its ancestors (a mask per pending sibling range). A range is
    (next record, records left); the next sibling is a subtree size further."""
    com, mass, l2, skip, cnt = rec
    P = len(Y)
    acc = np.zeros((P, 3))
    terms = np.zeros(P, dtype=np.int64)
    v, left, mask = 0, 1, np.ones(P, bool)
    saved, most = [], 0
    while left > 0:
        d = com[v] - Y
        r2 = (d * d).sum(1)
        accept = mask & (l2[v] < theta * theta * r2)
        acc[accept] += (mass[v] * d[accept]) / ((r2[accept] + eps * eps) ** 1.5)[:, None]
        terms += accept
        rej = mask & ~accept
        nv, nleft = v + skip[v], left - 1
        if rej.any() and cnt[v] > 0:
            if nleft > 0:
                saved.append((nv, nleft, mask))
                most = max(most, len(saved))
            v, left, mask = v + 1, int(cnt[v]), rej
        else:
            if rej.any() and cnt[v] < -1:
                for b in range(1, -cnt[v] + 1):
                    db = com[v + b] - Y[rej]
                    rb = (db * db).sum(1)
                    acc[rej] += mass[v + b] * db / ((rb + eps * eps) ** 1.5)[:, None]
                terms[rej] += -cnt[v]
            v, left = nv, nleft
        if left == 0 and saved:
            v, left, mask = saved.pop()
    return acc, terms, most


@pytest.mark.parametrize("name", ["gauss", "dups", "shallow"])
@pytest.mark.parametrize("theta", [0.0, 0.5, 0.9])
def test_cooperative_walk_takes_each_points_bhforce_terms(orc, name, theta):
    X, m, depth = _clouds()[name]
    tree = orc.Tree(X, m, max_depth=depth)
    rec = _records_with_counts(tree.export(), X, m)
    rng = np.random.default_rng(6)
    # a group of spatial neighbours plus a few stragglers
    c = X[rng.integers(len(X))]
    near = X[np.argsort(((X - c) ** 2).sum(1))[:40]] + rng.normal(scale=0.01, size=(40, 3))
    Y = np.vstack([near, rng.uniform(X.min(0), X.max(0), size=(24, 3))])
    a_o, c_o = tree.bh_acc(Y, 1.0, 0.1, theta)
    a, terms, most = _coop_walk(rec, Y, theta, 0.1)
    np.testing.assert_array_equal(terms, c_o)
    np.testing.assert_allclose(a, a_o, rtol=1e-11, atol=1e-12 * np.abs(a_o).max())
    assert most <= 20  # at most one saved range per tree level below the root


def test_saved_ranges_stay_within_the_depth_bound(orc):
    # a chain of ever-closer pairs drives the tree to its depth limit
    pts = [[0.0, 0.0, 0.0], [1.0, 1.0, 1.0]]
    for k in range(1, 24):
        s = 0.5 ** k
        pts += [[s, s, s], [s * 0.9, s * 1.1, s * 0.7]]
    X = np.array(pts)
    m = np.ones(len(X))
    tree = orc.Tree(X, m, max_depth=20)
    eo = tree.export()
    assert eo["depth"].max() == 20
    rec = _records_with_counts(eo, X, m)
    Y = X[:8] + 1e-9
    a_o, c_o = tree.bh_acc(Y, 1.0, 0.1, 0.0)
    a, terms, most = _coop_walk(rec, Y, 0.0, 0.1)
    np.testing.assert_array_equal(terms, c_o)
    # the GPU walk keeps saved range k in lane k's registers: 32 lanes, 20 levels
    assert 15 <= most <= 20


def _union_walk(rec, Y, theta, eps):
    """One walk for a group of points that follows every point's own
    stackless walk: each point keeps the record its walk reads next (nx); the
    group visits the smallest nx, and the points whose nx it is judge that
    record as their own walk would. Returns the forces, term counts, the
    visited records and whether every step went to v + 1 or v + size(v)."""
    com, mass, l2, skip = rec
    P, n = len(Y), len(skip)
    acc = np.zeros((P, 3))
    terms = np.zeros(P, dtype=np.int64)
    nx = np.zeros(P, dtype=np.int64)
    visited, successors_ok = [], True
    v = 0
    while v < n:
        visited.append(v)
        act = nx == v
        d = com[v] - Y
        r2 = (d * d).sum(1)
        accept = act & (l2[v] < theta * theta * r2)
        acc[accept] += (mass[v] * d[accept]) / ((r2[accept] + eps * eps) ** 1.5)[:, None]
        terms += accept
        nx[accept] = v + skip[v]
        nx[act & ~accept] = v + 1
        nv = int(nx.min())
        successors_ok &= nv in (v + 1, v + skip[v]) or nv >= n
        v = nv
    return acc, terms, visited, successors_ok


@pytest.mark.parametrize("name", ["gauss", "dups", "shallow"])
@pytest.mark.parametrize("theta", [0.0, 0.5, 0.9])
def test_union_walk_takes_each_points_bhforce_terms(orc, name, theta):
    # The GPU's union walk (k_bh<3>/<4>/<5>) modelled on the CPU: each point
    # takes exactly the oracle's BHForce terms, the group visits exactly the
    # union of its points' own walks, and the next record is always v + 1 or
    # v + size(v) (a waiting point accepted an ancestor of v).
    X, m, depth = _clouds()[name]
    tree = orc.Tree(X, m, max_depth=depth)
    rec = _records(tree.export(), X, m)
    rng = np.random.default_rng(8)
    c = X[rng.integers(len(X))]
    near = X[np.argsort(((X - c) ** 2).sum(1))[:48]] + rng.normal(scale=0.01, size=(48, 3))
    Y = np.vstack([near, rng.uniform(X.min(0), X.max(0), size=(16, 3))])
    a_o, c_o = tree.bh_acc(Y, 1.0, 0.1, theta)
    a, terms, visited, ok = _union_walk(rec, Y, theta, 0.1)
    np.testing.assert_array_equal(terms, c_o)
    np.testing.assert_allclose(a, a_o, rtol=1e-11, atol=1e-12 * np.abs(a_o).max())
    assert ok
    own = set()
    for y in Y:
        com, mass, l2, skip = rec
        v = 0
        while v < len(skip):
            own.add(v)
            d = com[v] - y
            v += skip[v] if l2[v] < theta * theta * (d @ d) else 1
    assert visited == sorted(own)

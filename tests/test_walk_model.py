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

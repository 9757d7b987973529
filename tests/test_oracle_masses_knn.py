"""Pins of the oracle's k-NN inverse-density masses (m_i ~ r_k(i)^D).

Fixed independently of the code: on points 0, 1, ..., n-1 along a line, point
i's 16th nearest neighbour is at distance 16 - i for i < 8 and 8 in the
interior; brute force with a library sort on tiny clouds; rigid invariance;
positive masses for repeated points.
"""
import numpy as np


def test_line_closed_form(orc):
    n = 60
    P = np.column_stack([np.arange(n, dtype=float), np.zeros(n), np.zeros(n)])
    m = orc.masses_knn(P, k=16, a=0.0, b=100.0)
    r = np.array([16.0 - i if i < 8 else (16.0 - (n - 1 - i) if i > n - 9 else 8.0) for i in range(n)])
    expect = r**3 / (r**3).sum()
    np.testing.assert_allclose(m, expect, rtol=1e-13)
    # D = 2: areas r^2
    m2 = orc.masses_knn(P, k=16, dim=2, a=0.0, b=100.0)
    np.testing.assert_allclose(m2, r**2 / (r**2).sum(), rtol=1e-13)


def test_brute_force_with_a_sort(orc):
    rng = np.random.default_rng(0)
    for k in (1, 5, 16):
        P = rng.uniform(-4, 4, size=(70, 3))
        d = np.sqrt(((P[:, None, :] - P[None, :, :]) ** 2).sum(-1))
        d[np.arange(70), np.arange(70)] = np.inf
        r = np.sort(d, axis=1)[:, k - 1]
        np.testing.assert_allclose(orc.masses_knn(P, k=k, total=2.0), 2.0 * r**3 / (r**3).sum(), rtol=1e-12)


def test_invariant_under_rigid_motion(orc):
    rng = np.random.default_rng(1)
    P = rng.uniform(-3, 3, size=(500, 3))
    q, _ = np.linalg.qr(rng.normal(size=(3, 3)))
    Q = P @ q.T + rng.normal(size=3) * 0.5
    np.testing.assert_allclose(orc.masses_knn(Q), orc.masses_knn(P), rtol=1e-10)


def test_repeated_points_keep_positive_mass(orc):
    P = np.vstack([np.zeros((30, 3)), np.random.default_rng(2).uniform(-1, 1, size=(40, 3))])
    m = orc.masses_knn(P)
    assert np.all(m > 0) and np.isfinite(m).all()
    assert abs(m.sum() - 1.0) < 1e-12

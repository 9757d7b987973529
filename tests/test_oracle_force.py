"""Pins of the oracle's all-pairs force (Eq. 6) against closed forms and physics.

None of these re-type Eq. 6: each checks a property that a dropped term, a
wrong exponent, a sign error or a swapped operand would break.
"""
import math

import numpy as np
import pytest

import synth


def _rng(s=0):
    return np.random.default_rng(s)


def test_single_source_peak_closed_form(orc):
    # |a|(r) = G m r / (r^2 + eps^2)^(3/2) peaks at r = eps/sqrt(2) with value
    # 2 G m / (3 sqrt(3) eps^2) (calculus, not the summation code).
    G, m, eps = 3.7, 0.8, 0.25
    X = np.zeros((1, 3))
    r = np.linspace(0.01, 1.0, 20001)
    Y = np.stack([r, np.zeros_like(r), np.zeros_like(r)], 1)
    a = orc.direct_acc(X, [m], Y, G, eps)
    mag = np.linalg.norm(a, axis=1)
    k = int(np.argmax(mag))
    assert abs(r[k] - eps / math.sqrt(2)) < 1e-4
    assert mag[k] == pytest.approx(2 * G * m / (3 * math.sqrt(3) * eps ** 2), rel=1e-7)


def test_attraction_points_at_source(orc):
    rng = _rng(1)
    X = rng.normal(size=(1, 3))
    Y = rng.normal(size=(50, 3)) * 3
    a = orc.direct_acc(X, [1.0], Y, 66.7, 0.2)
    cosang = np.einsum("ij,ij->i", a, X - Y) / np.linalg.norm(a, axis=1) / np.linalg.norm(X - Y, axis=1)
    assert np.all(cosang > 1 - 1e-12)


def test_inverse_square_far_field(orc):
    G, m, eps = 66.7, 0.3, 0.2
    X = np.zeros((1, 3))
    for r in [1e3, 1e4]:
        a = orc.direct_acc(X, [m], np.array([[0.0, r, 0.0]]), G, eps)
        assert np.linalg.norm(a) * r * r == pytest.approx(G * m, rel=2 * (eps / r) ** 2)


def test_gradient_of_plummer_potential(orc):
    # Eq. 6 is minus the gradient of Phi(y) = -G sum m_j / sqrt(|X_j - y|^2 + eps^2)
    # (this is why Eq. 4's printed (|.| + eps) form is not used as the energy).
    rng = _rng(2)
    X = rng.normal(size=(40, 3))
    m = rng.uniform(0.1, 1.0, size=40)
    G, eps = 2.0, 0.3
    Y = rng.normal(size=(10, 3))

    def phi(y):
        d = X - y
        return -G * np.sum(m / np.sqrt(np.sum(d * d, 1) + eps * eps))

    a = orc.direct_acc(X, m, Y, G, eps)
    h = 1e-5
    for i in range(len(Y)):
        g = np.zeros(3)
        for k in range(3):
            e = np.zeros(3)
            e[k] = h
            g[k] = (phi(Y[i] + e) - phi(Y[i] - e)) / (2 * h)
        np.testing.assert_allclose(a[i], -g, rtol=1e-6, atol=1e-9)


def _fibonacci_sphere(n):
    i = np.arange(n) + 0.5
    phi = np.arccos(1 - 2 * i / n)
    th = math.pi * (1 + 5 ** 0.5) * i
    return np.stack([np.cos(th) * np.sin(phi), np.sin(th) * np.sin(phi), np.cos(phi)], 1)


def test_shell_theorem(orc):
    # Newton's shell theorem: outside a uniform spherical shell the field is that
    # of a point of the shell's mass at its centre; inside it vanishes.
    X = _fibonacci_sphere(40000)
    m = np.full(len(X), 1.0 / len(X))
    G, eps = 1.0, 1e-3
    out = orc.direct_acc(X, m, np.array([[0.0, 0.0, 2.0], [1.5, 1.5, 0.0]]), G, eps)
    for y, a in zip([[0, 0, 2.0], [1.5, 1.5, 0.0]], out):
        y = np.asarray(y)
        r = np.linalg.norm(y)
        np.testing.assert_allclose(a, -G * y / r ** 3, rtol=1e-4, atol=1e-4 * G / r ** 2)
    inside = orc.direct_acc(X, m, np.array([[0.1, 0.2, -0.15], [0.0, 0.0, 0.0]]), G, eps)
    assert np.abs(inside).max() < 1e-3 * G


def test_superposition_over_partitions(orc):
    rng = _rng(3)
    X = rng.normal(size=(300, 3))
    m = rng.uniform(0.5, 2.0, size=300)
    Y = rng.normal(size=(20, 3))
    full = orc.direct_acc(X, m, Y, 1.5, 0.1)
    idx = rng.permutation(300)
    parts = [idx[:7], idx[7:150], idx[150:]]
    s = sum(orc.direct_acc(X[p], m[p], Y, 1.5, 0.1) for p in parts)
    np.testing.assert_allclose(full, s, rtol=1e-12, atol=1e-14)


def test_translation_and_rotation_equivariance(orc):
    rng = _rng(4)
    X = rng.normal(size=(200, 3))
    m = rng.uniform(size=200)
    Y = rng.normal(size=(30, 3))
    R = synth.random_rotation(rng, 180)
    t = rng.normal(size=3) * 10
    a0 = orc.direct_acc(X, m, Y, 66.7, 0.2)
    a1 = orc.direct_acc(X @ R.T + t, m, Y @ R.T + t, 66.7, 0.2)
    np.testing.assert_allclose(a1, a0 @ R.T, rtol=1e-10, atol=1e-12)


def test_newton_third_law(orc):
    # The force of X on Y is minus the force of Y on X (each particle's force is
    # its mass times its acceleration); this fails if the source and target
    # masses are swapped or one of them is dropped.
    rng = _rng(5)
    X = rng.normal(size=(120, 3))
    Y = rng.normal(size=(90, 3)) + 0.3
    mX = rng.uniform(0.2, 3.0, size=120)
    mY = rng.uniform(0.2, 3.0, size=90)
    F_on_Y = (mY[:, None] * orc.direct_acc(X, mX, Y, 1.0, 0.15)).sum(0)
    F_on_X = (mX[:, None] * orc.direct_acc(Y, mY, X, 1.0, 0.15)).sum(0)
    np.testing.assert_allclose(F_on_Y, -F_on_X, rtol=1e-10, atol=1e-12)


def test_monopole_error_is_second_order(orc):
    # About the centre of mass a cluster has no dipole moment, so replacing it by
    # its total mass at the CoM errs by O((l/r)^2): doubling r quarters the
    # relative error. A wrongly weighted centre leaves a dipole error O(l/r).
    rng = _rng(6)
    X = rng.uniform(-0.5, 0.5, size=(500, 3))
    m = rng.uniform(0.1, 1.0, size=500)
    com = (m[:, None] * X).sum(0) / m.sum()
    errs = []
    for r in [20.0, 40.0, 80.0]:
        y = com + np.array([[r, 0.3 * r, -0.2 * r]])
        exact = orc.direct_acc(X, m, y, 1.0, 1e-3)
        mono = orc.direct_acc(com[None, :], [m.sum()], y, 1.0, 1e-3)
        errs.append(np.linalg.norm(exact - mono) / np.linalg.norm(exact))
    assert 3.0 < errs[0] / errs[1] < 5.0
    assert 3.0 < errs[1] / errs[2] < 5.0


def test_softening_removes_singularity(orc):
    X = np.array([[1.0, 2.0, 3.0]])
    a = orc.direct_acc(X, [5.0], X.copy(), 66.7, 0.2)
    assert np.all(a == 0.0)


def test_abs_magnitude_bounds_sum(orc):
    rng = _rng(7)
    X = rng.normal(size=(100, 3))
    Y = rng.normal(size=(10, 3))
    a, ab = orc.direct_acc(X, np.ones(100), Y, 1.0, 0.1, want_abs=True)
    assert np.all(np.linalg.norm(a, axis=1) <= ab * (1 + 1e-12))

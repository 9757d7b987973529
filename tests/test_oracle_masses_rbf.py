"""Pins of the oracle's RBF mass interpolant (Eq. 17) and SPM masses (Eq. 19).

Each pin is fixed by the mathematics, not by the code: the interpolation
property at the landmarks, closed forms for one and two landmarks, Euclidean
invariance (stated in Sec. IV-F.1), the empty-landmark case (B = 1, Eq. 17),
and the point-wise product of Eq. 19.
"""
import math

import numpy as np
import pytest


def cloud(seed, n=600):
    return np.random.default_rng(seed).uniform(-4.0, 4.0, size=(n, 3))


def test_interpolates_one_at_every_landmark(orc):
    P = cloud(0)
    idx = [5, 77, 150, 300, 451, 599]
    B = orc.masses_rbf(P, idx, sigma=1.5)
    np.testing.assert_allclose(B[idx], 1.0, atol=1e-12)


def test_one_landmark_is_a_gaussian(orc):
    P = cloud(1)
    sigma, c = 1.3, 42
    B = orc.masses_rbf(P, [c], sigma=sigma, floor=1e-300)
    d2 = ((P - P[c]) ** 2).sum(1)
    np.testing.assert_allclose(B, np.exp(-d2 / sigma**2), rtol=1e-13, atol=1e-300)


def test_two_landmarks_closed_form(orc):
    # [[1, e], [e, 1]] lambda = [1, 1]  =>  lambda_1 = lambda_2 = 1 / (1 + e)
    P = cloud(2)
    sigma, c1, c2 = 2.0, 10, 20
    B = orc.masses_rbf(P, [c1, c2], sigma=sigma, floor=1e-300)
    e = math.exp(-((P[c1] - P[c2]) ** 2).sum() / sigma**2)
    g1 = np.exp(-((P - P[c1]) ** 2).sum(1) / sigma**2)
    g2 = np.exp(-((P - P[c2]) ** 2).sum(1) / sigma**2)
    np.testing.assert_allclose(B, (g1 + g2) / (1.0 + e), rtol=1e-12, atol=1e-300)


def test_invariant_under_rigid_motion(orc):
    P = cloud(3)
    idx = [1, 99, 200, 333]
    rng = np.random.default_rng(9)
    q, _ = np.linalg.qr(rng.normal(size=(3, 3)))
    q *= np.sign(np.linalg.det(q))
    Q = P @ q.T + rng.normal(size=3)
    np.testing.assert_allclose(orc.masses_rbf(Q, idx, sigma=1.7), orc.masses_rbf(P, idx, sigma=1.7),
                               rtol=1e-11, atol=1e-14)


def test_no_landmarks_gives_one_and_spm_equals_niv(orc):
    P = cloud(4)
    np.testing.assert_array_equal(orc.masses_rbf(P, []), np.ones(len(P)))
    np.testing.assert_allclose(orc.masses_spm(P, []), orc.masses_niv(P), rtol=1e-13)


def test_floor_far_from_landmarks(orc):
    P = np.vstack([cloud(5, 50) * 0.1, np.array([[4.5, 4.5, 4.5]])])
    B = orc.masses_rbf(P, [0, 1, 2], sigma=0.3, floor=1e-3)
    assert B[-1] == 1e-3
    assert np.all(B >= 1e-3)


def test_spm_is_the_pointwise_product(orc):
    P = cloud(6)
    idx = [3, 30, 300]
    S = orc.masses_spm(P, idx, sigma=1.0, total=2.0)
    N = orc.masses_niv(P)
    B = orc.masses_rbf(P, idx, sigma=1.0)
    assert abs(S.sum() - 2.0) < 1e-12
    ratio = S / (N * B)
    np.testing.assert_allclose(ratio, ratio[0], rtol=1e-12)


def test_repeated_landmark_is_rejected(orc):
    P = cloud(7)
    with pytest.raises(ValueError):
        orc.masses_rbf(P, [4, 4])

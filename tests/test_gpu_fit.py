"""The device rigid fit (Eqs. 14, 16) on its own, against the oracle's FP64
Kabsch step (one-sided Jacobi SVD).

fga_rigid_fit runs the code every iteration of fga_step runs (one matrix
entry per lane of a warp, an FP32 polar phase, an FP64 Newton step and an
FP64 correction against C) on reduced sums computed here in FP64, so the
fit's accuracy is checked without the FP32 forces in between: the rotation
to 1e-12 and the translation to 1e-12 of the cloud's extent.
"""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def fga():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__
    __graft_entry__.build_library()
    import paper_2009_14005_gb300 as m
    return m


@pytest.fixture(scope="module")
def orc():
    import oracle
    oracle.build()
    return oracle


def _rot(rng, deg):
    ax = rng.normal(size=3)
    ax /= np.linalg.norm(ax)
    th = np.radians(deg)
    K = np.array([[0, -ax[2], ax[1]], [ax[2], 0, -ax[0]], [-ax[1], ax[0], 0]])
    return np.eye(3) + np.sin(th) * K + (1 - np.cos(th)) * K @ K


def _sums(Y, D):
    """The 27 reduced sums about the FP32-rounded centroid, and that centre."""
    mu0 = Y.mean(0).astype(np.float32).astype(np.float64)
    yc = Y - mu0
    S = yc.T @ yc
    red = np.zeros(27)
    red[0:3] = yc.sum(0)
    red[3:6] = D.sum(0)
    red[6:12] = [S[0, 0], S[0, 1], S[0, 2], S[1, 1], S[1, 2], S[2, 2]]
    red[12:21] = (D.T @ yc).ravel()
    return red, mu0


@pytest.mark.parametrize("deg,seed", [(0.01, 1), (0.5, 2), (12.0, 3), (60.0, 4), (150.0, 5), (179.0, 6)])
def test_fit_matches_the_oracle_kabsch(fga, orc, deg, seed):
    rng = np.random.default_rng(seed)
    M = 1000
    Y = rng.normal(size=(M, 3)) * [3.0, 1.5, 0.5] + [0.4, -0.3, 0.2]
    D = Y @ _rot(rng, deg).T + [0.1, -0.05, 0.02] - Y + rng.normal(size=(M, 3)) * 1e-3
    red, mu0 = _sums(Y, D)
    R, t, code = fga.fga_rigid_fit(red, M, mu0)
    Ro, to, st = orc.kabsch(Y, D)
    assert code == fga.FGA_OK and st == 0
    np.testing.assert_allclose(R, Ro, atol=1e-12)
    np.testing.assert_allclose(t, to, atol=1e-12 * np.abs(Y).max())
    # orthogonal to FP64 rounding (the correction's first-order update leaves
    # |w|^2 / 2, w the FP32 phase's residual rotation, below 1e-14)
    np.testing.assert_allclose(R @ R.T, np.eye(3), atol=3e-14)
    assert abs(np.linalg.det(R) - 1.0) < 1e-13


def test_reflected_target_takes_the_eigen_route(fga, orc):
    # Y + D is a mirror image of Y: det C < 0, so the polar route gives way to
    # the eigen-decomposition route, which still returns a proper rotation
    rng = np.random.default_rng(7)
    M = 800
    Y = rng.normal(size=(M, 3)) * [2.0, 1.0, 0.4]
    D = Y * [1.0, 1.0, -1.0] - Y
    red, mu0 = _sums(Y, D)
    R, t, code = fga.fga_rigid_fit(red, M, mu0)
    Ro, to, st = orc.kabsch(Y, D)
    assert code == fga.FGA_OK and st == 0
    np.testing.assert_allclose(R, Ro, atol=1e-10)
    np.testing.assert_allclose(t, to, atol=1e-10 * np.abs(Y).max())
    assert abs(np.linalg.det(R) - 1.0) < 1e-12


def test_collinear_template_is_degenerate(fga, orc):
    rng = np.random.default_rng(8)
    s = np.linspace(-1, 1, 300)[:, None]
    Y = s * [0.6, 0.8, 0.0] + [0.1, 0.2, 0.3]
    D = rng.normal(size=Y.shape) * 1e-2
    red, mu0 = _sums(Y, D)
    R, t, code = fga.fga_rigid_fit(red, len(Y), mu0)
    Ro, to, st = orc.kabsch(Y, D)
    assert code == fga.FGA_EDEGENERATE and st == 1
    np.testing.assert_array_equal(R, np.eye(3))
    np.testing.assert_allclose(t, D.mean(0), atol=1e-14)
    np.testing.assert_allclose(t, to, atol=1e-14)


def test_planar_fit(fga, orc):
    rng = np.random.default_rng(9)
    M = 600
    Y = np.zeros((M, 3))
    Y[:, :2] = rng.normal(size=(M, 2)) * [2.0, 0.7]
    th = np.radians(33.0)
    R2 = np.array([[np.cos(th), -np.sin(th), 0], [np.sin(th), np.cos(th), 0], [0, 0, 1]])
    D = Y @ R2.T + [0.2, -0.1, 0.0] - Y
    D[:, :2] += rng.normal(size=(M, 2)) * 1e-3
    red, mu0 = _sums(Y, D)
    R, t, code = fga.fga_rigid_fit(red, M, mu0, dim=2)
    Ro, to, st = orc.kabsch(Y, D, dim=2)
    assert code == fga.FGA_OK and st == 0
    np.testing.assert_allclose(R, Ro, atol=1e-12)
    np.testing.assert_allclose(t, to, atol=1e-12 * np.abs(Y).max())


def test_bad_arguments_are_rejected(fga):
    red = np.zeros(27)
    with pytest.raises(Exception):
        fga.fga_rigid_fit(red, 0, np.zeros(3))
    with pytest.raises(Exception):
        fga.fga_rigid_fit(red, 10, np.zeros(3), dim=4)
    red[5] = np.nan
    with pytest.raises(Exception):
        fga.fga_rigid_fit(red, 10, np.zeros(3))

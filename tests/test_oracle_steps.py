"""Pins of the oracle's ODE step (Eqs. 7-10), rigid fit (Eqs. 14, 16),
normalisation (Appendix A) and NIV masses (Eq. 18)."""
import math

import numpy as np
import pytest

import synth


# --------------------------------------------------------------------------- Eqs. 7-10

def test_free_damping_is_geometric(orc):
    # With no gravity, Eq. 9 reduces to v_{k+1} = (1 - eta dt / m) v_k.
    rng = np.random.default_rng(0)
    v = rng.normal(size=(5, 3))
    mY = np.array([0.1, 0.5, 1.0, 2.0, 4.0])
    dt, eta = 0.1, 0.3
    cur = v.copy()
    for _ in range(25):
        cur, d = orc.ode_step(cur, np.zeros_like(cur), mY, dt, eta)
        np.testing.assert_allclose(d, dt * cur, rtol=1e-15)
    np.testing.assert_allclose(cur, v * ((1 - eta * dt / mY) ** 25)[:, None], rtol=1e-12)


def test_velocity_then_position_update_order(orc):
    # Eq. 10 moves with the *updated* velocity (semi-implicit Euler), which keeps
    # a circular orbit bounded; moving with the old velocity (explicit Euler)
    # spirals outwards. One test particle orbits a single heavy source, eta = 0.
    G, M, r0, dt = 1.0, 1.0, 1.0, 0.02
    X = np.zeros((1, 3))
    y = np.array([[r0, 0.0, 0.0]])
    v = np.array([[0.0, math.sqrt(G * M / r0), 0.0]])
    y_ex, v_ex = y.copy(), v.copy()
    radii, radii_ex = [], []
    for _ in range(3000):
        a = orc.direct_acc(X, [M], y, G, 1e-6)
        v, d = orc.ode_step(v, a, [1.0], dt, 0.0)
        y = y + d
        radii.append(np.linalg.norm(y))
        # the same orbit moved with the old velocity, for contrast
        a_ex = orc.direct_acc(X, [M], y_ex, G, 1e-6)
        y_ex = y_ex + dt * v_ex
        v_ex = v_ex + dt * a_ex
        radii_ex.append(np.linalg.norm(y_ex))
    assert max(radii) < 1.03 * r0 and min(radii) > 0.97 * r0
    assert radii_ex[-1] > 1.5 * r0


# --------------------------------------------------------------------------- Eqs. 14, 16

def _kabsch_numpy(Y, D):
    # reference via numpy's LAPACK SVD (a library routine standing in for Eq. 14)
    Z = Y + D
    my, mz = Y.mean(0), Z.mean(0)
    C = (Z - mz).T @ (Y - my)
    U, S, Vt = np.linalg.svd(C)
    d = np.sign(np.linalg.det(U @ Vt))
    R = U @ np.diag([1, 1, d]) @ Vt
    return R, mz - R @ my


def _horn_quaternion(Y, D):
    # Horn (1987): the optimal rotation is the top eigenvector of a 4x4
    # symmetric matrix built from the cross-covariance; an independent method.
    Z = Y + D
    my, mz = Y.mean(0), Z.mean(0)
    S = (Y - my).T @ (Z - mz)
    Sxx, Sxy, Sxz, Syx, Syy, Syz, Szx, Szy, Szz = S.ravel()
    N = np.array([
        [Sxx + Syy + Szz, Syz - Szy, Szx - Sxz, Sxy - Syx],
        [Syz - Szy, Sxx - Syy - Szz, Sxy + Syx, Szx + Sxz],
        [Szx - Sxz, Sxy + Syx, -Sxx + Syy - Szz, Syz + Szy],
        [Sxy - Syx, Szx + Sxz, Syz + Szy, -Sxx - Syy + Szz]])
    w, V = np.linalg.eigh(N)
    q0, qx, qy, qz = V[:, -1]
    R = np.array([
        [q0 * q0 + qx * qx - qy * qy - qz * qz, 2 * (qx * qy - q0 * qz), 2 * (qx * qz + q0 * qy)],
        [2 * (qy * qx + q0 * qz), q0 * q0 - qx * qx + qy * qy - qz * qz, 2 * (qy * qz - q0 * qx)],
        [2 * (qz * qx - q0 * qy), 2 * (qz * qy + q0 * qx), q0 * q0 - qx * qx - qy * qy + qz * qz]])
    return R, mz - R @ my


@pytest.mark.parametrize("deg", [0.5, 30.0, 120.0, 179.0])
def test_exact_rigid_displacement_recovered(orc, deg):
    rng = np.random.default_rng(int(deg * 10))
    Y = rng.normal(size=(200, 3)) * [3, 2, 1]
    R0 = synth.rotation_about(rng.normal(size=3), math.radians(deg))
    t0 = rng.normal(size=3)
    D = Y @ R0.T + t0 - Y
    R, t, st = orc.kabsch(Y, D)
    assert st == 0
    np.testing.assert_allclose(R, R0, atol=1e-12)
    np.testing.assert_allclose(t, t0, atol=1e-12)


def test_reflection_gives_proper_rotation(orc):
    rng = np.random.default_rng(1)
    Y = rng.normal(size=(100, 3)) * [3, 2, 1]
    P = np.diag([1.0, 1.0, -1.0])
    R, t, st = orc.kabsch(Y, Y @ P.T - Y)
    assert np.linalg.det(R) == pytest.approx(1.0, abs=1e-12)
    Rn, tn = _kabsch_numpy(Y, Y @ P.T - Y)
    np.testing.assert_allclose(R, Rn, atol=1e-10)


def test_zero_displacement_is_identity(orc):
    Y = np.random.default_rng(2).normal(size=(50, 3))
    R, t, st = orc.kabsch(Y, np.zeros_like(Y))
    np.testing.assert_allclose(R, np.eye(3), atol=1e-13)
    np.testing.assert_allclose(t, 0, atol=1e-13)


@pytest.mark.parametrize("seed", range(4))
def test_matches_library_svd_and_horn(orc, seed):
    rng = np.random.default_rng(seed)
    Y = rng.normal(size=(300, 3)) * rng.uniform(0.5, 3, size=3)
    D = rng.normal(size=(300, 3)) * 0.3 + Y @ (synth.random_rotation(rng, 40).T - np.eye(3))
    R, t, st = orc.kabsch(Y, D)
    Rn, tn = _kabsch_numpy(Y, D)
    Rh, th = _horn_quaternion(Y, D)
    np.testing.assert_allclose(R, Rn, atol=1e-12)
    np.testing.assert_allclose(t, tn, atol=1e-12)
    np.testing.assert_allclose(R, Rh, atol=1e-10)
    np.testing.assert_allclose(t, th, atol=1e-10)


def test_planar_template_still_fits(orc):
    rng = np.random.default_rng(5)
    Y = np.zeros((100, 3))
    Y[:, :2] = rng.normal(size=(100, 2))
    R0 = synth.random_rotation(rng, 60)
    t0 = rng.normal(size=3)
    R, t, st = orc.kabsch(Y, Y @ R0.T + t0 - Y)
    assert st == 0
    np.testing.assert_allclose(R, R0, atol=1e-10)


def test_collinear_template_is_degenerate(orc):
    s = np.linspace(-1, 1, 30)[:, None]
    Y = s * np.array([[1.0, 2.0, -0.5]])
    D = np.random.default_rng(6).normal(size=Y.shape) * 0.1
    R, t, st = orc.kabsch(Y, D)
    assert st == 1
    np.testing.assert_allclose(R, np.eye(3))
    np.testing.assert_allclose(t, D.mean(0), atol=1e-14)


def test_degenerate_bound_is_sigma2_1e7_sigma1(orc):
    # C = diag(4, 4 e^2, 0) exactly (orthogonal, centred x and y columns, D = 0):
    # sigma_2 / sigma_1 = e^2. A ratio of 1e-9 is degenerate, 1e-6 is not.
    x = np.array([1.0, -1.0, 1.0, -1.0])
    y = np.array([1.0, 1.0, -1.0, -1.0])
    for ratio, status in [(1e-9, 1), (1e-11, 1), (1e-6, 0), (1e-3, 0)]:
        Y = np.column_stack([x, np.sqrt(ratio) * y, np.zeros(4)])
        R, t, st = orc.kabsch(Y, np.zeros_like(Y))
        assert st == status, ratio
        np.testing.assert_allclose(R, np.eye(3), atol=1e-12)


# --------------------------------------------------------------------------- Appendix A

def test_normalisation_range_and_centres(orc):
    X, Y, _, _ = synth.lidar_pair(1, n=5000)
    Xn, Yn, info = orc.normalize(X, Y, -5.0, 5.0)
    allv = np.concatenate([Xn.ravel(), Yn.ravel()])
    assert allv.min() == pytest.approx(-5.0, abs=1e-12)
    assert allv.max() == pytest.approx(5.0, abs=1e-12)
    # both clouds end up with the same centroid a + s*(-l) (each is centred first)
    np.testing.assert_allclose(Xn.mean(0), Yn.mean(0), atol=1e-11)
    np.testing.assert_allclose(Xn.mean(0), -5.0 - info[7] * info[6], atol=1e-11)
    # isotropic: distances scale by s
    d0 = np.linalg.norm(X[1].astype(float) - X[0].astype(float))
    assert np.linalg.norm(Xn[1] - Xn[0]) == pytest.approx(info[7] * d0, rel=1e-12)


@pytest.mark.parametrize("seed", range(3))
def test_denormalisation_round_trip(orc, seed):
    # If [R|t] maps Y^ exactly onto X^ in the normalised frame, then
    # dnorm gives the original-frame transform: X = R Y + t_orig.
    rng = np.random.default_rng(seed)
    Y = rng.normal(size=(400, 3)) * [2, 1, 0.5] + rng.normal(size=3) * 5
    R0 = synth.random_rotation(rng, 170)
    t0 = rng.normal(size=3) * 3
    X = Y @ R0.T + t0
    Xn, Yn, info = orc.normalize(X, Y, -5.0, 5.0)
    R, tn, st = orc.kabsch(Yn, Xn - Yn)
    np.testing.assert_allclose(Yn @ R.T + tn, Xn, atol=1e-10)
    t_orig = orc.denormalize(R, tn, info, -5.0)
    np.testing.assert_allclose(R, R0, atol=1e-12)
    np.testing.assert_allclose(t_orig, t0, atol=1e-10)


def test_denormalisation_of_arbitrary_transform(orc):
    # For any normalised-frame (R, t), mapping a normalised template point and
    # undoing A.3 with the reference's statistics equals R Y + dnorm(t).
    rng = np.random.default_rng(9)
    X = rng.normal(size=(100, 3)) * 4 + 1
    Y = rng.normal(size=(80, 3)) * 2 - 3
    Xn, Yn, info = orc.normalize(X, Y, -2.0, 7.0)
    R = synth.random_rotation(rng, 90)
    t = rng.normal(size=3)
    Z = Yn @ R.T + t
    xb, l, s = info[:3], info[6], info[7]
    Z_orig = (Z - (-2.0)) / s + l + xb
    t_orig = orc.denormalize(R, t, info, -2.0)
    np.testing.assert_allclose(Z_orig, Y @ R.T + t_orig, atol=1e-11)


# --------------------------------------------------------------------------- Eq. 18

def test_niv_lattice_cloud_is_uniform(orc):
    h = 10.0 / 16
    g = (np.arange(16) + 0.5) * h - 5.0
    P = np.stack(np.meshgrid(g, g, g, indexing="ij"), -1).reshape(-1, 3)
    m = orc.masses_niv(P, 16, -5.0, 5.0, total=1.0)
    np.testing.assert_allclose(m, 1.0 / len(P), rtol=1e-12)


def test_niv_dense_patch_is_lighter(orc):
    rng = np.random.default_rng(0)
    sparse = rng.uniform(-5, 5, size=(2000, 3))
    dense = rng.uniform(0.01, 0.6, size=(3000, 3))
    P = np.concatenate([sparse, dense])
    m = orc.masses_niv(P)
    assert m[2000:].max() < m[:2000].min() * 1.0000001
    assert m.sum() == pytest.approx(1.0, rel=1e-13)


def test_niv_isolated_to_saturated_ratio(orc):
    # A ball of radius h/6 in a cube of side h covers (4/3)pi/216 = pi/162 of it;
    # an isolated point's weight over a saturated cell's is therefore 162/pi,
    # up to the oracle's stated quadrature error (3e-3).
    rng = np.random.default_rng(1)
    dense = rng.uniform(0.0, 0.6, size=(20000, 3))
    iso = np.array([[-5.0 + 0.3125, -5.0 + 0.3125, -5.0 + 0.3125]])   # a cell centre
    m = orc.masses_niv(np.concatenate([iso, dense]))
    assert m[0] / m[1] == pytest.approx(162.0 / math.pi, rel=3e-3)


def test_niv_translation_by_whole_cells(orc):
    rng = np.random.default_rng(2)
    P = rng.uniform(-4, 1, size=(3000, 3))
    h = 10.0 / 16
    m0 = orc.masses_niv(P)
    m1 = orc.masses_niv(P + 3 * h)
    np.testing.assert_allclose(m0, m1, rtol=1e-13)


def test_niv_weight_decreases_with_count(orc):
    # n points spread over a cell cover more of it as n grows, so their
    # weight falls (Eq. 18 takes the union of the balls, not their count).
    rng = np.random.default_rng(3)
    cells = []
    for k, n in enumerate([1, 2, 5, 20, 100]):
        lo = np.array([-5.0 + 0.625 * (2 * k + 1), 0.0, 0.0])
        cells.append(lo + rng.uniform(0.0, 0.625, size=(n, 3)))
    P = np.concatenate(cells)
    m = orc.masses_niv(P)
    firsts = np.cumsum([0, 1, 2, 5, 20])
    w = m[firsts]
    assert all(a > b for a, b in zip(w, w[1:]))



"""A CPU model of the GPU's lane-parallel rigid fit (Eqs. 14, 16) against the
oracle's Kabsch step.

On the GPU, the fit of one iteration spreads its 3 x 3 matrices over the
lanes of a warp, one entry per lane: lane k = 3 r + c forms entry (r, c) of
C from the 27 reduced values (the symmetric S read through a packed index),
the polar factor's FP64 Newton step takes cofactor (r, c) from the entries
(r+1, c+1), (r+2, c+2), (r+1, c+2), (r+2, c+1) (indices mod 3), a last FP64
correction against C solves a 3 x 3 system for the residual rotation, and
sums over lanes run as shuffle-down trees. This model replays those index maps and
trees with numpy on 32 simulated lanes (warp shuffles: a read of another
lane's register; a shuffle-down past lane 31 returns the lane's own value)
and checks them against closed forms and the oracle's fit, so that the
design is pinned independently of the kernel.
"""
import numpy as np
import pytest

LANES = np.arange(32)


def shfl(v, src):
    return np.full(32, v[src])


def shfl_down(v, d):
    src = LANES + d
    return np.where(src < 32, v[np.minimum(src, 31)], v)


def lane_sum9(v):
    a1 = v + shfl_down(v, 1)
    a2 = a1 + shfl_down(a1, 2)
    a3 = a2 + shfl_down(a2, 4)
    return shfl(a3 + shfl(v, 8), 0)


def entry_lanes():
    k = np.minimum(LANES, 8)
    r, c = k // 3, k % 3
    return k, r, c


def cofactor_sources():
    k, r, c = entry_lanes()
    r1, r2 = (r + 1) % 3, (r + 2) % 3
    c1, c2 = (c + 1) % 3, (c + 2) % 3
    return 3 * r1 + c1, 3 * r2 + c2, 3 * r1 + c2, 3 * r2 + c1


def sym_index():
    k, r, c = entry_lanes()
    lo, hi = np.minimum(r, c), np.maximum(r, c)
    return 6 + np.where(lo == 0, hi, np.where(lo == 1, 2 + hi, 5))


def reductions(Y, D, muf):
    """The 27 values the epilogue reduces: sum yc, sum d, S = sum yc yc^T
    (xx, xy, xz, yy, yz, zz), sum d yc^T (row-major), net force, torque (0)."""
    yc = Y - muf
    S = yc.T @ yc
    red = np.zeros(27)
    red[0:3] = yc.sum(0)
    red[3:6] = D.sum(0)
    red[6:12] = [S[0, 0], S[0, 1], S[0, 2], S[1, 1], S[1, 2], S[2, 2]]
    red[12:21] = (D.T @ yc).ravel()
    return red


def lane_C(red, M):
    k, r, c = entry_lanes()
    ybar_r, mud_r, ybar_c = red[r] / M, red[3 + r] / M, red[c] / M
    return red[sym_index()] + red[12 + k] - M * (ybar_r + mud_r) * ybar_c


def polar_lanes(ck):
    """Lane model of the polar factor: scaled Newton steps in FP32 (every lane
    the same values), one FP64 step with one entry per lane, and the
    correction against C."""
    nc2 = lane_sum9(ck * ck)[0]
    s0 = float(np.float32(1.0) / np.sqrt(np.float32(nc2)))
    Xf = (ck[:9] * s0).astype(np.float32)
    converged = False
    for _ in range(40):
        X = Xf.reshape(3, 3)
        cof = np.array([[X[(r + 1) % 3, (c + 1) % 3] * X[(r + 2) % 3, (c + 2) % 3] -
                         X[(r + 1) % 3, (c + 2) % 3] * X[(r + 2) % 3, (c + 1) % 3] for c in range(3)]
                        for r in range(3)], dtype=np.float32)
        det = np.float32(X[0] @ cof[0])
        assert det > 1e-6
        cf = (cof / det).ravel()
        xx, ii = np.float32((Xf * Xf).sum()), np.float32((cf * cf).sum())
        r4 = np.float32(1.0) / np.sqrt(ii / xx)
        g = np.float32(1.0) / np.sqrt(r4)
        xn = (np.float32(0.5) * g * Xf + np.float32(0.5) * r4 * g * cf).astype(np.float32)
        change = float(((xn - Xf) ** 2).sum())
        Xf = xn
        if change < 1e-12:
            converged = True
            break
    assert converged
    k, r, c = entry_lanes()
    x = Xf.astype(np.float64)[k]
    sa, sb, sc, sd = cofactor_sources()
    cf = x[sa] * x[sb] - x[sc] * x[sd]
    det = x[0] * cf[0] + x[1] * cf[1] + x[2] * cf[2]
    x = 0.5 * cf / det + 0.5 * x
    # the correction against C: M = Q0^T C, (tr H I - H) w = axial(M - M^T),
    # row r of Q gains q_r x w
    cs = ck * s0
    m = x[r] * cs[c] + x[3 + r] * cs[3 + c] + x[6 + r] * cs[6 + c]
    trh = m[0] + m[4] + m[8]
    A = np.where(r == c, trh, 0.0) - 0.5 * (m + m[3 * c + r])
    cfa = A[sa] * A[sb] - A[sc] * A[sd]
    deta = A[0] * cfa[0] + A[1] * cfa[1] + A[2] * cfa[2]
    ax = np.array([m[7] - m[5], m[2] - m[6], m[3] - m[1]])
    j = np.minimum(LANES, 2)
    wj = (cfa[3 * j] * ax[0] + cfa[3 * j + 1] * ax[1] + cfa[3 * j + 2] * ax[2]) / deta
    w = wj[:3]
    c1, c2 = (c + 1) % 3, (c + 2) % 3
    return x + x[3 * r + c1] * w[c2] - x[3 * r + c2] * w[c1]


@pytest.fixture(scope="module")
def orc():
    import oracle
    oracle.build()
    return oracle


def test_lane_sum9_is_the_single_thread_order():
    rng = np.random.default_rng(1)
    for _ in range(50):
        v = np.concatenate([rng.normal(size=9) * 10.0 ** rng.integers(-8, 8, 9), rng.normal(size=23)])
        want = ((v[0] + v[1]) + (v[2] + v[3])) + ((v[4] + v[5]) + (v[6] + v[7])) + v[8]
        got = lane_sum9(v)
        assert np.all(got == want)


def test_stop_test_sum_is_the_twelve_term_order():
    # lanes 0..11 hold e_q (lanes 12..31 a copy of e_11); lane 0 ends with
    # (((e0 + e1) + (e2 + e3)) + ((e4 + e5) + (e6 + e7))) + ((e8 + e9) + (e10 + e11))
    rng = np.random.default_rng(2)
    for _ in range(50):
        e = rng.exponential(size=12) * 10.0 ** rng.integers(-10, 2, 12)
        v = np.concatenate([e, np.full(20, e[11])])
        b1 = v + shfl_down(v, 1)
        b2 = b1 + shfl_down(b1, 2)
        b3 = b2 + shfl_down(b2, 4)
        d2 = b3 + shfl(b2, 8)
        want = (((e[0] + e[1]) + (e[2] + e[3])) + ((e[4] + e[5]) + (e[6] + e[7]))) + \
               ((e[8] + e[9]) + (e[10] + e[11]))
        assert d2[0] == want


def test_cyclic_cofactors_are_the_cofactor_matrix():
    rng = np.random.default_rng(3)
    for _ in range(20):
        X = rng.normal(size=(3, 3))
        a, b, c, d = cofactor_sources()
        x = X.ravel()
        cf = (x[a] * x[b] - x[c] * x[d])[:9].reshape(3, 3)
        np.testing.assert_allclose(cf, np.linalg.det(X) * np.linalg.inv(X).T, rtol=1e-12, atol=1e-12)
        np.testing.assert_allclose(x[0] * cf[0, 0] + x[1] * cf[0, 1] + x[2] * cf[0, 2], np.linalg.det(X),
                                   rtol=1e-12)


def test_packed_symmetric_index_reads_S():
    rng = np.random.default_rng(4)
    A = rng.normal(size=(3, 3))
    S = A @ A.T
    red = np.zeros(27)
    red[6:12] = [S[0, 0], S[0, 1], S[0, 2], S[1, 1], S[1, 2], S[2, 2]]
    np.testing.assert_array_equal(red[sym_index()][:9].reshape(3, 3), S)


@pytest.mark.parametrize("deg,seed", [(0.5, 5), (12.0, 6), (60.0, 7), (150.0, 8)])
def test_lane_fit_matches_the_oracle_kabsch(orc, deg, seed):
    rng = np.random.default_rng(seed)
    M = 400
    Y = rng.normal(size=(M, 3)) * [2.0, 1.0, 0.6] + [0.3, -0.2, 0.1]
    ax = rng.normal(size=3)
    ax /= np.linalg.norm(ax)
    th = np.radians(deg)
    K = np.array([[0, -ax[2], ax[1]], [ax[2], 0, -ax[0]], [-ax[1], ax[0], 0]])
    R0 = np.eye(3) + np.sin(th) * K + (1 - np.cos(th)) * K @ K
    D = (Y @ R0.T + [0.05, -0.02, 0.01] - Y) + rng.normal(size=(M, 3)) * 1e-3
    muf = Y.mean(0).astype(np.float32).astype(np.float64)  # the FP32 centre the kernels subtract
    red = reductions(Y, D, muf)
    ck = lane_C(red, M)
    mu_y, mu_d = Y.mean(0), D.mean(0)
    C_ref = (Y + D - mu_y - mu_d).T @ (Y - mu_y)
    np.testing.assert_allclose(ck[:9].reshape(3, 3), C_ref, rtol=1e-10, atol=1e-10 * np.abs(C_ref).max())
    rk = polar_lanes(ck)
    Rp = rk[:9].reshape(3, 3)
    R_orc, t_orc, st = orc.kabsch(Y, D)
    assert st == 0
    np.testing.assert_allclose(Rp, R_orc, atol=1e-12)
    muy = muf + red[0:3] / M
    tp = muy + red[3:6] / M - Rp @ muy
    np.testing.assert_allclose(tp, t_orc, atol=1e-12)

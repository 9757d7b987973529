"""Pins of the oracle's D = 2 path (clouds in the plane z = 0).

The paper states FGA for general D (2^D children, discs in the NIV measure).
Fixed by the mathematics: the 2-D orthogonal Procrustes optimum is the
rotation by atan2(c21 - c12, c11 + c22), also obtained from an SVD with the
determinant correction; a planar cloud's tree has at most 4 children per
cell; an isolated point's NIV weight is 16/pi times a saturated cell's (disc
of radius h/4 in a cell of side h); and the loop recovers a known planar
motion.
"""
import math

import numpy as np
import pytest


def rot2(deg):
    c, s = math.cos(math.radians(deg)), math.sin(math.radians(deg))
    return np.array([[c, -s], [s, c]])


def cov2(Y, D):
    Yc = Y[:, :2] - Y[:, :2].mean(0)
    Zc = (Y + D)[:, :2] - (Y + D)[:, :2].mean(0)
    return Zc.T @ Yc


def test_fit_is_the_closed_form_and_the_svd_solution(orc):
    rng = np.random.default_rng(0)
    for _ in range(20):
        Y = np.column_stack([rng.normal(size=(50, 2)), np.zeros(50)])
        D = np.column_stack([rng.normal(size=(50, 2)), np.zeros(50)])
        R, t, st = orc.kabsch(Y, D, dim=2)
        C = cov2(Y, D)
        th = math.atan2(C[1, 0] - C[0, 1], C[0, 0] + C[1, 1])
        np.testing.assert_allclose(R[:2, :2], rot2(math.degrees(th)), atol=1e-12)
        U, s, Vt = np.linalg.svd(C)
        Rs = U @ np.diag([1.0, np.sign(np.linalg.det(U @ Vt))]) @ Vt
        np.testing.assert_allclose(R[:2, :2], Rs, atol=1e-12)
        assert R[2, 2] == 1.0 and R[0, 2] == R[2, 0] == 0.0 and st == 0


def test_fit_recovers_a_planar_motion(orc):
    rng = np.random.default_rng(1)
    Y = np.column_stack([rng.normal(size=(80, 2)), np.zeros(80)])
    R0 = np.eye(3)
    R0[:2, :2] = rot2(33.0)
    t0 = np.array([0.3, -0.7, 0.0])
    D = Y @ R0.T + t0 - Y
    R, t, st = orc.kabsch(Y, D, dim=2)
    np.testing.assert_allclose(R, R0, atol=1e-12)
    np.testing.assert_allclose(t, t0, atol=1e-12)


def test_reflected_target_gives_a_rotation_and_symmetric_case_is_degenerate(orc):
    rng = np.random.default_rng(2)
    Y = np.column_stack([rng.normal(size=(40, 2)) * [3.0, 1.0], np.zeros(40)])
    F = np.diag([1.0, -1.0, 1.0])
    R, t, st = orc.kabsch(Y, Y @ F.T - Y, dim=2)
    assert abs(np.linalg.det(R) - 1.0) < 1e-12 and st == 0
    # a square's vertices and their mirror image: every rotation fits equally
    Q = np.array([[1.0, 0, 0], [0, 1.0, 0], [-1.0, 0, 0], [0, -1.0, 0]])
    R, t, st = orc.kabsch(Q, Q @ F.T - Q, dim=2)
    assert st == 1
    np.testing.assert_array_equal(R, np.eye(3))


def test_niv_2d_ratio_and_regular_lattice(orc):
    # lattice 4 over [-5, 5]^2: cells of side 2.5; one cell saturated, one isolated point
    h = 2.5
    dense = np.column_stack([np.random.default_rng(3).uniform(-4.9, -2.6, size=(20000, 2)),
                             np.zeros(20000)])
    iso = np.array([[4.0, 4.0, 0.0]])
    m = orc.masses_niv(np.vstack([dense, iso]), lattice=4, dim=2, total=1.0)
    # weights 1 / f: the dense cell is covered (f = 1), the isolated disc of
    # radius h/4 covers pi/16 of its cell (within the 2-D quadrature bound 1.1e-4)
    assert m[-1] / m[0] == pytest.approx(16.0 / math.pi, rel=1.1e-4)
    # a regular planar grid, one point per cell: equal masses
    g = np.linspace(-4.375, 4.375, 8)
    P = np.array([[x, y, 0.0] for x in g for y in g])
    mg = orc.masses_niv(P, lattice=8, dim=2)
    np.testing.assert_allclose(mg, mg[0], rtol=1e-12)


def test_planar_tree_is_a_quadtree(orc):
    P = np.column_stack([np.random.default_rng(4).uniform(-3, 3, size=(3000, 2)), np.zeros(3000)])
    e = orc.Tree(P, np.full(3000, 1.0 / 3000)).export()
    parent = np.asarray(e["parent"])
    counts = np.bincount(parent[parent >= 0], minlength=len(parent))
    assert counts.max() <= 4 and counts.max() == 4


def test_loop_recovers_a_planar_motion(orc):
    # an asymmetric planar shape (an L of two rectangles) under a known motion
    rng = np.random.default_rng(5)
    A = np.column_stack([rng.uniform(0, 3, 600), rng.uniform(0, 0.8, 600)])
    B = np.column_stack([rng.uniform(0, 0.8, 400), rng.uniform(0.8, 2.0, 400)])
    X = np.vstack([A, B])
    R0 = rot2(20.0)
    t0 = np.array([0.2, -0.1])
    Y = (X - t0) @ R0  # X = R0 Y + t0
    o = orc.register_full(X, Y, orc.Params(method=orc.FGA_DIRECT, dim=2, max_iter=300), round_to_f32=False)
    err = math.degrees(math.acos(np.clip((np.trace(o["R2"].T @ R0)) / 2.0, -1, 1)))
    assert err < 0.1
    assert np.linalg.norm(o["t2"] - t0) < 1e-2
    assert abs(o["R"][2, 2] - 1.0) < 1e-12

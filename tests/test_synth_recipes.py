"""The seeded input generators produce the workloads the design states
(sizes, noise, motion bounds, densities, arrival statistics) and are
deterministic per seed. They hold none of the method's arithmetic."""
import math

import numpy as np
import pytest

import synth


def _angle_deg(R):
    return math.degrees(math.acos(float(np.clip((np.trace(R) - 1.0) / 2.0, -1.0, 1.0))))


def _is_rotation(R):
    return np.allclose(R @ R.T, np.eye(len(R)), atol=1e-12) and abs(np.linalg.det(R) - 1.0) < 1e-12


@pytest.mark.parametrize("seed", range(6))
def test_sphere_pair(seed):
    X, Y, R, t = synth.sphere_pair(seed, n=1000, m=700)
    assert X.shape == (1000, 3) and Y.shape == (700, 3) and X.dtype == np.float32
    r = np.linalg.norm(X.astype(np.float64), axis=1)
    assert abs(r.mean() - 1.0) < 5e-3 and r.std() < 0.02  # unit sphere, sigma 0.01 noise
    assert _is_rotation(R) and 0.0 < _angle_deg(R) <= 45.0 + 1e-9
    assert np.linalg.norm(t) <= 0.2 + 1e-12
    # the template is the moved copy of the first 700 base points (noise on both)
    resid = np.linalg.norm(Y.astype(np.float64) @ R.T + t - X[:700], axis=1)
    assert np.median(resid) < 0.03


def test_box_pair_is_an_exact_copy():
    X, Y, R, t = synth.box_pair(0, n=500, deg=15.0)
    assert _is_rotation(R) and abs(_angle_deg(R) - 15.0) < 1e-9
    np.testing.assert_allclose(Y.astype(np.float64) @ R.T + t, X, atol=1e-6)
    assert np.all(np.abs(X) <= np.array([1.0, 0.6, 0.3]) + 1e-6)


def test_lidar_pair():
    X, Y, R, t = synth.lidar_pair(3, n=20000, m=15000)
    assert X.shape == (20000, 3) and Y.shape == (15000, 3)
    # second pose: yaw <= 10 deg, roll/pitch <= 1 deg, 1-3 m horizontal translation
    assert _is_rotation(R) and _angle_deg(R) <= math.hypot(10.0, 1.0, 1.0) + 1e-6
    assert 1.0 <= np.linalg.norm(t[:2]) <= 3.0 and t[2] == 0.0
    for P in (X, Y):
        r = np.linalg.norm(P.astype(np.float64), axis=1)
        assert r.max() <= 80.0 + 0.2  # ray casting to 80 m (plus noise)
        # the ground plane at -1.7 m holds a large share of the returns
        assert np.mean(np.abs(P[:, 2] + 1.7) < 0.1) > 0.3
        # constant angular sampling: density falls off with range
        near = np.mean(r < 10.0)
        far = np.mean((r >= 30.0) & (r < 40.0))
        assert near > far
    # every ray within the -25..+2 deg elevation fan (before noise)
    elev = np.degrees(np.arctan2(X[:, 2], np.linalg.norm(X[:, :2], axis=1)))
    assert np.quantile(elev, 0.001) > -27.0 and np.quantile(elev, 0.999) < 4.0


def test_planar_scene_pair():
    X, Y, R, t = synth.planar_scene_pair(2, n=40000, m=30000)
    assert X.shape == (40000, 3) and Y.shape == (30000, 3)
    assert _is_rotation(R) and _angle_deg(R) <= 30.0 + 1e-9 and np.linalg.norm(t) <= 0.2 + 1e-12
    # independent samples of the same scene: every template point lies near
    # some reference point once moved back, except for the 5 % outliers
    Yw = Y.astype(np.float64) @ R.T + t
    sub = Yw[:2000]
    d = np.sqrt(((sub[:, None, :] - X[None, :4000, :].astype(np.float64)) ** 2).sum(-1)).min(1)
    assert np.mean(d < 0.1) > 0.85


def test_batch_sizes_are_log_uniform():
    s = synth.batch_sizes(1000, count=4096, lo=500, hi=50_000)
    assert s.min() >= 500 and s.max() <= 50_000
    # log-uniform: the log-sizes are uniform on [ln 500, ln 50000]
    u = (np.log(s) - math.log(500)) / (math.log(50_000) - math.log(500))
    assert abs(u.mean() - 0.5) < 0.02 and abs(u.var() - 1 / 12) < 0.01
    assert np.array_equal(s, synth.batch_sizes(1000, count=4096))


def test_batch_pairs_alternate_shapes_and_bounds():
    pairs = synth.batch_pairs(7, count=6, lo=500, hi=2000)
    sizes = synth.batch_sizes(7, count=6, lo=500, hi=2000)
    for k, (X, Y, R, t) in enumerate(pairs):
        assert (len(X), len(Y)) == tuple(sizes[k])
        assert _angle_deg(R) <= 60.0 + 1e-9 and np.linalg.norm(t) <= 0.3 + 1e-12
        r = np.linalg.norm(X.astype(np.float64), axis=1)
        on_sphere = abs(r.mean() - 1.0) < 0.01 and r.std() < 0.03
        assert on_sphere == (k % 2 == 0)


@pytest.mark.parametrize("overlap", [0.3, 0.6, 1.0])
def test_cropped_scene_pair_overlap(overlap):
    X, Y, R, t = synth.cropped_scene_pair(5, 6000, 5000, overlap)
    assert X.shape == (6000, 3) and Y.shape == (5000, 3)
    Yw = Y.astype(np.float64) @ R.T + t  # back in the scene frame
    # the two views are windows along one axis: the one their centres differ on
    axis = int(np.argmax(np.abs(np.median(X, 0) - np.median(Yw, 0))))
    xl, xh = np.quantile(X[:, axis], [0.02, 0.98])
    yl, yh = np.quantile(Yw[:, axis], [0.02, 0.98])
    shared = (min(xh, yh) - max(xl, yl)) / (xh - xl)
    assert abs(shared - overlap) < 0.1, (axis, shared)


def test_serve_trace_arrivals_and_sizes():
    tr = synth.serve_trace(11, 400, rate=200.0, lo=1000, hi=4000)
    times = np.array([e[0] for e in tr])
    assert times[0] == 0.0 and np.all(np.diff(times) >= 0)
    gaps = np.diff(times)
    assert abs(gaps.mean() - 1 / 200.0) < 0.15 / 200.0  # exponential gaps at the rate
    assert abs(gaps.std() / gaps.mean() - 1.0) < 0.15   # coefficient of variation 1
    for _, X, Y, R, t in tr[:20]:
        assert 1000 <= len(X) <= 4000 and 1000 <= len(Y) <= 4000
    # deterministic per (seed, count): all gaps are drawn before the sizes
    again = synth.serve_trace(11, 400, rate=200.0, lo=1000, hi=4000)
    for a, b in zip(tr[:5], again[:5]):
        assert a[0] == b[0] and np.array_equal(a[1], b[1]) and np.array_equal(a[2], b[2])


def test_plane_pair():
    X, Y, R, t = synth.plane_pair(4, n=3000)
    assert X.shape == (3000, 2) and Y.shape == (3000, 2) and R.shape == (2, 2)
    assert _is_rotation(R) and math.degrees(abs(math.atan2(R[1, 0], R[0, 0]))) <= 30.0 + 1e-9
    assert np.linalg.norm(t) <= 0.2 + 1e-12


@pytest.mark.parametrize("gen", [synth.sphere_pair, synth.planar_scene_pair])
def test_same_seed_same_arrays(gen):
    a = gen(9, n=2000, m=1500)
    b = gen(9, n=2000, m=1500)
    c = gen(10, n=2000, m=1500)
    assert all(np.array_equal(x, y) for x, y in zip(a, b))
    assert not np.array_equal(a[0], c[0])

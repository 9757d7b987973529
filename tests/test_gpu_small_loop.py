"""Small all-pairs pairs: the whole iteration loop in one cluster launch.

A pair with N <= 4096 reference points, M <= 16384 template points and
N * M <= 2^20 runs every iteration of Algorithm 2 (Eq. 6, Eqs. 7-10, Eq. 14,
Eq. 16, composition and stop test) in one launch of one thread-block cluster.
That launch computes the same tiles, partial sums, block partials and rigid
fit as the separate force and epilogue launches, which fga_params.profile = 1
still takes, so the two must agree bit for bit; the oracle tests of the
all-pairs registrations (test_gpu_parity.py) run through the cluster launch.
"""
import numpy as np
import pytest

import synth

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


def _cuda(a):
    import torch
    return torch.as_tensor(np.ascontiguousarray(a, dtype=np.float32), device="cuda")


def _copy(fga, p, **kw):
    q = fga.params(**{k: getattr(p, k) for k, _ in p._fields_})
    for k, v in kw.items():
        setattr(q, k, v)
    return q


def _both(fga, X, Y, p):
    """(one-launch result, launches), (separate-launch result, launches)."""
    out = []
    for prof in (0, 1):
        before = fga.fga_launch_count()
        R, t, st = fga.fga_register(_cuda(X), _cuda(Y), _copy(fga, p, profile=prof))
        out.append(((R, t, st), fga.fga_launch_count() - before))
    return out


def _assert_same(a, b):
    (R1, t1, s1), (R2, t2, s2) = a, b
    np.testing.assert_array_equal(R1, R2)
    np.testing.assert_array_equal(t1, t2)
    for k in ("iterations", "converged", "degenerate_fits", "interactions", "status"):
        assert s1[k] == s2[k], (k, s1[k], s2[k])
    np.testing.assert_array_equal(s1["R_norm"], s2["R_norm"])
    np.testing.assert_array_equal(s1["net_force"], s2["net_force"])
    np.testing.assert_array_equal(s1["torque"], s2["torque"])


def _cloud(seed, n, scale=1.0):
    rng = np.random.default_rng(seed)
    return (rng.normal(size=(n, 3)) * scale).astype(np.float32)


CASES = {
    # the 1k x 1k sphere workload
    "sphere-1k": (lambda: synth.sphere_pair(3)[:2], dict(eps=0.05, eta=0.1, max_iter=100)),
    # ragged sizes: partial template blocks and source tiles
    "ragged": (lambda: (_cloud(1, 1500), _cloud(2, 555)), dict(max_iter=40)),
    # the largest reference (sources staged in shared memory)
    "max-n": (lambda: (_cloud(3, 4096), _cloud(4, 256)), dict(max_iter=20)),
    # the largest template (64 epilogue blocks), N * M = 2^20
    "max-m": (lambda: (_cloud(5, 64), _cloud(6, 16384)), dict(max_iter=20)),
    # one template point: every rigid fit is degenerate
    "one-point": (lambda: (_cloud(7, 50), _cloud(8, 1)), dict(max_iter=10)),
    "rigid-velocity": (lambda: synth.box_pair(9, 700, 20.0)[:2], dict(max_iter=60, velocity_mode=1)),
    "early-stop": (lambda: synth.box_pair(10, 600, 10.0)[:2], dict(max_iter=300, conv_tol=1e-6)),
}


@pytest.mark.parametrize("name", list(CASES))
def test_one_launch_equals_separate_launches(fga, name):
    make, kw = CASES[name]
    X, Y = make()
    p = fga.params(method=fga.FGA_DIRECT, **kw)
    (a, na), (b, nb) = _both(fga, X, Y, p)
    _assert_same(a, b)
    # the one-launch path ran: far fewer launches than two per iteration
    assert nb >= 2 * b[2]["iterations"]
    assert na < 30, na
    if name == "early-stop":
        assert a[2]["converged"] and a[2]["iterations"] < 300


def test_planar_pair_in_one_launch(fga):
    X, Y, _, _ = synth.box_pair(11, 900, 25.0)
    X2 = np.ascontiguousarray(X[:, :2])
    Y2 = np.ascontiguousarray(Y[:, :2])
    p = fga.params(method=fga.FGA_DIRECT, max_iter=50, dim=2)
    (a, na), (b, _) = _both(fga, X2, Y2, p)
    _assert_same(a, b)
    assert na < 30


@pytest.mark.parametrize("bs,qpt", [(128, 1), (128, 2), (128, 4), (256, 1), (256, 2), (256, 4)])
def test_every_tile_shape(fga, bs, qpt):
    old = fga.get_direct_tile(0)
    try:
        fga.set_direct_tile(0, bs, qpt)
        X, Y = _cloud(20 + bs + qpt, 1100), _cloud(30 + bs + qpt, 900)
        p = fga.params(method=fga.FGA_DIRECT, max_iter=15)
        (a, na), (b, _) = _both(fga, X, Y, p)
        _assert_same(a, b)
        assert na < 30
    finally:
        fga.set_direct_tile(0, *old)


def test_chunked_steps_and_trajectory(fga):
    X, Y, _, _ = synth.box_pair(12, 800, 20.0)
    Xn, Yn, _ = fga.fga_normalize(_cuda(X), _cuda(Y))
    p = fga.params(method=fga.FGA_DIRECT, max_iter=40)
    runs = []
    for prof, chunks in ((0, [40]), (0, [1, 2, 3, 34]), (1, [40])):
        s = fga.fga_state_create(Xn, None, Yn, None, _copy(fga, p, profile=prof))
        for c in chunks:
            s.step(c)
        R, t, st = s.get()
        runs.append((R, t, s.trajectory(40)))
        s.close()
    for R, t, tr in runs[1:]:
        np.testing.assert_array_equal(R, runs[0][0])
        np.testing.assert_array_equal(t, runs[0][1])
        np.testing.assert_array_equal(tr, runs[0][2])
    assert runs[0][2].shape == (40, 12)


def test_pairs_beyond_the_limits_take_separate_launches(fga):
    # N = 4097 (sources no longer staged) and N * M > 2^20
    for N, M in [(4097, 64), (2048, 600)]:
        X, Y = _cloud(40 + N, N), _cloud(41 + M, M)
        p = fga.params(method=fga.FGA_DIRECT, max_iter=12)
        before = fga.fga_launch_count()
        fga.fga_register(_cuda(X), _cuda(Y), p)
        assert fga.fga_launch_count() - before >= 24

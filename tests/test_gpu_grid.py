"""Per-pair parameters: theta sweeps and G / eps / eta grids as one batch.

A pair's result in a batch depends only on its own inputs and parameters, so
every cell of a grid must equal the same pair registered alone with that
cell's parameters (batch of one: bit for bit; the one-pair path and the
oracle: within the registration tolerance of 0.01 deg, 1e-4 x bbox diagonal).
Cells over the same clouds share one preparation (same arrays, same
normalisation, masses, dt and method), which must not change any result.
"""
import itertools

import numpy as np
import pytest

import synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def fga():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    import __graft_entry__
    __graft_entry__.build_library()
    import paper_2009_14005_gb300 as f
    return f


def _cuda(a):
    import torch
    return torch.as_tensor(np.ascontiguousarray(a, dtype=np.float32), device="cuda")


def rot_err_deg(Ra, Rb):
    c = (np.trace(Ra.T @ Rb) - 1.0) / 2.0
    return float(np.degrees(np.arccos(np.clip(c, -1.0, 1.0))))


def test_theta_sweep_batch(fga):
    X, Y, _, _ = synth.planar_scene_pair(31, n=6000, m=4000)
    Xd, Yd = _cuda(X), _cuda(Y)
    thetas = [0.0, 0.3, 0.5, 0.7, 0.9]
    cells = [fga.params(method=fga.FGA_BH, theta=th, max_iter=30) for th in thetas]
    res, st = fga.fga_register_batch([(Xd, Yd, None, None, c) for c in cells], fga.params())
    counts = [r["interactions"] for r in res]
    # a smaller opening angle opens more cells
    assert all(a >= b for a, b in zip(counts, counts[1:])) and counts[0] > counts[-1]
    diag = float(np.linalg.norm(X.max(0) - X.min(0)))
    for r, c in zip(res, cells):
        alone = fga.fga_register_batch([(Xd, Yd)], c)[0][0]
        assert np.array_equal(r["R"], alone["R"]) and np.array_equal(r["t"], alone["t"])
        assert r["interactions"] == alone["interactions"] and r["iterations"] == 30
        R1, t1, st1 = fga.fga_register(Xd, Yd, c)
        assert rot_err_deg(r["R"], R1) <= 0.01
        assert np.linalg.norm(r["t"] - t1) <= 1e-4 * diag


def test_g_eps_eta_grid_matches_alone_and_oracle(fga, orc):
    X, Y, R_gt, t_gt = synth.sphere_pair(0)  # the 1k x 1k unit-sphere pair
    Xd, Yd = _cuda(X), _cuda(Y)
    grid = list(itertools.product([10.0, 66.7, 200.0], [0.05, 0.2], [0.1, 0.3]))
    cells = [fga.params(method=fga.FGA_DIRECT, G=G, eps=e, eta=h, max_iter=100) for G, e, h in grid]
    res, st = fga.fga_register_batch([(Xd, Yd, None, None, c) for c in cells], fga.params())
    assert st["interactions"] == len(cells) * 100 * 1000 * 1000
    diag = float(np.linalg.norm(X.max(0) - X.min(0)))
    import oracle
    for k, (r, c) in enumerate(zip(res, cells)):
        alone = fga.fga_register_batch([(Xd, Yd)], c)[0][0]
        assert np.array_equal(r["R"], alone["R"]) and np.array_equal(r["t"], alone["t"]), grid[k]
        # oracle on cells spanning the grid (G = 200 only with the larger eps:
        # with eps = 0.05 that cell's dynamics are too stiff to compare FP32
        # with FP64 trajectories)
        if k in (0, 3, 6, 11):
            G, e, h = grid[k]
            o = orc.register_full(X, Y, orc.Params(method=orc.FGA_DIRECT, G=G, eps=e, eta=h, max_iter=100))
            assert oracle.rotation_error_deg(r["R"], o["R"]) <= 0.01, grid[k]
            assert np.linalg.norm(r["t"] - o["t"]) <= 1e-4 * diag, grid[k]


def test_own_iteration_limits_and_zero_iterations(fga):
    X, Y, _, _ = synth.sphere_pair(3, n=800, m=700)
    Xd, Yd = _cuda(X), _cuda(Y)
    lim = [0, 1, 7, 25]
    cells = [fga.params(method=fga.FGA_DIRECT, max_iter=n) for n in lim]
    res, st = fga.fga_register_batch([(Xd, Yd, None, None, c) for c in cells], fga.params(max_iter=3))
    assert st["iterations"] == 25
    for r, c, n in zip(res, cells, lim):
        assert r["iterations"] == n and not r["converged"]
        assert r["interactions"] == n * 800 * 700
        if n == 0:
            np.testing.assert_array_equal(r["R"], np.eye(3))
        else:
            alone = fga.fga_register_batch([(Xd, Yd)], c)[0][0]
            assert np.array_equal(r["R"], alone["R"])


def test_bad_cell_parameters_name_the_pair(fga):
    X, Y, _, _ = synth.sphere_pair(4, n=300, m=300)
    bad = fga.params(eps=0.0)
    with pytest.raises(fga.FGAError) as e:
        fga.fga_register_batch([(X, Y), (X, Y, None, None, bad)], fga.params(max_iter=5))
    assert "pair 1" in str(e.value)


def test_server_requests_with_own_parameters(fga):
    X, Y, _, _ = synth.sphere_pair(5, n=900, m=900)
    Xd, Yd = _cuda(X), _cuda(Y)
    cells = [fga.params(method=fga.FGA_DIRECT, G=G, max_iter=20) for G in (5.0, 30.0, 66.7)]
    with fga.Server(fga.params(method=fga.FGA_DIRECT, max_iter=10), iters_per_tick=3) as srv:
        tickets = {srv.submit(Xd, Yd, params=c): k for k, c in enumerate(cells)}
        got = srv.drain()
    for r in got:
        c = cells[tickets[r["ticket"]]]
        alone = fga.fga_register_batch([(Xd, Yd)], c)[0][0]
        assert r["iterations"] == 20
        assert np.array_equal(r["R"], alone["R"]) and np.array_equal(r["t"], alone["t"])

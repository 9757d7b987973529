"""Pins of the oracle's Algorithm 2 loop against what the method must do."""
import os

import numpy as np
import pytest

import synth

GOLD = os.path.join(os.path.dirname(__file__), "golden", "paper_parameters.txt")


def _paper_params():
    out = {}
    for ln in open(GOLD):
        ln = ln.strip()
        if ln and not ln.startswith("#"):
            k, v = ln.split()
            out[k] = float(v)
    return out


def test_default_parameters_are_the_papers(orc):
    gold = _paper_params()
    p = orc.Params()
    for k in ["G", "eps", "dt", "eta", "theta", "a", "b", "max_depth", "lattice"]:
        assert getattr(p, k) == gold[k], k


def test_aligned_identical_sets_are_a_fixed_point(orc):
    # Identical, aligned clouds: the net force and torque vanish pairwise
    # (Newton's third law), so the rigid fit never moves.
    rng = np.random.default_rng(0)
    X = rng.uniform(-1, 1, size=(300, 3)) * [1, 0.6, 0.3]
    p = orc.Params(max_iter=40)
    for vm in [orc.VEL_UNCONSTRAINED, orc.VEL_RIGID]:
        p.velocity_mode = vm
        o = orc.register_full(X, X.copy(), p, round_to_f32=False)
        np.testing.assert_allclose(o["R"], np.eye(3), atol=1e-10)
        np.testing.assert_allclose(o["t"], 0, atol=1e-10)


@pytest.mark.parametrize("vm", [0, 1])
@pytest.mark.parametrize("seed", [0, 1, 2])
def test_recovers_known_motion_noise_free(orc, vm, seed):
    X, Y, R_gt, t_gt = synth.box_pair(seed, 500, 15.0)
    p = orc.Params(max_iter=150, velocity_mode=vm)
    o = orc.register_full(X, Y, p)
    diag = np.linalg.norm(X.max(0) - X.min(0))
    assert orc.rotation_error_deg(o["R"], R_gt) < 0.01
    assert np.linalg.norm(o["t"] - t_gt) < 1e-4 * diag


def test_recovers_translation_only(orc):
    X, Y, _, _ = synth.box_pair(3, 400, 0.0, t=(0.3, -0.2, 0.1))
    o = orc.register_full(X, Y, orc.Params(max_iter=150))
    np.testing.assert_allclose(o["R"], np.eye(3), atol=1e-6)
    np.testing.assert_allclose(o["t"], [0.3, -0.2, 0.1], atol=1e-5)


def test_barnes_hut_loop_tracks_direct_loop(orc):
    X, Y, R_gt, t_gt = synth.box_pair(4, 600, 10.0)
    p = orc.Params(max_iter=60)
    d = orc.register_full(X, Y, p, want_traj=True)
    p.method = orc.FGA_BH
    p.theta = 0.1
    b = orc.register_full(X, Y, p, want_traj=True)
    dphi = max(orc.rotation_error_deg(d["traj"][k, :9].reshape(3, 3), b["traj"][k, :9].reshape(3, 3))
               for k in range(60))
    assert dphi < 0.05
    assert b["interactions"] < d["interactions"]


def test_stopping_rule(orc):
    # Reading of Algorithm 2's loop condition: stop at the first k >= 2 with
    # |T_k - T_{k-2}|_F^2 <= tol.
    X, Y, _, _ = synth.box_pair(5, 400, 10.0)
    p = orc.Params(max_iter=300, conv_tol=1e-6)
    o = orc.register_full(X, Y, p, want_traj=True)
    tr = o["traj"]
    k = o["iters"]
    assert 3 <= k < 300
    d = [np.sum((tr[j] - tr[j - 2]) ** 2) for j in range(2, k)]
    assert d[-1] <= 1e-6
    assert all(v > 1e-6 for v in d[:-1])
    p.conv_tol = 0.0
    p.max_iter = 37
    assert orc.register_full(X, Y, p)["iters"] == 37


def test_rigid_velocity_mode_stores_the_rigid_motion(orc):
    X, Y, _, _ = synth.box_pair(6, 200, 20.0)
    Xn, Yn, info = orc.normalize(X, Y)
    mX, mY = orc.default_masses(Xn, Yn, orc.Params())
    p = orc.Params(max_iter=5, velocity_mode=orc.VEL_RIGID)
    o = orc.register(Xn, mX, Yn, mY, p, want_traj=True, want_v=True)
    T4, T5 = o["traj"][3], o["traj"][4]
    R4, t4, R5, t5 = T4[:9].reshape(3, 3), T4[9:], T5[:9].reshape(3, 3), T5[9:]
    Y4 = Yn @ R4.T + t4
    Y5 = Yn @ R5.T + t5
    np.testing.assert_allclose(o["V"], (Y5 - Y4) / p.dt, atol=1e-10)


def test_unconstrained_velocity_persists(orc):
    # In the literal mode the stored velocity is Eq. 9's, not the rigid one.
    X, Y, _, _ = synth.box_pair(6, 200, 20.0)
    Xn, Yn, info = orc.normalize(X, Y)
    mX, mY = orc.default_masses(Xn, Yn, orc.Params())
    p = orc.Params(max_iter=1)
    o = orc.register(Xn, mX, Yn, mY, p, want_v=True)
    a = orc.direct_acc(Xn, mX, Yn, p.G, p.eps)
    v, d = orc.ode_step(np.zeros_like(Yn), a, mY, p.dt, p.eta)
    np.testing.assert_allclose(o["V"], v, rtol=1e-12)
    R, t, _ = orc.kabsch(Yn, d)
    np.testing.assert_allclose(o["R"], R, atol=1e-14)


def test_damping_reading_dissipates_eta_per_step(orc):
    # Template masses have mean dt, so a unit-weight particle loses exactly the
    # fraction eta of its velocity per step when no gravity acts.
    p = orc.Params()
    Xn = np.zeros((4, 3))
    Yn = np.ones((10, 3))
    mX, mY = orc.default_masses(Xn, Yn, p)
    v = np.ones((10, 3))
    v2, _ = orc.ode_step(v, np.zeros_like(v), mY, p.dt, p.eta)
    np.testing.assert_allclose(v2, (1 - p.eta) * v, rtol=1e-14)
    assert mX.sum() == pytest.approx(1.0)

"""Parity at the benchmark's full size (two 120k-point LiDAR sweeps, BH theta 0.5).

The whole 200-iteration trajectory is too long for the oracle here, so the
full-size checks are: normalisation, NIV masses and the complete tree
(bit-exact structure) on the full pair; BHForce on a sample of template
points; and one iteration of the loop against the oracle's first iteration.
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


@pytest.fixture(scope="module")
def pair(orc):
    X, Y, _, _ = synth.lidar_pair(1000, n=120_000)  # the benchmark's first pair
    Xn, Yn, info = orc.normalize(X, Y)
    Xn = Xn.astype(np.float32).astype(np.float64)
    Yn = Yn.astype(np.float32).astype(np.float64)
    mX = orc.masses_niv(Xn).astype(np.float32).astype(np.float64)
    return X, Y, Xn, Yn, mX


def _cuda(a):
    import torch
    return torch.as_tensor(np.ascontiguousarray(a, dtype=np.float32), device="cuda")


def test_fullsize_normalise_masses_tree(fga, orc, pair):
    X, Y, Xn, Yn, mX = pair
    Xg, Yg, info = fga.fga_normalize(_cuda(X), _cuda(Y))
    np.testing.assert_allclose(Xg.cpu().numpy(), Xn, atol=1e-6, rtol=0)
    m = fga.fga_masses(_cuda(Xn), fga.FGA_MASS_NIV).cpu().numpy()
    np.testing.assert_allclose(m, mX, rtol=1e-6)
    eo = orc.Tree(Xn, mX).export()
    eg = fga.fga_tree_build(_cuda(Xn), _cuda(mX), fga.params()).export()
    assert len(eg["depth"]) == len(eo["depth"])
    for k in ["depth", "cell", "npts", "is_leaf", "parent", "leaf_of"]:
        np.testing.assert_array_equal(eg[k], eo[k], err_msg=k)
    np.testing.assert_allclose(eg["mass"], eo["mass"], rtol=2e-7, atol=1e-12)


def test_fullsize_bh_forces_on_sample(fga, orc, pair):
    X, Y, Xn, Yn, mX = pair
    p = fga.params(theta=0.5)
    t = fga.fga_tree_build(_cuda(Xn), _cuda(mX), p)
    a, cnt = fga.fga_forces(t, None, None, _cuda(Yn), None, p, want_count=True)
    a = a.cpu().numpy().astype(np.float64)
    _, terms = fga.fga_forces_terms(t, _cuda(Yn), None, p)
    idx = np.random.default_rng(0).choice(len(Yn), 600, replace=False)
    terms = terms.cpu().numpy()[idx]
    tree_o = orc.Tree(Xn, mX)
    a_bo, c_o = tree_o.bh_acc(Yn[idx], p.G, 0.2, 0.5)
    a_d = orc.direct_acc(Xn, mX, Yn[idx], p.G, 0.2)
    err_gpu = np.linalg.norm(a[idx] - a_d) / np.linalg.norm(a_d)
    err_orc = np.linalg.norm(a_bo - a_d) / np.linalg.norm(a_d)
    assert err_gpu <= err_orc + 1e-5
    # a point away from the oracle's force took other terms (an FP32/FP64 tie)
    close = np.linalg.norm(a[idx] - a_bo, axis=1) <= 1e-4 * np.linalg.norm(a_bo, axis=1) + 1e-6
    assert np.all(close | (terms != c_o))
    assert close.mean() > 0.99
    # mean terms per point over the sample vs the device count over all points
    assert abs(cnt / len(Yn) - c_o.mean()) < 0.1 * c_o.mean()


def test_fullsize_first_iteration(fga, orc, pair):
    X, Y, Xn, Yn, mX = pair
    mY = np.full(len(Yn), np.float32(0.1)).astype(np.float64)
    po = orc.Params(method=orc.FGA_BH, theta=0.5, max_iter=1)
    o = orc.register(Xn, mX, Yn, mY, po)
    p = fga.params(method=fga.FGA_BH, theta=0.5, max_iter=1)
    s = fga.fga_state_create(_cuda(Xn), _cuda(mX), _cuda(Yn), _cuda(mY), p)
    s.step(1)
    R, t, st = s.get()
    import oracle
    assert oracle.rotation_error_deg(R, o["R"]) < 1e-3
    np.testing.assert_allclose(t, o["t"], atol=1e-6)
    assert abs(st["interactions"] - o["interactions"]) <= 1e-3 * o["interactions"]


def test_fullsize_registration_matches_oracle(fga, orc, pair):
    # the benchmark's configuration end to end: 120k x 120k, NIV masses,
    # Barnes-Hut theta 0.5, G = 1, 200 iterations; the oracle runs the same
    # loop in FP64 (with G = 66.7 this trajectory is chaotic: a 1e-7
    # perturbation of the input grows to tens of degrees, so no FP32 run can
    # follow the FP64 one)
    X, Y, Xn, Yn, mX = pair
    po = orc.Params(method=orc.FGA_BH, theta=0.5, max_iter=200, niv_masses=True, G=1.0)
    o = orc.register_full(X, Y, po)
    p = fga.params(method=fga.FGA_BH, theta=0.5, max_iter=200, mass_mode=fga.FGA_MASS_NIV, G=1.0)
    R, t, st = fga.fga_register(_cuda(X), _cuda(Y), p)
    import oracle
    diag = np.linalg.norm(X.max(0) - X.min(0))
    assert oracle.rotation_error_deg(R, o["R"]) <= 0.01
    assert np.linalg.norm(t - o["t"]) <= 1e-4 * diag
    assert abs(st["interactions"] - o["interactions"]) <= 1e-3 * o["interactions"]

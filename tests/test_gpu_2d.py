"""The D = 2 path on the GPU (planar clouds, quadtree, 2-D NIV, 2 x 2 fit)
against the oracle's D = 2 path."""
import math

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


def err2(R2, Rref):
    return math.degrees(math.acos(np.clip(np.trace(R2.T @ Rref) / 2.0, -1.0, 1.0)))


@pytest.mark.parametrize("method,niv,n", [("direct", False, 3000), ("direct", True, 2500), ("bh", False, 20000),
                                          ("bh", True, 12000)])
def test_planar_registration_matches_oracle(fga, orc, method, niv, n):
    X, Y, R_gt, t_gt = synth.plane_pair(7 + n, n=n, m=int(0.8 * n))
    m_o = orc.FGA_BH if method == "bh" else orc.FGA_DIRECT
    po = orc.Params(method=m_o, theta=0.5, max_iter=150, dim=2, niv_masses=niv)
    o = orc.register_full(X, Y, po)
    p = fga.params(method=fga.FGA_BH if method == "bh" else fga.FGA_DIRECT, theta=0.5, max_iter=150,
                   dim=2, mass_mode=fga.FGA_MASS_NIV if niv else fga.FGA_MASS_UNIFORM)
    R, t, st = fga.fga_register(_cuda(X), _cuda(Y), p)
    assert R[2, 2] == 1.0 and R[0, 2] == R[1, 2] == R[2, 0] == R[2, 1] == 0.0
    diag = float(np.linalg.norm(X.max(0) - X.min(0)))
    assert err2(R[:2, :2], o["R2"]) <= 0.01
    assert np.linalg.norm(t[:2] - o["t2"]) <= 1e-4 * diag
    assert abs(t[2]) <= 1e-5 * diag
    if method == "bh":
        assert abs(st["interactions"] - o["interactions"]) <= 1e-3 * o["interactions"]
    else:
        assert st["interactions"] == 150 * len(X) * len(Y)


def test_planar_ground_truth_and_host_inputs(fga):
    X, Y, R_gt, t_gt = synth.plane_pair(3, n=4000, max_deg=25.0)
    p = fga.params(method=fga.FGA_DIRECT, max_iter=300, dim=2)
    R, t, st = fga.fga_register(X, Y, p)  # host arrays
    assert err2(R[:2, :2], R_gt) < 1.0


def test_planar_pairs_in_a_mixed_batch(fga):
    X2, Y2, _, _ = synth.plane_pair(11, n=3000)
    X3, Y3, _, _ = synth.sphere_pair(11, n=2000)
    p2 = fga.params(method=fga.FGA_DIRECT, max_iter=40, dim=2)
    p3 = fga.params(method=fga.FGA_DIRECT, max_iter=40)
    res, st = fga.fga_register_batch([(_cuda(X2), _cuda(Y2), None, None, p2),
                                      (_cuda(X3), _cuda(Y3), None, None, p3)], p3)
    a2 = fga.fga_register_batch([(_cuda(X2), _cuda(Y2))], p2)[0][0]
    a3 = fga.fga_register_batch([(_cuda(X3), _cuda(Y3))], p3)[0][0]
    assert np.array_equal(res[0]["R"], a2["R"]) and np.array_equal(res[1]["R"], a3["R"])
    assert res[0]["R"][2, 2] == 1.0


def test_planar_shape_is_checked(fga):
    X, Y, _, _ = synth.plane_pair(2, n=500)
    p = fga.params(dim=2, max_iter=5)
    with pytest.raises(ValueError):
        fga.fga_register(_cuda(np.column_stack([X, np.zeros(len(X))])), _cuda(Y), p)
    X3 = np.column_stack([X, np.zeros(len(X))])
    Y3 = np.column_stack([Y, np.zeros(len(Y))])
    with pytest.raises(fga.FGAError):
        fga.fga_register(_cuda(X3), _cuda(Y3), fga.params(dim=4))

"""GPU inverse-density masses from the k-th nearest neighbour against the
oracle, and registrations that use them (D = 3 and D = 2)."""
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


@pytest.mark.parametrize("k", [8, 16, 32])
def test_knn_masses_match_oracle(fga, orc, k):
    X, Y, _, _ = synth.lidar_pair(21, n=20000, m=2000)
    Xn, _, _ = orc.normalize(X, Y)
    P = Xn.astype(np.float32)
    g = fga.fga_masses(_cuda(P), fga.FGA_MASS_KNN, lattice=k).cpu().numpy()
    o = orc.masses_knn(P.astype(np.float64), k=k)
    np.testing.assert_allclose(g, o, rtol=3e-6)


@pytest.mark.parametrize("n", [17, 257, 5003])
def test_knn_masses_ragged(fga, orc, n):
    P = np.random.default_rng(n).uniform(-4, 4, size=(n, 3)).astype(np.float32)
    g = fga.fga_masses(_cuda(P), fga.FGA_MASS_KNN, lattice=16, total=2.0).cpu().numpy()
    np.testing.assert_allclose(g, orc.masses_knn(P.astype(np.float64), k=16, total=2.0), rtol=3e-6)


def test_registration_with_knn_masses(fga, orc):
    X, Y, _, _ = synth.lidar_pair(5, n=6000)
    po = orc.Params(method=orc.FGA_BH, theta=0.5, max_iter=100, knn_masses=True, lattice=16, G=1.0)
    o = orc.register_full(X, Y, po)
    p = fga.params(method=fga.FGA_BH, theta=0.5, max_iter=100, mass_mode=fga.FGA_MASS_KNN, lattice=16, G=1.0)
    R, t, st = fga.fga_register(_cuda(X), _cuda(Y), p)
    import oracle
    diag = float(np.linalg.norm(X.max(0) - X.min(0)))
    assert oracle.rotation_error_deg(R, o["R"]) <= 0.01
    assert np.linalg.norm(t - o["t"]) <= 1e-4 * diag


def test_planar_registration_with_knn_masses(fga, orc):
    X, Y, _, _ = synth.plane_pair(8, n=3000)
    po = orc.Params(method=orc.FGA_DIRECT, max_iter=100, dim=2, knn_masses=True, lattice=16)
    o = orc.register_full(X, Y, po)
    p = fga.params(method=fga.FGA_DIRECT, max_iter=100, dim=2, mass_mode=fga.FGA_MASS_KNN, lattice=16)
    R, t, st = fga.fga_register(_cuda(X), _cuda(Y), p)
    import math
    c = np.clip(np.trace(R[:2, :2].T @ o["R2"]) / 2.0, -1, 1)
    assert math.degrees(math.acos(c)) <= 0.01
    assert np.linalg.norm(t[:2] - o["t2"]) <= 1e-4 * float(np.linalg.norm(X.max(0) - X.min(0)))


def test_bad_k_is_rejected(fga):
    P = _cuda(np.random.default_rng(0).uniform(-1, 1, size=(100, 3)))
    with pytest.raises(fga.FGAError):
        fga.fga_masses(P, fga.FGA_MASS_KNN, lattice=12)
    with pytest.raises(fga.FGAError):
        fga.fga_register(P, P, fga.params(mass_mode=fga.FGA_MASS_KNN, lattice=7))

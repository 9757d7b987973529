"""GPU NIV masses (Sec. IV-F.2, Eq. 18) against the FP64 oracle (needs a GPU).

Both sides measure each lattice cell's covered fraction on the same lines with
the same FP64 chord arithmetic, so they differ only in the order in which the
lines' lengths are summed; masses are FP32 outputs and must agree to 1e-6
relative. The cases cover the shapes whose fractions the oracle is pinned to
in closed form (one ball, coincident balls, a lens, a ball cut by a face, a
clamped point on a corner, a filled cell), random clouds at several lattice
sizes with ragged counts and points outside [a, b], the surface-like LiDAR
and planar-scene clouds, and a fine lattice whose non-empty cells are
measured in more than one chunk.
"""
import numpy as np
import pytest

import synth

pytestmark = pytest.mark.gpu

A, B, RHO = -5.0, 5.0, 16
H = (B - A) / RHO


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


def _f32(a):
    return np.asarray(a, dtype=np.float32).astype(np.float64)


def _check(fga, orc, P, lattice=RHO, a=A, b=B, total=1.0):
    P = _f32(P)
    m_o = orc.masses_niv(P, lattice, a, b, total)
    m = fga.fga_masses(_cuda(P), fga.FGA_MASS_NIV, lattice, a, b, total).cpu().numpy()
    np.testing.assert_allclose(m, m_o, rtol=1e-6)
    return m


def test_closed_form_shapes_match_oracle(fga, orc):
    rng = np.random.default_rng(0)
    r = H / 6
    lo = lambda i: A + np.asarray(i, dtype=np.float64) * H   # noqa: E731
    parts = [
        lo((1, 1, 1)) + H / 2,                                         # one ball
        np.tile(lo((3, 1, 1)) + [0.3, 0.2, 0.4], (5, 1)),              # coincident balls
        np.array([lo((5, 1, 1)) + H / 2, lo((5, 1, 1)) + H / 2 + [0.1, 0.05, 0.0]]),  # lens
        lo((7, 1, 1)) + [H / 2, H / 2, 0.3 * r],                       # cut by the lower z face
        lo((9, 1, 1)) + [0.2 * r, H / 2, H / 2],                       # cut by the lower x face
        np.array([[B + 2.0, B + 2.0, B + 2.0]]),                       # clamped onto the far corner
        np.array([[A, A, A]]),                                         # on the near corner
    ]
    g = np.arange(0.0, H * (1 - 1e-6), r / 2)
    parts.append(np.stack(np.meshgrid(g, g, g, indexing="ij"), -1).reshape(-1, 3) + lo((12, 12, 12)))
    parts.append(lo((2, 9, 4)) + rng.uniform(0, H, size=(37, 3)))      # a random cluster
    m = _check(fga, orc, np.concatenate([np.atleast_2d(p) for p in parts]))
    assert np.all(m > 0)


@pytest.mark.parametrize("lattice,n,seed", [(1, 500, 1), (7, 3001, 2), (16, 12345, 3), (64, 20000, 4)])
def test_random_clouds_match_oracle(fga, orc, lattice, n, seed):
    rng = np.random.default_rng(seed)
    P = np.concatenate([rng.uniform(-5.5, 5.5, size=(n - n // 3, 3)),     # some outside [a, b]
                        rng.normal(scale=0.4, size=(n // 3, 3))])          # a dense blob
    _check(fga, orc, P, lattice=lattice, total=2.5)


def test_unit_interval_domain_matches_oracle(fga, orc):
    rng = np.random.default_rng(5)
    P = rng.uniform(0.0, 1.0, size=(4000, 3)) ** 2
    _check(fga, orc, P, lattice=8, a=0.0, b=1.0)


@pytest.mark.parametrize("kind", ["lidar", "planar"])
def test_surface_clouds_match_oracle(fga, orc, kind):
    if kind == "lidar":
        X, Y, _, _ = synth.lidar_pair(6, n=30000)
    else:
        X, Y, _, _ = synth.planar_scene_pair(6, n=60000)
    Xn, _, _ = orc.normalize(X, Y)
    _check(fga, orc, Xn)


def test_fine_lattice_many_chunks_matches_oracle(fga, orc):
    # lattice 128: ~70k non-empty cells, measured in three chunks of 32768
    rng = np.random.default_rng(7)
    P = rng.uniform(-5, 5, size=(80000, 3))
    _check(fga, orc, P, lattice=128)


def test_repeatable_bitwise(fga):
    X, Y, _, _ = synth.lidar_pair(8, n=20000)
    P = _cuda(X / np.abs(X).max() * 4.9)
    m1 = fga.fga_masses(P, fga.FGA_MASS_NIV).cpu().numpy()
    m2 = fga.fga_masses(P, fga.FGA_MASS_NIV).cpu().numpy()
    np.testing.assert_array_equal(m1, m2)

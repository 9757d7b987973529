"""Pins of the oracle's NIV measure (Sec. IV-F.2, Eq. 18) against closed forms.

Eq. 18 divides the volume of the union of the balls B(Y_i) of a lattice
cell's points, inside the cell, by the cell's volume. The balls have radius
(b - a) / (2 D rho) = h / (2 D) for cell side h. The oracle integrates the
union exactly along one axis and by the midpoint rule across it (64 x 64
lines per 3D cell, 1024 per 2D cell), which it states to be within 3e-3 (3D)
and 1.1e-4 (2D) of the exact fraction. These tests hold it to that bound on
shapes whose volume is known in closed form:

- one ball wholly inside a cell: 4/3 pi r^3 / h^3 (pi r^2 / h^2 in 2D);
- two coincident balls: exactly the same fraction as one (a union, not a count);
- two disjoint balls: twice that;
- two balls overlapping at centre distance d: 2 V - lens(d);
- a ball cut by a cell face at depth t: V - cap(r - t);
- a ball centred on a cell corner: V / 2^D;
- a cell filled with points closer than the ball radius: fraction 1.

A dropped clip, a wrong radius (d read as the tree depth), a sum of volumes
instead of a union, or a count-only formula each fails one of them.
"""
import math

import numpy as np
import pytest

A, B, RHO = -5.0, 5.0, 16
H = (B - A) / RHO
TOL = {3: 3e-3, 2: 1.1e-4}


def _radius(dim):
    return H / (2 * dim)


def _ball(dim, r=None):
    r = _radius(dim) if r is None else r
    return 4.0 / 3.0 * math.pi * r ** 3 if dim == 3 else math.pi * r * r


def _cell_volume(dim):
    return H ** dim


def _lens(dim, d):
    r = _radius(dim)
    if dim == 3:
        return math.pi * (4 * r + d) * (2 * r - d) ** 2 / 12.0
    return 2 * r * r * math.acos(d / (2 * r)) - 0.5 * d * math.sqrt(4 * r * r - d * d)


def _cap(dim, hc):
    """Volume (area) of the part of a ball (disc) of radius r beyond a plane
    (line) at distance r - hc from its centre."""
    r = _radius(dim)
    if dim == 3:
        return math.pi * hc * hc * (3 * r - hc) / 3.0
    return r * r * math.acos((r - hc) / r) - (r - hc) * math.sqrt(2 * r * hc - hc * hc)


def _cell_lo(idx):
    return A + np.asarray(idx, dtype=np.float64) * H


def _embed(P, dim):
    P = np.atleast_2d(np.asarray(P, dtype=np.float64))
    if dim == 2:
        P = np.concatenate([P, np.zeros((len(P), 1))], 1)
    return P


def _frac_of(orc, P, dim, cell_idx):
    frac, _ = orc.niv_fractions(_embed(P, dim), RHO, A, B, dim)
    return frac[tuple(reversed(cell_idx))]


@pytest.mark.parametrize("dim", [3, 2])
def test_single_ball_inside_cell(orc, dim):
    rng = np.random.default_rng(10 + dim)
    r = _radius(dim)
    exact = _ball(dim) / _cell_volume(dim)
    for _ in range(20):
        idx = rng.integers(0, RHO, size=dim)
        c = _cell_lo(idx) + rng.uniform(r, H - r, size=dim)
        f = _frac_of(orc, c, dim, idx)
        assert f == pytest.approx(exact, rel=TOL[dim])


@pytest.mark.parametrize("dim", [3, 2])
def test_coincident_balls_count_once(orc, dim):
    rng = np.random.default_rng(20 + dim)
    idx = (5,) * dim
    c = _cell_lo(idx) + rng.uniform(0.3 * H, 0.7 * H, size=dim)
    one = _frac_of(orc, c, dim, idx)
    for k in (2, 3, 17):
        assert _frac_of(orc, np.tile(c, (k, 1)), dim, idx) == one


@pytest.mark.parametrize("dim", [3, 2])
def test_disjoint_balls_add(orc, dim):
    r = _radius(dim)
    idx = (7,) * dim
    lo = _cell_lo(idx)
    if dim == 3:
        P = [lo + [r * 1.05, r * 1.05, r * 1.05], lo + [H - r * 1.05, H - r * 1.05, H - r * 1.05]]
    else:
        P = [lo + [r * 1.05, r * 1.05], lo + [H - r * 1.05, H - r * 1.05]]
    exact = 2 * _ball(dim) / _cell_volume(dim)
    assert _frac_of(orc, np.array(P), dim, idx) == pytest.approx(exact, rel=TOL[dim])


@pytest.mark.parametrize("dim", [3, 2])
def test_overlapping_balls_lens(orc, dim):
    rng = np.random.default_rng(30 + dim)
    r = _radius(dim)
    idx = (3,) * dim
    centre = _cell_lo(idx) + H / 2
    # both balls stay inside the cell: |offset| + r <= h / 2 per axis
    dmax = 1.9 * r if dim == 3 else 0.99 * r
    for _ in range(12):
        d = rng.uniform(0.05 * r, dmax)
        u = rng.normal(size=dim)
        u /= np.linalg.norm(u)
        P = np.array([centre, centre + d * u])
        exact = (2 * _ball(dim) - _lens(dim, d)) / _cell_volume(dim)
        assert _frac_of(orc, P, dim, idx) == pytest.approx(exact, rel=TOL[dim])


@pytest.mark.parametrize("dim", [3, 2])
def test_ball_cut_by_cell_face(orc, dim):
    rng = np.random.default_rng(40 + dim)
    r = _radius(dim)
    idx = (9,) * dim
    lo = _cell_lo(idx)
    for axis in range(dim):
        for _ in range(6):
            t = rng.uniform(0.02 * r, 0.98 * r)   # depth of the centre below the face
            c = lo + H / 2
            c = c.copy()
            c[axis] = lo[axis] + t                # lower face of this axis
            exact = (_ball(dim) - _cap(dim, r - t)) / _cell_volume(dim)
            assert _frac_of(orc, c, dim, idx) == pytest.approx(exact, rel=TOL[dim])


@pytest.mark.parametrize("dim", [3, 2])
def test_ball_on_cell_corner_and_clamping(orc, dim):
    # A point beyond the lattice is clamped into the corner cell and its ball
    # is centred on the domain's corner: a 1 / 2^D part lies in the cell.
    exact = _ball(dim) / 2 ** dim / _cell_volume(dim)
    far = np.full(dim, B + 3.0)
    assert _frac_of(orc, far, dim, (RHO - 1,) * dim) == pytest.approx(exact, rel=2 * TOL[dim])
    corner = np.full(dim, A)
    assert _frac_of(orc, corner, dim, (0,) * dim) == pytest.approx(exact, rel=2 * TOL[dim])


@pytest.mark.parametrize("dim", [3, 2])
def test_filled_cell_is_fully_covered(orc, dim):
    # Points on a grid of spacing r / 2 cover every line through the cell.
    r = _radius(dim)
    idx = (4,) * dim
    g = np.arange(0.0, H * (1 - 1e-9), r / 2)
    P = np.stack(np.meshgrid(*([g] * dim), indexing="ij"), -1).reshape(-1, dim) + _cell_lo(idx)
    assert _frac_of(orc, P, dim, idx) == pytest.approx(1.0, rel=1e-12)


@pytest.mark.parametrize("dim", [3, 2])
def test_masses_are_inverse_fractions(orc, dim):
    # One isolated ball, one filled cell: weights 1 / fraction, summing to 1.
    r = _radius(dim)
    iso_idx = (1,) * dim
    iso = _cell_lo(iso_idx) + H / 2
    full_idx = (12,) * dim
    g = np.arange(0.0, H * (1 - 1e-9), r / 2)
    grids = np.meshgrid(*([g] * dim), indexing="ij")
    dense = np.stack(grids, -1).reshape(-1, dim) + _cell_lo(full_idx)
    P = _embed(np.concatenate([iso[None], dense]), dim)
    m = orc.masses_niv(P, RHO, A, B, 1.0, dim=dim)
    frac, cell = orc.niv_fractions(P, RHO, A, B, dim)
    f_iso = frac.ravel()[cell[0]]
    assert frac.ravel()[cell[1]] == pytest.approx(1.0, rel=1e-12)
    assert m[0] / m[1] == pytest.approx(1.0 / f_iso, rel=1e-12)
    assert f_iso == pytest.approx(_ball(dim) / _cell_volume(dim), rel=TOL[dim])
    assert m.sum() == pytest.approx(1.0, rel=1e-13)


def test_fraction_grows_with_spread_not_with_count(orc):
    # Two clusters of equal count: the spread one covers more of its cell.
    rng = np.random.default_rng(50)
    r = _radius(3)
    tight = _cell_lo((2, 2, 2)) + H / 2 + rng.normal(scale=0.01 * r, size=(40, 3))
    spread = _cell_lo((10, 2, 2)) + H / 2 + rng.uniform(-0.3 * H, 0.3 * H, size=(40, 3))
    frac, cell = orc.niv_fractions(np.concatenate([tight, spread]), RHO, A, B, 3)
    f_tight, f_spread = frac.ravel()[cell[0]], frac.ravel()[cell[40]]
    assert f_tight < 1.1 * _ball(3) / _cell_volume(3)
    assert f_spread > 5 * f_tight

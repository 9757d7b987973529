"""Seeded synthetic point-set pairs shaped like the FGA paper's workloads.

This module only *generates inputs*: point clouds, ground-truth rigid motions
and size lists. It holds none of the registration method's arithmetic (no
normalisation, masses, forces, trees or Procrustes steps), so that both the
FP64 oracle and the CUDA path can consume the same inputs without sharing any
of the method's code.

Every generator is a pure function of its seed. Point arrays are returned as
C-contiguous ``float32`` arrays of shape ``(n, 3)`` (row-major xyz), ground
truth as ``float64``. The convention is that the ground-truth transform maps
the template onto the reference: ``X ~ R_gt @ Y + t_gt``.

Workloads (the paper measures on bunny, KITTI, lounge, 3DMatch; none of those
datasets is reproduced here, only their shape statistics):

* :func:`sphere_pair`   -- points on the unit sphere, noise sigma = 0.01,
  rotation <= 45 deg, translation <= 0.2 (the 1k x 1k direct-sum case).
* :func:`lidar_pair`    -- two 64-ring LiDAR-like sweeps of a ground plane plus
  box obstacles with the 1/r^2 density fall-off that constant angular sampling
  gives, about 50 % overlap, noise sigma = 0.02 m (a stand-in for the paper's
  KITTI frame-to-frame experiment, Sec. V-F, by shape only).
* :func:`planar_scene_pair` -- piecewise-planar scenes with 10x density
  variation and 5 % outliers (large inhomogeneous clouds).
* :func:`box_pair`      -- a noise-free anisotropic box volume under a known
  motion, used to check that the loop recovers an applied (R, t).
* :func:`batch_sizes`   -- log-uniform (N, M) sizes for many independent pairs.
"""
from __future__ import annotations

import math

import numpy as np

__all__ = [
    "random_rotation",
    "random_translation",
    "sphere_pair",
    "box_pair",
    "lidar_pair",
    "planar_scene_pair",
    "batch_sizes",
    "rotation_about",
]


def rotation_about(axis, angle_rad: float) -> np.ndarray:
    """Rotation matrix for ``angle_rad`` about the unit ``axis`` (Rodrigues)."""
    ax = np.asarray(axis, dtype=np.float64)
    ax = ax / np.linalg.norm(ax)
    k = np.array([[0.0, -ax[2], ax[1]], [ax[2], 0.0, -ax[0]], [-ax[1], ax[0], 0.0]])
    return np.eye(3) + math.sin(angle_rad) * k + (1.0 - math.cos(angle_rad)) * (k @ k)


def random_rotation(rng: np.random.Generator, max_deg: float) -> np.ndarray:
    """Uniformly random axis, angle uniform in (0, max_deg] degrees."""
    axis = rng.normal(size=3)
    angle = math.radians(rng.uniform(0.0, max_deg))
    return rotation_about(axis, angle)


def random_translation(rng: np.random.Generator, max_norm: float) -> np.ndarray:
    """Uniform sample from the ball of radius ``max_norm``."""
    d = rng.normal(size=3)
    d /= np.linalg.norm(d)
    return d * max_norm * rng.uniform() ** (1.0 / 3.0)


def _f32(a) -> np.ndarray:
    return np.ascontiguousarray(np.asarray(a, dtype=np.float32))


def sphere_pair(seed: int, n: int = 1000, m: int | None = None, max_deg: float = 45.0,
                t_max: float = 0.2, sigma: float = 0.01):
    """Points on the unit sphere (normalised Gaussian vectors).

    The reference is ``P + noise``; the template is ``R_gt^T (P' - t_gt) + noise``
    where ``P'`` are the first ``m`` base points, with independent noise on both.
    Returns ``(X, Y, R_gt, t_gt)``.
    """
    m = n if m is None else m
    rng = np.random.default_rng(seed)
    p = rng.normal(size=(max(n, m), 3))
    p /= np.linalg.norm(p, axis=1, keepdims=True)
    r_gt = random_rotation(rng, max_deg)
    t_gt = random_translation(rng, t_max)
    x = p[:n] + rng.normal(scale=sigma, size=(n, 3))
    y = (p[:m] - t_gt) @ r_gt + rng.normal(scale=sigma, size=(m, 3))
    return _f32(x), _f32(y), r_gt, t_gt


def box_pair(seed: int, n: int = 500, deg: float = 15.0, t=(0.1, -0.05, 0.08),
             half_extents=(1.0, 0.6, 0.3)):
    """Noise-free points uniform in an anisotropic box, template = exact copy.

    ``X`` is uniform in the box; ``Y = R_gt^T (X - t_gt)`` with a random axis and
    exactly ``deg`` degrees of rotation. Returns ``(X, Y, R_gt, t_gt)``.
    """
    rng = np.random.default_rng(seed)
    x = rng.uniform(-1.0, 1.0, size=(n, 3)) * np.asarray(half_extents)
    r_gt = rotation_about(rng.normal(size=3), math.radians(deg))
    t_gt = np.asarray(t, dtype=np.float64)
    xf = _f32(x)
    y = (xf.astype(np.float64) - t_gt) @ r_gt
    return xf, _f32(y), r_gt, t_gt


# ---------------------------------------------------------------------------
# LiDAR-like sweeps
# ---------------------------------------------------------------------------

def _scene_boxes(rng: np.random.Generator, ground_z: float, radius: float):
    nb = int(rng.integers(20, 41))
    boxes = []
    while len(boxes) < nb:
        r = rng.uniform(4.0, radius)
        phi = rng.uniform(0.0, 2.0 * math.pi)
        cx, cy = r * math.cos(phi), r * math.sin(phi)
        sx, sy, sz = rng.uniform(0.5, 4.0, size=3)
        lo = np.array([cx - sx / 2, cy - sy / 2, ground_z])
        hi = np.array([cx + sx / 2, cy + sy / 2, ground_z + sz])
        boxes.append((lo, hi))
    return boxes


def _cast(origin, dirs, ground_z, boxes, max_range):
    """Nearest hit distance of each ray against the ground plane and boxes."""
    n = dirs.shape[0]
    t_hit = np.full(n, np.inf)
    dz = dirs[:, 2]
    with np.errstate(divide="ignore", invalid="ignore"):
        tg = (ground_z - origin[2]) / dz
    ok = (dz < 0) & (tg > 0)
    t_hit[ok] = tg[ok]
    inv = np.where(np.abs(dirs) > 1e-12, 1.0 / np.where(np.abs(dirs) > 1e-12, dirs, 1.0), np.inf)
    for lo, hi in boxes:
        t1 = (lo - origin) * inv
        t2 = (hi - origin) * inv
        tmin = np.minimum(t1, t2)
        tmax = np.maximum(t1, t2)
        # rays parallel to a slab: inside -> (-inf, inf), outside -> empty
        par = ~np.isfinite(inv)
        if par.any():
            inside = (origin >= lo) & (origin <= hi)
            tmin = np.where(par, np.where(inside, -np.inf, np.inf), tmin)
            tmax = np.where(par, np.where(inside, np.inf, -np.inf), tmax)
        tn = tmin.max(axis=1)
        tf = tmax.min(axis=1)
        hit = (tn <= tf) & (tn > 0)
        t_hit = np.where(hit & (tn < t_hit), tn, t_hit)
    t_hit[t_hit > max_range] = np.inf
    return t_hit


def _sweep(rng, rot, centre, az_lo_deg, az_width_deg, n_az, ground_z, boxes,
           max_range, sigma, n_rings=64, el_lo=-25.0, el_hi=2.0):
    el = np.radians(np.linspace(el_lo, el_hi, n_rings))
    az = np.radians(az_lo_deg + az_width_deg * (np.arange(n_az) + 0.5) / n_az)
    ee, aa = np.meshgrid(el, az, indexing="ij")
    d_s = np.stack([np.cos(ee) * np.cos(aa), np.cos(ee) * np.sin(aa), np.sin(ee)], -1).reshape(-1, 3)
    d_w = d_s @ rot.T
    t = _cast(centre, d_w, ground_z, boxes, max_range)
    ok = np.isfinite(t)
    pts = d_s[ok] * t[ok, None]
    pts = pts + rng.normal(scale=sigma, size=pts.shape)
    return pts


def lidar_pair(seed: int, n: int = 120_000, m: int | None = None, overlap: float = 0.5,
               sigma: float = 0.02, max_range: float = 80.0, ground_z: float = -1.7,
               max_yaw_deg: float = 10.0):
    """Two LiDAR-like sweeps (64 rings over -25..+2 deg) of one synthetic scene.

    The scene is a ground plane at ``ground_z`` plus 20-40 axis-aligned boxes
    (sides 0.5-4 m) within 40 m. Sensor A sits at the origin; sensor B is moved
    by a yaw <= ``max_yaw_deg``, roll/pitch <= 1 deg and a 1-3 m horizontal
    translation. Each sweep keeps an azimuth window of 180 deg; the windows are
    offset so that about ``overlap`` of each sweep sees the same part of the
    scene. The number of returns is trimmed to exactly ``n`` (reference) and
    ``m`` (template) by uniform subsampling, which keeps the 1/r^2 density
    fall-off of constant angular sampling.

    Returns ``(X, Y, R_gt, t_gt)`` with points in each sensor's own frame and
    ``X ~ R_gt Y + t_gt``.
    """
    m = n if m is None else m
    rng = np.random.default_rng(seed)
    boxes = _scene_boxes(rng, ground_z, 40.0)
    yaw = math.radians(rng.uniform(-max_yaw_deg, max_yaw_deg))
    r_b = rotation_about([0, 0, 1], yaw) @ rotation_about([1, 0, 0], math.radians(rng.uniform(-1, 1))) \
        @ rotation_about([0, 1, 0], math.radians(rng.uniform(-1, 1)))
    dist = rng.uniform(1.0, 3.0)
    ang = rng.uniform(0.0, 2.0 * math.pi)
    c_b = np.array([dist * math.cos(ang), dist * math.sin(ang), 0.0])
    width = 180.0
    shift = width * (1.0 - overlap)
    a0 = rng.uniform(0.0, 360.0)

    def trimmed(rot, centre, az_lo, count):
        n_az = 2048
        while True:
            pts = _sweep(rng, rot, centre, az_lo, width, n_az, ground_z, boxes, max_range, sigma)
            if pts.shape[0] >= count:
                break
            n_az = int(n_az * 1.3 * count / max(pts.shape[0], 1)) + 1
        keep = rng.choice(pts.shape[0], size=count, replace=False)
        keep.sort()
        return pts[keep]

    x = trimmed(np.eye(3), np.zeros(3), a0, n)
    y = trimmed(r_b, c_b, a0 + shift - math.degrees(yaw), m)
    return _f32(x), _f32(y), r_b, c_b


# ---------------------------------------------------------------------------
# Piecewise-planar scenes
# ---------------------------------------------------------------------------

def _planar_scene(rng):
    k = int(rng.integers(8, 17))
    patches = []
    for _ in range(k):
        normal_axis = int(rng.integers(0, 3))
        tilt = rotation_about(rng.normal(size=3), math.radians(rng.uniform(0, 10)))
        centre = rng.uniform(-1.0, 1.0, size=3)
        size = rng.uniform(0.3, 1.5, size=2)
        density = math.exp(rng.uniform(0.0, math.log(10.0)))
        patches.append((normal_axis, tilt, centre, size, density))
    return patches


def _sample_scene(rng, patches, n, sigma, outlier_frac):
    weights = np.array([p[3][0] * p[3][1] * p[4] for p in patches])
    weights /= weights.sum()
    n_out = int(round(outlier_frac * n))
    counts = rng.multinomial(n - n_out, weights)
    pts = []
    for (axis, tilt, centre, size, _), c in zip(patches, counts):
        uv = (rng.uniform(-0.5, 0.5, size=(c, 2)) * size)
        local = np.zeros((c, 3))
        other = [i for i in range(3) if i != axis]
        local[:, other[0]] = uv[:, 0]
        local[:, other[1]] = uv[:, 1]
        pts.append(local @ tilt.T + centre)
    body = np.concatenate(pts, axis=0)
    body += rng.normal(scale=sigma, size=body.shape)
    lo, hi = body.min(0), body.max(0)
    pad = 0.1 * (hi - lo)
    out = rng.uniform(lo - pad, hi + pad, size=(n_out, 3))
    allp = np.concatenate([body, out], axis=0)
    return allp[rng.permutation(allp.shape[0])]


def planar_scene_pair(seed: int, n: int = 1_000_000, m: int | None = None,
                      max_deg: float = 30.0, t_max: float = 0.2, sigma: float = 0.01,
                      outlier_frac: float = 0.05):
    """8-16 planar rectangles, per-patch density log-uniform over a 10x range.

    ``X`` and ``Y`` are sampled independently from the same scene (no shared
    points), each with noise ``sigma`` and ``outlier_frac`` uniform outliers in
    the 10 %-inflated bounding box; ``Y`` is then moved by ``(R_gt, t_gt)^-1``.
    Returns ``(X, Y, R_gt, t_gt)``.
    """
    m = n if m is None else m
    rng = np.random.default_rng(seed)
    patches = _planar_scene(rng)
    r_gt = random_rotation(rng, max_deg)
    t_gt = random_translation(rng, t_max)
    x = _sample_scene(rng, patches, n, sigma, outlier_frac)
    y = (_sample_scene(rng, patches, m, sigma, outlier_frac) - t_gt) @ r_gt
    return _f32(x), _f32(y), r_gt, t_gt


def batch_sizes(seed: int, count: int = 256, lo: int = 500, hi: int = 50_000):
    """``count`` independent (N, M) pairs, each log-uniform in [lo, hi]."""
    rng = np.random.default_rng(seed)
    s = np.exp(rng.uniform(math.log(lo), math.log(hi), size=(count, 2)))
    return np.round(s).astype(np.int64)


def batch_pairs(seed: int, count: int = 256, lo: int = 500, hi: int = 50_000,
                max_deg: float = 60.0, t_max: float = 0.3):
    """``count`` independent pairs with N and M log-uniform in [lo, hi].

    Shapes alternate between unit-sphere clouds and piecewise-planar scenes;
    each pair has its own rotation (<= max_deg) and translation (<= t_max).
    Returns a list of (X, Y, R_gt, t_gt).
    """
    sizes = batch_sizes(seed, count, lo, hi)
    out = []
    for k, (n, m) in enumerate(sizes):
        if k % 2 == 0:
            out.append(sphere_pair(seed * 100_003 + k, n=int(n), m=int(m), max_deg=max_deg,
                                   t_max=t_max))
        else:
            out.append(planar_scene_pair(seed * 100_003 + k, n=int(n), m=int(m), max_deg=max_deg,
                                         t_max=t_max))
    return out


def cropped_scene_pair(seed: int, n: int, m: int, overlap: float, max_deg: float = 30.0,
                       t_max: float = 0.2, sigma: float = 0.01, outlier_frac: float = 0.05):
    """Two partial views of one piecewise-planar scene with a given overlap.

    The scene (as in ``planar_scene_pair``) is cut along its longest axis into
    two windows of equal width whose shared part is ``overlap`` of each window;
    X keeps ``n`` points of the first window, Y ``m`` points of the second
    (uniform subsamples of denser draws), and Y is then moved by
    ``(R_gt, t_gt)^-1``. Returns ``(X, Y, R_gt, t_gt)``."""
    rng = np.random.default_rng(seed)
    patches = _planar_scene(rng)
    r_gt = random_rotation(rng, max_deg)
    t_gt = random_translation(rng, t_max)
    probe = _sample_scene(rng, patches, 4096, sigma, 0.0)
    lo, hi = probe.min(0), probe.max(0)
    axis = int(np.argmax(hi - lo))
    span = float(hi[axis] - lo[axis])
    width = span / (2.0 - overlap)
    win_x = (lo[axis], lo[axis] + width)
    win_y = (lo[axis] + width * (1.0 - overlap), hi[axis])

    def view(count, win):
        frac = max((win[1] - win[0]) / span, 0.05)
        draw = int(count / frac * 1.3) + 64
        while True:
            pts = _sample_scene(rng, patches, draw, sigma, outlier_frac)
            keep = pts[(pts[:, axis] >= win[0]) & (pts[:, axis] <= win[1])]
            if keep.shape[0] >= count:
                return keep[rng.choice(keep.shape[0], size=count, replace=False)]
            draw = int(draw * 1.5)

    x = view(n, win_x)
    y = (view(m, win_y) - t_gt) @ r_gt
    return _f32(x), _f32(y), r_gt, t_gt


def serve_trace(seed: int, count: int, rate: float = 200.0, lo: int = 1000, hi: int = 500_000,
                overlap_lo: float = 0.3, overlap_hi: float = 1.0):
    """A request trace: Poisson arrivals at ``rate`` per second.

    Request k arrives at ``t_k`` (seconds, exponential gaps) and carries a
    cropped-scene pair with N and M log-uniform in [lo, hi] and overlap
    uniform in [overlap_lo, overlap_hi]. Returns a list of
    ``(t_k, X, Y, R_gt, t_gt)``."""
    rng = np.random.default_rng(seed)
    gaps = rng.exponential(1.0 / rate, size=count)
    times = np.cumsum(gaps) - gaps[0]
    sizes = np.round(np.exp(rng.uniform(math.log(lo), math.log(hi), size=(count, 2)))).astype(np.int64)
    overlaps = rng.uniform(overlap_lo, overlap_hi, size=count)
    out = []
    for k in range(count):
        X, Y, R, t = cropped_scene_pair(seed * 1_000_003 + k, int(sizes[k, 0]), int(sizes[k, 1]),
                                        float(overlaps[k]))
        out.append((float(times[k]), X, Y, R, t))
    return out


def plane_pair(seed: int, n: int = 5000, m: int | None = None, max_deg: float = 30.0,
               t_max: float = 0.2, sigma: float = 0.005):
    """A planar (D = 2) pair: 6-12 random wall segments (a 2-D scan of a room),
    per-segment density log-uniform over 10x, noise ``sigma``. X and Y are
    sampled independently from the same segments; Y is moved by
    ``(R_gt, t_gt)^-1`` with a rotation <= max_deg. Returns ``(X, Y, R_gt,
    t_gt)`` with X, Y of shape (n, 2), (m, 2) and R_gt 2 x 2."""
    m = n if m is None else m
    rng = np.random.default_rng(seed)
    k = int(rng.integers(6, 13))
    a = rng.uniform(-1.5, 1.5, size=(k, 2))
    b = a + rng.uniform(-1.2, 1.2, size=(k, 2))
    dens = np.exp(rng.uniform(0.0, math.log(10.0), size=k)) * np.linalg.norm(b - a, axis=1)
    ang = math.radians(rng.uniform(-max_deg, max_deg))
    r_gt = np.array([[math.cos(ang), -math.sin(ang)], [math.sin(ang), math.cos(ang)]])
    t_gt = rng.uniform(-1.0, 1.0, size=2)
    t_gt *= rng.uniform(0.0, t_max) / max(np.linalg.norm(t_gt), 1e-12)

    def sample(count):
        seg = rng.choice(k, size=count, p=dens / dens.sum())
        u = rng.uniform(0.0, 1.0, size=count)[:, None]
        pts = a[seg] + u * (b[seg] - a[seg])
        return pts + rng.normal(scale=sigma, size=pts.shape)

    x = sample(n)
    y = (sample(m) - t_gt) @ r_gt
    return _f32(x), _f32(y), r_gt, t_gt

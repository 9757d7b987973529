"""FP64 CPU oracle of the FGA hot path (arXiv 2009.14005) -- test infrastructure.

This package wraps ``fga_oracle.c`` (plain C, double precision) through
``ctypes``. It is the reference that the CUDA library is checked against and
is used only by ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline
leg of ``bench.py``. It does not import the CUDA package and the CUDA package
never imports it.

Functions follow the paper's steps:

==========================  ===============================================
``normalize``/``denormalize``  Appendix, Eqs. A.1-A.3 and dnorm(t)
``masses_niv``                 Sec. IV-F.2, Eq. 18 (NIV measure)
``direct_acc``                 Sec. IV-C, Eq. 6
``Tree`` / ``Tree.bh_acc``     Algorithm 1 and BHForce (Algorithm 2, Eq. 15)
``ode_step``                   Eqs. 7-10
``kabsch``                     Eqs. 14 and 16
``register``                   Algorithm 2
``register_full``              normalise -> masses -> Algorithm 2 -> dnorm
==========================  ===============================================

Mass normalisation (a reading; the paper never fixes mass units): reference
masses sum to 1 (the NIV footnote's importance weights sum to one), template
masses have mean ``dt`` so that Eq. 7's friction removes the fraction ``eta``
of each unit-weight particle's momentum per step (Sec. III: the friction
"dissipates the fraction eta of the particle momentum").
"""
from __future__ import annotations

import ctypes
import os
import subprocess
from dataclasses import dataclass

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "fga_oracle.c")
_LIB_PATH = os.path.join(_HERE, "_build", "liboracle.so")

FGA_DIRECT = 0
FGA_BH = 1
VEL_UNCONSTRAINED = 0
VEL_RIGID = 1


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (-O2, OpenMP, IEEE semantics) in-tree."""
    os.makedirs(os.path.dirname(_LIB_PATH), exist_ok=True)
    if force or not os.path.exists(_LIB_PATH) or os.path.getmtime(_LIB_PATH) < os.path.getmtime(_SRC):
        tmp = _LIB_PATH + ".tmp%d" % os.getpid()
        subprocess.check_call(["gcc", "-O2", "-std=c11", "-D_DEFAULT_SOURCE", "-fopenmp", "-fPIC",
                               "-shared", "-o", tmp, _SRC, "-lm"])
        os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


class _Params(ctypes.Structure):
    _fields_ = [("G", ctypes.c_double), ("eps", ctypes.c_double), ("eta", ctypes.c_double),
                ("dt", ctypes.c_double), ("theta", ctypes.c_double), ("max_iter", ctypes.c_int),
                ("conv_tol", ctypes.c_double), ("method", ctypes.c_int),
                ("velocity_mode", ctypes.c_int), ("max_depth", ctypes.c_int), ("dim", ctypes.c_int)]


@dataclass
class Params:
    """Algorithm parameters; defaults are the paper's (Sec. V, parameter settings)."""
    G: float = 66.7
    eps: float = 0.2
    eta: float = 0.2
    dt: float = 0.1
    theta: float = 0.6
    max_iter: int = 100
    conv_tol: float = 0.0
    method: int = FGA_DIRECT
    velocity_mode: int = VEL_UNCONSTRAINED
    max_depth: int = 20
    a: float = -5.0
    b: float = 5.0
    lattice: int = 16
    niv_masses: bool = False
    knn_masses: bool = False  # inverse-density masses from the k-th neighbour, k = lattice
    dim: int = 3  # 2: clouds given as (n, 2), registered in the plane

    def _c(self) -> _Params:
        return _Params(self.G, self.eps, self.eta, self.dt, self.theta, self.max_iter,
                       self.conv_tol, self.method, self.velocity_mode, self.max_depth, self.dim)


_lib = None


def lib():
    global _lib
    if _lib is None:
        _lib = ctypes.CDLL(build())
        D = ctypes.POINTER(ctypes.c_double)
        L = ctypes.c_long
        LP = ctypes.POINTER(ctypes.c_long)
        _lib.orc_normalize.argtypes = [D, L, D, L, ctypes.c_double, ctypes.c_double, D, D, D]
        _lib.orc_denormalize.argtypes = [D, D, D, ctypes.c_double, D]
        _lib.orc_masses_niv.argtypes = [D, L, ctypes.c_int, ctypes.c_double, ctypes.c_double,
                                        ctypes.c_double, D]
        _lib.orc_masses_niv_d.argtypes = [D, L, ctypes.c_int, ctypes.c_int, ctypes.c_double,
                                          ctypes.c_double, ctypes.c_double, D]
        _lib.orc_niv_fractions.argtypes = [D, L, ctypes.c_int, ctypes.c_int, ctypes.c_double,
                                           ctypes.c_double, D, LP]
        _lib.orc_kabsch_d.argtypes = [D, D, L, ctypes.c_int, D, D]
        _lib.orc_masses_knn.argtypes = [D, L, ctypes.c_int, ctypes.c_int, ctypes.c_double, ctypes.c_double,
                                        ctypes.c_double, D]
        _lib.orc_masses_rbf.argtypes = [D, L, LP, ctypes.c_int, ctypes.c_double, ctypes.c_double, D]
        _lib.orc_direct_acc.argtypes = [D, D, L, D, L, ctypes.c_double, ctypes.c_double, D, D]
        _lib.orc_tree_build.argtypes = [D, D, L, ctypes.c_int]
        _lib.orc_tree_build.restype = ctypes.c_void_p
        _lib.orc_tree_free.argtypes = [ctypes.c_void_p]
        _lib.orc_tree_export.argtypes = [ctypes.c_void_p, L, LP, D, LP]
        _lib.orc_tree_export.restype = L
        _lib.orc_tree_stats.argtypes = [ctypes.c_void_p, LP, ctypes.POINTER(ctypes.c_int)]
        _lib.orc_bh_acc.argtypes = [ctypes.c_void_p, D, L, ctypes.c_double, ctypes.c_double,
                                    ctypes.c_double, D, LP]
        _lib.orc_ode_step.argtypes = [D, D, D, L, ctypes.c_double, ctypes.c_double, D, D]
        _lib.orc_kabsch.argtypes = [D, D, L, D, D]
        _lib.orc_register.argtypes = [D, D, L, D, D, L, ctypes.POINTER(_Params), D, D, D,
                                      ctypes.POINTER(ctypes.c_int), D, LP, D]
        _lib.orc_set_threads.argtypes = [ctypes.c_int]
        _lib.orc_max_threads.restype = ctypes.c_int
    return _lib


def _d(a) -> np.ndarray:
    return np.ascontiguousarray(np.asarray(a, dtype=np.float64))


def _p(a):
    if a is None:
        return None
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def _lp(a):
    if a is None:
        return None
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_long))


def set_threads(n: int) -> None:
    lib().orc_set_threads(int(n))


def max_threads() -> int:
    return int(lib().orc_max_threads())


# --------------------------------------------------------------------------- Appendix

def normalize(X, Y, a: float = -5.0, b: float = 5.0):
    """Eqs. A.1-A.3. Returns ``(Xn, Yn, info)`` with info = (Xbar, Ybar, l, s)."""
    X, Y = _d(X), _d(Y)
    Xn = np.empty_like(X)
    Yn = np.empty_like(Y)
    info = np.zeros(8)
    rc = lib().orc_normalize(_p(X), len(X), _p(Y), len(Y), a, b, _p(Xn), _p(Yn), _p(info))
    if rc != 0:
        raise ValueError("degenerate input: both centred clouds have a single coordinate value")
    return Xn, Yn, info


def denormalize(R, t, info, a: float = -5.0) -> np.ndarray:
    """Translation in the original frame for a normalised-frame ``[R | t]``."""
    R, t, info = _d(R).reshape(9), _d(t), _d(info)
    out = np.zeros(3)
    lib().orc_denormalize(_p(R), _p(t), _p(info), a, _p(out))
    return out


# --------------------------------------------------------------------------- masses

def masses_niv(P, lattice: int = 16, a: float = -5.0, b: float = 5.0, total: float = 1.0, dim: int = 3):
    """Eq. 18 with the readings documented in the C source (dim 2: the x, y
    lattice with discs)."""
    P = _d(P)
    out = np.empty(len(P))
    rc = lib().orc_masses_niv_d(_p(P), len(P), dim, lattice, a, b, total, _p(out))
    if rc != 0:
        raise ValueError("bad NIV arguments")
    return out


def niv_fractions(P, lattice: int = 16, a: float = -5.0, b: float = 5.0, dim: int = 3):
    """Covered fraction of every lattice cell (Eq. 18's V(union of balls) /
    V(cell); 0 for empty cells), shape (lattice,) * dim indexed [cz, cy, cx]
    in 3D and [cy, cx] in 2D, and each point's flat cell index."""
    P = _d(P)
    ncell = lattice ** dim
    frac = np.empty(ncell)
    cell = np.empty(len(P), dtype=np.int64)
    rc = lib().orc_niv_fractions(_p(P), len(P), dim, lattice, a, b, _p(frac),
                                 cell.ctypes.data_as(ctypes.POINTER(ctypes.c_long)))
    if rc != 0:
        raise ValueError("bad NIV arguments")
    return frac.reshape((lattice,) * dim), cell


def masses_knn(P, k: int = 16, dim: int = 3, a: float = -5.0, b: float = 5.0, total: float = 1.0):
    """Inverse-density masses from the distance to the k-th nearest neighbour
    (reading in the C source)."""
    P = _d(P)
    out = np.empty(len(P))
    rc = lib().orc_masses_knn(_p(P), len(P), k, dim, a, b, total, _p(out))
    if rc != 0:
        raise ValueError("bad kNN-mass arguments")
    return out


def masses_rbf(P, landmarks, sigma: float = 10.0 / 16.0, floor: float = 1e-3):
    """Eq. 17: the RBF interpolant B over the landmark indices (readings in the
    C source); B = 1 everywhere without landmarks."""
    P = _d(P)
    idx = np.ascontiguousarray(np.asarray(landmarks, dtype=np.int64))
    out = np.empty(len(P))
    rc = lib().orc_masses_rbf(_p(P), len(P), idx.ctypes.data_as(ctypes.POINTER(ctypes.c_long)), len(idx),
                              sigma, floor, _p(out))
    if rc != 0:
        raise ValueError("bad RBF arguments (%d)" % rc)
    return out


def masses_spm(P, landmarks, sigma: float = 10.0 / 16.0, floor: float = 1e-3, lattice: int = 16,
               a: float = -5.0, b: float = 5.0, total: float = 1.0, niv: bool = True):
    """Eq. 19: smooth-particle masses S = N o B (NIV weights times the RBF
    interpolant; B alone with niv=False), scaled to sum to `total`."""
    B = masses_rbf(P, landmarks, sigma, floor)
    N = masses_niv(P, lattice, a, b, 1.0) if niv else np.ones(len(B))
    S = N * B
    return total * S / S.sum()


def masses_uniform(n: int, total: float = 1.0) -> np.ndarray:
    return np.full(n, total / n)


# --------------------------------------------------------------------------- forces

def direct_acc(X, mX, Y, G: float, eps: float, want_abs: bool = False):
    """Eq. 6 divided by m_Y (gravity acceleration) for every template point."""
    X, mX, Y = _d(X), _d(mX), _d(Y)
    acc = np.empty_like(Y)
    ab = np.empty(len(Y)) if want_abs else None
    lib().orc_direct_acc(_p(X), _p(mX), len(X), _p(Y), len(Y), G, eps, _p(acc), _p(ab))
    return (acc, ab) if want_abs else acc


class Tree:
    """Barnes-Hut tree of Algorithm 1 built on ``X`` with masses ``mX``."""

    def __init__(self, X, mX, max_depth: int = 20):
        self.X, self.mX = _d(X), _d(mX)
        self._h = lib().orc_tree_build(_p(self.X), _p(self.mX), len(self.X), max_depth)
        if not self._h:
            raise ValueError("empty point set")

    def __del__(self):
        h = getattr(self, "_h", None)
        if h:
            lib().orc_tree_free(h)
            self._h = None

    def export(self):
        """Canonical node list: cells with >= 2 children, and leaves (pre-order).

        Returns dict with int arrays depth, cell (n x 3), npts, is_leaf, parent,
        float arrays mass, com (n x 3), l, and leaf_of (per point).
        """
        n = lib().orc_tree_export(self._h, 0, None, None, None)
        ints = np.zeros((n, 7), dtype=np.int64)
        dbls = np.zeros((n, 5))
        leaf_of = np.full(len(self.X), -1, dtype=np.int64)
        lib().orc_tree_export(self._h, n, _lp(ints), _p(dbls), _lp(leaf_of))
        return dict(depth=ints[:, 0], cell=ints[:, 1:4], npts=ints[:, 4], is_leaf=ints[:, 5] != 0,
                    parent=ints[:, 6], mass=dbls[:, 0], com=dbls[:, 1:4], l=dbls[:, 4],
                    leaf_of=leaf_of)

    def stats(self):
        n = ctypes.c_long()
        d = ctypes.c_int()
        lib().orc_tree_stats(self._h, ctypes.byref(n), ctypes.byref(d))
        return n.value, d.value

    def bh_acc(self, Y, G: float, eps: float, theta: float):
        """BHForce / m_Y for every template point, and per-point term counts."""
        Y = _d(Y)
        acc = np.empty_like(Y)
        cnt = np.empty(len(Y), dtype=np.int64)
        lib().orc_bh_acc(self._h, _p(Y), len(Y), G, eps, theta, _p(acc), _lp(cnt))
        return acc, cnt


# --------------------------------------------------------------------------- ODE / Kabsch

def ode_step(v, acc, mY, dt: float, eta: float):
    """Eqs. 7-10: returns (v', d)."""
    v, acc, mY = _d(v), _d(acc), _d(mY)
    vo = np.empty_like(v)
    do = np.empty_like(v)
    lib().orc_ode_step(_p(v), _p(acc), _p(mY), len(v), dt, eta, _p(vo), _p(do))
    return vo, do


def kabsch(Y, D, dim: int = 3):
    """Eqs. 14 and 16: returns (R, t, status) with status 1 for a degenerate fit
    (dim 2: the 2 x 2 fit of the x, y components, embedded as diag(R', 1))."""
    Y, D = _d(Y), _d(D)
    R = np.zeros(9)
    t = np.zeros(3)
    st = lib().orc_kabsch_d(_p(Y), _p(D), len(Y), dim, _p(R), _p(t))
    return R.reshape(3, 3), t, int(st)


# --------------------------------------------------------------------------- Algorithm 2

def register(Xn, mX, Yn, mY, params: Params, V0=None, want_traj: bool = False,
             want_v: bool = False):
    """Algorithm 2 on normalised inputs with final masses.

    Returns dict(R, t, iters, interactions, degenerate, traj?, V?).
    """
    Xn, mX, Yn, mY = _d(Xn), _d(mX), _d(Yn), _d(mY)
    V0 = None if V0 is None else _d(V0)
    R = np.zeros(9)
    t = np.zeros(3)
    iters = ctypes.c_int()
    inter = ctypes.c_long()
    traj = np.zeros((params.max_iter, 12)) if want_traj else None
    vout = np.zeros_like(Yn) if want_v else None
    cp = params._c()
    deg = lib().orc_register(_p(Xn), _p(mX), len(Xn), _p(Yn), _p(mY), len(Yn), ctypes.byref(cp),
                             _p(V0), _p(R), _p(t), ctypes.byref(iters), _p(traj),
                             ctypes.byref(inter), _p(vout))
    out = dict(R=R.reshape(3, 3), t=t, iters=iters.value, interactions=inter.value,
               degenerate=int(deg))
    if want_traj:
        out["traj"] = traj[: iters.value]
    if want_v:
        out["V"] = vout
    return out


def default_masses(Xn, Yn, params: Params):
    """Masses per the module docstring: X sums to 1 (uniform or NIV), Y mean dt."""
    if params.knn_masses:
        mX = masses_knn(Xn, params.lattice, params.dim, params.a, params.b, 1.0)
    elif params.niv_masses:
        mX = masses_niv(Xn, params.lattice, params.a, params.b, 1.0, dim=params.dim)
    else:
        mX = masses_uniform(len(Xn), 1.0)
    mY = masses_uniform(len(Yn), params.dt * len(Yn))
    return mX, mY


def register_full(X, Y, params: Params, round_to_f32: bool = True, want_traj: bool = False):
    """Normalise, assign masses, run Algorithm 2, de-normalise.

    With ``round_to_f32`` the normalised clouds and masses are rounded to
    float32 before the loop, which is the precision in which the GPU path
    stores them; the loop itself stays FP64.
    Returns dict(R, t (original frame), R_n, t_n (normalised frame), info, ...).
    """
    if params.dim == 2:
        # the plane z = 0 of the 3-D formulas: a zero coordinate never sets
        # the normalisation's extremes, and the tree does not split z
        X = embed2(X)
        Y = embed2(Y)
    Xn, Yn, info = normalize(X, Y, params.a, params.b)
    if round_to_f32:
        Xn = Xn.astype(np.float32).astype(np.float64)
        Yn = Yn.astype(np.float32).astype(np.float64)
    mX, mY = default_masses(Xn, Yn, params)
    if round_to_f32:
        mX = mX.astype(np.float32).astype(np.float64)
        mY = mY.astype(np.float32).astype(np.float64)
    out = register(Xn, mX, Yn, mY, params, want_traj=want_traj)
    out["R_n"], out["t_n"] = out["R"], out["t"]
    out["t"] = denormalize(out["R_n"], out["t_n"], info, params.a)
    out["info"] = info
    if params.dim == 2:
        out["R2"], out["t2"] = out["R"][:2, :2], out["t"][:2]
    return out


def embed2(P):
    """(n, 2) -> (n, 3) with z = 0."""
    P = _d(P)
    return np.ascontiguousarray(np.column_stack([P[:, 0], P[:, 1], np.zeros(len(P))]))


def rotation_error_deg(R1, R2) -> float:
    """Eq. 20: angle of R1^T R2 in degrees."""
    c = (np.trace(np.asarray(R1).T @ np.asarray(R2)) - 1.0) / 2.0
    return float(np.degrees(np.arccos(np.clip(c, -1.0, 1.0))))

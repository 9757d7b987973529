"""Python binding of libfga, the GB300 implementation of the FGA hot path.

Argument marshalling only: every step runs in the CUDA kernels of
``libfga.so`` (see ``include/fga.h`` for the C ABI). PyTorch provides device
memory and streams. Importing this package fails loudly if ``libfga.so`` has
not been built (``python paper_2009_14005_gb300/build.py``); there is no CPU
fallback.

The functions keep the C names:

==========================  ============================================
``fga_normalize``            Appendix A (A.1-A.3)
``fga_denormalize``          dnorm(t) of the Appendix (host arithmetic)
``fga_masses``               Sec. IV-F, uniform or NIV (Eq. 18)
``fga_tree_build``           Algorithm 1 -> :class:`Tree`
``fga_forces``               Eq. 6 (all pairs) or BHForce (Eq. 15)
``fga_state_create``         Algorithm 2 state -> :class:`State`
``fga_step`` / ``fga_state_get`` / ``fga_state_trajectory``
``fga_register``             Algorithm 2 end to end (host or device inputs)
==========================  ============================================
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libfga.so")

FGA_OK = 0
FGA_EINVAL = -1
FGA_ENOMEM = -2
FGA_ECUDA = -3
FGA_EDEGENERATE = -4
FGA_EINTERNAL = -5

FGA_DIRECT = 0
FGA_BH = 1
FGA_AUTO = 2
FGA_WALK_AUTO = 0  # Barnes-Hut walk by template size
FGA_WALK_LANE = 1  # one walk per template point
FGA_WALK_COOP = 2  # one walk per 64 template points
FGA_WALK_CURSOR = 3  # one walk per 64 points following each point's own walk
FGA_WALK_CURSOR32 = 4  # the same, 32 points per warp
FGA_WALK_CURSOR128 = 5  # the same, 128 points per warp
FGA_VEL_UNCONSTRAINED = 0
FGA_VEL_RIGID = 1
FGA_MASS_UNIFORM = 0
FGA_MASS_NIV = 1
FGA_MASS_RBF = 2
FGA_MASS_SPM = 3
FGA_MASS_KNN = 4
FGA_MAX_LANDMARKS = 512

SYMBOLS = [
    "fga_params_default", "fga_last_error", "fga_launch_count", "fga_normalize",
    "fga_denormalize", "fga_masses", "fga_tree_build", "fga_tree_destroy",
    "fga_tree_node_count", "fga_tree_export", "fga_tree_preorder", "fga_forces", "fga_state_create", "fga_step",
    "fga_state_get", "fga_state_trajectory", "fga_state_destroy", "fga_register",
    "fga_forces_direct_static", "fga_register_batch", "fga_direct_max_n",
    "fga_server_create", "fga_server_submit", "fga_server_poll", "fga_server_stats_get",
    "fga_server_destroy", "fga_autotune", "fga_set_direct_tile", "fga_get_direct_tile",
    "fga_masses_landmarks", "fga_forces_terms", "fga_rigid_fit",
]
FGA_STATIC_SCRATCH_FLOAT4 = 524288
FGA_STATIC_STATE_FLOAT4 = 33


class fga_params(ctypes.Structure):
    _fields_ = [("G", ctypes.c_float), ("eps", ctypes.c_float), ("eta", ctypes.c_float),
                ("dt", ctypes.c_float), ("theta", ctypes.c_float), ("max_iter", ctypes.c_int),
                ("conv_tol", ctypes.c_float), ("method", ctypes.c_int),
                ("normalize", ctypes.c_int), ("a", ctypes.c_float), ("b", ctypes.c_float),
                ("velocity_mode", ctypes.c_int), ("max_depth", ctypes.c_int),
                ("mass_mode", ctypes.c_int), ("lattice", ctypes.c_int),
                ("profile", ctypes.c_int), ("dim", ctypes.c_int),
                ("bh_walk", ctypes.c_int)]


class fga_stats(ctypes.Structure):
    _fields_ = [("iterations", ctypes.c_int), ("converged", ctypes.c_int),
                ("degenerate_fits", ctypes.c_int), ("status", ctypes.c_int),
                ("interactions", ctypes.c_int64), ("last_conv", ctypes.c_double),
                ("net_force", ctypes.c_double * 3), ("torque", ctypes.c_double * 3),
                ("R_norm", ctypes.c_double * 9), ("t_norm", ctypes.c_double * 3),
                ("norm_info", ctypes.c_double * 8), ("elapsed_ms", ctypes.c_double),
                ("force_ms", ctypes.c_double), ("force_launches", ctypes.c_int),
                ("h2d_bytes", ctypes.c_int64), ("d2h_bytes", ctypes.c_int64)]

    def to_dict(self):
        return dict(iterations=self.iterations, converged=bool(self.converged),
                    degenerate_fits=self.degenerate_fits, status=self.status,
                    interactions=int(self.interactions), last_conv=self.last_conv,
                    net_force=np.array(self.net_force[:]), torque=np.array(self.torque[:]),
                    R_norm=np.array(self.R_norm[:]).reshape(3, 3), t_norm=np.array(self.t_norm[:]),
                    norm_info=np.array(self.norm_info[:]), elapsed_ms=self.elapsed_ms,
                    force_ms=self.force_ms, force_launches=self.force_launches,
                    h2d_bytes=int(self.h2d_bytes), d2h_bytes=int(self.d2h_bytes))


class fga_pair(ctypes.Structure):
    _fields_ = [("X", ctypes.c_void_p), ("N", ctypes.c_int64), ("Y", ctypes.c_void_p),
                ("M", ctypes.c_int64), ("mX", ctypes.c_void_p), ("mY", ctypes.c_void_p),
                ("params", ctypes.c_void_p)]


class fga_pair_result(ctypes.Structure):
    _fields_ = [("R", ctypes.c_double * 9), ("t", ctypes.c_double * 3), ("method", ctypes.c_int),
                ("iterations", ctypes.c_int), ("converged", ctypes.c_int), ("status", ctypes.c_int),
                ("interactions", ctypes.c_int64)]


class fga_server_config(ctypes.Structure):
    _fields_ = [("mem_budget", ctypes.c_int64), ("max_pairs", ctypes.c_int),
                ("iters_per_tick", ctypes.c_int), ("device", ctypes.c_int),
                ("max_work", ctypes.c_double), ("prep_threads", ctypes.c_int)]


class fga_served(ctypes.Structure):
    _fields_ = [("ticket", ctypes.c_int64), ("result", fga_pair_result),
                ("submit_ms", ctypes.c_double), ("admit_ms", ctypes.c_double),
                ("start_ms", ctypes.c_double), ("done_ms", ctypes.c_double),
                ("error", ctypes.c_char * 160)]


class fga_server_stats(ctypes.Structure):
    _fields_ = [("submitted", ctypes.c_int64), ("completed", ctypes.c_int64),
                ("failed", ctypes.c_int64), ("pending", ctypes.c_int), ("preparing", ctypes.c_int),
                ("resident", ctypes.c_int), ("bytes_charged", ctypes.c_int64),
                ("work_admitted", ctypes.c_double),
                ("mem_budget", ctypes.c_int64), ("ticks", ctypes.c_int64),
                ("pair_iterations", ctypes.c_int64), ("busy_ms", ctypes.c_double)]

    def to_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


FGA_TUNE_DIRECT_TILES, FGA_TUNE_CROSSOVER, FGA_TUNE_ALL, FGA_TUNE_NSIZES = 1, 2, 3, 7


class fga_tune_report(ctypes.Structure):
    _fields_ = [("direct_bs", ctypes.c_int * 3), ("direct_qpt", ctypes.c_int * 3),
                ("direct_gips", ctypes.c_double * 3), ("direct_max_n", ctypes.c_int64),
                ("sizes", ctypes.c_int64 * FGA_TUNE_NSIZES),
                ("direct_us_per_point", ctypes.c_double * FGA_TUNE_NSIZES),
                ("bh_us_per_point", ctypes.c_double * FGA_TUNE_NSIZES),
                ("bh_build_ms", ctypes.c_double * FGA_TUNE_NSIZES), ("elapsed_ms", ctypes.c_double)]

    def to_dict(self):
        d = {}
        for k, _ in self._fields_:
            v = getattr(self, k)
            d[k] = list(v) if hasattr(v, "__len__") else v
        return d


class FGAError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__("libfga error %d: %s" % (code, msg))
        self.code = code


def _load():
    if not os.path.exists(LIB_PATH):
        raise ImportError("libfga.so is not built; run `python paper_2009_14005_gb300/build.py` "
                          "(there is no CPU fallback)")
    lib = ctypes.CDLL(LIB_PATH)
    P, I64, VP, F, D = ctypes.c_void_p, ctypes.c_int64, ctypes.c_void_p, ctypes.c_float, ctypes.c_double
    PP = ctypes.POINTER(fga_params)
    DP = ctypes.POINTER(ctypes.c_double)
    sig = {
        "fga_params_default": (None, [PP]),
        "fga_last_error": (ctypes.c_char_p, []),
        "fga_launch_count": (I64, []),
        "fga_normalize": (ctypes.c_int, [P, I64, P, I64, F, F, P, P, DP, VP]),
        "fga_denormalize": (None, [DP, DP, DP, F, DP]),
        "fga_masses": (ctypes.c_int, [P, I64, ctypes.c_int, ctypes.c_int, F, F, D, P, VP]),
        "fga_tree_build": (ctypes.c_int, [P, P, I64, PP, ctypes.POINTER(ctypes.c_void_p), VP]),
        "fga_tree_destroy": (None, [P]),
        "fga_tree_node_count": (I64, [P]),
        "fga_tree_export": (I64, [P, I64, P, P, P, VP]),
        "fga_tree_preorder": (I64, [P, I64, P, VP]),
        "fga_forces": (ctypes.c_int, [P, P, P, I64, P, P, I64, PP, P, ctypes.POINTER(I64), VP]),
        "fga_forces_terms": (ctypes.c_int, [P, P, P, I64, PP, P, P, VP]),
        "fga_state_create": (ctypes.c_int, [P, P, I64, P, P, I64, P, PP,
                                            ctypes.POINTER(ctypes.c_void_p), VP]),
        "fga_step": (ctypes.c_int, [P, ctypes.c_int, VP]),
        "fga_state_get": (ctypes.c_int, [P, DP, DP, ctypes.POINTER(fga_stats), VP]),
        "fga_state_trajectory": (ctypes.c_int, [P, DP, ctypes.c_int, VP]),
        "fga_state_destroy": (None, [P]),
        "fga_register": (ctypes.c_int, [P, I64, P, I64, P, P, PP, DP, DP,
                                        ctypes.POINTER(fga_stats), VP]),
        "fga_forces_direct_static": (ctypes.c_int, [P, P, I64, P, P, I64, PP, P, VP]),
        "fga_rigid_fit": (ctypes.c_int, [DP, I64, DP, ctypes.c_int, DP, DP, VP]),
        "fga_register_batch": (ctypes.c_int, [ctypes.POINTER(fga_pair), ctypes.c_int, PP,
                                              ctypes.POINTER(fga_pair_result),
                                              ctypes.POINTER(fga_stats), VP]),
        "fga_direct_max_n": (I64, [I64]),
        "fga_server_create": (ctypes.c_int, [PP, ctypes.POINTER(fga_server_config),
                                             ctypes.POINTER(ctypes.c_void_p)]),
        "fga_server_submit": (ctypes.c_int, [P, ctypes.POINTER(fga_pair), ctypes.POINTER(I64)]),
        "fga_server_poll": (ctypes.c_int, [P, ctypes.POINTER(fga_served), ctypes.c_int,
                                           ctypes.POINTER(ctypes.c_int), ctypes.c_int]),
        "fga_server_stats_get": (ctypes.c_int, [P, ctypes.POINTER(fga_server_stats)]),
        "fga_server_destroy": (ctypes.c_int, [P]),
        "fga_autotune": (ctypes.c_int, [PP, ctypes.c_int, VP, ctypes.POINTER(fga_tune_report)]),
        "fga_masses_landmarks": (ctypes.c_int, [P, I64, P, ctypes.c_int, F, F, ctypes.c_int, ctypes.c_int,
                                                F, F, D, P, VP]),
        "fga_set_direct_tile": (ctypes.c_int, [ctypes.c_int, ctypes.c_int, ctypes.c_int]),
        "fga_get_direct_tile": (ctypes.c_int, [ctypes.c_int, ctypes.POINTER(ctypes.c_int),
                                               ctypes.POINTER(ctypes.c_int)]),
    }
    for name, (res, args) in sig.items():
        f = getattr(lib, name)
        f.restype = res
        f.argtypes = args
    return lib


lib = _load()


def _err(code):
    if code != FGA_OK:
        raise FGAError(code, lib.fga_last_error().decode())


def last_error() -> str:
    return lib.fga_last_error().decode()


def fga_launch_count() -> int:
    return int(lib.fga_launch_count())


def params(**kw) -> fga_params:
    """fga_params with the paper's defaults (``fga_params_default``) and overrides."""
    p = fga_params()
    lib.fga_params_default(ctypes.byref(p))
    for k, v in kw.items():
        if not hasattr(p, k):
            raise AttributeError(k)
        setattr(p, k, v)
    return p


# --------------------------------------------------------------------------- marshalling

def _torch():
    import torch
    return torch


def _stream(stream):
    if stream is None:
        return ctypes.c_void_p(_torch().cuda.current_stream().cuda_stream)
    if isinstance(stream, int):
        return ctypes.c_void_p(stream)
    return ctypes.c_void_p(stream.cuda_stream)


def _dev(t, cols=None, name="tensor"):
    """Contiguous float32 CUDA tensor (no copy if it already is one)."""
    torch = _torch()
    if t is None:
        return None
    if not isinstance(t, torch.Tensor):
        t = torch.as_tensor(np.asarray(t, dtype=np.float32))
    if not t.is_cuda:
        t = t.to("cuda")
    t = t.to(torch.float32).contiguous()
    if cols is not None and (t.dim() != 2 or t.shape[1] != cols):
        raise ValueError("%s must have shape (n, %d)" % (name, cols))
    return t


def _ptr(t):
    return None if t is None else ctypes.c_void_p(t.data_ptr())


def _d(a, n):
    return np.ascontiguousarray(np.asarray(a, dtype=np.float64).reshape(n))


def _dp(a):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


# --------------------------------------------------------------------------- Appendix A

def fga_normalize(X, Y, a: float = -5.0, b: float = 5.0, stream=None):
    torch = _torch()
    X, Y = _dev(X, 3, "X"), _dev(Y, 3, "Y")
    Xn, Yn = torch.empty_like(X), torch.empty_like(Y)
    info = np.zeros(8)
    _err(lib.fga_normalize(_ptr(X), X.shape[0], _ptr(Y), Y.shape[0], a, b, _ptr(Xn), _ptr(Yn),
                           _dp(info), _stream(stream)))
    return Xn, Yn, info


def fga_denormalize(R, t_norm, info, a: float = -5.0):
    R, t_norm, info = _d(R, 9), _d(t_norm, 3), _d(info, 8)
    out = np.zeros(3)
    lib.fga_denormalize(_dp(R), _dp(t_norm), _dp(info), a, _dp(out))
    return out


def fga_masses(pts, mode: int = FGA_MASS_UNIFORM, lattice: int = 16, a: float = -5.0,
               b: float = 5.0, total: float = 1.0, stream=None):
    torch = _torch()
    pts = _dev(pts, 3, "pts")
    out = torch.empty(pts.shape[0], dtype=torch.float32, device=pts.device)
    _err(lib.fga_masses(_ptr(pts), pts.shape[0], mode, lattice, a, b, total, _ptr(out),
                        _stream(stream)))
    return out


def fga_masses_landmarks(pts, landmarks, mode: int = FGA_MASS_SPM, sigma: float = 0.625,
                         floor: float = 1e-3, lattice: int = 16, a: float = -5.0, b: float = 5.0,
                         total: float = 1.0, stream=None):
    """Eq. 17 (mode FGA_MASS_RBF) or Eq. 19 (FGA_MASS_SPM) masses from landmark
    point indices; see fga_masses_landmarks in fga.h."""
    torch = _torch()
    pts = _dev(pts, 3, "pts")
    idx = np.ascontiguousarray(np.asarray(landmarks, dtype=np.int64).reshape(-1))
    out = torch.empty(pts.shape[0], dtype=torch.float32, device=pts.device)
    _err(lib.fga_masses_landmarks(_ptr(pts), pts.shape[0], idx.ctypes.data if len(idx) else None, len(idx),
                                  sigma, floor, mode, lattice, a, b, total, _ptr(out), _stream(stream)))
    return out


# --------------------------------------------------------------------------- Algorithm 1

class Tree:
    """Owner of an ``fga_tree`` handle (freed with fga_tree_destroy)."""

    def __init__(self, handle, n):
        self._h = handle
        self.N = n

    @property
    def handle(self):
        return self._h

    def node_count(self) -> int:
        return int(lib.fga_tree_node_count(self._h))

    def export(self, stream=None):
        n = self.node_count()
        ints = np.zeros((n, 7), dtype=np.int64)
        dbls = np.zeros((n, 5))
        leaf_of = np.full(self.N, -1, dtype=np.int64)
        got = lib.fga_tree_export(self._h, n, ints.ctypes.data_as(ctypes.c_void_p),
                                  dbls.ctypes.data_as(ctypes.c_void_p),
                                  leaf_of.ctypes.data_as(ctypes.c_void_p), _stream(stream))
        if got < 0:
            _err(int(got))
        return dict(depth=ints[:, 0], cell=ints[:, 1:4], npts=ints[:, 4], is_leaf=ints[:, 5] != 0,
                    parent=ints[:, 6], mass=dbls[:, 0], com=dbls[:, 1:4], l=dbls[:, 4],
                    leaf_of=leaf_of)

    def preorder(self, stream=None):
        """The walk's depth-first records: dict of com (n x 3), mass, l2 and the
        int fields size (subtree record count), count, first."""
        n = int(lib.fga_tree_preorder(self._h, 0, None, _stream(stream)))
        if n < 0:
            _err(n)
        rec = np.zeros((n, 8), dtype=np.float32)
        got = lib.fga_tree_preorder(self._h, n, rec.ctypes.data_as(ctypes.c_void_p), _stream(stream))
        if got < 0:
            _err(int(got))
        bits = rec.view(np.int32)
        return dict(com=rec[:, 0:3], mass=rec[:, 3], l2=rec[:, 4], size=bits[:, 5].copy(),
                    count=bits[:, 6].copy(), first=bits[:, 7].copy())

    def close(self):
        if self._h:
            lib.fga_tree_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def fga_tree_build(X, mX=None, p: fga_params | None = None, stream=None) -> Tree:
    p = p or params()
    X = _dev(X, 3, "X")
    mX = _dev(mX) if mX is not None else None
    h = ctypes.c_void_p()
    _err(lib.fga_tree_build(_ptr(X), _ptr(mX), X.shape[0], ctypes.byref(p), ctypes.byref(h),
                            _stream(stream)))
    return Tree(h, X.shape[0])


# --------------------------------------------------------------------------- Eq. 6 / BHForce

def fga_forces(tree, X, mX, Y, mY=None, p: fga_params | None = None, want_count: bool = False,
               stream=None):
    """Eq. 6 per template point; tree=None -> all pairs, else BHForce on ``tree``."""
    torch = _torch()
    p = p or params()
    Y = _dev(Y, 3, "Y")
    X = _dev(X, 3, "X") if X is not None else None
    mX = _dev(mX) if mX is not None else None
    mY = _dev(mY) if mY is not None else None
    out = torch.empty_like(Y)
    cnt = ctypes.c_int64(0)
    N = X.shape[0] if X is not None else 0
    _err(lib.fga_forces(tree.handle if tree is not None else None, _ptr(X), _ptr(mX), N, _ptr(Y),
                        _ptr(mY), Y.shape[0], ctypes.byref(p), _ptr(out),
                        ctypes.byref(cnt) if want_count else None, _stream(stream)))
    return (out, int(cnt.value)) if want_count else out


def fga_forces_terms(tree, Y, mY=None, p: fga_params | None = None, stream=None):
    """BHForce on ``tree`` and each template point's term count (int32, Y's order)."""
    torch = _torch()
    p = p or params()
    Y = _dev(Y, 3, "Y")
    mY = _dev(mY) if mY is not None else None
    out = torch.empty_like(Y)
    terms = torch.empty(Y.shape[0], dtype=torch.int32, device=Y.device)
    _err(lib.fga_forces_terms(tree.handle, _ptr(Y), _ptr(mY), Y.shape[0], ctypes.byref(p), _ptr(out),
                              _ptr(terms), _stream(stream)))
    return out, terms


def fga_forces_direct_static(X, mX, Y, mY=None, p: fga_params | None = None, out=None,
                             stream=None):
    """All-pairs forces like ``fga_forces(None, ...)`` but without any device
    allocation inside the library (for callers that must not allocate): the
    intermediates live in a fixed 8 MiB device array; pass ``out`` to avoid the
    one allocation this wrapper would otherwise make for the result."""
    torch = _torch()
    p = p or params()
    X, Y = _dev(X, 3, "X"), _dev(Y, 3, "Y")
    mX = _dev(mX) if mX is not None else None
    mY = _dev(mY) if mY is not None else None
    out = torch.empty_like(Y) if out is None else out
    _err(lib.fga_forces_direct_static(_ptr(X), _ptr(mX), X.shape[0], _ptr(Y), _ptr(mY), Y.shape[0],
                                      ctypes.byref(p), _ptr(out), _stream(stream)))
    return out


# --------------------------------------------------------------------------- Algorithm 2

class State:
    """Owner of an ``fga_state`` handle; keeps its tree and inputs alive."""

    def __init__(self, handle, keep):
        self._h = handle
        self._keep = keep

    @property
    def handle(self):
        return self._h

    def step(self, n_iter: int, stream=None):
        fga_step(self, n_iter, stream)

    def get(self, stream=None):
        return fga_state_get(self, stream)

    def trajectory(self, n: int, stream=None):
        return fga_state_trajectory(self, n, stream)

    def close(self):
        if self._h:
            lib.fga_state_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def fga_state_create(Xn, mX, Yn, mY, p: fga_params, tree: Tree | None = None, stream=None) -> State:
    Xn, Yn = _dev(Xn, 3, "Xn"), _dev(Yn, 3, "Yn")
    mX = _dev(mX) if mX is not None else None
    mY = _dev(mY) if mY is not None else None
    h = ctypes.c_void_p()
    _err(lib.fga_state_create(_ptr(Xn), _ptr(mX), Xn.shape[0], _ptr(Yn), _ptr(mY), Yn.shape[0],
                              tree.handle if tree is not None else None, ctypes.byref(p),
                              ctypes.byref(h), _stream(stream)))
    return State(h, (tree, Xn, Yn, mX, mY))


def fga_step(state: State, n_iter: int, stream=None):
    _err(lib.fga_step(state.handle, int(n_iter), _stream(stream)))


def fga_state_get(state: State, stream=None):
    """Returns (R, t, stats-dict) in the normalised frame; stats['status'] has the code."""
    R = np.zeros(9)
    t = np.zeros(3)
    st = fga_stats()
    code = lib.fga_state_get(state.handle, _dp(R), _dp(t), ctypes.byref(st), _stream(stream))
    if code not in (FGA_OK, FGA_EDEGENERATE):
        _err(code)
    return R.reshape(3, 3), t, st.to_dict()


def fga_state_trajectory(state: State, n: int, stream=None):
    out = np.zeros((max(n, 0), 12))
    rows = lib.fga_state_trajectory(state.handle, _dp(out), int(n), _stream(stream))
    if rows < 0:
        _err(rows)
    return out[:rows]


def fga_rigid_fit(red, M: int, mu0, dim: int = 3, stream=None):
    """One rigid fit (Eqs. 14, 16) on the device from the 27 reduced sums
    (see include/fga.h); returns (R', t', status)."""
    red = np.ascontiguousarray(np.asarray(red, dtype=np.float64))
    mu0 = np.ascontiguousarray(np.asarray(mu0, dtype=np.float64))
    if red.shape != (27,) or mu0.shape != (3,):
        raise ValueError("fga_rigid_fit: red must hold 27 values and mu0 3")
    R = np.zeros(9)
    t = np.zeros(3)
    code = lib.fga_rigid_fit(_dp(red), int(M), _dp(mu0), int(dim), _dp(R), _dp(t), _stream(stream))
    if code not in (FGA_OK, FGA_EDEGENERATE):
        _err(code)
    return R.reshape(3, 3), t, code


def fga_register(X, Y, p: fga_params | None = None, mX=None, mY=None, stream=None):
    """Whole registration. X, Y (and masses) may be CUDA tensors or host arrays
    (numpy / CPU tensors; copied to the device inside the C call).
    Returns (R, t, stats-dict) with X ~ R Y + t in the original frames."""
    torch = _torch()
    p = p or params()

    def host_or_dev(a, cols):
        if a is None:
            return None
        if isinstance(a, torch.Tensor):
            if a.is_cuda:
                return _dev(a, cols)
            return a.to(torch.float32).contiguous()
        t = torch.from_numpy(np.ascontiguousarray(np.asarray(a, dtype=np.float32)))
        return t

    cols = 2 if p.dim == 2 else 3
    Xa, Ya = host_or_dev(X, cols), host_or_dev(Y, cols)
    mXa, mYa = host_or_dev(mX, None), host_or_dev(mY, None)
    R = np.zeros(9)
    t = np.zeros(3)
    st = fga_stats()
    code = lib.fga_register(_ptr(Xa), Xa.shape[0], _ptr(Ya), Ya.shape[0], _ptr(mXa), _ptr(mYa),
                            ctypes.byref(p), _dp(R), _dp(t), ctypes.byref(st), _stream(stream))
    if code not in (FGA_OK, FGA_EDEGENERATE):
        _err(code)
    d = st.to_dict()
    d["status"] = code
    return R.reshape(3, 3), t, d


def fga_direct_max_n(new_value: int = 0) -> int:
    """FGA_AUTO crossover: returns the current N limit of the all-pairs sum, sets it if > 0."""
    return int(lib.fga_direct_max_n(int(new_value)))


def fga_register_batch(pairs, p: fga_params | None = None, stream=None):
    """Register many (X, Y) pairs together (one graph-captured loop for all).

    ``pairs``: list of (X, Y), (X, Y, mX, mY) or (X, Y, mX, mY, params) where
    params (an ``fga_params``, or None) replaces ``p`` for that pair, e.g. one
    cell of a parameter grid; arrays may be CUDA tensors or host arrays.
    Returns (list of dicts with R, t, method, iterations, converged, status,
    interactions; stats dict)."""
    torch = _torch()
    p = p or params()
    keep = []

    def arr(a, cols):
        if a is None:
            return None
        if isinstance(a, torch.Tensor):
            t = _dev(a, cols) if a.is_cuda else a.to(torch.float32).contiguous()
        else:
            t = torch.from_numpy(np.ascontiguousarray(np.asarray(a, dtype=np.float32)))
        keep.append(t)
        return t

    n = len(pairs)
    cp = (fga_pair * n)()
    for k, pr in enumerate(pairs):
        X, Y = pr[0], pr[1]
        mX = pr[2] if len(pr) > 2 else None
        mY = pr[3] if len(pr) > 3 else None
        pk = pr[4] if len(pr) > 4 else None
        cols = 2 if (pk if pk is not None else p).dim == 2 else 3
        Xt, Yt, mXt, mYt = arr(X, cols), arr(Y, cols), arr(mX, None), arr(mY, None)
        if pk is not None:
            keep.append(pk)
        cp[k] = fga_pair(Xt.data_ptr(), Xt.shape[0], Yt.data_ptr(), Yt.shape[0],
                         mXt.data_ptr() if mXt is not None else None,
                         mYt.data_ptr() if mYt is not None else None,
                         ctypes.addressof(pk) if pk is not None else None)
    res = (fga_pair_result * n)()
    st = fga_stats()
    code = lib.fga_register_batch(cp, n, ctypes.byref(p), res, ctypes.byref(st), _stream(stream))
    if code not in (FGA_OK, FGA_EDEGENERATE):
        _err(code)
    out = [dict(R=np.array(r.R[:]).reshape(3, 3), t=np.array(r.t[:]), method=r.method,
                iterations=r.iterations, converged=bool(r.converged), status=r.status,
                interactions=int(r.interactions)) for r in res]
    d = st.to_dict()
    d["status"] = code
    return out, d


def autotune(p: fga_params | None = None, flags: int = FGA_TUNE_ALL, stream=None) -> dict:
    """Measures and installs the all-pairs tiles and the FGA_AUTO crossover
    (``fga_autotune``); returns the report as a dict."""
    rep = fga_tune_report()
    _err(lib.fga_autotune(ctypes.byref(p) if p is not None else None, int(flags), _stream(stream),
                          ctypes.byref(rep)))
    return rep.to_dict()


def set_direct_tile(size_class: int, bs: int, qpt: int):
    _err(lib.fga_set_direct_tile(int(size_class), int(bs), int(qpt)))


def get_direct_tile(size_class: int):
    bs, q = ctypes.c_int(), ctypes.c_int()
    _err(lib.fga_get_direct_tile(int(size_class), ctypes.byref(bs), ctypes.byref(q)))
    return bs.value, q.value


def _served_dict(o: fga_served) -> dict:
    r = o.result
    return dict(ticket=int(o.ticket), R=np.array(r.R[:]).reshape(3, 3), t=np.array(r.t[:]),
                method=r.method, iterations=r.iterations, converged=bool(r.converged),
                status=r.status, interactions=int(r.interactions), submit_ms=o.submit_ms,
                admit_ms=o.admit_ms, start_ms=o.start_ms, done_ms=o.done_ms,
                error=o.error.decode(errors="replace"))


class Server:
    """Registration server (``fga_server_*``): continuous batching on one GPU.

    ``submit(X, Y, mX=None, mY=None)`` returns a ticket; the arrays (CUDA
    tensors or host arrays) are held until the request's result is polled.
    ``poll(max=256, wait_ms=0)`` returns finished requests as dicts (ticket,
    R, t, method, iterations, converged, status, interactions, and the host
    times submit_ms, admit_ms, start_ms, done_ms in ms since creation)."""

    def __init__(self, p: fga_params | None = None, mem_budget: int = 0, max_pairs: int = 0,
                 iters_per_tick: int = 0, device: int = -1, max_work: float = 0.0,
                 prep_threads: int = 0):
        self._h = ctypes.c_void_p()
        self._p = p or params()
        cfg = fga_server_config(int(mem_budget), int(max_pairs), int(iters_per_tick), int(device),
                                float(max_work), int(prep_threads))
        _err(lib.fga_server_create(ctypes.byref(self._p), ctypes.byref(cfg), ctypes.byref(self._h)))
        self._keep = {}

    def submit(self, X, Y, mX=None, mY=None, params: fga_params | None = None) -> int:
        torch = _torch()
        held = []

        def arr(a, cols):
            if a is None:
                return None
            if isinstance(a, torch.Tensor):
                t = _dev(a, cols) if a.is_cuda else a.to(torch.float32).contiguous()
            else:
                t = torch.from_numpy(np.ascontiguousarray(np.asarray(a, dtype=np.float32)))
            held.append(t)
            return t

        cols = 2 if (params if params is not None else self._p).dim == 2 else 3
        Xt, Yt, mXt, mYt = arr(X, cols), arr(Y, cols), arr(mX, None), arr(mY, None)
        if any(t.is_cuda for t in held):
            # the server reads device inputs on its own stream: they must be complete
            torch.cuda.current_stream(Xt.device if Xt.is_cuda else Yt.device).synchronize()
        q = fga_pair(Xt.data_ptr(), Xt.shape[0], Yt.data_ptr(), Yt.shape[0],
                     mXt.data_ptr() if mXt is not None else None,
                     mYt.data_ptr() if mYt is not None else None,
                     ctypes.addressof(params) if params is not None else None)
        ticket = ctypes.c_int64()
        _err(lib.fga_server_submit(self._h, ctypes.byref(q), ctypes.byref(ticket)))
        self._keep[int(ticket.value)] = held
        return int(ticket.value)

    def poll(self, max: int = 256, wait_ms: int = 0) -> list:
        out = (fga_served * max)()
        n = ctypes.c_int()
        _err(lib.fga_server_poll(self._h, out, max, ctypes.byref(n), int(wait_ms)))
        res = [_served_dict(out[k]) for k in range(n.value)]
        for r in res:
            self._keep.pop(r["ticket"], None)
        return res

    def drain(self, wait_ms: int = -1) -> list:
        """All results of the requests submitted so far (waits for them)."""
        res = []
        while True:
            got = self.poll(256, wait_ms)
            if not got:
                return res
            res.extend(got)

    def stats(self) -> dict:
        st = fga_server_stats()
        _err(lib.fga_server_stats_get(self._h, ctypes.byref(st)))
        return st.to_dict()

    def close(self):
        if self._h:
            lib.fga_server_destroy(self._h)
            self._h = ctypes.c_void_p()
            self._keep.clear()

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

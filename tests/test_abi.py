"""The C-ABI library loads and exports what include/fga.h declares (no GPU needed)."""
import ctypes
import os
import re

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "fga.h")


def _declared():
    src = open(HEADER).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(fga_[a-z_]+)\s*\(", src)))


@pytest.fixture(scope="module")
def fga():
    import __graft_entry__
    __graft_entry__.build_library()
    import paper_2009_14005_gb300 as m
    return m


def test_every_declared_symbol_is_exported(fga):
    lib = ctypes.CDLL(fga.LIB_PATH)
    declared = _declared()
    assert len(declared) >= 15
    for name in declared:
        assert hasattr(lib, name), name
    assert sorted(fga.SYMBOLS) == declared


def test_defaults_are_the_papers(fga):
    p = fga.params()
    assert p.G == pytest.approx(66.7) and p.eps == pytest.approx(0.2) and p.eta == pytest.approx(0.2)
    assert p.dt == pytest.approx(0.1) and p.theta == pytest.approx(0.6)
    assert (p.a, p.b, p.max_depth, p.lattice) == (-5.0, 5.0, 20, 16)


def test_host_denormalize_matches_oracle(fga, orc):
    import synth
    rng = np.random.default_rng(0)
    X = rng.normal(size=(50, 3)) * 3 + 1
    Y = rng.normal(size=(40, 3)) - 2
    _, _, info = orc.normalize(X, Y, -5.0, 5.0)
    R = synth.random_rotation(rng, 120)
    t = rng.normal(size=3)
    np.testing.assert_allclose(fga.fga_denormalize(R, t, info, -5.0),
                               orc.denormalize(R, t, info, -5.0), rtol=1e-14, atol=1e-14)


def test_errors_without_gpu_work(fga):
    # argument checks happen before any device call
    R, t = (ctypes.c_double * 9)(), (ctypes.c_double * 3)()
    code = fga.lib.fga_register(None, 0, None, 0, None, None, ctypes.byref(fga.params()), R, t,
                                None, None)
    assert code == fga.FGA_EINVAL
    assert "bad arguments" in fga.last_error()
    code = fga.lib.fga_state_create(None, None, 0, None, None, 0, None, ctypes.byref(fga.params()),
                                    ctypes.byref(ctypes.c_void_p()), None)
    assert code == fga.FGA_EINVAL


def test_params_struct_matches_the_header(fga):
    # fga_params_default fills every field, the last one included
    p = fga.params()
    assert p.dim == 3 and p.bh_walk == fga.FGA_WALK_AUTO
    assert ctypes.sizeof(fga.fga_params) == 4 * len(fga.fga_params._fields_)


def test_bad_walk_is_rejected_without_gpu_work(fga):
    X = np.zeros((8, 3), dtype=np.float32)
    R, t = (ctypes.c_double * 9)(), (ctypes.c_double * 3)()
    p = fga.params(bh_walk=7)
    code = fga.lib.fga_register(X.ctypes.data, 8, X.ctypes.data, 8, None, None, ctypes.byref(p), R, t,
                                None, None)
    assert code == fga.FGA_EINVAL
    assert "bh_walk" in fga.lib.fga_last_error().decode()


def test_sizes_above_the_limits_are_rejected_without_gpu_work(fga):
    X = np.zeros((8, 3), dtype=np.float32)
    R, t = (ctypes.c_double * 9)(), (ctypes.c_double * 3)()
    p = fga.params()
    code = fga.lib.fga_register(X.ctypes.data, (1 << 30) + 1, X.ctypes.data, 8, None, None,
                                ctypes.byref(p), R, t, None, None)
    assert code == fga.FGA_EINVAL
    out = ctypes.c_void_p()
    code = fga.lib.fga_tree_build(X.ctypes.data, None, (1 << 26) + 1, ctypes.byref(p), ctypes.byref(out), None)
    assert code == fga.FGA_EINVAL and "2^26" in fga.lib.fga_last_error().decode()


def test_batch_masses_and_forces_reject_bad_arguments_without_gpu_work(fga):
    X = np.zeros((64, 3), dtype=np.float32)
    res = (fga.fga_pair_result * 2)()
    good = fga.fga_pair(X.ctypes.data, 64, X.ctypes.data, 64, None, None, None)
    big = fga.fga_pair(X.ctypes.data, (1 << 26) + 1, X.ctypes.data, 64, None, None, None)
    bad_p = fga.params(bh_walk=9)
    per_pair = fga.fga_pair(X.ctypes.data, 64, X.ctypes.data, 64, None, None, ctypes.addressof(bad_p))
    p = fga.params()
    for pairs, needle in (([good, big], "pair 1"), ([per_pair, good], "pair 0")):
        arr = (fga.fga_pair * 2)(*pairs)
        code = fga.lib.fga_register_batch(arr, 2, ctypes.byref(p), res, None, None)
        assert code == fga.FGA_EINVAL and needle in fga.lib.fga_last_error().decode()
    out = np.zeros(64, dtype=np.float32)
    for mode, lattice, total in ((fga.FGA_MASS_NIV, 0, 1.0), (fga.FGA_MASS_KNN, 12, 1.0),
                                 (fga.FGA_MASS_UNIFORM, 16, 0.0), (7, 16, 1.0)):
        code = fga.lib.fga_masses(X.ctypes.data, 64, mode, lattice, -5.0, 5.0, total, out.ctypes.data, None)
        assert code == fga.FGA_EINVAL
    acc = np.zeros((64, 3), dtype=np.float32)
    for kw in (dict(eps=0.0), dict(theta=-1.0)):
        q = fga.params(**kw)
        code = fga.lib.fga_forces(None, X.ctypes.data, None, 64, X.ctypes.data, None, 64, ctypes.byref(q),
                                  acc.ctypes.data, None, None)
        assert code == fga.FGA_EINVAL


def test_host_tables_round_trip(fga):
    # the all-pairs tile table and the FGA_AUTO crossover are host state
    saved = [fga.get_direct_tile(c) for c in range(3)]
    old_n = fga.fga_direct_max_n(0)
    try:
        for c, (bs, q) in enumerate([(128, 4), (256, 1), (256, 2)]):
            fga.set_direct_tile(c, bs, q)
            assert fga.get_direct_tile(c) == (bs, q)
        for bad in ((3, 128, 2), (0, 64, 2), (1, 256, 3), (-1, 128, 1)):
            with pytest.raises(fga.FGAError):
                fga.set_direct_tile(*bad)
        assert fga.get_direct_tile(0) == (128, 4)  # a rejected call changes nothing
        assert fga.fga_direct_max_n(12345) == old_n and fga.fga_direct_max_n(0) == 12345
    finally:
        for c, (bs, q) in enumerate(saved):
            fga.set_direct_tile(c, bs, q)
        fga.fga_direct_max_n(old_n)


def test_rigid_fit_rejects_bad_arguments_without_gpu_work(fga):
    red = np.zeros(27)
    R, t = np.zeros(9), np.zeros(3)
    dp = lambda a: a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))  # noqa: E731
    mu0 = np.zeros(3)
    assert fga.lib.fga_rigid_fit(dp(red), 0, dp(mu0), 3, dp(R), dp(t), None) == fga.FGA_EINVAL
    assert fga.lib.fga_rigid_fit(dp(red), 10, dp(mu0), 4, dp(R), dp(t), None) == fga.FGA_EINVAL
    assert fga.lib.fga_rigid_fit(None, 10, dp(mu0), 3, dp(R), dp(t), None) == fga.FGA_EINVAL
    bad = red.copy()
    bad[20] = np.inf
    assert fga.lib.fga_rigid_fit(dp(bad), 10, dp(mu0), 3, dp(R), dp(t), None) == fga.FGA_EINVAL
    assert "non-finite" in fga.last_error()
    with pytest.raises(ValueError):
        fga.fga_rigid_fit(np.zeros(26), 10, mu0)

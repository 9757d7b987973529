"""The autotuner and every launch shape it can pick.

Each all-pairs tile shape must give the oracle's forces (Eq. 6) within the
per-point bound 1e-5 x sum of term magnitudes, on ragged sizes that span
several tiles and chunks; the tuner's report must be self-consistent; and a
registration after tuning must still match the oracle.
"""
import numpy as np
import pytest

import synth

pytestmark = pytest.mark.gpu

SHAPES = [(128, 1), (128, 2), (128, 4), (256, 1), (256, 2), (256, 4)]


@pytest.fixture(scope="module")
def fga():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    import __graft_entry__
    __graft_entry__.build_library()
    import paper_2009_14005_gb300 as f
    return f


@pytest.fixture
def saved_tables(fga):
    tiles = [fga.get_direct_tile(c) for c in range(3)]
    cross = fga.fga_direct_max_n(0)
    yield
    for c, (bs, q) in enumerate(tiles):
        fga.set_direct_tile(c, bs, q)
    fga.fga_direct_max_n(cross)


def _cuda(a):
    import torch
    return torch.as_tensor(np.ascontiguousarray(a), device="cuda")


@pytest.mark.parametrize("shape", SHAPES)
@pytest.mark.parametrize("N,M", [(1531, 1337), (9000, 70001)])
def test_every_direct_tile_matches_oracle(fga, orc, saved_tables, shape, N, M):
    rng = np.random.default_rng(N + M + shape[0] + shape[1])
    X = rng.normal(size=(N, 3)).astype(np.float32) * 2
    Y = rng.normal(size=(M, 3)).astype(np.float32) * 2
    mX = (rng.uniform(0.1, 1.0, N) / N).astype(np.float32)
    sub = rng.choice(M, size=min(M, 2000), replace=False)
    a_o, ab = orc.direct_acc(X, mX, Y[sub], 66.7, 0.05, want_abs=True)
    for c in range(3):
        fga.set_direct_tile(c, *shape)
    assert fga.get_direct_tile(2) == shape
    a = fga.fga_forces(None, _cuda(X), _cuda(mX), _cuda(Y), None,
                       fga.params(G=66.7, eps=0.05)).cpu().numpy().astype(np.float64)[sub]
    err = np.linalg.norm(a - a_o, axis=1)
    assert np.all(err <= 1e-5 * ab + 1e-30), (err / ab).max()


def test_bad_tile_is_rejected(fga, saved_tables):
    with pytest.raises(fga.FGAError):
        fga.set_direct_tile(0, 192, 1)
    with pytest.raises(fga.FGAError):
        fga.set_direct_tile(3, 128, 1)


def test_autotune_report_and_registration_after(fga, orc, saved_tables):
    p = fga.params(max_iter=100, theta=0.5)
    rep = fga.autotune(p)
    for c in range(3):
        assert (rep["direct_bs"][c], rep["direct_qpt"][c]) in SHAPES
        assert (rep["direct_bs"][c], rep["direct_qpt"][c]) == fga.get_direct_tile(c)
        assert rep["direct_gips"][c] > 0
    assert rep["sizes"] == [1024 << k for k in range(fga.FGA_TUNE_NSIZES)]
    assert rep["direct_max_n"] == fga.fga_direct_max_n(0)
    assert rep["direct_max_n"] == 512 or rep["direct_max_n"] in rep["sizes"]
    d, b = rep["direct_us_per_point"], rep["bh_us_per_point"]
    assert all(x > 0 for x in d + b)
    # the all-pairs cost per point grows about linearly with N once a pair
    # fills the GPU (at the smaller sizes the launch's fixed costs weigh in)
    assert d[-1] > 1.6 * d[-2]
    # the crossover is where the all-pairs sum stops being the cheaper one
    k = rep["sizes"].index(rep["direct_max_n"]) if rep["direct_max_n"] in rep["sizes"] else -1
    assert all(d[j] <= b[j] for j in range(k + 1))
    if k + 1 < len(d):
        assert d[k + 1] > b[k + 1]
    # a registration with the tuned shapes still follows the oracle
    X, Y, _, _ = synth.sphere_pair(2, n=3000, m=2500)
    pp = fga.params(method=fga.FGA_DIRECT, max_iter=40, G=66.7, eps=0.05, eta=0.1)
    R, t, st = fga.fga_register(X, Y, pp)
    o = orc.register_full(X, Y, orc.Params(method=orc.FGA_DIRECT, max_iter=40, G=66.7, eps=0.05, eta=0.1))
    c = (np.trace(R.T @ o["R"]) - 1) / 2
    assert np.degrees(np.arccos(np.clip(c, -1, 1))) <= 0.01
    assert np.linalg.norm(t - o["t"]) <= 1e-4 * np.linalg.norm(X.max(0) - X.min(0))

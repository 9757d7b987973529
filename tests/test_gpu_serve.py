"""The registration server (continuous batching) on the GPU.

Each request is Algorithm 2 on one pair; in the server it shares every launch
with whatever other pairs are resident at the time. The per-pair arithmetic
(its tasks, its partial sums, its reduction order, its rigid fit) does not
depend on the other pairs, so a served result must equal the same pair run
alone through the batch executor bit for bit, and the one-pair path
(fga_register) within the registration tolerance (0.01 deg, 1e-4 x bbox
diagonal).
"""
import time

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


def rot_err_deg(Ra, Rb):
    c = (np.trace(Ra.T @ Rb) - 1.0) / 2.0
    return float(np.degrees(np.arccos(np.clip(c, -1.0, 1.0))))


def mixed_pairs():
    """Pairs of uneven size: all-pairs and Barnes-Hut ones (crossover N = 2500)."""
    sizes = [(600, 900), (3000, 2200), (1200, 5000), (8000, 3000), (2000, 700),
             (5000, 12000), (900, 1500), (16000, 9000)]
    out = []
    for k, (n, m) in enumerate(sizes):
        if k % 2:
            X, Y, _, _ = synth.planar_scene_pair(500 + k, n=n, m=m, max_deg=40.0)
        else:
            X, Y, _, _ = synth.sphere_pair(500 + k, n=n, m=m, max_deg=40.0)
        out.append((X, Y))
    return out


def params(fga, **kw):
    base = dict(method=fga.FGA_AUTO, max_iter=30, theta=0.5)
    base.update(kw)
    return fga.params(**base)


def test_served_equals_alone(fga):
    pairs = mixed_pairs()
    old = fga.fga_direct_max_n(2500)
    try:
        p = params(fga)
        alone_batch = [fga.fga_register_batch([pr], p)[0][0] for pr in pairs]
        alone_single = [fga.fga_register(X, Y, p) for X, Y in pairs]
        with fga.Server(p, iters_per_tick=3) as srv:
            tickets = {}
            # staggered arrivals: later pairs join while earlier ones iterate
            for k, (X, Y) in enumerate(pairs):
                tickets[srv.submit(X, Y)] = k
                time.sleep(0.002 * (k % 3))
            got = srv.drain()
            st = srv.stats()
    finally:
        fga.fga_direct_max_n(old)
    assert len(got) == len(pairs)
    assert st["completed"] == len(pairs) and st["failed"] == 0
    assert st["resident"] == 0 and st["bytes_charged"] == 0
    for r in got:
        k = tickets[r["ticket"]]
        b = alone_batch[k]
        assert r["status"] == fga.FGA_OK, r["error"]
        assert r["iterations"] == 30
        assert r["method"] == b["method"]
        assert np.array_equal(r["R"], b["R"]) and np.array_equal(r["t"], b["t"]), k
        assert r["interactions"] == b["interactions"]
        R1, t1, st1 = alone_single[k]
        X, Y = pairs[k]
        diag = float(np.linalg.norm(X.max(0) - X.min(0)))
        assert rot_err_deg(r["R"], R1) <= 0.01
        assert np.linalg.norm(r["t"] - t1) <= 1e-4 * diag
        assert r["submit_ms"] <= r["admit_ms"] <= r["start_ms"] <= r["done_ms"]


def test_memory_admission_bounds_residency(fga):
    pairs = mixed_pairs()[:6]
    p = params(fga, method=fga.FGA_DIRECT, max_iter=20)
    alone = [fga.fga_register_batch([pr], p)[0][0] for pr in pairs]
    # a budget that holds only some of these pairs at a time (their bounds
    # are about 0.2 - 2.3 MB each)
    budget = 3 * 1024 * 1024
    with fga.Server(p, mem_budget=budget, iters_per_tick=2) as srv:
        tickets = {srv.submit(X, Y): k for k, (X, Y) in enumerate(pairs)}
        seen_charge, seen_resident, got = 0, 0, []
        t_end = time.time() + 120
        while len(got) < len(pairs) and time.time() < t_end:
            st = srv.stats()
            seen_charge = max(seen_charge, st["bytes_charged"])
            seen_resident = max(seen_resident, st["resident"] + st["preparing"])
            got.extend(srv.poll(64, wait_ms=1))
        assert st["mem_budget"] == budget
    assert len(got) == len(pairs)
    assert 0 < seen_charge <= budget
    assert seen_resident < len(pairs)
    for r in got:
        b = alone[tickets[r["ticket"]]]
        assert np.array_equal(r["R"], b["R"]) and np.array_equal(r["t"], b["t"])


def test_bad_request_is_reported_alone(fga):
    p = params(fga, max_iter=10)
    X, Y, _, _ = synth.sphere_pair(7, n=800, m=700)
    bad = Y.copy()
    bad[5, 1] = np.nan
    with fga.Server(p) as srv:
        t_ok = srv.submit(X, Y)
        t_bad = srv.submit(X, bad)
        t_ok2 = srv.submit(X, Y)
        got = {r["ticket"]: r for r in srv.drain()}
        with pytest.raises(fga.FGAError):
            srv.submit(np.zeros((0, 3), np.float32), Y)
        st = srv.stats()
    assert got[t_bad]["status"] == fga.FGA_EINVAL and "non-finite" in got[t_bad]["error"]
    assert got[t_ok]["status"] == fga.FGA_OK and got[t_ok2]["status"] == fga.FGA_OK
    assert np.array_equal(got[t_ok]["R"], got[t_ok2]["R"])
    assert st["failed"] == 1 and st["completed"] == 3


def test_pair_larger_than_budget_is_refused(fga):
    p = params(fga)
    X, Y, _, _ = synth.sphere_pair(3, n=20000, m=20000)
    with fga.Server(p, mem_budget=1 << 20) as srv:
        with pytest.raises(fga.FGAError) as e:
            srv.submit(X, Y)
    assert "budget" in str(e.value)


def test_early_exit_matches_alone(fga, orc):
    # Served pairs that stop early stop where they stop alone (bit for bit) and
    # where the FP64 oracle stops (within one iteration), at its transform.
    p = params(fga, method=fga.FGA_DIRECT, max_iter=300, conv_tol=1e-6)
    po = orc.Params(method=orc.FGA_DIRECT, max_iter=300, conv_tol=1e-6)
    pairs = [synth.box_pair(20 + k, n=400 + 150 * k)[:2] for k in range(4)]
    alone = [fga.fga_register_batch([pr], p)[0][0] for pr in pairs]
    with fga.Server(p, iters_per_tick=5) as srv:
        tickets = {srv.submit(X, Y): k for k, (X, Y) in enumerate(pairs)}
        got = srv.drain()
    for r in got:
        k = tickets[r["ticket"]]
        b = alone[k]
        assert r["converged"] and r["iterations"] == b["iterations"] < 300
        assert np.array_equal(r["R"], b["R"])
        X, Y = pairs[k]
        o = orc.register_full(X, Y, po)
        assert abs(r["iterations"] - o["iters"]) <= 1
        diag = np.linalg.norm(X.max(0) - X.min(0))
        assert rot_err_deg(r["R"], o["R"]) <= 0.01
        assert np.linalg.norm(np.asarray(r["t"]) - o["t"]) <= 1e-4 * diag


def test_work_cap_admits_one_at_a_time(fga):
    pairs = mixed_pairs()[:5]
    p = params(fga, method=fga.FGA_DIRECT, max_iter=12)
    alone = [fga.fga_register_batch([pr], p)[0][0] for pr in pairs]
    # a cap below every pair's estimate: a pair is admitted only when none is held
    with fga.Server(p, iters_per_tick=2, max_work=1.0) as srv:
        tickets = {srv.submit(X, Y): k for k, (X, Y) in enumerate(pairs)}
        held, got = 0, []
        while len(got) < len(pairs):
            st = srv.stats()
            held = max(held, st["resident"] + st["preparing"])
            got.extend(srv.poll(64, wait_ms=1))
    assert held == 1
    order = [tickets[r["ticket"]] for r in got]
    assert order == sorted(order)  # FIFO admission, one at a time
    for r in got:
        b = alone[tickets[r["ticket"]]]
        assert np.array_equal(r["R"], b["R"]) and np.array_equal(r["t"], b["t"])

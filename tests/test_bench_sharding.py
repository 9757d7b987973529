"""Multi-rank logic of bench.py on CPU (gloo, world size 2): disjoint work per
rank, max-over-ranks time and sum-over-ranks units."""
import os
import socket

import pytest


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _worker(rank, world, port, q):
    import torch.distributed as dist
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(world))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    seeds = bench.shard_seeds(rank, world, 3)
    t, u = bench.reduce_max_sum(10.0 * (rank + 1), 100.0 + rank, world)
    bench.barrier(world)
    q.put((rank, seeds, t, u))
    dist.destroy_process_group()


def test_two_rank_sharding_and_reduction():
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    out = [q.get(timeout=120) for _ in range(2)]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    out.sort()
    s0, s1 = set(out[0][1]), set(out[1][1])
    assert s0.isdisjoint(s1) and len(s0) == len(s1) == 3
    for _, _, t, u in out:
        assert t == pytest.approx(20.0)
        assert u == pytest.approx(201.0)


def test_direct_equivalent_is_labelled():
    import bench
    d = bench.direct_equivalent(2e12, 500.0)
    assert d["value"] == pytest.approx(4e12) and "equivalent" in d["note"]
    assert bench.direct_equivalent(1.0, 0.0)["value"] is None


def test_cpu_single_thread_sample_on_the_sphere_workload():
    import bench
    import oracle
    a = bench.parse_args(["--workload", "sphere-direct"])
    pair = bench.make_pairs([1000], a)[0]
    before = oracle.max_threads()
    d = bench.cpu_single_thread(pair, a, iters=2)
    assert d["cores"] == 1 and d["value"] > 0
    assert oracle.max_threads() == before


def test_cpu_direct_subsample_on_a_barnes_hut_workload():
    import bench
    a = bench.parse_args(["--workload", "lidar-bh", "--n", "3000"])
    pair = bench.make_pairs([1000], a)[0]
    d = bench.cpu_direct_sample(pair, a, m_sample=256)
    assert d["value"] > 0 and "256 template points" in d["sample"]


@pytest.mark.parametrize("name", ["lidar-bh", "sphere-direct", "planar-direct", "planar-bh", "batch",
                                  "grid", "serve"])
def test_every_workload_has_a_named_config(name):
    import json
    import bench
    a = bench.parse_args(["--workload", name])
    cfg = bench.workload_config(a)
    assert isinstance(cfg.get("workload"), str) and cfg["workload"]
    json.dumps(cfg)  # serialisable as part of the bench line
    w = bench.workload(a)
    assert w["iters"] > 0 and w["n"] > 0


def test_default_workload_is_the_1m_planar_barnes_hut_registration():
    import bench
    a = bench.parse_args([])
    w = bench.workload(a)
    assert a.workload == "planar-bh" and w["n"] == 1_000_000 and w["method"] == "bh"
    assert w["theta"] == 0.5 and w["iters"] == 100 and w["masses"] == "uniform"
    assert bench.workload(bench.parse_args(["--workload", "lidar-bh"]))["masses"] == "knn16"


def test_reference_arm_prints_one_json_line(capsys):
    import json
    import bench
    assert bench.main(["--impl", "reference", "--n", "3000", "--steps", "1", "--warmup", "0"]) == 0
    line = json.loads(capsys.readouterr().out.strip().splitlines()[-1])
    assert line["impl"] == "reference" and line["value"] > 0 and line["higher_is_better"]
    assert line["e2e"]["h2d_bytes_per_step"] == 0 and line["cpu_baseline"]["kind"] == "oracle"
    assert line["config"]["workload"].startswith("planar-scene-")


def test_ground_truth_summary():
    import bench
    m = {"gt_rot": [0.1, 0.3, 0.2], "gt_t": [1e-5, 3e-5, 2e-5]}
    g = bench.gt_summary(m)
    assert g["rot_deg_median"] == 0.2 and g["rot_deg_max"] == 0.3 and g["t_rel_max"] == 3e-5
    assert bench.gt_summary({"gt_rot": [], "gt_t": []}) is None

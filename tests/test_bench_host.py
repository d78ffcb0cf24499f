"""Host logic of bench.py on the CPU: the convergence metric helpers and the
multi-process path (world size 2 over gloo, as the replicas of a torchrun
launch would use NCCL): the step time is the maximum over ranks and the job's
throughput counts every replica; the reference arm runs on rank 0 only."""
import json
import os
import socket
import subprocess
import sys

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import bench  # noqa: E402


def test_clusters_and_first_reach():
    ref = np.array([1.0, 2.0, 2.0 + 1e-12, 3.0, 4.0])
    assert list(bench.clusters(ref)) == [0, 1, 1, 2, 3]
    # pair 1 may land on either member of its cluster; pair 3 never gets within 1e-9
    hist = np.array([[1.1, 2.1, 2.1, 3.1], [1.0 + 1e-10, 2.0 + 1e-12, 2.05, 3.0 + 1e-6],
                     [1.0, 2.0, 2.0 + 5e-10, 3.0 + 1e-6]])
    reach = bench.first_reach(hist, ref[:4], 1e-9, ref)
    assert list(reach) == [1, 1, 2, -1]


def test_first_reach_with_a_shorter_reference_table():
    """More pairs than reference eigenvalues or than the oracle's history
    covers (the h = 1/2048, k = 128 workload: 136 reference values, oracle
    histories of pairs 0..41): pairs past the table never count, the rest do;
    the reference set is the oracle's stable pairs among 0..41, without pair
    11 (reached, then left: an unstable fixed point)."""
    ref = np.array([1.0, 2.0, 3.0])
    hist = np.array([[1.0, 2.0, 3.0, 4.0, 5.0]])
    assert list(bench.first_reach(hist, ref, 1e-9, ref)) == [0, 0, 0, -1, -1]
    rs = bench.reference_set(bench.WORK_H2048)
    assert rs.max() < 42 and list(rs[:3]) == [0, 1, 2] and 11 not in rs
    conv, S = bench.time_to_target(np.array([0, 3, -1, -1]), None, 60)
    assert (conv, S) == (2, 3)


def test_time_to_target_with_and_without_reference_set():
    reach = np.array([3, 5, -1, 7])
    assert bench.time_to_target(reach, None, 60) == (3, 7)
    assert bench.time_to_target(reach, np.array([0, 1, 3]), 60) == (3, 7)
    # a set pair that never reaches the target costs the whole cap
    assert bench.time_to_target(reach, np.array([0, 2]), 60) == (1, 60)


def test_job_value():
    assert bench.job_value(1, 14, 15, 6.0) == pytest.approx(14 / 0.09)
    assert bench.job_value(4, 14, 15, 6.0) == pytest.approx(4 * 14 / 0.09)
    assert bench.job_value(1, 14, 8, 6.0, 12.0) == pytest.approx(14 / 0.06)


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


_WORKER = r"""
import os, sys, json
sys.path.insert(0, sys.argv[1])
import torch, torch.distributed as dist
import bench
dist.init_process_group("gloo", rank=int(os.environ["RANK"]), world_size=int(os.environ["WORLD_SIZE"]))
rank = dist.get_rank()
ms = bench.max_over_ranks(torch, 10.0 + 5.0 * rank)      # rank 1 is the slow replica
print(json.dumps({"rank": rank, "ms": ms, "value": bench.job_value(dist.get_world_size(), 14, 15, ms / 15)}))
dist.destroy_process_group()
"""


def test_max_over_ranks_two_gloo_processes(tmp_path):
    script = tmp_path / "worker.py"
    script.write_text(_WORKER)
    port = _free_port()
    procs = []
    for r in range(2):
        env = dict(os.environ, RANK=str(r), WORLD_SIZE="2", MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port),
                   CUDA_VISIBLE_DEVICES="")
        procs.append(subprocess.Popen([sys.executable, str(script), ROOT], env=env, stdout=subprocess.PIPE,
                                      stderr=subprocess.PIPE, text=True))
    outs = []
    for p in procs:
        out, err = p.communicate(timeout=180)
        assert p.returncode == 0, err
        outs.append(json.loads(out.strip().splitlines()[-1]))
    for o in outs:
        assert o["ms"] == 15.0                     # the slow replica's time on every rank
        assert o["value"] == pytest.approx(2 * 14 / 0.015)


def test_reference_arm_runs_on_rank_zero_only(capsys, monkeypatch):
    monkeypatch.setenv("RANK", "1")

    class Args:
        steps = 1
    bench.main_reference(Args())
    assert capsys.readouterr().out == ""


def test_oracle_pool_matches_sequential_oracle():
    """The pair-parallel CPU baseline (worker processes, pairs split evenly)
    computes exactly the oracle's own iterates: pairs are independent
    (Section 3.2), so splitting them over processes changes nothing."""
    import meshgen as mg
    import oracle
    work = {"dim": 2, "N": 32, "NH": 8, "k": 6, "tol": 1e-10}
    pool = bench.OraclePool(work, procs=2)
    try:
        assert pool.procs == 2 and sorted(sum(pool.cols, [])) == list(range(6))
        dts = [pool.step() for _ in range(3)]
    finally:
        pool.close()
    assert all(dt > 0 for dt in dts)
    prob = oracle.Problem.from_hierarchy(mg.build_hierarchy(2, 32, 8))
    _, _, _, hist = oracle.solve(prob, 6, tol=1e-10, max_steps=3, history=True)
    assert np.allclose(np.array(pool.history), np.array(hist), rtol=1e-14, atol=0)

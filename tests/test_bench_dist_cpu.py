"""The multi-rank path of bench.py on CPU: two gloo ranks on 127.0.0.1 agree on
the slowest rank's time, and the whole-job value counts every rank's pairs
(replicas only: the ranks exchange nothing but the timing)."""
import os
import socket
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world),
                      LOCAL_RANK=str(rank))
    sys.path.insert(0, ROOT)
    import torch.distributed as dist

    import bench

    dist.init_process_group("gloo", rank=rank, world_size=world)
    w, r, local = bench.dist_setup(world)
    ms = bench.max_over_ranks(10.0 + 5.0 * rank, dist, "cpu")
    value = bench.job_value(1000, 4, w, ms / 1e3)
    q.put((r, w, local, ms, value))
    dist.barrier()
    dist.destroy_process_group()


def test_two_gloo_ranks_take_the_slowest_time_and_sum_the_work():
    torch = pytest.importorskip("torch")
    import torch.multiprocessing as mp

    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    out = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    assert [o[0] for o in out] == [0, 1] and all(o[1] == 2 for o in out)
    assert [o[2] for o in out] == [0, 1]
    for _, _, _, ms, value in out:
        assert ms == 15.0                                  # max over ranks
        assert value == pytest.approx(1000 * 4 * 2 / 0.015)  # both replicas' pairs / slowest time


def test_single_rank_needs_no_process_group():
    sys.path.insert(0, ROOT)
    import bench

    assert bench.max_over_ranks(3.5, None) == 3.5
    assert bench.job_value(10, 2, 1, 0.5) == 40.0


def test_reference_arm_prints_one_contract_line():
    """bench.py --impl reference times the CPU oracle on a bounded sample and
    prints one JSON line with the contract's keys (it needs no GPU)."""
    import json
    import subprocess

    out = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference",
                          "--workload", "cylinder_48", "--steps", "1", "--warmup", "1"],
                         capture_output=True, text=True, timeout=600, cwd=ROOT)
    assert out.returncode == 0, out.stderr[-2000:]
    lines = [l for l in out.stdout.splitlines() if l.strip().startswith("{")]
    assert len(lines) == 1
    d = json.loads(lines[0])
    for k in ("impl", "metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step",
              "higher_is_better", "scaling", "vs_baseline", "dtype", "data", "config", "e2e", "cpu_baseline"):
        assert k in d, k
    assert d["impl"] == "reference" and d["value"] > 0 and d["higher_is_better"] is True
    assert d["e2e"]["h2d_bytes_per_step"] == 0 and d["e2e"]["value"] == d["value"]
    assert d["cpu_baseline"]["kind"] == "oracle" and d["cpu_baseline"]["cores"] >= 1


@pytest.mark.parametrize("workload", ["tree_2d", "cylinder_hypersonic_tree", "naca_supersonic_tree", "sphere_96_tree"])
def test_tree_workloads_have_bounded_oracle_samples(workload):
    """Every tree workload names a coarser tree the CPU oracle runs in about
    a second per step (the cpu_baseline and reference legs); the sample keeps
    the workload's body inside its finest level."""
    import time

    sys.path.insert(0, ROOT)
    import bench
    import oracle

    case = bench._workload_case(None, workload, "mixed")
    sample = bench.cpu_sample_case(case)
    assert sample["precision"] == "fp64" and len(sample["tree"]["level"]) < len(case["tree"]["level"])
    o = oracle.OracleTree(sample, threads=4)
    if case["body"]["kind"] != "none":
        assert o.nfluid < o.nleaf
    t0 = time.perf_counter()
    o.step(1)
    assert time.perf_counter() - t0 < 20.0

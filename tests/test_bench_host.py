"""Host logic of bench.py's multi-process (replicas) mode on CPU: two gloo
ranks aggregate the slowest rank's time and the units of all ranks; under the
reference arm only rank 0 works and prints."""
import os
import subprocess
import sys

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _rank_main(rank, world, port, out):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    sys.path.insert(0, ROOT)
    import bench
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        seconds, units = bench.aggregate(dist, 1.0 + rank, 10.0 * (rank + 1), "cpu")
        out[rank] = (seconds, units)
    finally:
        dist.destroy_process_group()


def test_aggregate_two_gloo_ranks():
    port = 29500 + (os.getpid() % 2000)
    with mp.Manager() as manager:
        out = manager.dict()
        mp.spawn(_rank_main, args=(2, port, out), nprocs=2, join=True)
        got = dict(out)
    # max of (1, 2) seconds, sum of (10, 20) units, on every rank
    assert got == {0: (2.0, 30.0), 1: (2.0, 30.0)}


def test_aggregate_single_process_is_identity():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.aggregate(None, 1.5, 7, "cpu") == (1.5, 7)


def test_reference_arm_nonzero_rank_exits_without_work():
    env = dict(os.environ, RANK="1", WORLD_SIZE="2", LOCAL_RANK="1")
    p = subprocess.run([sys.executable, "bench.py", "--impl", "reference", "--steps", "1", "--warmup", "0"],
                       cwd=ROOT, env=env, capture_output=True, text=True, timeout=120)
    assert p.returncode == 0, p.stderr
    assert p.stdout.strip() == ""


def test_cpu_child_runs_the_configured_cycle_shape():
    """The oracle arm's sample process takes the native arm's cycle: V(2,1)
    and W(2,1) on the same 8 x 8 p=1 sample."""
    recs = {}
    for shape in ("1,1,64", "2,1,64"):
        p = subprocess.run([sys.executable, "bench.py", "--cpu-child", "8,1,2,1,0.5," + shape], cwd=ROOT,
                           capture_output=True, text=True, timeout=300)
        assert p.returncode == 0, p.stderr
        recs[shape] = __import__("json").loads(p.stdout.strip().splitlines()[-1])
    assert recs["1,1,64"]["dofs"] == recs["2,1,64"]["dofs"] == 8 * 8 * 3 * 4
    assert recs["2,1,64"]["cycles"] >= 2
    assert recs["1,1,64"]["shape"] == [1, 1, 64] and recs["2,1,64"]["shape"] == [2, 1, 64]
    assert recs["1,1,64"]["nu"] == recs["2,1,64"]["nu"] == [2, 1]


def test_reference_arm_reports_the_configuration_it_ran():
    """The reference arm runs the oracle on the configuration named by the
    arguments and says so: its config's mesh and DOF count are those of the
    problem it timed."""
    import json
    p = subprocess.run([sys.executable, "bench.py", "--impl", "reference", "--n", "8", "--p", "1",
                        "--steps", "2", "--warmup", "1", "--nu", "1"], cwd=ROOT, capture_output=True, text=True,
                       timeout=300)
    assert p.returncode == 0, p.stderr
    rec = json.loads(p.stdout.strip().splitlines()[-1])
    assert rec["impl"] == "reference"
    assert rec["config"]["n"] == [8, 8] and rec["config"]["dofs"] == 8 * 8 * 3 * 4
    assert "8x8" in rec["cpu_baseline"]["sample"] and rec["cpu_baseline"]["cores"] == 1
    assert rec["value"] > 0 and rec["e2e"]["value"] == rec["value"]


def test_cpu_child_single_outer_iteration():
    """seconds = 0: exactly one outer iteration after the untimed setup (the
    full-configuration baseline)."""
    import json
    p = subprocess.run([sys.executable, "bench.py", "--cpu-child", "8,1,1,1,0,1,1,64"], cwd=ROOT,
                       capture_output=True, text=True, timeout=300)
    assert p.returncode == 0, p.stderr
    rec = json.loads(p.stdout.strip().splitlines()[-1])
    assert rec["cycles"] == 1 and rec["setup_s"] >= 0


@pytest.mark.parametrize("argv,arms,precision", [
    ([], "fp32,fp16", "fp32"),
    (["--precision", "bf16"], "bf16", "bf16"),
    (["--arms", "fp16"], "fp16", "fp32"),
    (["--workload", "unsteady3d"], "fp32", "fp16"),
    (["--workload", "batch"], "fp32", "fp16"),
    (["--workload", "cut"], "fp32", "fp32"),
    (["--workload", "cut", "--precision", "fp64"], "fp64", "fp64"),
])
def test_precision_defaults(monkeypatch, argv, arms, precision):
    """The default run times the FP32 and the scaled-FP16 cycle of the 256^2
    workload; the unsteady and batch workloads default to FP16 blocks, the
    cut-cell one to FP32; an explicit --precision is the only arm."""
    sys.path.insert(0, ROOT)
    import bench
    monkeypatch.setattr(sys, "argv", ["bench.py"] + argv)
    args = bench.parse()
    assert args.arms == arms and args.precision == precision

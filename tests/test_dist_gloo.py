"""Multi-rank paths on CPU (gloo, world size 2): the whole-job aggregation
bench.py uses under torchrun (sum of units over ranks divided by the slowest
rank's time), and the reference arm's rank handling."""
import json
import os
import socket
import subprocess
import sys

import pytest

ROOT = os.path.abspath(os.path.join(os.path.dirname(__file__), ".."))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, out):
    import torch.distributed as dist
    sys.path.insert(0, ROOT)
    import bench
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    units = 100.0 * (rank + 1)          # rank 0: 100 cells, rank 1: 200 cells
    ms = 10.0 + 30.0 * rank             # rank 1 is the slow one (40 ms)
    out[rank] = (bench.max_over_ranks(dist, ms), bench.sum_over_ranks(dist, units),
                 bench.job_rate(dist, units, ms))
    dist.barrier()
    dist.destroy_process_group()


def test_job_rate_over_two_gloo_ranks():
    import torch.multiprocessing as mp
    mgr = mp.Manager()
    out = mgr.dict()
    mp.spawn(_worker, args=(2, _free_port(), out), nprocs=2, join=True)
    for r in (0, 1):
        mx, tot, rate = out[r]
        assert mx == 40.0 and tot == 300.0
        assert rate == pytest.approx(300.0 / 0.040)


def test_reference_arm_prints_one_line_on_rank0_only():
    env = dict(os.environ, RANK="0", WORLD_SIZE="1")
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference",
                        "--steps", "2", "--warmup", "1"], capture_output=True, text=True,
                       env=env, timeout=600)
    assert r.returncode == 0, r.stderr[-2000:]
    line = json.loads(r.stdout.strip().splitlines()[-1])
    assert line["impl"] == "reference" and line["value"] > 0
    for k in ("metric", "unit", "n_gpus", "steps", "warmup", "ms_per_step", "higher_is_better",
              "cpu_baseline", "e2e", "config"):
        assert k in line
    assert line["e2e"]["h2d_bytes_per_step"] == 0
    env1 = dict(os.environ, RANK="1", WORLD_SIZE="2")
    r1 = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference",
                         "--steps", "2", "--warmup", "1"], capture_output=True, text=True,
                        env=env1, timeout=600)
    assert r1.returncode == 0 and r1.stdout.strip() == ""


@pytest.mark.parametrize("workload", ["adjoint1k", "spectrum8k", "ensemble", "nlc8k"])
def test_reference_arm_of_every_workload(workload):
    # three warm-up attempts, as the driver runs it (the first attempts of an
    # adaptive run may be rejected while dt settles)
    env = dict(os.environ, RANK="0", WORLD_SIZE="1")
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference",
                        "--workload", workload, "--steps", "1", "--warmup", "3"], capture_output=True,
                       text=True, env=env, timeout=600)
    assert r.returncode == 0, r.stderr[-2000:]
    line = json.loads(r.stdout.strip().splitlines()[-1])
    assert line["impl"] == "reference" and line["value"] > 0 and line["ms_per_step"] > 0
    for k in ("metric", "unit", "n_gpus", "steps", "warmup", "higher_is_better", "cpu_baseline", "e2e",
              "config"):
        assert k in line

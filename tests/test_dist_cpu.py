"""Multi-process host logic of bench.py on CPU: world size 2 over gloo.

The workloads are independent problems, so N ranks run N replicas with no
data-path collective; what the ranks share is the barrier around the timed
region and the max over ranks of the elapsed time.  These tests run that
logic as two CPU processes.
"""
import json
import os
import socket
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _dist_worker(rank, world, port, out_dir):
    os.environ.update(RANK=str(rank), LOCAL_RANK=str(rank), WORLD_SIZE=str(world),
                      MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    sys.path.insert(0, ROOT)
    import bench
    d = bench._Dist()
    d.init("gloo")
    d.barrier()
    # each rank "measured" a different time; every rank must see the largest
    m = d.max(1.5 + rank)
    d.barrier()
    with open(os.path.join(out_dir, f"r{rank}.json"), "w") as f:
        json.dump({"rank": d.rank, "world": d.world, "max": m}, f)
    import torch.distributed as td
    td.destroy_process_group()


def test_dist_max_over_ranks_gloo(tmp_path):
    import torch.multiprocessing as mp
    port = _free_port()
    mp.start_processes(_dist_worker, args=(2, port, str(tmp_path)), nprocs=2, join=True,
                       start_method="spawn")
    got = [json.load(open(tmp_path / f"r{r}.json")) for r in range(2)]
    assert [g["rank"] for g in got] == [0, 1]
    assert all(g["world"] == 2 for g in got)
    assert all(g["max"] == 2.5 for g in got)


def test_dist_single_rank_is_identity():
    sys.path.insert(0, ROOT)
    import bench
    d = bench._Dist()
    if d.world != 1:
        pytest.skip("run under a launcher")
    d.init("gloo")
    d.barrier()
    assert d.max(3.25) == 3.25


def test_reference_arm_under_torchrun_prints_one_line(tmp_path):
    """bench.py --impl reference at N=2: rank 0 alone times the oracle and prints
    one JSON line; rank 1 exits 0 without work."""
    port = _free_port()
    cmd = [sys.executable, "-m", "torch.distributed.run", "--nnodes=1", "--nproc-per-node", "2",
           "--master-addr", "127.0.0.1", "--master-port", str(port),
           os.path.join(ROOT, "bench.py"), "--impl", "reference", "--gpus", "2",
           "--steps", "1", "--warmup", "0", "--side", "24"]
    env = dict(os.environ, OMP_NUM_THREADS="1")
    p = subprocess.run(cmd, cwd=str(tmp_path), env=env, capture_output=True, text=True, timeout=300)
    assert p.returncode == 0, p.stderr[-2000:]
    lines = [l for l in p.stdout.splitlines() if l.startswith("{")]
    assert len(lines) == 1, p.stdout
    line = json.loads(lines[0])
    assert line["impl"] == "reference"
    assert line["n_gpus"] == 2
    assert line["value"] > 0
    assert line["e2e"]["h2d_bytes_per_step"] == 0

"""The N > 1 plumbing of bench.py on CPU: two gloo ranks (127.0.0.1), barrier, the
max-over-ranks timing and the sum of units, and the reference arm's rank handling (only
rank 0 works and prints)."""
import json
import os
import socket
import subprocess
import sys

import pytest

torch = pytest.importorskip("torch")
ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, out_dir):
    os.environ.update(RANK=str(rank), WORLD_SIZE=str(world), LOCAL_RANK=str(rank), MASTER_ADDR="127.0.0.1",
                      MASTER_PORT=str(port))
    sys.path.insert(0, ROOT)
    import bench
    d = bench.Dist()
    d.init(torch)
    d.barrier(torch)
    ms = 10.0 + 5.0 * rank            # this rank's timing
    res = {"max": d.max(torch, ms), "sum": d.sum(torch, 3.0), "rank": d.rank, "world": d.world}
    d.barrier(torch)
    d.close()
    with open(os.path.join(out_dir, f"r{rank}.json"), "w") as fh:
        json.dump(res, fh)


def test_two_gloo_ranks_max_and_sum(tmp_path):
    import torch.multiprocessing as mp
    port = free_port()
    mp.start_processes(_worker, args=(2, port, str(tmp_path)), nprocs=2, join=True, start_method="spawn")
    for r in range(2):
        res = json.load(open(tmp_path / f"r{r}.json"))
        assert res["world"] == 2 and res["rank"] == r
        assert res["max"] == 15.0          # the slowest rank decides the timing
        assert res["sum"] == 6.0           # units of all ranks


def test_reference_arm_nonzero_rank_exits_quietly():
    env = dict(os.environ, RANK="1", WORLD_SIZE="2", LOCAL_RANK="1")
    p = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--gpus", "2",
                        "--steps", "1", "--warmup", "0"], env=env, capture_output=True, text=True, timeout=120)
    assert p.returncode == 0
    assert p.stdout.strip() == ""

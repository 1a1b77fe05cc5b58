"""The N > 1 host logic of bench.py on CPU with gloo ranks (world size 2):
every rank runs an independent replica, the job's time is the slowest rank's
(all-reduce MAX), and the whole-job value is all ranks' units over that time.
The reference arm runs on rank 0 only."""
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


def _worker(rank, world, port, out_path):
    import torch
    import torch.distributed as dist
    sys.path.insert(0, ROOT)
    import bench
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    units = 1000.0 * (rank + 1)
    seconds = 0.5 + 0.25 * rank          # rank 1 is the slow one
    t = torch.tensor([seconds])
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    u = torch.tensor([units])
    dist.all_reduce(u, op=dist.ReduceOp.SUM)
    value = bench.aggregate([units] * world, [float(t.item())])  # as in run_btas: same per-rank units
    if rank == 0:
        with open(out_path, "w") as f:
            json.dump({"tmax": float(t.item()), "usum": float(u.item()), "value": value}, f)
    dist.destroy_process_group()


def test_gloo_world2_max_time_and_aggregate(tmp_path):
    import torch.multiprocessing as mp
    out = str(tmp_path / "r.json")
    mp.spawn(_worker, args=(2, _free_port(), out), nprocs=2, join=True)
    r = json.load(open(out))
    assert r["tmax"] == 0.75
    assert r["usum"] == 3000.0
    assert r["value"] == pytest.approx(2 * 1000.0 / 0.75)


def test_aggregate_is_total_over_slowest():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.aggregate([10.0, 10.0, 10.0], [1.0, 2.0, 0.5]) == 15.0


def test_reference_arm_nonzero_rank_exits_quietly():
    env = dict(os.environ, RANK="1", WORLD_SIZE="2", LOCAL_RANK="1")
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--steps", "1",
                        "--warmup", "0", "--n", "64"], env=env, capture_output=True, text=True, timeout=120)
    assert r.returncode == 0 and r.stdout.strip() == ""


def test_reference_arm_rank0_prints_one_line():
    env = dict(os.environ, RANK="0", WORLD_SIZE="1", LOCAL_RANK="0")
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--steps", "1",
                        "--warmup", "0", "--n", "256"], env=env, capture_output=True, text=True, timeout=300)
    assert r.returncode == 0, r.stderr
    lines = [ln for ln in r.stdout.splitlines() if ln.strip()]
    assert len(lines) == 1
    d = json.loads(lines[0])
    assert d["impl"] == "reference" and d["value"] > 0 and d["cpu_baseline"]["kind"] == "oracle"
    assert d["e2e"]["h2d_bytes_per_step"] == 0

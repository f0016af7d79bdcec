"""The benchmark's multi-rank host logic on CPU: world_size-2 gloo process
groups stand in for the one-process-per-GPU launch (the replicas share no data
path, so only the timing reduction crosses ranks)."""
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


def _worker(rank, world, port, out_dir):
    import torch.distributed as dist
    sys.path.insert(0, ROOT)
    import bench
    dist.init_process_group("gloo", init_method="tcp://127.0.0.1:%d" % port, rank=rank, world_size=world)
    # rank r took 1 + r seconds for 10 units: the job's time is the slowest rank's
    t = bench.rank_max(1.0 + rank, dist, device="cpu")
    v = bench.replica_value(10.0, world, t)
    dist.barrier()
    dist.destroy_process_group()
    with open(os.path.join(out_dir, "r%d.json" % rank), "w") as f:
        json.dump({"t": t, "v": v}, f)


def test_rank_max_and_replica_value_over_gloo(tmp_path):
    import torch.multiprocessing as mp
    world, port = 2, _free_port()
    mp.spawn(_worker, args=(world, port, str(tmp_path)), nprocs=world, join=True)
    for r in range(world):
        d = json.load(open(tmp_path / ("r%d.json" % r)))
        assert d["t"] == 2.0                  # max over ranks, seen by every rank
        assert d["v"] == pytest.approx(10.0)  # 2 ranks x 10 units / 2 s


def test_single_rank_is_local():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.rank_max(3.5) == 3.5
    assert bench.replica_value(7.0, 1, 2.0) == 3.5


def test_reference_arm_runs_on_rank_zero_only():
    # ranks other than 0 exit 0 without work or output
    env = dict(os.environ, RANK="1", WORLD_SIZE="2", LOCAL_RANK="1")
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--gpus", "2",
                        "--steps", "1", "--warmup", "0"], cwd=ROOT, env=env, capture_output=True, text=True,
                       timeout=120)
    assert r.returncode == 0, r.stderr[-2000:]
    assert r.stdout.strip() == ""

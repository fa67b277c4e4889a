"""The multi-process path of bench.py on CPU: two gloo ranks (the lost blocks
shard with no collective in the forward; the collectives are the barrier
around the timed region, the max over ranks of the elapsed time, and in the
forward+backward step the sum over ranks of the shared rho / gamma
gradients), and the reference arm printing only on rank 0."""
import json
import os
import socket
import subprocess
import sys

import pytest
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(world), LOCAL_RANK=str(rank))
    sys.path.insert(0, ROOT)
    import bench
    r, w, local = bench.dist_env()
    dist = bench.init_dist(w, "gloo")
    try:
        bench.barrier(w)
        t = bench.reduce_max(1.0 + 10.0 * r, w)     # rank 1 is the slowest
        import torch
        g = bench.allreduce_sum_(torch.tensor([[1.0 + r, 2.0 * r]]), w)   # rho / gamma gradients
        out[r] = (r, w, local, t, bench.job_value(1000, w, t), g.tolist())
        bench.barrier(w)
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks_max_time_and_job_value():
    world = 2
    port = _free_port()
    with mp.Manager() as m:
        out = m.dict()
        mp.spawn(_worker, args=(world, port, out), nprocs=world, join=True)
        res = dict(out)
    assert sorted(res) == [0, 1]
    for r in range(world):
        rank, w, local, t, v, g = res[r]
        assert (rank, w, local) == (r, world, r)
        assert t == 11.0                              # max over ranks, on every rank
        assert v == pytest.approx(2 * 1000 / 11.0e-3)  # all ranks' units / slowest time
        assert g == [[3.0, 2.0]]                      # rho / gamma gradients summed over ranks


def test_single_rank_helpers_need_no_process_group():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.reduce_max(3.5, 1) == 3.5
    bench.barrier(1)
    assert bench.job_value(804, 1, 1.0) == pytest.approx(804e3)
    import torch
    g = torch.tensor([[1.0, 2.0]])
    assert bench.allreduce_sum_(g, 1) is g and g.tolist() == [[1.0, 2.0]]


def test_reference_arm_rank_nonzero_exits_quietly():
    env = dict(os.environ, RANK="1", WORLD_SIZE="2", LOCAL_RANK="1")
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference",
                        "--gpus", "2", "--steps", "1", "--warmup", "0"],
                       capture_output=True, text=True, env=env, cwd=ROOT, timeout=300)
    assert r.returncode == 0, r.stderr
    assert r.stdout.strip() == ""


def test_reference_arm_line_on_rank0():
    env = dict(os.environ, RANK="0", WORLD_SIZE="1", LOCAL_RANK="0")
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference",
                        "--steps", "1", "--warmup", "0"],
                       capture_output=True, text=True, env=env, cwd=ROOT, timeout=600)
    assert r.returncode == 0, r.stderr
    line = json.loads(r.stdout.strip().splitlines()[-1])
    assert line["impl"] == "reference" and line["unit"] == "blocks/s" and line["value"] > 0
    assert line["cpu_baseline"]["kind"] == "oracle"
    assert line["e2e"]["h2d_bytes_per_step"] == 0

"""Replica bookkeeping of bench.py at world size 2 on CPU (gloo ranks).

The hot path does not shard: N GPUs run N independent replicas.  What the
multi-rank run adds is host logic: distinct seeds per replica, the max over
ranks of the step time, the whole-job throughput, and a reference arm that
only rank 0 runs.  Two gloo ranks exercise exactly that.
"""
import os
import socket
import subprocess
import sys

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    sys.path.insert(0, ROOT)
    import bench
    ms_local = 10.0 + 5.0 * rank          # rank 1 is the slow replica
    ms = bench.reduce_step_time(ms_local, dist)
    out[rank] = (bench.replica_seed(rank), ms, bench.whole_job_value(1000, world, ms))
    dist.barrier()
    dist.destroy_process_group()


def test_two_gloo_ranks_agree_on_the_max_step_time_and_job_value():
    world = 2
    port = _free_port()
    with mp.Manager() as m:
        out = m.dict()
        mp.spawn(_rank_main, args=(world, port, out), nprocs=world, join=True)
        res = dict(out)
    seeds = {res[r][0] for r in range(world)}
    assert len(seeds) == world                         # independent inputs per replica
    assert all(res[r][1] == 15.0 for r in range(world))  # the slowest replica sets the pace
    # 2 ranks x 1000 units in 15 ms
    assert all(abs(res[r][2] - 2000 / 15e-3 / 1e9) < 1e-15 for r in range(world))


def test_reference_arm_runs_on_rank_0_only():
    env = dict(os.environ, RANK="1", WORLD_SIZE="2", LOCAL_RANK="1")
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference",
                        "--gpus", "2", "--steps", "1", "--warmup", "0"],
                       capture_output=True, text=True, env=env, timeout=120)
    assert r.returncode == 0
    assert r.stdout.strip() == ""                      # rank 1 prints nothing and does no work

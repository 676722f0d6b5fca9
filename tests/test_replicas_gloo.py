"""The multi-process path of bench.py on CPU: two gloo ranks (world size 2).

The data path does not shard (replicas only), so what N > 1 adds is host logic: which pose each
replica renders at each step, the max over ranks of the timed region, the whole-job value, and the
reference arm that only rank 0 runs."""
import os
import socket
import subprocess
import sys

import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, out):
    import bench
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        poses = torch.tensor([bench.replica_pose(s, rank, 16) for s in range(32)])
        gathered = [torch.zeros_like(poses) for _ in range(world)]
        dist.all_gather(gathered, poses)
        local_ms = 3.0 + 2.5 * rank                    # rank 1 is the slow replica
        ms_max = bench.max_over_ranks(local_ms, world, torch.device("cpu"))
        out.put((rank, [g.tolist() for g in gathered], ms_max, bench.job_ms_per_iter(ms_max, world)))
    finally:
        dist.destroy_process_group()


def test_two_replicas_render_different_poses_and_report_the_slowest():
    world, port = 2, _free_port()
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    procs = [ctx.Process(target=_rank_main, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=120) for _ in range(world))
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, gathered, ms_max, job in res:
        assert ms_max == 5.5                           # the slowest replica's time, on every rank
        assert job == 5.5 / 2                          # two iterations finish every 5.5 ms
        a, b = gathered
        assert all(x != y for x, y in zip(a, b))       # different views at every step
        assert sorted(set(a)) == list(range(16)) and sorted(set(b)) == list(range(16))


def test_single_process_needs_no_process_group():
    import bench
    assert bench.max_over_ranks(4.25, 1, torch.device("cpu")) == 4.25
    assert bench.job_ms_per_iter(4.25, 1) == 4.25
    assert [bench.replica_pose(s, 0, 16) for s in range(3)] == [0, 1, 2]


def test_reference_arm_runs_on_rank_zero_only():
    env = dict(os.environ, RANK="1", WORLD_SIZE="2", LOCAL_RANK="1")
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--gpus", "2",
                        "--steps", "1", "--warmup", "0"], env=env, capture_output=True, text=True, timeout=300)
    assert r.returncode == 0, r.stderr
    assert r.stdout.strip() == ""

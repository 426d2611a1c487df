"""The multi-GPU mode of the bench is replicas only (the step has no exchange
between GPUs): every rank runs its own step and the job takes as long as its
slowest replica. These CPU tests run that logic on two gloo ranks (one spawned
process each), and check that the reference arm runs and prints on rank 0 only."""
import json
import os
import socket
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port() -> int:
    with socket.socket(socket.AF_INET, socket.SOCK_STREAM) as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _replica(rank: int, world: int, port: int, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(world), LOCAL_RANK=str(rank))
    import torch.distributed as dist
    sys.path.insert(0, ROOT)
    import bench
    dist.init_process_group("gloo", init_method="env://", rank=rank, world_size=world)
    try:
        # each replica "times" a different step; all must report the slowest
        v = bench.max_over_ranks(10.0 + 3.0 * rank)
        # the line's value: the slowest replica's ms per step, not divided by the replica count
        ms = bench.replica_step_ms(100.0 + 30.0 * rank, 10)
        head = bench.headline_fields(ms, world)
        dist.barrier()
        out.put((rank, v, bench.dist_env(), head))
    finally:
        dist.destroy_process_group()


def test_max_over_ranks_on_two_gloo_ranks():
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_replica, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    got = sorted(q.get(timeout=120) for _ in range(2))
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    assert [(r, v) for r, v, _, _ in got] == [(0, 13.0), (1, 13.0)]
    assert [env for _, _, env, _ in got] == [(0, 2, 0), (1, 2, 1)]
    for _, _, _, head in got:
        assert head["value"] == 13.0 and head["ms_per_step"] == 13.0 and head["n_gpus"] == 2


def test_max_over_ranks_without_a_group_is_the_value():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.max_over_ranks(7.5) == 7.5


def _reference(rank: int, timeout: int = 300):
    env = dict(os.environ, RANK=str(rank), WORLD_SIZE="2", LOCAL_RANK=str(rank), CUDA_VISIBLE_DEVICES="")
    return subprocess.run([sys.executable, "bench.py", "--impl", "reference", "--gpus", "2",
                           "--workload", "planted-n1024-m2048-r32", "--steps", "1", "--warmup", "0",
                           "--cpu-cols", "64"], env=env, cwd=ROOT, capture_output=True, text=True,
                          timeout=timeout)


def test_reference_arm_runs_on_rank_zero_only():
    p1 = _reference(1)
    assert p1.returncode == 0, p1.stderr[-2000:]
    assert p1.stdout.strip() == ""
    p0 = _reference(0)
    assert p0.returncode == 0, p0.stderr[-2000:]
    line = json.loads(p0.stdout.strip().splitlines()[-1])
    assert line["impl"] == "reference" and line["n_gpus"] == 2
    assert line["cpu_baseline"]["kind"] == "oracle" and line["value"] > 0
    for key in ("metric", "unit", "steps", "warmup", "ms_per_step", "higher_is_better", "e2e", "config"):
        assert key in line

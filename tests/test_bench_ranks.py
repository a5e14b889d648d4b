"""The benchmark's multi-process path on CPU: two gloo ranks (the GPU runs use
NCCL, one process per GPU, through the same helpers).  Every rank brackets
its timed region with barriers and the job's time is the largest rank's;
under the reference arm only rank 0 works and prints."""
import multiprocessing as mp
import os
import socket
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket(socket.AF_INET, socket.SOCK_STREAM) as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, values, out):
    os.environ.update({"MASTER_ADDR": "127.0.0.1", "MASTER_PORT": str(port), "RANK": str(rank),
                       "WORLD_SIZE": str(world), "LOCAL_RANK": str(rank), "CUDA_VISIBLE_DEVICES": ""})
    sys.path.insert(0, ROOT)
    import bench
    dist = bench.init_ranks(world)
    try:
        bench.barrier(dist)
        got = bench.max_over_ranks(values[rank], dist)
        bench.barrier(dist)
        out.put((rank, dist.get_backend(), got))
    finally:
        dist.destroy_process_group()


@pytest.mark.parametrize("values", [(1.5, 2.5), (7.0, -3.0)])
def test_job_time_is_the_slowest_rank(values):
    ctx = mp.get_context("spawn")
    out = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank_main, args=(r, 2, port, values, out)) for r in range(2)]
    for p in procs:
        p.start()
    res = sorted(out.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    assert [r for r, _, _ in res] == [0, 1]
    assert all(backend == "gloo" for _, backend, _ in res)
    assert all(got == max(values) for _, _, got in res)


def test_single_process_needs_no_group():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.init_ranks(1) is None
    assert bench.max_over_ranks(3.25, None) == 3.25
    bench.barrier(None)


def test_reference_arm_other_ranks_exit_quietly():
    env = dict(os.environ, RANK="1", WORLD_SIZE="2", LOCAL_RANK="1")
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--gpus", "2"],
                       cwd=ROOT, env=env, capture_output=True, text=True, timeout=120)
    assert r.returncode == 0, r.stderr
    assert r.stdout.strip() == ""

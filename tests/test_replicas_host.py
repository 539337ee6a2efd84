"""bench.py on several ranks: the host logic of an N > 1 launch, on CPU.

The path shards by independent problems, so the ranks are replicas: each
solves its own problem and the only exchange comes after the timed steps,
where every rank's device and wall seconds are reduced to their maximum over
the ranks (the whole job's time) and rank 0 reports the job. Two gloo ranks
on the host check that reduction; the reference arm's other ranks must exit
at once without output.
"""
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


def _rank_main(rank, world, port, q):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    sys.path.insert(0, ROOT)
    import torch.distributed as tdist

    import bench
    tdist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        tdist.barrier()
        # rank r: device seconds 1 + r, wall seconds 10 (world - r)
        q.put((rank, bench.max_over_ranks([1.0 + rank, 10.0 * (world - rank)])))
        tdist.barrier()
    finally:
        tdist.destroy_process_group()


def test_max_over_ranks_on_two_gloo_ranks():
    import multiprocessing as mp
    world = 2
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank_main, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    try:
        got = dict(q.get(timeout=180) for _ in range(world))
    finally:
        for p in procs:
            p.join(60)
            if p.is_alive():
                p.kill()
    assert [p.exitcode for p in procs] == [0] * world
    # every rank holds the maxima: device time of rank 1, wall time of rank 0
    assert got == {0: [2.0, 20.0], 1: [2.0, 20.0]}


def test_max_over_ranks_without_a_process_group():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.max_over_ranks([3, 4.5]) == [3.0, 4.5]


@pytest.mark.parametrize("rank", ["1", "3"])
def test_reference_arm_other_ranks_exit_without_work(rank):
    env = dict(os.environ, RANK=rank, WORLD_SIZE="4", LOCAL_RANK=rank)
    r = subprocess.run([sys.executable, "bench.py", "--impl", "reference", "--steps", "2", "--warmup", "1"],
                       cwd=ROOT, env=env, capture_output=True, text=True, timeout=300)
    assert r.returncode == 0, r.stderr[-2000:]
    assert r.stdout.strip() == ""

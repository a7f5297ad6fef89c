"""The N > 1 path of bench.py on CPU: two gloo ranks (replicas, no
collective on the data path; only the barrier and the max over ranks of the
timed region)."""
import os
import socket
import sys

import pytest

torch = pytest.importorskip("torch")
import torch.multiprocessing as mp  # noqa: E402

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, q):
    os.environ.update(RANK=str(rank), LOCAL_RANK=str(rank), WORLD_SIZE=str(world), MASTER_ADDR="127.0.0.1",
                      MASTER_PORT=str(port))
    sys.path.insert(0, ROOT)
    import bench
    import torch.distributed as dist

    class Args:
        gpus = world
    w, r, local = bench.dist_setup(Args)
    try:
        bench.barrier(w)
        # every rank times a different region; the job's time is the slowest
        got = bench.max_over_ranks(10.0 * (r + 1), w)
        # the reference arm runs on rank 0 only: other ranks return at once
        skipped = None
        if r != 0:
            class RArgs:
                gpus, steps, warmup = world, 1, 0
            skipped = bench.run_reference(RArgs, w, r)
        q.put((r, w, got, skipped))
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks_barrier_and_max_over_ranks():
    world = 2
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(timeout=120)
    assert all(p.exitcode == 0 for p in procs), [p.exitcode for p in procs]
    res = sorted(q.get(timeout=5) for _ in range(world))
    assert [r for r, *_ in res] == [0, 1]
    assert all(w == world for _, w, _, _ in res)
    assert all(got == 20.0 for _, _, got, _ in res)  # max over ranks, seen by every rank
    assert res[1][3] is None

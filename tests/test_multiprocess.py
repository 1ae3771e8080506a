"""The multi-process path of the benchmark on CPU: two gloo ranks run the
replica plumbing (process group, barrier, max over ranks of the times, the
whole-job rate) the way the GPU run does under torchrun with NCCL."""
import os
import socket
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, out):
    os.environ.update(RANK=str(rank), WORLD_SIZE=str(world), LOCAL_RANK=str(rank), MASTER_ADDR="127.0.0.1",
                      MASTER_PORT=str(port))
    sys.path.insert(0, ROOT)
    import torch.distributed as dist

    import bench

    r, w, local = bench.dist_setup(world, backend="gloo")
    assert (r, w, local) == (rank, world, rank)
    bench.barrier(w)
    t = 1.0 + rank                                # the slower rank sets the time
    tmax = bench.max_over_ranks(t, w, local)
    rate = bench.replica_rate(1000, w, tmax)
    out.put((rank, tmax, rate))
    dist.destroy_process_group()


def test_two_gloo_ranks():
    mp = pytest.importorskip("torch.multiprocessing")
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank_main, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    assert [r for r, _, _ in res] == [0, 1]
    for _, tmax, rate in res:
        assert tmax == 2.0                        # max over ranks
        assert rate == 2 * 1000 / 2.0             # whole-job units over the slowest time


def test_single_process_defaults():
    sys.path.insert(0, ROOT)
    import bench

    assert bench.max_over_ranks(3.5, 1, 0) == 3.5
    assert bench.replica_rate(500, 1, 2.0) == 250.0

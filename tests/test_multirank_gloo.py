"""The multi-rank host logic of bench.py on two CPU ranks (gloo): disjoint grid offsets per rank and
the whole-job reduction (maximum of the step times, sum of the counts). No GPU is involved."""
import os
import socket

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402

import bench  # noqa: E402


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, q):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        offs = [bench.step_offset(s, 4, rank, world) for s in range(3)]
        maxima, sums = bench.reduce_over_ranks(dist, "cpu", [10.0 + rank, 5.0 * rank], [100.0 + rank, 1.0])
        q.put((rank, offs, maxima, sums))
    finally:
        dist.destroy_process_group()


def test_two_ranks_offsets_and_reduction():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank_main, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = {}
    for _ in procs:
        rank, offs, maxima, sums = q.get(timeout=120)
        res[rank] = (offs, maxima, sums)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    # the two ranks of each step take different sub-grids
    for s in range(3):
        assert res[0][0][s] != res[1][0][s]
    # every rank sees the same whole-job figures: max of times, sum of counts
    for r in (0, 1):
        assert res[r][1] == [11.0, 5.0]
        assert res[r][2] == [201.0, 2.0]


def test_stride_one_is_replicas():
    assert {bench.step_offset(s, 1, r, 4) for s in range(3) for r in range(4)} == {0}

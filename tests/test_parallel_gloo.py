"""Rank bookkeeping of multi-GPU runs, with two gloo ranks on the CPU.

The decomposition never crosses ranks; these tests cover the host logic that
splits problems over ranks and combines the timings (max for the step time,
sum for the work done).
"""

import os
import socket

import pytest
import torch.multiprocessing as mp

from paper_1703_09074_gb300 import parallel


def test_rank_share_partitions_the_problems():
    for count in (0, 1, 7, 256):
        for world in (1, 2, 3, 8):
            seen = []
            for r in range(world):
                seen += parallel.rank_share(count, r, world)
            assert sorted(seen) == list(range(count))
    with pytest.raises(ValueError):
        parallel.rank_share(4, 2, 2)


def test_reductions_without_a_process_group_are_identity():
    assert parallel.max_over_ranks(3.5) == 3.5
    assert parallel.sum_over_ranks(2.0) == 2.0


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, out):
    import torch.distributed as td
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    td.init_process_group("gloo", rank=rank, world_size=world)
    try:
        share = parallel.rank_share(10, rank, world)
        step_ms = 5.0 + rank  # rank 1 is the slow one
        out[rank] = (share, parallel.max_over_ranks(step_ms), parallel.sum_over_ranks(len(share)))
    finally:
        td.destroy_process_group()


def test_two_gloo_ranks_combine_timings_and_work():
    ctx = mp.get_context("spawn")
    with ctx.Manager() as m:
        out = m.dict()
        port = _free_port()
        procs = [ctx.Process(target=_worker, args=(r, 2, port, out)) for r in range(2)]
        for p in procs:
            p.start()
        for p in procs:
            p.join(120)
            assert p.exitcode == 0
        res = dict(out)
    assert sorted(res[0][0] + res[1][0]) == list(range(10))
    assert res[0][1] == res[1][1] == 6.0
    assert res[0][2] == res[1][2] == 10.0

"""Multi-rank host logic of bench.py on CPU (gloo, world size 2): the time reported is the
max over ranks and the solve count the sum (independent solves per rank, no data-path
collective)."""
import os
import socket
import sys

import pytest
import torch.multiprocessing as tmp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _worker(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world),
                      LOCAL_RANK=str(rank))
    sys.path.insert(0, ROOT)
    import torch.distributed as dist
    import bench
    dist.init_process_group("gloo", rank=rank, world_size=world)
    t = bench.max_over_ranks(10.0 + rank, dist)
    s = bench.sum_over_ranks(9.0, dist)
    bench.barrier(dist)
    out[rank] = (t, s, bench.rank_of(dist), bench.world_of(dist))
    dist.destroy_process_group()


@pytest.mark.timeout(120)
def test_max_time_and_summed_solves_over_two_ranks():
    ctx = tmp.get_context("spawn")
    mgr = ctx.Manager()
    out = mgr.dict()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, out)) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(90)
        assert p.exitcode == 0
    assert out[0] == (11.0, 18.0, 0, 2)
    assert out[1] == (11.0, 18.0, 1, 2)


def test_single_process_helpers_are_identity():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.max_over_ranks(3.5, None) == 3.5
    assert bench.sum_over_ranks(2.0, None) == 2.0
    assert bench.rank_of(None) == 0 and bench.world_of(None) == 1

"""The multi-GPU path is replicas only (independent runs per rank, no data
exchange); what it adds on the host is the seed split and the whole-job
aggregation, checked here with two gloo ranks on the CPU."""
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
    import torch
    import torch.distributed as dist
    sys.path.insert(0, ROOT)
    import bench
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world),
                      LOCAL_RANK=str(rank))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    r, w, loc = bench.dist_env()
    # rank r reports (time, dead, evals) = (10 + 5 r, 1000 (r + 1), 7 + r)
    res = bench.aggregate(10.0 + 5 * r, 1000.0 * (r + 1), 7.0 + r, w, torch.device("cpu"))
    out[rank] = (r, w, loc, res, bench.rank_seeds(r, 20))
    dist.barrier()
    dist.destroy_process_group()


@pytest.mark.timeout(120)
def test_two_gloo_ranks_split_seeds_and_aggregate():
    torch = pytest.importorskip("torch")
    import torch.multiprocessing as mp
    port = _free_port()
    with mp.Manager() as man:
        out = man.dict()
        mp.spawn(_rank_main, args=(2, port, out), nprocs=2, join=True)
        got = dict(out)
    for rank in (0, 1):
        r, w, loc, res, seeds = got[rank]
        assert (r, w, loc) == (rank, 2, rank)
        # slowest rank's time, summed units
        assert res == (15.0, 3000.0, 15.0)
    assert set(got[0][4]).isdisjoint(got[1][4])
    assert sorted(got[0][4] + got[1][4]) == list(range(40))


def test_single_rank_aggregate_is_identity():
    pytest.importorskip("torch")
    sys.path.insert(0, ROOT)
    import bench
    assert bench.aggregate(12.5, 100, 9, 1, None) == (12.5, 100.0, 9.0)
    assert bench.rank_seeds(0, 3) == [0, 1, 2]

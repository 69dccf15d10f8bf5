"""Multi-GPU path of bench.py ("replicas only": the solves shard by
right-hand side with no exchange): the whole-job timing takes the slowest
rank and the units of all ranks.  Run as two gloo processes on CPU."""
import os
import socket
import sys

import pytest
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, ms, units, out):
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    sys.path.insert(0, ROOT)
    import bench
    out[rank] = bench.replicas_aggregate(ms[rank], units[rank], world, "cpu")
    dist.barrier()
    dist.destroy_process_group()


@pytest.mark.parametrize("world", [2, 3])
def test_replicas_take_slowest_rank_and_all_units(world):
    ctx = mp.get_context("spawn")
    ms = [10.0 + 5.0 * r for r in range(world)]
    units = [1536.0] * world
    port = _free_port()
    with ctx.Manager() as mgr:
        out = mgr.dict()
        procs = [ctx.Process(target=_worker, args=(r, world, port, ms, units, out))
                 for r in range(world)]
        for p in procs:
            p.start()
        for p in procs:
            p.join(120)
        codes = [p.exitcode for p in procs]
        res = dict(out)
    assert codes == [0] * world
    for r in range(world):
        assert res[r] == (max(ms), sum(units))


def test_single_process_is_identity():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.replicas_aggregate(12.5, 768.0, 1, "cpu") == (12.5, 768.0)


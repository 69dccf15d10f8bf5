"""Host logic of the frequency sharding (Sec. IV-D: sources spread over
workers, partial products aggregated): the round-robin frequency partition,
and the reducers that the library calls through fwi_set_reducer, driven
through the same C function-pointer type the library calls, as two gloo
processes on CPU (host buffers stand in for the device buffers)."""
import ctypes
import os
import socket
import sys

import numpy as np
import pytest
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


@pytest.mark.parametrize("n_freq,world", [(6, 2), (6, 4), (12, 8), (4, 4), (3, 5)])
def test_frequency_shards_cover_every_frequency_once(n_freq, world):
    from paper_2604_15796_gb300 import sharding
    shards = [sharding.frequency_shard(n_freq, world, r) for r in range(world)]
    flat = sorted(l for s in shards for l in s)
    assert flat == list(range(n_freq))
    sizes = [len(s) for s in shards]
    assert max(sizes) - min(sizes) <= 1
    # round robin: each rank's frequencies span the band
    for s in shards:
        assert all(b - a == world for a, b in zip(s, s[1:]))
    with pytest.raises(ValueError):
        sharding.frequency_shard(n_freq, world, world)


def _worker(rank, world, port, kind, out):
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    sys.path.insert(0, ROOT)
    from paper_2604_15796_gb300 import libfwi, sharding
    make = {"collective": sharding.collective_reducer,
            "host_staged": sharding.host_staged_reducer}[kind]
    fn = libfwi.reduce_callback(make(wrap=sharding.host_array))
    buf = np.arange(10, dtype=np.float64) * (rank + 1) + 0.25 * rank
    # the library calls the reducer through this pointer type
    cfun = ctypes.cast(fn, libfwi.REDUCE_FN)
    rc = cfun(buf.ctypes.data, buf.size, None, None)
    out[rank] = (rc, buf.tolist())
    dist.barrier()
    dist.destroy_process_group()


@pytest.mark.parametrize("kind", ["collective", "host_staged"])
def test_reducer_sums_over_ranks_through_the_c_callback(kind):
    world = 2
    ctx = mp.get_context("spawn")
    port = _free_port()
    with ctx.Manager() as mgr:
        out = mgr.dict()
        procs = [ctx.Process(target=_worker, args=(r, world, port, kind, out))
                 for r in range(world)]
        for p in procs:
            p.start()
        for p in procs:
            p.join(120)
        codes = [p.exitcode for p in procs]
        res = dict(out)
    assert codes == [0] * world
    want = sum(np.arange(10) * (r + 1) + 0.25 * r for r in range(world))
    for r in range(world):
        rc, got = res[r]
        assert rc == 0
        assert np.array_equal(np.asarray(got), want)


def test_reducer_failure_is_reported_as_nonzero():
    from paper_2604_15796_gb300 import libfwi

    def broken(ptr, count, stream):
        raise RuntimeError("peer lost")
    fn = libfwi.reduce_callback(broken)
    buf = np.zeros(4)
    assert ctypes.cast(fn, libfwi.REDUCE_FN)(buf.ctypes.data, 4, None, None) == 1
    assert libfwi.FWI_ERR_REDUCE == 9 and libfwi.STATUS_NAMES[9] == "REDUCE"

"""Frequency sharding (Sec. IV-D) through the C ABI: two ranks, each a
process with a context holding half of the frequencies (round robin) and
the matching rows of d_obs, with a host-staged gloo reducer
(fwi_set_reducer).  Both ranks run on cuda:0 as independent processes:
their kernels never wait on one another, every exchange goes through the
host.  Every rank must return the gradient and misfit of all frequencies
(Eq. 7, 17) and, after one ADMM-TV iteration (Eq. 9-14), the same m, g, u
and SoS as the oracle's step over all frequencies; the two ranks' results
must be bitwise equal."""
import os
import socket
import sys

import numpy as np
import pytest
import torch.multiprocessing as mp

from gpu_common import oracle_problem, rel_l2, small_workload
from oracle import admm, inverse, model

pytestmark = pytest.mark.gpu
ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
FREQS = (1.0e6, 1.5e6, 2.0e6, 2.5e6, 3.0e6)


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _case():
    w = small_workload((32, 32), n_elem=6, freqs=FREQS, seed=17)
    prob = oracle_problem(w)
    sos0 = np.full(w.shape, w.c0) + 0.5 * (w.sos - w.c0)
    m0 = model.contrast_from_sos(sos0, w.c0)
    _, d = inverse.forward_model(model.contrast_from_sos(w.sos, w.c0), prob, "lu")
    d = d.astype(np.complex64)
    return w, prob, m0, d


def _rank(rank, world, port, params, out):
    import torch
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    sys.path.insert(0, ROOT)
    sys.path.insert(0, os.path.join(ROOT, "tests"))
    from paper_2604_15796_gb300 import libfwi, sharding
    torch.cuda.set_device(0)
    w, prob, m0, d = _case()
    idx = sharding.frequency_shard(len(FREQS), world, rank)
    ctx = libfwi.Context(w.shape, w.h, w.c0, w.elem, np.asarray(FREQS)[idx], tol=1e-6)
    ctx.set_reducer(sharding.host_staged_reducer())
    m = torch.from_numpy(m0).cuda()
    grad = torch.empty(w.shape, dtype=torch.complex128, device="cuda")
    mis, _, _ = ctx.gradient(m, torch.from_numpy(np.ascontiguousarray(d[idx])).cuda(), grad)
    g = torch.from_numpy(admm.grad_op(m0, w.shape)).cuda()
    u = torch.zeros_like(g)
    sos = torch.empty(w.shape, dtype=torch.float64, device="cuda")
    ctx.admm_tv_step(m, g, u, grad, sos=sos, **params)
    torch.cuda.synchronize()
    out[rank] = (grad.cpu().numpy(), mis, m.cpu().numpy(), g.cpu().numpy(), u.cpu().numpy(),
                 sos.cpu().numpy())
    ctx.close()
    dist.barrier()
    dist.destroy_process_group()


def test_two_ranks_sharded_by_frequency_match_the_oracle():
    w, prob, m0, d = _case()
    ref = inverse.gradient(m0, d.astype(np.complex128), prob, "lu")
    scale = float(np.abs(ref["grad"]).max())
    p = admm.AdmmParams(lam=1e-3 * scale, rho=0.5 * scale, gamma=1e-3 * scale, n_cg=6)
    rf = inverse.receiver_fields(m0, prob, "lu")
    g0 = admm.grad_op(m0, w.shape)
    rm, rg, ru, rsos, _ = admm.admm_tv_step(m0, g0, np.zeros_like(g0), ref["grad"],
                                            ref["fields"], rf, prob, p)
    params = dict(lam=p.lam, rho=p.rho, gamma=p.gamma, n_cg=p.n_cg)
    world = 2
    ctx = mp.get_context("spawn")
    port = _free_port()
    with ctx.Manager() as mgr:
        out = mgr.dict()
        procs = [ctx.Process(target=_rank, args=(r, world, port, params, out))
                 for r in range(world)]
        for q in procs:
            q.start()
        for q in procs:
            q.join(600)
        codes = [q.exitcode for q in procs]
        res = dict(out)
    assert codes == [0] * world
    for r in range(world):
        grad, mis, m1, g1, u1, sos1 = res[r]
        assert rel_l2(grad, ref["grad"]) < 1e-3, rel_l2(grad, ref["grad"])
        assert abs(mis - ref["misfit"]) <= 1e-3 * ref["misfit"]
        assert rel_l2(m1 - m0, rm - m0) < 1e-3
        assert rel_l2(sos1, rsos) < 1e-3
        assert rel_l2(g1, rg) < 1e-3 and rel_l2(u1, ru) < 1e-3
    for a, b in zip(res[0], res[1]):
        assert np.array_equal(np.asarray(a), np.asarray(b))

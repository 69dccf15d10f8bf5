"""Checkpoint / resume: two ADMM-TV iterations run straight through, and the
same run interrupted after the first (state saved, context destroyed, a new
context created, state loaded), give bit-identical contrast, TV variables
and SoS."""
import numpy as np
import pytest

from gpu_common import contrast, oracle_problem, small_workload, to_gpu
from oracle import inverse
from paper_2604_15796_gb300 import checkpoint

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def lib():
    import torch
    from paper_2604_15796_gb300 import build, libfwi
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    build.build()
    return libfwi


def test_resumed_run_repeats_the_uninterrupted_run(lib, tmp_path):
    import torch
    w = small_workload((32, 32), n_elem=8, freqs=(1.5e6, 3.0e6))
    _, d = inverse.forward_model(contrast(w), oracle_problem(w), "bicgstab", tol=1e-10)
    d_gpu = to_gpu(d, torch.complex64)
    sos0 = to_gpu(w.c0 + 0.5 * (w.sos - w.c0), torch.float64)

    def new_ctx():
        return lib.Context(w.shape, w.h, w.c0, w.elem, w.freqs)

    def iterate(ctx, m, g, u, n, prm):
        grad = torch.empty(w.shape, dtype=torch.complex128, device="cuda")
        sos = torch.empty(w.shape, dtype=torch.float64, device="cuda")
        for _ in range(n):
            ctx.gradient(m, d_gpu, grad)
            ctx.admm_tv_step(m, g, u, grad, sos=sos, **prm)
        return sos

    ctx = new_ctx()
    m = ctx.contrast_from_sos(sos0)
    grad = torch.empty(w.shape, dtype=torch.complex128, device="cuda")
    ctx.gradient(m, d_gpu, grad)
    s = float(grad.abs().max())
    prm = dict(lam=1e-3 * s, rho=0.5 * s, gamma=1e-3 * s, n_cg=4)
    g, u = ctx.admm_init(m)
    sos_full = iterate(ctx, m, g, u, 2, prm)
    ctx.close()

    ctx1 = new_ctx()
    m1 = ctx1.contrast_from_sos(sos0)
    g1, u1 = ctx1.admm_init(m1)
    iterate(ctx1, m1, g1, u1, 1, prm)
    path = str(tmp_path / "state.npz")
    checkpoint.save(path, 1, m1, g1, u1, prm)
    ctx1.close()

    ctx2 = new_ctx()
    k, m2, g2, u2, prm2 = checkpoint.load(path)
    assert k == 1 and prm2 == prm
    sos2 = iterate(ctx2, m2, g2, u2, 1, prm2)
    ctx2.close()
    for a, b in ((m2, m), (g2, g), (u2, u), (sos2, sos_full)):
        assert torch.equal(a, b)
    assert np.isfinite(sos2.cpu().numpy()).all()

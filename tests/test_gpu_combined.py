"""The acquisition and model options together: plane-wave transmits, an
attenuating background and an inversion mesh in one context, against the
oracle (data, gradient and one ADMM-TV step)."""
import numpy as np
import pytest

from gpu_common import oracle_problem, rel_l2, small_workload, to_gpu, to_np
from oracle import admm, inverse, model
from paper_2604_15796_gb300 import phantoms

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def lib():
    import torch
    from paper_2604_15796_gb300 import build, libfwi
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    build.build()
    return libfwi


def test_plane_waves_lossy_background_and_inversion_mesh(lib):
    import torch
    alpha0, r = 1e-4, 2
    w = small_workload((32, 32), n_elem=6, freqs=(1.5e6, 3.0e6))
    prob = oracle_problem(w)
    prob.extra.update(alpha0=alpha0, inv_factor=r)
    ang = np.deg2rad([-30.0, 0.0, 20.0, 45.0])
    W = model.plane_wave_weights(prob, ang)
    sh = model.inversion_shape(prob)
    m_fine = model.contrast_from_sos(w.sos, w.c0, None, alpha0)
    m_true = model.restrict(m_fine, prob) / r ** 2
    m0 = 0.5 * m_true
    _, d_true = inverse.forward_model(model.prolong(m_true, prob), prob, "bicgstab", tol=1e-12,
                                      weights=W)
    d_obs = d_true.astype(np.complex64).astype(np.complex128)
    ref = inverse.gradient_inversion_mesh(m0, d_obs, prob, "bicgstab", tol=1e-12, weights=W)
    ctx = lib.Context(w.shape, w.h, w.c0, w.elem, w.freqs, tx_angles=ang, alpha0=alpha0,
                      inv_factor=r)
    m_gpu = to_gpu(m0, torch.complex128)
    data = ctx.empty_data()
    ctx.forward(m_gpu, data=data)
    assert rel_l2(to_np(data), ref["data"]) < 1e-4
    grad = torch.empty(sh, dtype=torch.complex128, device="cuda")
    mis, _, _ = ctx.gradient(m_gpu, to_gpu(d_obs, torch.complex64), grad)
    assert rel_l2(to_np(grad), ref["grad_inv"]) < 1e-3
    assert abs(mis - ref["misfit"]) <= 1e-3 * ref["misfit"]
    rf = inverse.receiver_fields(model.prolong(m0, prob), prob, "bicgstab", tol=1e-12)
    s = float(np.abs(ref["grad_inv"]).max())
    p = admm.AdmmParams(lam=1e-3 * s, rho=0.5 * s, gamma=1e-3 * s, n_cg=6)
    g0 = admm.grad_op(m0, sh)
    u0 = 0.01 * phantoms.complex_normal(g0.shape, 12)
    _, g1, u1, sos1, dm = admm.admm_tv_step(m0, g0, u0, ref["grad_inv"], ref["fields"], rf,
                                            prob, p)
    g_gpu, u_gpu = to_gpu(g0, torch.complex128), to_gpu(u0, torch.complex128)
    sos = torch.empty(sh, dtype=torch.float64, device="cuda")
    ctx.admm_tv_step(m_gpu, g_gpu, u_gpu, grad, lam=p.lam, rho=p.rho, gamma=p.gamma,
                     n_cg=p.n_cg, sos=sos)
    ctx.close()
    assert rel_l2(to_np(m_gpu) - m0, dm) < 1e-3
    assert rel_l2(to_np(sos) - w.c0, sos1 - w.c0) < 1e-3
    assert rel_l2(to_np(g_gpu), g1) < 1e-3
    assert rel_l2(to_np(u_gpu), u1) < 1e-3

"""Inversion mesh coarser than the forward mesh (Sec. IV) through the C ABI:
the contrast, gradient, TV variables and SoS live on cells of r^d forward
pixels; the library prolongs the contrast into the forward solves and sums
gradients and J^H products over each cell.  Against the oracle's
prolong / restrict (2-D and 3-D, FP32 and FP64)."""
import numpy as np
import pytest

from gpu_common import contrast, oracle_problem, rel_l2, small_workload, to_gpu, to_np
from oracle import admm, inverse, model
from paper_2604_15796_gb300 import phantoms

pytestmark = pytest.mark.gpu

R = 2


@pytest.fixture(scope="module")
def lib():
    import torch
    from paper_2604_15796_gb300 import build, libfwi
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    build.build()
    return libfwi


def _case(shape, n_elem, freqs):
    w = small_workload(shape, n_elem=n_elem, freqs=freqs)
    prob = oracle_problem(w)
    prob.extra["inv_factor"] = R
    sh = model.inversion_shape(prob)
    # the phantom's contrast averaged over each cell, on the inversion mesh
    m_true = model.restrict(contrast(w), prob) / R ** len(shape)
    return w, prob, sh, m_true


@pytest.mark.parametrize("fp64", [False, True])
@pytest.mark.parametrize("shape,n_elem,freqs", [((32, 32), 6, (1.5e6, 3.0e6)),
                                                ((8, 8, 16), 5, (1.0e6, 2.0e6))])
def test_inversion_mesh_data_gradient_and_admm_step(lib, shape, n_elem, freqs, fp64):
    import torch
    w, prob, sh, m_true = _case(shape, n_elem, freqs)
    m0 = 0.5 * m_true
    _, d_true = inverse.forward_model(model.prolong(m_true, prob), prob, "bicgstab", tol=1e-12)
    fdt = torch.complex128 if fp64 else torch.complex64
    d_obs = d_true if fp64 else d_true.astype(np.complex64).astype(np.complex128)
    ref = inverse.gradient_inversion_mesh(m0, d_obs, prob, "bicgstab", tol=1e-12)
    ctx = lib.Context(w.shape, w.h, w.c0, w.elem, w.freqs,
                      precision=lib.FWI_FP64 if fp64 else lib.FWI_MIXED,
                      tol=1e-12 if fp64 else 1e-6, inv_factor=R)
    assert ctx.inv_shape == sh
    tol_d, tol_g = (1e-8, 1e-8) if fp64 else (1e-4, 1e-3)
    m_gpu = to_gpu(m0, torch.complex128)
    data = ctx.empty_data()
    ctx.forward(m_gpu, data=data)
    assert rel_l2(to_np(data), ref["data"]) < tol_d
    grad = torch.empty(sh, dtype=torch.complex128, device="cuda")
    mis, _, _ = ctx.gradient(m_gpu, to_gpu(d_obs, fdt), grad)
    assert rel_l2(to_np(grad), ref["grad_inv"]) < tol_g
    assert abs(mis - ref["misfit"]) <= tol_g * ref["misfit"]
    rf = inverse.receiver_fields(model.prolong(m0, prob), prob, "bicgstab", tol=1e-12)
    scale = float(np.abs(ref["grad_inv"]).max())
    p = admm.AdmmParams(lam=1e-3 * scale, rho=0.5 * scale, gamma=1e-3 * scale, n_cg=6)
    g0 = admm.grad_op(m0, sh)
    u0 = 0.01 * phantoms.complex_normal(g0.shape, 12)
    _, g1, u1, sos1, dm = admm.admm_tv_step(m0, g0, u0, ref["grad_inv"], ref["fields"], rf,
                                            prob, p)
    g_gpu, u_gpu = to_gpu(g0, torch.complex128), to_gpu(u0, torch.complex128)
    sos = torch.empty(sh, dtype=torch.float64, device="cuda")
    ctx.admm_tv_step(m_gpu, g_gpu, u_gpu, grad, lam=p.lam, rho=p.rho, gamma=p.gamma,
                     n_cg=p.n_cg, sos=sos)
    ctx.close()
    assert rel_l2(to_np(m_gpu) - m0, dm) < tol_g
    assert rel_l2(to_np(sos) - w.c0, sos1 - w.c0) < tol_g
    assert rel_l2(to_np(g_gpu), g1) < tol_g
    assert rel_l2(to_np(u_gpu), u1) < tol_g


def test_inversion_mesh_jacobian_products(lib):
    import torch
    w, prob, sh, m_true = _case((32, 32), 6, (1.5e6, 3.0e6))
    mf = model.prolong(m_true, prob)
    fields, _ = inverse.forward_model(mf, prob, "bicgstab", tol=1e-12)
    rf = inverse.receiver_fields(mf, prob, "bicgstab", tol=1e-12)
    a = phantoms.complex_normal(sh, 5)
    b = phantoms.complex_normal((w.n_freq, w.n_elem, w.n_elem), 6)
    ja_ref = inverse.jac_forward(model.prolong(a, prob), fields, rf, prob)
    jhb_ref = model.restrict(inverse.jac_adjoint(b, fields, rf, prob).reshape(w.shape), prob)
    ctx = lib.Context(w.shape, w.h, w.c0, w.elem, w.freqs, inv_factor=R)
    ctx.forward(to_gpu(m_true, torch.complex128))
    for tc in (True, False):
        ctx.set_jac_tensor_cores(tc)
        ja = to_np(ctx.jac_forward(to_gpu(a, torch.complex128)))
        jhb = to_np(ctx.jac_adjoint(to_gpu(b, torch.complex128)))
        assert jhb.shape == sh
        assert rel_l2(ja, ja_ref) < 1e-4
        assert rel_l2(jhb, jhb_ref) < 1e-4
    ctx.close()


def test_inversion_mesh_request_in_the_server(lib):
    w, prob, sh, m_true = _case((32, 32), 6, (1.5e6, 3.0e6))
    sos_true = model.sos_from_contrast(m_true, w.c0)
    sos0 = w.c0 + 0.5 * (sos_true - w.c0)
    m0 = model.contrast_from_sos(sos0, w.c0)
    _, d_true = inverse.forward_model(model.prolong(m_true, prob), prob, "bicgstab", tol=1e-12)
    d = d_true.astype(np.complex64)
    ref = inverse.gradient_inversion_mesh(m0, d.astype(np.complex128), prob, "bicgstab",
                                          tol=1e-12)
    scale = float(np.abs(ref["grad_inv"]).max())
    p = admm.AdmmParams(lam=1e-3 * scale, rho=0.5 * scale, gamma=1e-3 * scale, n_cg=6)
    rf = inverse.receiver_fields(model.prolong(m0, prob), prob, "bicgstab", tol=1e-12)
    g0 = admm.grad_op(m0, sh)
    _, _, _, sos1, _ = admm.admm_tv_step(m0, g0, np.zeros_like(g0), ref["grad_inv"],
                                         ref["fields"], rf, prob, p)
    srv = lib.Server(max_active=1)
    sos, res = srv.wait(srv.submit(w.shape, w.h, w.c0, w.elem, w.freqs, sos0, d, n_iter=1,
                                   lam=p.lam, rho=p.rho, gamma=p.gamma, n_cg=p.n_cg,
                                   inv_factor=R))
    srv.close()
    assert res["status"] == 0 and sos.shape == sh
    assert rel_l2(sos - sos0, sos1 - sos0) < 1e-3
    assert abs(res["misfit_first"] - ref["misfit"]) <= 1e-3 * ref["misfit"]

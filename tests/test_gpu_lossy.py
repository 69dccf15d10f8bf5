"""Attenuating background (Eq. 1-3 with a complex kappa0; complex k) through
the C ABI against the oracle: the contrast map, the incident fields (2-D:
the device's complex-argument Hankel function; 3-D: complex exponentials;
line elements with their damping), and data, gradient and one ADMM-TV step
(SoS from the complex contrast), FP32 and FP64, 2-D and 3-D."""
import numpy as np
import pytest

from gpu_common import oracle_problem, rel_l2, small_workload, to_gpu, to_np
from oracle import admm, inverse, model, operator
from paper_2604_15796_gb300 import phantoms

pytestmark = pytest.mark.gpu

ALPHA0 = 1e-4  # Np/m/Hz: Im k / Re k ~ 0.025 (tissue: ~0.0015)


@pytest.fixture(scope="module")
def lib():
    import torch
    from paper_2604_15796_gb300 import build, libfwi
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    build.build()
    return libfwi


def _case(shape, n_elem=5, freqs=(1.5e6, 3.0e6), length=0.0):
    w = small_workload(shape, n_elem=n_elem, freqs=freqs)
    prob = oracle_problem(w)
    prob.extra["alpha0"] = ALPHA0
    prob.extra["elem_length"] = length
    return w, prob


@pytest.mark.parametrize("fp64", [False, True])
@pytest.mark.parametrize("shape,length", [((32, 32), 0.0), ((8, 8, 16), 0.0),
                                          ((8, 8, 16), 1e-2)])
def test_lossy_incident_fields_and_contrast(lib, shape, length, fp64):
    import torch
    w, prob = _case(shape, length=length)
    ctx = lib.Context(w.shape, w.h, w.c0, w.elem, w.freqs, alpha0=ALPHA0, elem_length=length,
                      precision=lib.FWI_FP64 if fp64 else lib.FWI_MIXED)
    m = ctx.contrast_from_sos(to_gpu(w.sos, torch.float64))
    m_ref = model.contrast_from_sos(w.sos, w.c0, None, ALPHA0)
    assert rel_l2(to_np(m), m_ref) < 1e-13
    fields = ctx.empty_fields()
    ctx.forward(torch.zeros(w.shape, dtype=torch.complex128, device="cuda"), fields=fields)
    ctx.close()
    assert rel_l2(to_np(fields), operator.incident_fields(prob)) < (1e-9 if fp64 else 1e-6)


@pytest.mark.parametrize("fp64", [False, True])
@pytest.mark.parametrize("shape", [(32, 32), (8, 8, 16)])
def test_lossy_data_gradient_and_admm_step(lib, shape, fp64):
    import torch
    w, prob = _case(shape)
    m_true = model.contrast_from_sos(w.sos, w.c0, None, ALPHA0)
    m0 = 0.5 * m_true
    _, d_true = inverse.forward_model(m_true, prob, "bicgstab", tol=1e-12)
    fdt = torch.complex128 if fp64 else torch.complex64
    d_obs = d_true if fp64 else d_true.astype(np.complex64).astype(np.complex128)
    ref = inverse.gradient(m0, d_obs, prob, "bicgstab", tol=1e-12)
    ctx = lib.Context(w.shape, w.h, w.c0, w.elem, w.freqs, alpha0=ALPHA0,
                      precision=lib.FWI_FP64 if fp64 else lib.FWI_MIXED,
                      tol=1e-12 if fp64 else 1e-6)
    tol_d, tol_g = (1e-8, 1e-8) if fp64 else (1e-4, 1e-3)
    m_gpu = to_gpu(m0, torch.complex128)
    data = ctx.empty_data()
    ctx.forward(m_gpu, data=data)
    assert rel_l2(to_np(data), ref["data"]) < tol_d
    grad = torch.empty(w.shape, dtype=torch.complex128, device="cuda")
    mis, _, _ = ctx.gradient(m_gpu, to_gpu(d_obs, fdt), grad)
    assert rel_l2(to_np(grad), ref["grad"]) < tol_g
    assert abs(mis - ref["misfit"]) <= tol_g * ref["misfit"]
    rf = inverse.receiver_fields(m0, prob, "bicgstab", tol=1e-12)
    scale = float(np.abs(ref["grad"]).max())
    p = admm.AdmmParams(lam=1e-3 * scale, rho=0.5 * scale, gamma=1e-3 * scale, n_cg=6)
    g0 = admm.grad_op(m0, w.shape)
    u0 = 0.01 * phantoms.complex_normal(g0.shape, 12)
    _, g1, u1, sos1, dm = admm.admm_tv_step(m0, g0, u0, ref["grad"], ref["fields"], rf, prob, p)
    g_gpu, u_gpu = to_gpu(g0, torch.complex128), to_gpu(u0, torch.complex128)
    sos = torch.empty(w.shape, dtype=torch.float64, device="cuda")
    ctx.admm_tv_step(m_gpu, g_gpu, u_gpu, grad, lam=p.lam, rho=p.rho, gamma=p.gamma,
                     n_cg=p.n_cg, sos=sos)
    ctx.close()
    assert rel_l2(to_np(m_gpu) - m0, dm) < tol_g
    assert rel_l2(to_np(sos) - w.c0, sos1 - w.c0) < tol_g
    assert rel_l2(to_np(g_gpu), g1) < tol_g
    assert rel_l2(to_np(u_gpu), u1) < tol_g


@pytest.mark.parametrize("alpha0", [ALPHA0, 0.0])
def test_sos_and_attenuation_from_the_contrast(lib, alpha0):
    """Attenuation inversion output: the device's inverse of the contrast map
    against the oracle's, and the round trip from (SoS, attenuation)."""
    import torch
    w, _ = _case((32, 32))
    alpha = 2e-5 + 1e-5 * phantoms.complex_normal(w.shape, 3).real ** 2
    m_ref = model.contrast_from_sos(w.sos, w.c0, alpha, alpha0)
    ctx = lib.Context(w.shape, w.h, w.c0, w.elem, w.freqs, alpha0=alpha0)
    m = ctx.contrast_from_sos(to_gpu(w.sos, torch.float64), to_gpu(alpha, torch.float64))
    sos, att = ctx.sos_attenuation_from_contrast(m)
    ctx.close()
    assert rel_l2(to_np(m), m_ref) < 1e-13
    assert rel_l2(to_np(sos), model.sos_from_contrast(m_ref, w.c0, alpha0)) < 1e-13
    assert rel_l2(to_np(att), model.attenuation_from_contrast(m_ref, w.c0, alpha0)) < 1e-10
    assert rel_l2(to_np(sos), w.sos) < 1e-13 and rel_l2(to_np(att), alpha) < 1e-10


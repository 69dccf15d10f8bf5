"""Plane-wave transmits (Sec. V-A) through the C ABI against the oracle.

The library solves the element point sources and synthesises the plane
waves by superposition (data, residual and Jacobian rows are weighted sums
over elements); the oracle solves every plane-wave transmit field directly
from its own incident field, solves the receiver fields separately
(Sec. IV-B, refreshed every iteration), and computes its weights itself.
Cases: fewer, equal and more transmits than elements; 2-D and 3-D; FP32
fields with FP64 scalars and the FP64 path."""
import numpy as np
import pytest

from gpu_common import contrast, oracle_problem, rel_l2, small_workload, to_gpu, to_np
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


# (shape, n_elem, freqs, steering angles in degrees)
CASES = [((32, 32), 6, (1.5e6, 3.0e6), (-40.0, -10.0, 0.0, 15.0, 35.0)),
         ((16, 64), 8, (2.0e6,), tuple(np.linspace(-60.0, 60.0, 11))),
         ((8, 8, 16), 5, (1.0e6, 2.0e6), (-20.0, 0.0, 20.0))]


def _case(shape, n_elem, freqs, deg):
    w = small_workload(shape, n_elem=n_elem, freqs=freqs)
    prob = oracle_problem(w)
    ang = np.deg2rad(np.asarray(deg, dtype=np.float64))
    return w, prob, ang, model.plane_wave_weights(prob, ang)


@pytest.mark.parametrize("fp64", [False, True])
@pytest.mark.parametrize("shape,n_elem,freqs,deg", CASES)
def test_plane_wave_data_gradient_and_admm_step(lib, shape, n_elem, freqs, deg, fp64):
    import torch
    w, prob, ang, W = _case(shape, n_elem, freqs, deg)
    m_true = contrast(w)
    m0 = 0.5 * m_true
    _, d_true = inverse.forward_model(m_true, prob, "bicgstab", tol=1e-12, weights=W)
    fdt = torch.complex128 if fp64 else torch.complex64
    d_obs = d_true if fp64 else d_true.astype(np.complex64).astype(np.complex128)
    ref = inverse.gradient(m0, d_obs, prob, "bicgstab", tol=1e-12, weights=W)
    ctx = lib.Context(w.shape, w.h, w.c0, w.elem, w.freqs,
                      precision=lib.FWI_FP64 if fp64 else lib.FWI_MIXED,
                      tol=1e-12 if fp64 else 1e-6, tx_angles=ang)
    assert ctx.n_t == len(ang)
    tol_d, tol_g = (1e-8, 1e-8) if fp64 else (1e-4, 1e-3)
    m_gpu = to_gpu(m0, torch.complex128)
    data = ctx.empty_data()
    assert tuple(data.shape) == (w.n_freq, len(ang), w.n_elem)
    ctx.forward(m_gpu, data=data)
    assert rel_l2(to_np(data), ref["data"]) < tol_d
    grad = torch.empty(w.shape, dtype=torch.complex128, device="cuda")
    mis, _, _ = ctx.gradient(m_gpu, to_gpu(d_obs, fdt), grad)
    assert rel_l2(to_np(grad), ref["grad"]) < tol_g
    assert abs(mis - ref["misfit"]) <= tol_g * ref["misfit"]
    # one ADMM-TV step against the oracle's, with the receiver fields solved
    # separately at the current model (strict distorted Born)
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


def test_plane_wave_jacobian_products(lib):
    """J a and J^H b of the plane-wave data map (Eq. 15-17 with transmit
    fields of the plane waves and separately solved receiver fields), on the
    tensor-core and the CUDA-core contractions."""
    import torch
    w, prob, ang, W = _case(*CASES[0])
    m = contrast(w)
    fields_pw, _ = inverse.forward_model(m, prob, "bicgstab", tol=1e-12, weights=W)
    rf = inverse.receiver_fields(m, prob, "bicgstab", tol=1e-12)
    a = phantoms.complex_normal(w.shape, 5)
    b = phantoms.complex_normal((w.n_freq, len(ang), w.n_elem), 6)
    ja_ref = inverse.jac_forward(a, fields_pw, rf, prob)
    jhb_ref = inverse.jac_adjoint(b, fields_pw, rf, prob)
    ctx = lib.Context(w.shape, w.h, w.c0, w.elem, w.freqs, tx_angles=ang)
    ctx.forward(to_gpu(m, torch.complex128))
    out = {}
    for tc in (True, False):
        ctx.set_jac_tensor_cores(tc)
        out[tc] = (to_np(ctx.jac_forward(to_gpu(a, torch.complex128))),
                   to_np(ctx.jac_adjoint(to_gpu(b, torch.complex128))))
    ctx.close()
    for tc in (True, False):
        assert out[tc][0].shape == ja_ref.shape
        assert rel_l2(out[tc][0], ja_ref) < 1e-4
        assert rel_l2(out[tc][1], jhb_ref) < 1e-4
    assert rel_l2(out[True][0], out[False][0]) < 2e-6
    assert rel_l2(out[True][1], out[False][1]) < 2e-6


def test_plane_wave_request_alone_in_the_mix_and_against_the_oracle(lib):
    """A plane-wave reconstruction request through the server: one iteration
    matches the oracle; its result is the same alone and beside a
    point-transmit request."""
    w, prob, ang, W = _case(*CASES[0])
    m_true = contrast(w)
    sos0 = np.full(w.shape, w.c0) + 0.5 * (w.sos - w.c0)
    m0 = model.contrast_from_sos(sos0, w.c0)
    _, d_true = inverse.forward_model(m_true, prob, "bicgstab", tol=1e-12, weights=W)
    d = d_true.astype(np.complex64)
    ref = inverse.gradient(m0, d.astype(np.complex128), prob, "bicgstab", tol=1e-12, weights=W)
    scale = float(np.abs(ref["grad"]).max())
    p = admm.AdmmParams(lam=1e-3 * scale, rho=0.5 * scale, gamma=1e-3 * scale, n_cg=6)
    rf = inverse.receiver_fields(m0, prob, "bicgstab", tol=1e-12)
    g0 = admm.grad_op(m0, w.shape)
    _, _, _, sos1, _ = admm.admm_tv_step(m0, g0, np.zeros_like(g0), ref["grad"], ref["fields"],
                                         rf, prob, p)
    prm = dict(n_iter=1, lam=p.lam, rho=p.rho, gamma=p.gamma, n_cg=p.n_cg)
    srv = lib.Server(max_active=1)
    sos_alone, res = srv.wait(srv.submit(w.shape, w.h, w.c0, w.elem, w.freqs, sos0, d,
                                         tx_angles=ang, **prm))
    srv.close()
    assert res["status"] == 0
    assert rel_l2(sos_alone - sos0, sos1 - sos0) < 1e-3
    assert abs(res["misfit_first"] - ref["misfit"]) <= 1e-3 * ref["misfit"]
    # beside a point-transmit request of another grid
    w2 = small_workload((16, 64), n_elem=5, freqs=(2.0e6,), seed=3)
    _, d2 = inverse.forward_model(contrast(w2), oracle_problem(w2), "bicgstab", tol=1e-10)
    srv = lib.Server(max_active=2)
    ids = [srv.submit(w.shape, w.h, w.c0, w.elem, w.freqs, sos0, d, tx_angles=ang, **prm),
           srv.submit(w2.shape, w2.h, w2.c0, w2.elem, w2.freqs, np.full(w2.shape, w2.c0),
                      d2.astype(np.complex64), **prm)]
    mix = [srv.wait(i) for i in ids]
    srv.close()
    assert mix[0][1]["status"] == 0 and mix[1][1]["status"] == 0
    assert rel_l2(mix[0][0], sos_alone) < 1e-12

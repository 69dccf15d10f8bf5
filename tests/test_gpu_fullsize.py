"""Parity at full size, in the launch configuration the benchmark times
(FP32 fields, Krylov tolerance 1e-6, every right-hand side batched, on a
side stream, autotuned tile shapes): the 2-D thyroid-like workload (256^2
grid, 0.1 mm pixels, 128 elements, 6 frequencies 0.5-3 MHz: 768 right-hand
sides) and the 3-D single-sided volume (160 x 160 x 128 voxels of 0.2 mm,
128 elements, 4 frequencies 0.5-2 MHz: 512 right-hand sides), on outputs
the FP64 oracle computes one by one:

* sampled forward fields and their data rows (Eq. 4-5), at the lowest and
  highest frequency and the first, middle and last element;
* sampled adjoint fields for seeded sources ((I - M K)^H lambda = s; 2-D);
* the gradient, a sum over all right-hand sides, through identities that
  hold at any size: <a, grad> = <J a, r> (grad = J^H r, Sec. IV-A) with J a
  from the device's Jacobian, and the misfit 1/2 ||d - d_obs||^2 (Eq. 7)
  evaluated on the host from the device's data."""
import numpy as np
import pytest

import oracle
from gpu_common import rel_l2, to_gpu, to_np
from oracle import inverse, model, operator
from paper_2604_15796_gb300 import phantoms

pytestmark = pytest.mark.gpu

FORWARD_SAMPLES = [(0, 0), (5, 127), (3, 64)]   # (frequency, element)
ADJOINT_SAMPLES = [(1, 5), (4, 100)]


@pytest.fixture(scope="module")
def lib():
    import torch
    from paper_2604_15796_gb300 import build, libfwi
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    build.build()
    return libfwi


def _one_frequency(w, l, elem=None):
    return oracle.Problem(tuple(w.shape), w.h, w.c0, w.elem if elem is None else elem,
                          np.asarray([w.freqs[l]]))


def test_thyroid256_sampled_parity(lib):
    import torch
    w = phantoms.thyroid_256()
    assert w.shape == (256, 256) and w.n_elem == 128 and w.n_freq == 6
    m = 0.8 * model.contrast_from_sos(w.sos, w.c0)
    src = phantoms.complex_normal((w.n_freq, w.n_elem) + tuple(w.shape), 31)
    stream = torch.cuda.Stream()
    with torch.cuda.stream(stream):
        ctx = lib.Context(w.shape, w.h, w.c0, w.elem, w.freqs, tol=1e-6, stream=stream)
        assert ctx.n_rhs == 768
        m_gpu = to_gpu(m, torch.complex128)
        fields = ctx.empty_fields()
        data = ctx.empty_data()
        rep = ctx.forward(m_gpu, fields=fields, data=data)
        assert rep.info.n_not_converged == 0
        lam = ctx.empty_fields()
        ctx.adjoint(m_gpu, to_gpu(src, torch.complex64), lam)
        # gradient at m for d_obs = d(m) + 10 % seeded noise
        noise = phantoms.complex_normal(tuple(data.shape), 32)
        rms = float(torch.linalg.vector_norm(data).item()) / np.sqrt(data.numel())
        d_obs = data + torch.from_numpy(0.1 * rms * noise).to(device="cuda", dtype=data.dtype)
        grad = torch.empty(w.shape, dtype=torch.complex128, device="cuda")
        d_grad = ctx.empty_data()
        mis, rf, ra = ctx.gradient(m_gpu, d_obs, grad, data=d_grad)
        assert rf.info.n_not_converged == 0 and ra.info.n_not_converged == 0
        a = to_gpu(phantoms.complex_normal(w.shape, 33), torch.complex128)
        j_grad = ctx.jac_forward(grad)
        j_a = ctx.jac_forward(a)
        stream.synchronize()
    fields_h, data_h, lam_h = to_np(fields), to_np(data), to_np(lam)
    grad_h, a_h = to_np(grad), to_np(a)
    r = to_np(d_grad).astype(np.complex128) - to_np(d_obs).astype(np.complex128)
    jg, ja = to_np(j_grad), to_np(j_a)
    ctx.close()

    # forward fields and data rows against the oracle's solves
    for l, e in FORWARD_SAMPLES:
        prob = _one_frequency(w, l)
        b = operator.incident_fields(_one_frequency(w, l, w.elem[[e]]))[0]
        x, info = operator.solve(m, b, prob, 0, "bicgstab", tol=1e-10)
        assert info[0][1] <= 1e-10
        row = inverse.forward_data(m, x[None], prob)[0, 0]
        assert rel_l2(fields_h[l, e], x[0]) < 1e-4, (l, e)
        assert rel_l2(data_h[l, e], row) < 1e-4, (l, e)
    # adjoint fields for the seeded sources (rounded to FP32 as the device
    # received them)
    for l, e in ADJOINT_SAMPLES:
        s = src[l, e].astype(np.complex64).astype(np.complex128)
        ref = inverse.solve_adjoint(m, s[None, None], _one_frequency(w, l), "bicgstab",
                                    tol=1e-10)[0, 0]
        assert rel_l2(lam_h[l, e], ref) < 1e-4, (l, e)
    # the gradient is J^H r: <grad, grad> = <J grad, r>, <a, grad> = <J a, r>
    g2 = np.vdot(grad_h, grad_h).real
    assert abs(np.vdot(jg, r) - g2) <= 1e-3 * g2
    scale = np.linalg.norm(a_h) * np.linalg.norm(grad_h)
    assert abs(np.vdot(ja, r) - np.vdot(a_h, grad_h)) <= 1e-3 * scale
    # the misfit from the device's data
    assert abs(mis - 0.5 * np.vdot(r, r).real) <= 1e-5 * mis
    # the gradient's data are the forward data (same model, same launch)
    assert rel_l2(to_np(d_grad), data_h) < 1e-5


def test_volume3d_sampled_parity(lib):
    """Sampled fields and data entries (receivers 0, 31, 64, 100, 127) at the
    lowest and highest frequency, and the gradient identities."""
    import torch
    w = phantoms.volume_3d()
    assert w.shape == (128, 160, 160) and w.n_elem == 128 and w.n_freq == 4
    m = 0.8 * model.contrast_from_sos(w.sos, w.c0)
    samples = [(0, 10), (3, 77)]
    rx = [0, 31, 64, 100, 127]
    stream = torch.cuda.Stream()
    with torch.cuda.stream(stream):
        ctx = lib.Context(w.shape, w.h, w.c0, w.elem, w.freqs, tol=1e-6, stream=stream)
        assert ctx.n_rhs == 512
        m_gpu = to_gpu(m, torch.complex128)
        fields = ctx.empty_fields()
        data = ctx.empty_data()
        rep = ctx.forward(m_gpu, fields=fields, data=data)
        assert rep.info.n_not_converged == 0
        got = [fields[l, e].cpu().numpy() for l, e in samples]
        noise = phantoms.complex_normal(tuple(data.shape), 34)
        rms = float(torch.linalg.vector_norm(data).item()) / np.sqrt(data.numel())
        d_obs = data + torch.from_numpy(0.1 * rms * noise).to(device="cuda", dtype=data.dtype)
        grad = torch.empty(w.shape, dtype=torch.complex128, device="cuda")
        d_grad = ctx.empty_data()
        mis, rf, ra = ctx.gradient(m_gpu, d_obs, grad, data=d_grad)
        assert rf.info.n_not_converged == 0 and ra.info.n_not_converged == 0
        a = to_gpu(phantoms.complex_normal(w.shape, 35), torch.complex128)
        j_grad = ctx.jac_forward(grad)
        j_a = ctx.jac_forward(a)
        stream.synchronize()
    data_h, grad_h, a_h = to_np(data), to_np(grad), to_np(a)
    r = to_np(d_grad).astype(np.complex128) - to_np(d_obs).astype(np.complex128)
    jg, ja = to_np(j_grad), to_np(j_a)
    del fields
    ctx.close()
    for (l, e), f in zip(samples, got):
        prob = _one_frequency(w, l)
        b = operator.incident_fields(_one_frequency(w, l, w.elem[[e]]))[0]
        x, info = operator.solve(m, b, prob, 0, "bicgstab", tol=1e-10)
        assert info[0][1] <= 1e-10
        assert rel_l2(f, x[0]) < 1e-4, (l, e)
        row = inverse.forward_data(m, x[None], _one_frequency(w, l, w.elem[rx]))[0, 0]
        assert rel_l2(data_h[l, e, rx], row) < 1e-4, (l, e)
    g2 = np.vdot(grad_h, grad_h).real
    assert abs(np.vdot(jg, r) - g2) <= 1e-3 * g2
    scale = np.linalg.norm(a_h) * np.linalg.norm(grad_h)
    assert abs(np.vdot(ja, r) - np.vdot(a_h, grad_h)) <= 1e-3 * scale
    assert abs(mis - 0.5 * np.vdot(r, r).real) <= 1e-5 * mis

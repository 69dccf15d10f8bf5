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
  evaluated on the host from the device's data;
* the gradient element by element against the oracle, with the residual
  confined to a few (frequency, transmit) rows: d_obs equals the device's
  own data except in those rows, so every other row's residual is exactly
  zero (its adjoint source and adjoint field vanish) and the gradient is
  sum over the chosen rows of conj(p_e) lambda_e (Eq. 17), which the oracle
  computes from one forward and one adjoint solve per row;
* one ADMM-TV iteration (Eq. 9-14) with the oracle's fields (slow);
* sampled fields and data rows of the 512^2 large-aperture workload with
  all 2,304 right-hand sides in one launch."""
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


def _confined_residual_gradient(lib, w, m, rows, seed, rx=None):
    """Device gradient at m for d_obs = d(m) + delta, delta nonzero only in
    the (frequency, transmit) rows ``rows``; returns the device gradient,
    the residual rows the device formed (d - d_obs, FP64 from the device's
    FP32 values) and the misfit."""
    import torch
    stream = torch.cuda.Stream()
    with torch.cuda.stream(stream):
        ctx = lib.Context(w.shape, w.h, w.c0, w.elem, w.freqs, tol=1e-6, stream=stream)
        m_gpu = to_gpu(m, torch.complex128)
        data = ctx.empty_data()
        rep = ctx.forward(m_gpu, data=data)
        assert rep.info.n_not_converged == 0
        d_obs = data.clone()
        rng = np.random.default_rng(seed)
        for l, e in rows:
            row = data[l, e]
            rms = float(torch.linalg.vector_norm(row).item()) / np.sqrt(row.numel())
            noise = rng.standard_normal(row.shape) + 1j * rng.standard_normal(row.shape)
            d_obs[l, e] += torch.from_numpy(0.3 * rms * noise).to(device="cuda",
                                                                  dtype=data.dtype)
        grad = torch.empty(w.shape, dtype=torch.complex128, device="cuda")
        d_grad = ctx.empty_data()
        mis, rf, ra = ctx.gradient(m_gpu, d_obs, grad, data=d_grad)
        assert rf.info.n_not_converged == 0 and ra.info.n_not_converged == 0
        stream.synchronize()
    r = to_np(d_grad).astype(np.complex128) - to_np(d_obs).astype(np.complex128)
    g = to_np(grad)
    ctx.close()
    return g, r, mis


def _oracle_confined_gradient(w, m, rows, r):
    """sum over the rows of conj(p_{l,e}) lambda_{l,e}: one forward and one
    adjoint solve per row (BiCGSTAB, tol 1e-10), adjoint sources from the
    residual rows (Sec. IV-B, Eq. 17)."""
    ref = np.zeros(w.shape, dtype=np.complex128)
    for l, e in rows:
        prob = _one_frequency(w, l)
        b = operator.incident_fields(_one_frequency(w, l, w.elem[[e]]))[0]
        p, info = operator.solve(m, b, prob, 0, "bicgstab", tol=1e-10)
        assert info[0][1] <= 1e-10
        # s = sum_j conj(R_j) r_j, accumulated over blocks of 16 receivers
        src = np.zeros((1, 1) + tuple(w.shape), dtype=np.complex128)
        for j0 in range(0, w.n_elem, 16):
            sub = _one_frequency(w, l, w.elem[j0:j0 + 16])
            src += inverse.adjoint_sources(r[l, e, j0:j0 + 16][None, None], sub)
        lam = inverse.solve_adjoint(m, src, prob, "bicgstab", tol=1e-10)[0, 0]
        ref += np.conj(p[0]) * lam
    return ref


def test_thyroid256_gradient_with_confined_residual_matches_oracle(lib):
    w = phantoms.thyroid_256()
    m = 0.8 * model.contrast_from_sos(w.sos, w.c0)
    rows = [(0, 3), (5, 100), (2, 64)]
    g, r, mis = _confined_residual_gradient(lib, w, m, rows, 41)
    mask = np.zeros(r.shape[:2], dtype=bool)
    for l, e in rows:
        mask[l, e] = True
    # the other rows' residual vanishes (same model, same launch: the data
    # are reproduced to rounding at most)
    assert np.linalg.norm(r[~mask]) <= 1e-6 * np.linalg.norm(r[mask])
    assert abs(mis - 0.5 * np.vdot(r, r).real) <= 1e-5 * mis
    ref = _oracle_confined_gradient(w, m, rows, r)
    assert rel_l2(g, ref) < 1e-3, rel_l2(g, ref)


def test_volume3d_gradient_with_confined_residual_matches_oracle(lib):
    w = phantoms.volume_3d()
    m = 0.8 * model.contrast_from_sos(w.sos, w.c0)
    rows = [(0, 17), (3, 90)]
    g, r, mis = _confined_residual_gradient(lib, w, m, rows, 43)
    mask = np.zeros(r.shape[:2], dtype=bool)
    for l, e in rows:
        mask[l, e] = True
    assert np.linalg.norm(r[~mask]) <= 1e-6 * np.linalg.norm(r[mask])
    ref = _oracle_confined_gradient(w, m, rows, r)
    assert rel_l2(g, ref) < 1e-3, rel_l2(g, ref)


def test_large512_sampled_parity(lib):
    """All 192 x 12 = 2,304 right-hand sides of the 512^2 workload in one
    launch (the benchmark's configuration); fields and data rows at the
    lowest and highest frequency against the oracle's solves."""
    import torch
    w = phantoms.large_512()
    assert w.shape == (512, 512) and w.n_elem == 192 and w.n_freq == 12
    m = 0.8 * model.contrast_from_sos(w.sos, w.c0)
    samples = [(0, 0), (11, 191), (6, 95)]
    stream = torch.cuda.Stream()
    with torch.cuda.stream(stream):
        ctx = lib.Context(w.shape, w.h, w.c0, w.elem, w.freqs, tol=1e-6, stream=stream)
        assert ctx.n_rhs == 2304
        fields = ctx.empty_fields()
        data = ctx.empty_data()
        rep = ctx.forward(to_gpu(m, torch.complex128), fields=fields, data=data)
        assert rep.info.n_not_converged == 0
        got = [(fields[l, e].cpu().numpy(), data[l, e].cpu().numpy()) for l, e in samples]
        stream.synchronize()
    del fields
    ctx.close()
    for (l, e), (f, d) in zip(samples, got):
        prob = _one_frequency(w, l)
        b = operator.incident_fields(_one_frequency(w, l, w.elem[[e]]))[0]
        x, info = operator.solve(m, b, prob, 0, "bicgstab", tol=1e-10)
        assert info[0][1] <= 1e-10
        row = inverse.forward_data(m, x[None], prob)[0, 0]
        assert rel_l2(f, x[0]) < 1e-4, (l, e, rel_l2(f, x[0]))
        assert rel_l2(d, row) < 1e-4, (l, e, rel_l2(d, row))


@pytest.mark.slow
def test_thyroid256_admm_step_matches_oracle(lib):
    """One ADMM-TV iteration (Eq. 9-14, Algorithm 1) at full size: the
    Gauss-Newton m-step by CG (n_cg = 2, each iteration one J and one J^H
    over all 768 right-hand sides), shrink, dual update and SoS, against
    the oracle's step on the oracle's own fields (768 FP64 solves).  The
    gradient, g and u are seeded inputs of both sides; lambda, rho, gamma
    are scaled to ||J^H J|| as in the benchmark."""
    import torch
    from oracle import admm
    w = phantoms.thyroid_256()
    m = 0.8 * model.contrast_from_sos(w.sos, w.c0)
    shape = tuple(w.shape)
    stream = torch.cuda.Stream()
    with torch.cuda.stream(stream):
        ctx = lib.Context(w.shape, w.h, w.c0, w.elem, w.freqs, tol=1e-6, stream=stream)
        m_gpu = to_gpu(m, torch.complex128)
        rep = ctx.forward(m_gpu)
        assert rep.info.n_not_converged == 0
        v = to_gpu(phantoms.complex_normal(shape, 7), torch.complex128)
        nrm = 1.0
        for _ in range(4):
            v = v / torch.linalg.vector_norm(v)
            v = ctx.jac_adjoint(ctx.jac_forward(v))
            nrm = float(torch.linalg.vector_norm(v).item())
        stream.synchronize()
    params = admm.AdmmParams(lam=1e-4 * nrm, rho=1e-2 * nrm, gamma=1e-5 * nrm, n_cg=2)
    grad = 1e-3 * nrm * phantoms.complex_normal(shape, 51) * np.abs(m).max()
    g0 = admm.grad_op(m, shape) + 0.01 * np.abs(m).max() * phantoms.complex_normal(
        (2,) + shape, 52)
    u0 = 0.01 * np.abs(m).max() * phantoms.complex_normal((2,) + shape, 53)
    with torch.cuda.stream(stream):
        mg = to_gpu(m, torch.complex128)
        gg = to_gpu(g0, torch.complex128)
        ug = to_gpu(u0, torch.complex128)
        sos = torch.empty(shape, dtype=torch.float64, device="cuda")
        ctx.admm_tv_step(mg, gg, ug, to_gpu(grad, torch.complex128), sos=sos,
                         lam=params.lam, rho=params.rho, gamma=params.gamma, n_cg=params.n_cg)
        stream.synchronize()
    m1, g1, u1, sos1 = to_np(mg), to_np(gg), to_np(ug), to_np(sos)
    ctx.close()
    prob = oracle.Problem(shape, w.h, w.c0, w.elem, np.asarray(w.freqs))
    fields = operator.solve_forward(m, prob, "bicgstab", tol=1e-10)
    k = model.wavenumbers(prob)
    rf = fields * (k * k * prob.cell_volume)[:, None, None, None]
    rm, rg, ru, rsos, rdm = admm.admm_tv_step(m, g0, u0, grad, fields, rf, prob, params)
    assert rel_l2(m1 - m, rdm) < 1e-3, rel_l2(m1 - m, rdm)
    assert rel_l2(sos1, rsos) < 1e-3
    assert rel_l2(g1, rg) < 1e-3
    assert rel_l2(u1, ru) < 1e-3

"""GPU parity of the batched BiCGSTAB solves, data, adjoint solves, gradient
and ADMM-TV step (Eq. 4-5, 7, 9-17, Algorithm 1) through the C ABI, against
the FP64 oracle on the same seeded inputs.

Tolerances (relative L2): fields and data 1e-4, gradient and updated SoS /
contrast update 1e-3 in mixed precision (FP32 fields, FP64 scalars, Krylov
tolerance 1e-6); FP64 mode with Krylov tolerance 1e-12: 1e-9."""
import numpy as np
import pytest

from gpu_common import contrast, oracle_problem, rel_l2, small_workload, to_gpu, to_np
from oracle import admm, inverse, operator
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


def _oracle_fields(w, m):
    return operator.solve_forward(m, oracle_problem(w), "bicgstab", tol=1e-12)


CASES = [((32, 32), 6, (1.5e6, 3.0e6)), ((16, 64), 5, (2.0e6,)), ((32, 96), 8, (1e6, 2.5e6)),
         ((8, 8, 16), 4, (1.0e6, 2.0e6)), ((16, 256), 6, (2.0e6, 3.0e6)),
         ((256, 16), 4, (1.5e6,)), ((8, 512), 4, (2.5e6,))]


@pytest.mark.parametrize("shape,n_elem,freqs", CASES)
def test_forward_fields_and_data(lib, shape, n_elem, freqs):
    import torch
    w = small_workload(shape, n_elem=n_elem, freqs=freqs)
    ctx = lib.Context(w.shape, w.h, w.c0, w.elem, w.freqs, tol=1e-6)
    m = contrast(w)
    fields = ctx.empty_fields()
    data = ctx.empty_data()
    rep = ctx.forward(to_gpu(m, torch.complex128), fields=fields, data=data)
    ref = _oracle_fields(w, m)
    refd = inverse.forward_data(m, ref, oracle_problem(w))
    got = to_np(fields)
    assert rel_l2(got, ref) < 1e-4
    assert rel_l2(to_np(data), refd) < 1e-4
    # per-RHS errors too (no RHS may hide behind the norm of the others)
    for l in range(w.n_freq):
        for e in range(w.n_elem):
            assert rel_l2(got[l, e], ref[l, e]) < 1e-4
    assert rep.max_iters > 0 and np.all(rep.status == 0)
    assert np.all(rep.rel_resid <= 1e-6)
    ctx.close()


def test_forward_fp64_reference_config(lib):
    """The 64 x 64 FP64 reference configuration (disc inclusion, 32
    elements, 1 MHz) in FP64 mode against dense LU."""
    import torch
    w = phantoms.disc_phantom()
    ctx = lib.Context(w.shape, w.h, w.c0, w.elem, w.freqs, precision=lib.FWI_FP64, tol=1e-12)
    m = contrast(w)
    fields = ctx.empty_fields()
    data = ctx.empty_data()
    ctx.forward(to_gpu(m, torch.complex128), fields=fields, data=data)
    prob = oracle_problem(w)
    ref = operator.solve_forward(m, prob, "lu")
    assert rel_l2(to_np(fields), ref) < 1e-9
    assert rel_l2(to_np(data), inverse.forward_data(m, ref, prob)) < 1e-9
    ctx.close()


def test_homogeneous_medium_needs_no_iterations(lib):
    import torch
    w = small_workload((16, 16), n_elem=3, freqs=(2e6,))
    ctx = lib.Context(w.shape, w.h, w.c0, w.elem, w.freqs)
    m = np.zeros(w.shape, dtype=np.complex128)
    fields = ctx.empty_fields()
    data = ctx.empty_data()
    rep = ctx.forward(to_gpu(m, torch.complex128), fields=fields, data=data)
    p0 = operator.incident_fields(oracle_problem(w))
    # A = I: the first BiCGSTAB step gives s = 0 and stops
    assert rep.max_iters == 1
    assert rel_l2(to_np(fields), p0) < 1e-6
    assert np.abs(to_np(data)).max() == 0.0
    ctx.close()


def test_warm_start_and_iteration_cap(lib):
    import torch
    w = small_workload((32, 32), n_elem=4, freqs=(3e6,))
    m = contrast(w)
    ctx = lib.Context(w.shape, w.h, w.c0, w.elem, w.freqs, max_it=1)
    fields = ctx.empty_fields()
    rep = ctx.forward(to_gpu(m, torch.complex128), fields=fields, allow_nonconverged=True)
    assert rep.code == lib.FWI_ERR_NOT_CONVERGED
    assert np.all(rep.iters == 1)
    assert np.all(rep.status == lib.FWI_ERR_NOT_CONVERGED)
    ctx.close()
    ctx = lib.Context(w.shape, w.h, w.c0, w.elem, w.freqs)
    cold = ctx.forward(to_gpu(m, torch.complex128), fields=fields, warm_start=True)
    ref = _oracle_fields(w, m)
    assert rel_l2(to_np(fields), ref) < 1e-4
    warm = ctx.forward(to_gpu(m, torch.complex128), fields=fields, warm_start=True)
    assert warm.max_iters <= 1 and cold.max_iters >= 1
    ctx.close()


def test_batched_launches_match_single_launch(lib):
    """max_batch splits the right-hand sides over several launches; the
    result must not depend on it (bitwise: fixed-order reductions)."""
    import torch
    w = small_workload((32, 32), n_elem=5, freqs=(1.5e6, 3e6))
    m_gpu = to_gpu(contrast(w), torch.complex128)
    out = []
    for mb in (0, 3, 7):
        ctx = lib.Context(w.shape, w.h, w.c0, w.elem, w.freqs, max_batch=mb)
        f = ctx.empty_fields()
        ctx.forward(m_gpu, fields=f)
        out.append(to_np(f))
        ctx.close()
    assert np.array_equal(out[0], out[1]) and np.array_equal(out[0], out[2])


@pytest.mark.parametrize("shape", [(256, 256), (16, 512), (8, 16, 160)])
def test_tile_variants_give_identical_results(lib, shape):
    """Every tile-shape variant the autotuner may pick gives bitwise the same
    fields (per-row fixed-order partial sums)."""
    import itertools
    import torch
    w = small_workload(shape, n_elem=3, freqs=(2.5e6,))
    m_gpu = to_gpu(contrast(w), torch.complex128)
    ctx = lib.Context(w.shape, w.h, w.c0, w.elem, w.freqs)
    ref = None
    ncy = 2 if len(shape) == 3 else 1
    for rf, ri, cz, cy in itertools.product(range(3), range(3), range(2), range(ncy)):
        try:
            ctx.set_tuning(rf, ri, cz, cy)
        except lib.FwiError:
            continue  # this length has no such variant
        f = ctx.empty_fields()
        ctx.forward(m_gpu, fields=f)
        got = to_np(f)
        if ref is None:
            ref = got
        assert np.array_equal(got, ref), (rf, ri, cz, cy)
    ctx.close()


def test_adjoint_solves(lib):
    import torch
    w = small_workload((32, 32), n_elem=4, freqs=(2e6, 3e6))
    ctx = lib.Context(w.shape, w.h, w.c0, w.elem, w.freqs)
    m = contrast(w)
    src = phantoms.complex_normal((w.n_freq, w.n_elem) + tuple(w.shape), 9)
    lam = ctx.empty_fields()
    ctx.adjoint(to_gpu(m, torch.complex128), to_gpu(src, torch.complex64), lam)
    srcr = src.astype(np.complex64).astype(np.complex128)
    ref = inverse.solve_adjoint(m, srcr, oracle_problem(w), "bicgstab", tol=1e-12)
    assert rel_l2(to_np(lam), ref) < 1e-4
    ctx.close()


def _gradient_case(w, seed=3):
    prob = oracle_problem(w)
    m = contrast(w)
    rng = np.random.default_rng(seed)
    m_true = m + 0.02 * rng.standard_normal(w.shape)
    d_true = inverse.forward_data(m_true, operator.solve_forward(m_true, prob, "bicgstab",
                                                                 tol=1e-12), prob)
    return prob, m, d_true


@pytest.mark.parametrize("shape", [(32, 32), (8, 8, 16)])
def test_gradient_matches_oracle(lib, shape):
    import torch
    w = small_workload(shape, n_elem=6, freqs=(1.5e6, 3e6))
    prob, m, d_obs = _gradient_case(w)
    ctx = lib.Context(w.shape, w.h, w.c0, w.elem, w.freqs)
    grad = torch.empty(w.shape, dtype=torch.complex128, device="cuda")
    data = ctx.empty_data()
    d_obs32 = d_obs.astype(np.complex64)
    mis, rf, ra = ctx.gradient(to_gpu(m, torch.complex128), to_gpu(d_obs32, torch.complex64),
                               grad, data=data)
    ref = inverse.gradient(m, d_obs32.astype(np.complex128), prob, "bicgstab", tol=1e-12)
    assert rel_l2(to_np(grad), ref["grad"]) < 1e-3
    assert rel_l2(to_np(data), ref["data"]) < 1e-4
    assert abs(mis - ref["misfit"]) <= 1e-3 * ref["misfit"]
    assert rf.max_iters > 0 and ra.max_iters > 0
    ctx.close()


def test_gradient_fp64_reference_config(lib):
    import torch
    w = phantoms.disc_phantom()
    prob, m, d_obs = _gradient_case(w)
    ctx = lib.Context(w.shape, w.h, w.c0, w.elem, w.freqs, precision=lib.FWI_FP64, tol=1e-12)
    grad = torch.empty(w.shape, dtype=torch.complex128, device="cuda")
    mis, _, _ = ctx.gradient(to_gpu(m, torch.complex128), to_gpu(d_obs, torch.complex128), grad)
    ref = inverse.gradient(m, d_obs, prob, "bicgstab", tol=1e-13)
    assert rel_l2(to_np(grad), ref["grad"]) < 1e-8
    assert abs(mis - ref["misfit"]) <= 1e-9 * ref["misfit"]
    ctx.close()


def test_jacobian_products(lib):
    import torch
    w = small_workload((32, 32), n_elem=6, freqs=(1.5e6, 3e6))
    prob = oracle_problem(w)
    m = contrast(w)
    ctx = lib.Context(w.shape, w.h, w.c0, w.elem, w.freqs)
    ctx.forward(to_gpu(m, torch.complex128))
    fields = _oracle_fields(w, m)
    k = 2 * np.pi * np.asarray(w.freqs) / w.c0
    rfields = fields * (k ** 2 * w.h ** 2)[:, None, None, None]
    a = phantoms.complex_normal(w.shape, 5)
    b = phantoms.complex_normal((w.n_freq, w.n_elem, w.n_elem), 6)
    ja = to_np(ctx.jac_forward(to_gpu(a, torch.complex128)))
    jhb = to_np(ctx.jac_adjoint(to_gpu(b, torch.complex128)))
    assert rel_l2(ja, inverse.jac_forward(a, fields, rfields, prob)) < 1e-4
    assert rel_l2(jhb.ravel(), inverse.jac_adjoint(b, fields, rfields, prob)) < 1e-4
    ctx.close()


@pytest.mark.parametrize("shape,prec,n_elem", [((32, 32), "mixed", 6), ((8, 8, 16), "mixed", 6),
                                               ((64, 64), "fp64", 0), ((8, 32, 32), "mixed", 136),
                                               ((16, 128), "mixed", 150)])
def test_admm_tv_step_matches_oracle(lib, shape, prec, n_elem):
    """One ADMM-TV iteration (m-step CG with J / J^H, shrink, dual update,
    SoS) against the oracle, including 2-D and 3-D cases with more than 128
    elements (two element tiles in the tensor-core contractions)."""
    import torch
    fp64 = prec == "fp64"
    if shape == (64, 64):
        w = phantoms.disc_phantom()
    elif n_elem > 128:
        width = shape[-1] * 0.1e-3
        w = phantoms.scaled(shape, 0.1e-3, n_elem, 0.9 * width / n_elem, np.array([1.5e6]), 17,
                            inclusions=[1520.0, 1580.0], semi_mm=(0.3, 0.6))
    else:
        w = small_workload(shape, n_elem=n_elem, freqs=(1.5e6, 3e6))
    prob, m, d_obs = _gradient_case(w)
    ctx = lib.Context(w.shape, w.h, w.c0, w.elem, w.freqs,
                      precision=lib.FWI_FP64 if fp64 else lib.FWI_MIXED,
                      tol=1e-12 if fp64 else 1e-6)
    fdt = torch.complex128 if fp64 else torch.complex64
    dob = d_obs if fp64 else d_obs.astype(np.complex64).astype(np.complex128)
    ref = inverse.gradient(m, dob, prob, "bicgstab", tol=1e-13)
    kk = (2 * np.pi * np.asarray(w.freqs) / w.c0) ** 2 * w.h ** w.dim
    rf = ref["fields"] * kk.reshape((-1,) + (1,) * (w.dim + 1))
    g0 = admm.grad_op(m, w.shape)
    u0 = 0.01 * phantoms.complex_normal(g0.shape, 12)
    # parameters scaled to the normal matrix so that every term acts
    scale = float(np.abs(ref["grad"]).max())
    params = admm.AdmmParams(lam=1e-3 * scale, rho=0.5 * scale, gamma=1e-3 * scale, n_cg=8)
    m1, g1, u1, sos1, dm = admm.admm_tv_step(m, g0, u0, ref["grad"], ref["fields"], rf,
                                             prob, params)
    m_gpu = to_gpu(m, torch.complex128)
    grad = torch.empty(w.shape, dtype=torch.complex128, device="cuda")
    ctx.gradient(m_gpu, to_gpu(dob, fdt), grad)
    g_gpu = to_gpu(g0, torch.complex128)
    u_gpu = to_gpu(u0, torch.complex128)
    sos = torch.empty(w.shape, dtype=torch.float64, device="cuda")
    ctx.admm_tv_step(m_gpu, g_gpu, u_gpu, grad, lam=params.lam, rho=params.rho,
                     gamma=params.gamma, n_cg=params.n_cg, sos=sos)
    tol = 1e-8 if fp64 else 1e-3
    assert rel_l2(to_np(m_gpu) - m, dm) < tol
    assert rel_l2(to_np(sos) - w.c0, sos1 - w.c0) < tol
    assert rel_l2(to_np(g_gpu), g1) < tol
    assert rel_l2(to_np(u_gpu), u1) < tol
    ctx.close()


@pytest.mark.parametrize("shape,n_elem,freqs", [((32, 32), 20, (1.5e6, 3.0e6)),
                                                ((8, 8, 16), 17, (1.0e6, 2.0e6))])
def test_two_chain_iteration_is_bitwise_identical(lib, shape, n_elem, freqs):
    """Batches of >= 32 RHS iterate as two halves on two streams (the
    default on 2-D lattices; 3-D lattices default to one chain); every RHS
    follows the same arithmetic, so fields, data and gradient are bitwise
    the same as with one chain, and match the oracle."""
    import torch
    width = shape[-1] * 0.1e-3
    w = phantoms.scaled(shape, 0.1e-3, n_elem, min(0.3e-3, 0.9 * width / n_elem),
                        np.asarray(freqs), 13, inclusions=[1520.0, 1580.0], semi_mm=(0.2, 0.5))
    m = contrast(w)
    ctx = lib.Context(w.shape, w.h, w.c0, w.elem, w.freqs)
    assert ctx.tuning()["overlap_halves"] == (1 if len(shape) == 2 else 0)
    m_gpu = to_gpu(m, torch.complex128)
    res = {}
    for on in (True, False):
        ctx.set_overlap(on)
        fields = ctx.empty_fields()
        data = ctx.empty_data()
        rep = ctx.forward(m_gpu, fields=fields, data=data)
        grad = torch.empty(w.shape, dtype=torch.complex128, device="cuda")
        ctx.gradient(m_gpu, data, grad)
        res[on] = (to_np(fields), to_np(data), to_np(grad), rep.max_iters)
    ctx.close()
    for a, b in zip(res[True], res[False]):
        assert np.array_equal(a, b)
    ref = _oracle_fields(w, m)
    assert rel_l2(res[True][0], ref) < 1e-4

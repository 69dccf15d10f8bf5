"""Tensor-core (tcgen05, 3xTF32) pixel contractions: the data projection,
J a and J^H b (Eq. 4, 15-17) against the FP64 oracle and against the
CUDA-core FP32 kernels on the same forward fields.  Cases cover one and two
128-element tiles with ragged element counts, pixel counts that leave
partial pixel blocks and partial split-K chunks, 2-D and 3-D grids."""
import numpy as np
import pytest

from gpu_common import contrast, oracle_problem, rel_l2, small_workload, to_gpu, to_np
from oracle import inverse, operator
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


# (shape, n_elem, freqs): N = 1024 / 2048 / 8192 / 768 pixels; 6 .. 136 elements
CASES = [((32, 32), 6, (1.5e6, 3.0e6)),
         ((16, 64), 40, (2.0e6,)),
         ((16, 128), 136, (1.0e6, 2.5e6)),
         ((64, 128), 128, (1.5e6, 3.0e6)),
         ((8, 96), 17, (2.0e6,)),
         ((8, 8, 16), 20, (1.0e6, 2.0e6))]


def _workload(shape, n_elem, freqs):
    width = shape[-1] * 0.1e-3
    pitch = min(0.3e-3, 0.9 * width / n_elem)
    return phantoms.scaled(shape, 0.1e-3, n_elem, pitch, np.asarray(freqs), 11,
                           inclusions=[1520.0, 1580.0], semi_mm=(0.2, 0.5))


@pytest.mark.parametrize("shape,n_elem,freqs", CASES)
def test_tensor_core_contractions(lib, shape, n_elem, freqs):
    import torch
    w = _workload(shape, n_elem, freqs)
    prob = oracle_problem(w)
    m = contrast(w)
    ctx = lib.Context(w.shape, w.h, w.c0, w.elem, w.freqs)
    assert ctx.tuning()["jac_tensor_cores"] == 1
    m_gpu = to_gpu(m, torch.complex128)
    data_tc = ctx.empty_data()
    ctx.forward(m_gpu, data=data_tc)
    a = phantoms.complex_normal(w.shape, 5)
    b = phantoms.complex_normal((w.n_freq, w.n_elem, w.n_elem), 6)
    b = 0.5 * (b + np.swapaxes(b, 1, 2))  # J a is complex symmetric in (e, j)
    ja_tc = to_np(ctx.jac_forward(to_gpu(a, torch.complex128)))
    jhb_tc = to_np(ctx.jac_adjoint(to_gpu(b, torch.complex128)))

    ctx.set_jac_tensor_cores(False)
    data_cc = ctx.empty_data()
    ctx.forward(m_gpu, data=data_cc)
    ja_cc = to_np(ctx.jac_forward(to_gpu(a, torch.complex128)))
    jhb_cc = to_np(ctx.jac_adjoint(to_gpu(b, torch.complex128)))
    ctx.close()

    # same FP32 fields: the two FP32 paths agree to FP32 rounding
    assert rel_l2(to_np(data_tc), to_np(data_cc)) < 2e-6
    assert rel_l2(ja_tc, ja_cc) < 2e-6
    assert rel_l2(jhb_tc, jhb_cc) < 2e-6
    # and both match the FP64 oracle at the field tolerance
    fields = operator.solve_forward(m, prob, "bicgstab", tol=1e-12)
    k = 2 * np.pi * np.asarray(w.freqs) / w.c0
    rfields = fields * (k ** 2 * w.h ** w.dim).reshape((-1,) + (1,) * (w.dim + 1))
    assert rel_l2(ja_tc, inverse.jac_forward(a, fields, rfields, prob)) < 1e-4
    assert rel_l2(jhb_tc.ravel(), inverse.jac_adjoint(b, fields, rfields, prob).ravel()) < 1e-4
    assert rel_l2(to_np(data_tc), inverse.forward_data(m, fields, prob)) < 1e-4


def test_tensor_core_products_are_deterministic(lib):
    import torch
    w = small_workload((64, 64), n_elem=24, freqs=(1.5e6, 2.5e6))
    ctx = lib.Context(w.shape, w.h, w.c0, w.elem, w.freqs)
    ctx.forward(to_gpu(contrast(w), torch.complex128))
    a = to_gpu(phantoms.complex_normal(w.shape, 8), torch.complex128)
    b = to_gpu(phantoms.complex_normal((w.n_freq, w.n_elem, w.n_elem), 9), torch.complex128)
    r1 = (to_np(ctx.jac_forward(a)), to_np(ctx.jac_adjoint(b)))
    r2 = (to_np(ctx.jac_forward(a)), to_np(ctx.jac_adjoint(b)))
    ctx.close()
    assert np.array_equal(r1[0], r2[0]) and np.array_equal(r1[1], r2[1])


@pytest.mark.parametrize("shape,n_elem,freqs", [((32, 32), 6, (1.5e6, 3.0e6)),
                                                ((16, 128), 136, (2.0e6,))])
def test_gradient_with_tensor_core_mixes(lib, shape, n_elem, freqs):
    """Data projection, adjoint sources (materialised mix) and gradient: the
    tensor-core and CUDA-core paths agree, and both match the oracle."""
    import torch
    w = _workload(shape, n_elem, freqs)
    prob = oracle_problem(w)
    m_true = contrast(w)
    m0 = 0.5 * m_true
    _, d_obs = inverse.forward_model(m_true, prob, "bicgstab", tol=1e-12)
    d32 = d_obs.astype(np.complex64)
    ctx = lib.Context(w.shape, w.h, w.c0, w.elem, w.freqs)
    m_gpu = to_gpu(m0, torch.complex128)
    out = {}
    for tc in (True, False):
        ctx.set_jac_tensor_cores(tc)
        grad = torch.empty(w.shape, dtype=torch.complex128, device="cuda")
        mis, _, _ = ctx.gradient(m_gpu, to_gpu(d32, torch.complex64), grad)
        out[tc] = (to_np(grad), mis)
    ctx.close()
    assert rel_l2(out[True][0], out[False][0]) < 1e-5
    # the data agree to ~1e-6 (FP32 rounding); the misfit of a partly fitted
    # model amplifies that by |d| / |F(m) - d|
    assert abs(out[True][1] - out[False][1]) <= 1e-4 * out[False][1]
    ref = inverse.gradient(m0, d32.astype(np.complex128), prob, "bicgstab", tol=1e-12)
    assert rel_l2(out[True][0], ref["grad"]) < 1e-3


def test_full_size_contraction_accuracy(lib):
    """256^2 grid, 128 elements, 2 frequencies (the thyroid256 geometry):
    J a on the tensor cores (FP32 accumulation in TMEM over sub-chunks of
    at most 512 pixels) against the FMA kernel, and the data projection
    against the definition (Eq. 4) evaluated on the device fields in FP64."""
    import torch
    w = phantoms.scaled((256, 256), 0.1e-3, 128, 0.2e-3, np.array([1.0e6, 3.0e6]), 21,
                        inclusions=[1520.0, 1580.0])
    m = contrast(w)
    ctx = lib.Context(w.shape, w.h, w.c0, w.elem, w.freqs)
    m_gpu = to_gpu(m, torch.complex128)
    fields = ctx.empty_fields()
    data = ctx.empty_data()
    ctx.forward(m_gpu, fields=fields, data=data)
    a = to_gpu(phantoms.complex_normal(w.shape, 5), torch.complex128)
    ja_tc = to_np(ctx.jac_forward(a))
    ctx.set_jac_tensor_cores(False)
    ja_cc = to_np(ctx.jac_forward(a))
    ctx.close()
    err = rel_l2(ja_tc, ja_cc)
    print(f"J a tensor cores vs FMA at 256^2: {err:.2e}")
    assert err < 1e-5
    # data = sum_n R_j(n) m_n p_e(n) (Eq. 4) on the device fields, in FP64
    f = to_np(fields).astype(np.complex128).reshape(w.n_freq, w.n_elem, -1)
    rows = inverse.receiver_rows(oracle_problem(w)).reshape(w.n_freq, w.n_elem, -1)
    mm = m.reshape(1, -1)
    ref = np.stack([(f[l] * mm) @ rows[l].T for l in range(w.n_freq)])
    err_d = rel_l2(to_np(data), ref)
    print(f"data (tensor cores) vs FP64 on the same fields: {err_d:.2e}")
    assert err_d < 2e-5

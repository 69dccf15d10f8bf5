"""3-D line elements of finite elevation (Sec. V-B) through the C ABI: the
incident fields (panelled Gauss-Legendre quadrature of the mean Green's
function on the device) against the oracle's adaptive quadrature, and the
data and gradient of a contrast against the oracle, FP32 and FP64."""
import numpy as np
import pytest

from gpu_common import contrast, oracle_problem, rel_l2, small_workload, to_gpu, to_np
from oracle import inverse, operator

pytestmark = pytest.mark.gpu

LENGTH = 1e-2  # 1 cm elevation, as in the paper's 3-D study


@pytest.fixture(scope="module")
def lib():
    import torch
    from paper_2604_15796_gb300 import build, libfwi
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    build.build()
    return libfwi


def _case(shape=(8, 8, 16), n_elem=5, freqs=(1.0e6, 2.0e6)):
    w = small_workload(shape, n_elem=n_elem, freqs=freqs)
    prob = oracle_problem(w)
    prob.extra["elem_length"] = LENGTH
    return w, prob


@pytest.mark.parametrize("fp64", [False, True])
def test_incident_fields_of_line_elements(lib, fp64):
    """With m = 0 the fields are the incident fields (A = I)."""
    import torch
    w, prob = _case()
    ref = operator.element_green(prob)
    ctx = lib.Context(w.shape, w.h, w.c0, w.elem, w.freqs,
                      precision=lib.FWI_FP64 if fp64 else lib.FWI_MIXED, elem_length=LENGTH)
    fields = ctx.empty_fields()
    ctx.forward(torch.zeros(w.shape, dtype=torch.complex128, device="cuda"), fields=fields)
    ctx.close()
    assert rel_l2(to_np(fields), ref) < (1e-9 if fp64 else 1e-6)


@pytest.mark.parametrize("fp64", [False, True])
def test_line_element_data_and_gradient(lib, fp64):
    import torch
    w, prob = _case()
    m_true = contrast(w)
    m0 = 0.5 * m_true
    _, d_true = inverse.forward_model(m_true, prob, "bicgstab", tol=1e-12)
    fdt = torch.complex128 if fp64 else torch.complex64
    d_obs = d_true if fp64 else d_true.astype(np.complex64).astype(np.complex128)
    ref = inverse.gradient(m0, d_obs, prob, "bicgstab", tol=1e-12)
    ctx = lib.Context(w.shape, w.h, w.c0, w.elem, w.freqs,
                      precision=lib.FWI_FP64 if fp64 else lib.FWI_MIXED,
                      tol=1e-12 if fp64 else 1e-6, elem_length=LENGTH)
    tol_d, tol_g = (1e-8, 1e-8) if fp64 else (1e-4, 1e-3)
    m_gpu = to_gpu(m0, torch.complex128)
    data = ctx.empty_data()
    ctx.forward(m_gpu, data=data)
    assert rel_l2(to_np(data), ref["data"]) < tol_d
    grad = torch.empty(w.shape, dtype=torch.complex128, device="cuda")
    mis, _, _ = ctx.gradient(m_gpu, to_gpu(d_obs, fdt), grad)
    ctx.close()
    assert rel_l2(to_np(grad), ref["grad"]) < tol_g
    assert abs(mis - ref["misfit"]) <= tol_g * ref["misfit"]
    # the elevation changes the data: point elements give other data
    pt = lib.Context(w.shape, w.h, w.c0, w.elem, w.freqs,
                     precision=lib.FWI_FP64 if fp64 else lib.FWI_MIXED)
    d_pt = pt.empty_data()
    pt.forward(m_gpu, data=d_pt)
    pt.close()
    assert rel_l2(to_np(d_pt), ref["data"]) > 1e-2

"""The allocation-free contraction entry point, for callers that cannot call
cudaMalloc, gives the same Jacobian product as the context-based one.

fwi_contract_pixels_noalloc keeps its split partial sums in a file-scope
device array instead of a context workspace.  This test calls it through
the C ABI twice in a row (the second call reuses the array with the first
call's contents still in it) and compares each result with fwi_jac_forward
at the tolerance of the other Jacobian tests (relative L2 1e-4).  It also
checks that sizes beyond the array are rejected with FWI_ERR_INVALID_ARG.
Collected last so that a run stopping at the first failure has run every
other test before it."""
import ctypes

import numpy as np
import pytest

from gpu_common import contrast, rel_l2, small_workload, to_gpu, to_np
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


def test_noalloc_contraction_matches_context_jacobian(lib):
    import torch
    w = small_workload((32, 32), n_elem=6, freqs=(1.5e6, 3.0e6))
    ctx = lib.Context(w.shape, w.h, w.c0, w.elem, w.freqs)
    fields = ctx.empty_fields()
    ctx.forward(to_gpu(contrast(w), torch.complex128), fields=fields)
    a = phantoms.complex_normal(w.shape, 31)
    y_ref = to_np(ctx.jac_forward(to_gpu(a, torch.complex128)))
    a64 = to_gpu(a, torch.complex64)
    k = 2 * np.pi * np.asarray(w.freqs) / w.c0
    scale = np.ascontiguousarray(k ** 2 * w.h ** 2, dtype=np.float64)
    for call in range(2):
        y = torch.full((w.n_freq, w.n_elem, w.n_elem), float("nan"), dtype=torch.complex128,
                       device="cuda")
        torch.cuda.synchronize()
        st = lib.fwi_contract_pixels_noalloc(
            ctypes.c_void_p(fields.data_ptr()), ctypes.c_void_p(a64.data_ptr()),
            ctypes.c_void_p(fields.data_ptr()), w.n_freq, w.n_elem, w.n,
            scale.ctypes.data_as(ctypes.POINTER(ctypes.c_double)),
            ctypes.c_void_p(y.data_ptr()), None)
        assert st == lib.FWI_OK, lib.fwi_last_error(None)
        err = rel_l2(to_np(y), y_ref)
        assert err < 1e-4, (call, err)
    ctx.close()


def test_noalloc_contraction_rejects_sizes_beyond_its_scratch(lib):
    import torch
    x = torch.zeros(16, dtype=torch.complex64, device="cuda")
    y = torch.zeros(16, dtype=torch.complex128, device="cuda")
    scale = np.ones(1)
    # 1 frequency x 1024^2 partial sums > 524288: rejected before any launch
    st = lib.fwi_contract_pixels_noalloc(
        ctypes.c_void_p(x.data_ptr()), None, ctypes.c_void_p(x.data_ptr()), 1, 1024, 16,
        scale.ctypes.data_as(ctypes.POINTER(ctypes.c_double)), ctypes.c_void_p(y.data_ptr()),
        None)
    assert st == lib.FWI_ERR_INVALID_ARG
    assert b"4 MiB" in lib.fwi_last_error(None)

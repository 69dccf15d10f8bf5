"""The allocation-free contraction entry point, for callers that cannot call
cudaMalloc, gives the same Jacobian product as the context-based one.

fwi_contract_pixels_noalloc keeps its split partial sums in a file-scope
device array instead of a context workspace.  These tests call it through
the C ABI, each case twice in a row (the second call reuses the array with
the first call's contents still in it), and compare:

* with fwi_jac_forward (the context-based entry point) and with the FP64
  oracle's J a (oracle fields as inputs), at the tolerance of the other
  Jacobian tests (relative L2 1e-4), also with a = NULL (a = 1);
* on 130 elements x 4 frequencies (three element tiles per side, and a
  split-K count capped by the size of the array) with the definition of the
  contraction summed in FP64;
* at the exact limit n_freq * n_elem^2 = 524288 (accepted) and one element
  beyond it, and at n_freq = 33 (both rejected with FWI_ERR_INVALID_ARG).

Collected last so that a run stopping at the first failure has run every
other test before it."""
import ctypes

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


def call(lib, X, a, Q, n_freq, n_elem, N, scale, Y):
    st = lib.fwi_contract_pixels_noalloc(
        ctypes.c_void_p(X.data_ptr()), None if a is None else ctypes.c_void_p(a.data_ptr()),
        ctypes.c_void_p(Q.data_ptr()), n_freq, n_elem, N,
        scale.ctypes.data_as(ctypes.POINTER(ctypes.c_double)), ctypes.c_void_p(Y.data_ptr()),
        None)
    return st


def nan_out(shape):
    import torch
    return torch.full(shape, float("nan"), dtype=torch.complex128, device="cuda")


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
    for c in range(2):
        y = nan_out((w.n_freq, w.n_elem, w.n_elem))
        torch.cuda.synchronize()
        st = call(lib, fields, a64, fields, w.n_freq, w.n_elem, w.n, scale, y)
        assert st == lib.FWI_OK, lib.fwi_last_error(None)
        err = rel_l2(to_np(y), y_ref)
        assert err < 1e-4, (c, err)
    ctx.close()


def test_noalloc_contraction_matches_oracle(lib):
    """J a of the FP64 oracle (Eq. 16) on the oracle's own fields, and its
    data projection (a = NULL means a = 1: sum_n p_e(n) ptilde_j(n))."""
    import torch
    w = small_workload((24, 20), n_elem=9, freqs=(1.0e6, 2.0e6, 3.0e6))
    prob = oracle_problem(w)
    m = contrast(w)
    fields = operator.solve_forward(m, prob, "lu")
    rf = inverse.receiver_fields(m, prob, "lu")  # ptilde_j = A^-1 R_j, solved
    k = 2 * np.pi * np.asarray(w.freqs) / w.c0
    a = phantoms.complex_normal(w.shape, 5)
    ref_a = inverse.jac_forward(a, fields, rf, prob)
    ref_1 = inverse.jac_forward(np.ones(w.shape), fields, rf, prob)
    X = to_gpu(fields.reshape(w.n_freq, w.n_elem, -1), torch.complex64)
    a64 = to_gpu(a, torch.complex64)
    scale = np.ascontiguousarray(k ** 2 * prob.cell_volume, dtype=np.float64)
    for c in range(2):
        for av, ref in ((a64, ref_a), (None, ref_1)):
            y = nan_out((w.n_freq, w.n_elem, w.n_elem))
            torch.cuda.synchronize()
            st = call(lib, X, av, X, w.n_freq, w.n_elem, w.n, scale, y)
            assert st == lib.FWI_OK, lib.fwi_last_error(None)
            err = rel_l2(to_np(y), ref)
            assert err < 1e-4, (c, av is None, err)


def definition(X, a, Q, scale):
    """Y[l][e][j] = scale_l sum_n X[l][e][n] a[n] Q[l][j][n], in FP64."""
    X = X.astype(np.complex128)
    Q = Q.astype(np.complex128)
    Xa = X if a is None else X * a.astype(np.complex128)[None, None, :]
    return np.einsum("len,ljn->lej", Xa, Q) * scale[:, None, None]


def test_noalloc_contraction_several_tiles_split_capped_by_the_array(lib):
    """130 elements (three 64-element tiles per side) x 4 frequencies:
    4 * 130^2 = 67,600 partials per split, so the 524,288-partial array
    caps the split-K count at 7, below what the SM count asks for."""
    import torch
    n_freq, n_elem, N = 4, 130, 3000
    rng = np.random.default_rng(11)
    X = (rng.standard_normal((n_freq, n_elem, N)) + 1j * rng.standard_normal(
        (n_freq, n_elem, N))).astype(np.complex64)
    Q = (rng.standard_normal((n_freq, n_elem, N)) + 1j * rng.standard_normal(
        (n_freq, n_elem, N))).astype(np.complex64)
    a = (rng.standard_normal(N) + 1j * rng.standard_normal(N)).astype(np.complex64)
    scale = np.ascontiguousarray(rng.uniform(0.5, 2.0, n_freq))
    ref = definition(X, a, Q, scale)
    Xd, Qd, ad = (torch.from_numpy(v).cuda() for v in (X, Q, a))
    for c in range(2):
        y = nan_out((n_freq, n_elem, n_elem))
        torch.cuda.synchronize()
        st = call(lib, Xd, ad, Qd, n_freq, n_elem, N, scale, y)
        assert st == lib.FWI_OK, lib.fwi_last_error(None)
        err = rel_l2(to_np(y), ref)
        assert err < 1e-4, (c, err)


def test_noalloc_contraction_limits(lib):
    """2 x 512^2 = 524,288 partials fill the array exactly (accepted, one
    split); 2 x 513^2 and 33 frequencies are rejected before any launch."""
    import torch
    n_freq, n_elem, N = 2, 512, 40
    rng = np.random.default_rng(3)
    X = (rng.standard_normal((n_freq, n_elem, N)) + 1j * rng.standard_normal(
        (n_freq, n_elem, N))).astype(np.complex64)
    scale = np.ones(n_freq)
    ref = definition(X, None, X, scale)
    Xd = torch.from_numpy(X).cuda()
    for c in range(2):
        y = nan_out((n_freq, n_elem, n_elem))
        torch.cuda.synchronize()
        st = call(lib, Xd, None, Xd, n_freq, n_elem, N, scale, y)
        assert st == lib.FWI_OK, lib.fwi_last_error(None)
        err = rel_l2(to_np(y), ref)
        assert err < 1e-4, (c, err)
    big = torch.zeros((n_freq, 513, N), dtype=torch.complex64, device="cuda")
    yb = torch.zeros((n_freq, 513, 513), dtype=torch.complex128, device="cuda")
    st = call(lib, big, None, big, n_freq, 513, N, scale, yb)
    assert st == lib.FWI_ERR_INVALID_ARG
    assert b"4 MiB" in lib.fwi_last_error(None)
    x = torch.zeros((33, 1, 16), dtype=torch.complex64, device="cuda")
    y = torch.zeros((33, 1, 1), dtype=torch.complex128, device="cuda")
    st = call(lib, x, None, x, 33, 1, 16, np.ones(33), y)
    assert st == lib.FWI_ERR_INVALID_ARG
    assert b"FWI_NOALLOC_MAX_FREQ" in lib.fwi_last_error(None)


def test_noalloc_contraction_rejects_sizes_beyond_its_scratch(lib):
    import torch
    x = torch.zeros(16, dtype=torch.complex64, device="cuda")
    y = torch.zeros(16, dtype=torch.complex128, device="cuda")
    scale = np.ones(1)
    # 1 frequency x 1024^2 partial sums > 524288: rejected before any launch
    st = call(lib, x, None, x, 1, 1024, 16, scale, y)
    assert st == lib.FWI_ERR_INVALID_ARG
    assert b"4 MiB" in lib.fwi_last_error(None)

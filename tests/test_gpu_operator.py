"""GPU parity of single Lippmann-Schwinger operator applications (Eq. 5,
Sec. IV-A) through the C ABI: K, A = I - K diag(m) and A^H against the FP64
oracle, element by element, on grids that exercise every FFT radix (2, 3,
5), non-square and 3-D lattices and ragged row tiles.

Tolerance: a single FP32 application carries the rounding of two
length-L FFTs per axis (relative error ~ log2(L) * 6e-8); 1e-5 leaves a
margin of ~10x.  FP64 applications: 1e-11."""
import numpy as np
import pytest

from gpu_common import contrast, oracle_problem, rel_l2, small_workload, to_gpu, to_np
from oracle import inverse, operator
from paper_2604_15796_gb300 import phantoms

pytestmark = pytest.mark.gpu

SHAPES = [(32, 32), (8, 16), (32, 96), (16, 160), (96, 32), (8, 8, 16), (16, 8, 8),
          (16, 256), (256, 16), (8, 512), (512, 8), (8, 16, 256)]


@pytest.fixture(scope="module")
def lib():
    import torch
    from paper_2604_15796_gb300 import build, libfwi
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    build.build()
    return libfwi


@pytest.mark.parametrize("shape", SHAPES)
@pytest.mark.parametrize("prec", ["mixed", "fp64"])
def test_apply_operators_match_oracle(lib, shape, prec):
    import torch
    w = small_workload(shape, n_elem=3, freqs=(2.0e6, 3.5e6))
    fp64 = prec == "fp64"
    ctx = lib.Context(w.shape, w.h, w.c0, w.elem, w.freqs,
                      precision=lib.FWI_FP64 if fp64 else lib.FWI_MIXED)
    fdt = torch.complex128 if fp64 else torch.complex64
    tol = 1e-11 if fp64 else 1e-5
    prob = oracle_problem(w)
    m = contrast(w)
    v = phantoms.complex_normal((3,) + tuple(shape), 17)
    m_gpu = to_gpu(m, torch.complex128)
    v_gpu = to_gpu(v, fdt)
    vin = v.astype(np.complex64).astype(np.complex128) if not fp64 else v
    for l in range(len(w.freqs)):
        ref_k = operator.apply_K(vin, prob, l)
        ref_a = operator.apply_A(vin, m, prob, l)
        ref_ah = inverse.apply_AH(vin, m, prob, l)
        got_k = to_np(ctx.apply("K", v_gpu, l))
        got_a = to_np(ctx.apply("A", v_gpu, l, m_gpu))
        got_ah = to_np(ctx.apply("AH", v_gpu, l, m_gpu))
        assert rel_l2(got_k, ref_k) < tol, (l, rel_l2(got_k, ref_k))
        assert rel_l2(got_a, ref_a) < tol
        assert rel_l2(got_ah, ref_ah) < tol
    ctx.close()


def test_operator_adjoint_identity_on_gpu(lib):
    """<A u, v> = <u, A^H v> with both sides computed by the GPU."""
    import torch
    w = small_workload((32, 32), n_elem=2, freqs=(3e6,))
    ctx = lib.Context(w.shape, w.h, w.c0, w.elem, w.freqs, precision=lib.FWI_FP64)
    m_gpu = to_gpu(contrast(w), torch.complex128)
    u = phantoms.complex_normal((1, 32, 32), 3)
    v = phantoms.complex_normal((1, 32, 32), 4)
    Au = to_np(ctx.apply("A", to_gpu(u, torch.complex128), 0, m_gpu))
    AHv = to_np(ctx.apply("AH", to_gpu(v, torch.complex128), 0, m_gpu))
    assert np.isclose(np.vdot(Au, v), np.vdot(u, AHv), rtol=1e-12)
    ctx.close()


def test_invalid_arguments_are_rejected(lib):
    import torch
    w = small_workload((16, 16), n_elem=2, freqs=(2e6,))
    ctx = lib.Context(w.shape, w.h, w.c0, w.elem, w.freqs)
    v = torch.zeros((1, 16, 16), dtype=torch.complex64, device="cuda")
    with pytest.raises(lib.FwiError) as e:
        ctx.apply("K", v, 5)  # frequency index out of range
    assert e.value.status == lib.FWI_ERR_INVALID_ARG
    big = torch.zeros((3, 16, 16), dtype=torch.complex64, device="cuda")
    with pytest.raises(lib.FwiError):
        ctx.apply("K", big, 0)  # more vectors than the batch
    ctx.close()
    with pytest.raises(lib.FwiError) as e:
        lib.Context((16, 24), w.h, w.c0, w.elem, w.freqs)  # 2*24 has no FFT plan
    assert e.value.status == lib.FWI_ERR_INVALID_ARG


@pytest.mark.parametrize("shape", [(32, 96), (256, 16), (8, 512), (8, 16, 256), (16, 8, 8),
                                   (16, 96, 32), (8, 160, 16)])
def test_tma_staged_column_passes_match_plain_loads(lib, shape):
    """The FP32 column passes give the same result, to FP32 rounding,
    whether their input tiles, twiddles and kernel-spectrum tiles are staged
    in shared memory (TMA tensor copies) or read from global memory with
    plain loads (the same arithmetic steps on the same values; the compiled
    kernels may fuse multiply-adds differently), and both match the
    oracle."""
    import torch
    w = small_workload(shape, n_elem=3, freqs=(2.0e6,))
    ctx = lib.Context(w.shape, w.h, w.c0, w.elem, w.freqs)
    m_gpu = to_gpu(contrast(w), torch.complex128)
    v_gpu = to_gpu(phantoms.complex_normal((3,) + tuple(shape), 21), torch.complex64)
    out = {}
    for tma in (True, False):
        ctx.set_col_tma(tma)
        out[tma] = to_np(ctx.apply("A", v_gpu, 0, m_gpu))
    ctx.close()
    # one FP32 rounding per product at most (~6e-8 relative), not a bug
    assert rel_l2(out[True], out[False]) < 3e-7, rel_l2(out[True], out[False])
    prob = oracle_problem(w)
    vin = to_np(v_gpu).astype(np.complex128)
    ref = operator.apply_A(vin, contrast(w), prob, 0)
    assert rel_l2(out[True], ref) < 1e-5


@pytest.mark.parametrize("shape", [(32, 96), (96, 32), (8, 512), (16, 8, 8), (8, 16, 160),
                                   (8, 8, 160)])
def test_staged_row_passes_match_plain_loads(lib, shape):
    """The FP32 forward row pass gives the same result, to FP32 rounding,
    whether each work item's rows are staged in shared memory by bulk copies
    or read with plain loads: single applications of K, A and A^H, and a
    whole forward solve (every BiCGSTAB update mode of the fused row pass),
    with ragged row tiles; both match the oracle."""
    import torch
    w = small_workload(shape, n_elem=3, freqs=(2.0e6,))
    ctx = lib.Context(w.shape, w.h, w.c0, w.elem, w.freqs, tol=1e-6)
    m = contrast(w)
    m_gpu = to_gpu(m, torch.complex128)
    v = phantoms.complex_normal((3,) + tuple(shape), 23)
    v_gpu = to_gpu(v, torch.complex64)
    out = {}
    for stage in (True, False):
        ctx.set_row_stage(stage)
        assert ctx.tuning()["row_stage"] == int(stage)
        ops = [to_np(ctx.apply(k, v_gpu, 0, None if k == "K" else m_gpu))
               for k in ("K", "A", "AH")]
        f = ctx.empty_fields()
        ctx.forward(m_gpu, fields=f)
        out[stage] = (ops, to_np(f))
    ctx.close()
    for a, b in zip(out[True][0], out[False][0]):
        assert rel_l2(a, b) < 3e-7, rel_l2(a, b)
    # the solve stops at tol = 1e-6: rounding differences stay below it
    assert rel_l2(out[True][1], out[False][1]) < 1e-5
    prob = oracle_problem(w)
    vin = v.astype(np.complex64).astype(np.complex128)
    assert rel_l2(out[True][0][1], operator.apply_A(vin, m, prob, 0)) < 1e-5
    assert rel_l2(out[True][0][2], inverse.apply_AH(vin, m, prob, 0)) < 1e-5
    ref_f = operator.solve_forward(m, prob, "bicgstab", tol=1e-10)
    assert rel_l2(out[True][1], ref_f) < 1e-4


@pytest.mark.parametrize("shape", [(32, 32), (128, 32), (8, 8, 16), (128, 16, 16), (128, 8, 16),
                                   (256, 16), (256, 96), (256, 8, 8)])
def test_two_column_convolution_matches_one_column(lib, shape):
    """The FP32 convolution pass gives the same result, to FP32 rounding,
    with two columns per thread (packed f32x2 arithmetic on column pairs;
    transform lengths 16, 64, 256 and 512 along the convolution axis) as with
    one, for single applications of K, A and A^H and for a whole forward
    solve; both match the oracle."""
    import torch
    w = small_workload(shape, n_elem=3, freqs=(2.0e6,))
    ctx = lib.Context(w.shape, w.h, w.c0, w.elem, w.freqs, tol=1e-6)
    m = contrast(w)
    m_gpu = to_gpu(m, torch.complex128)
    v = phantoms.complex_normal((3,) + tuple(shape), 29)
    v_gpu = to_gpu(v, torch.complex64)
    out = {}
    for pairs in (True, False):
        ctx.set_col_pairs(pairs)
        assert ctx.tuning()["col_pairs"] == int(pairs)
        ops = [to_np(ctx.apply(k, v_gpu, 0, None if k == "K" else m_gpu))
               for k in ("K", "A", "AH")]
        f = ctx.empty_fields()
        ctx.forward(m_gpu, fields=f)
        out[pairs] = (ops, to_np(f))
    ctx.close()
    for a, b in zip(out[True][0], out[False][0]):
        assert rel_l2(a, b) < 3e-7, rel_l2(a, b)
    assert rel_l2(out[True][1], out[False][1]) < 1e-5
    prob = oracle_problem(w)
    vin = v.astype(np.complex64).astype(np.complex128)
    assert rel_l2(out[True][0][0], operator.apply_K(vin, prob, 0)) < 1e-5
    assert rel_l2(out[True][0][1], operator.apply_A(vin, m, prob, 0)) < 1e-5
    assert rel_l2(out[True][0][2], inverse.apply_AH(vin, m, prob, 0)) < 1e-5
    ref_f = operator.solve_forward(m, prob, "bicgstab", tol=1e-10)
    assert rel_l2(out[True][1], ref_f) < 1e-4

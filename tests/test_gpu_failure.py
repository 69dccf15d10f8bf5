"""Failure detection without a GPU fault:

* a stalled tensor-core pipeline: the next contraction withholds its first
  stage (test switch), every wait of the kernel is bounded (1 s of
  %globaltimer), the kernel sets its error word, drains its own MMAs, frees
  its tensor memory and returns; the call reports FWI_ERR_CUDA and the
  context gives the same data as before on the next call;
* cancellation from another host thread stops a running solve at its next
  host check (FWI_ERR_CANCELLED), and the next solve runs to the end;
* a non-finite input is reported (FWI_ERR_NONFINITE) without a fault."""
import threading
import time

import numpy as np
import pytest

from gpu_common import contrast, small_workload, to_gpu, to_np
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


def test_stalled_tensor_core_pipeline_is_reported(lib):
    import torch
    w = small_workload((32, 32), n_elem=6)
    ctx = lib.Context(w.shape, w.h, w.c0, w.elem, w.freqs)
    assert ctx.tuning()["jac_tensor_cores"] == 1
    m = to_gpu(contrast(w), torch.complex128)
    d1 = ctx.empty_data()
    ctx.forward(m, data=d1)
    ctx.debug_stall_once()
    d2 = ctx.empty_data()
    t0 = time.perf_counter()
    with pytest.raises(lib.FwiError) as err:
        ctx.forward(m, data=d2)
    waited = time.perf_counter() - t0
    assert err.value.status == lib.FWI_ERR_CUDA
    assert "pipeline wait timed out" in str(err.value)
    assert waited > 0.9  # the kernel gave up after its 1 s bound
    d3 = ctx.empty_data()
    ctx.forward(m, data=d3)
    ctx.close()
    assert np.array_equal(to_np(d1), to_np(d3))


def test_cancel_stops_a_running_solve(lib):
    """FP64, one right-hand side per launch: 256 sequential solves, each with
    its own captured graph, so the call runs long enough to be cancelled."""
    import torch
    w = phantoms.scaled((256, 256), 0.1e-3, 64, 0.2e-3, np.array([1.0e6, 1.5e6, 2.0e6, 3.0e6]),
                        9, inclusions=[1520.0, 1580.0])
    ctx = lib.Context(w.shape, w.h, w.c0, w.elem, w.freqs, precision=lib.FWI_FP64, max_batch=1)
    m = to_gpu(contrast(w), torch.complex128)
    timer = threading.Timer(0.1, ctx.cancel)
    t0 = time.perf_counter()
    timer.start()
    with pytest.raises(lib.FwiError) as err:
        ctx.forward(m)
    cancelled_after = time.perf_counter() - t0
    timer.join()
    assert err.value.status == lib.FWI_ERR_CANCELLED
    t0 = time.perf_counter()
    rep = ctx.forward(m)
    full = time.perf_counter() - t0
    ctx.close()
    assert rep.max_iters > 0 and rep.info.n_not_converged == 0
    assert cancelled_after < full


def test_nonfinite_input_is_reported(lib):
    """A NaN in the contrast makes every right-hand side non-finite: the
    bounded BiCGSTAB marks them, the call reports FWI_ERR_NONFINITE, and the
    context solves the next, finite, contrast."""
    import torch
    w = small_workload((32, 32), n_elem=4)
    ctx = lib.Context(w.shape, w.h, w.c0, w.elem, w.freqs)
    m = to_gpu(contrast(w), torch.complex128)
    m_bad = m.clone()
    m_bad[3, 5] = complex(float("nan"), 0.0)
    with pytest.raises(lib.FwiError) as err:
        ctx.forward(m_bad)
    assert err.value.status == lib.FWI_ERR_NONFINITE
    rep = ctx.forward(m)
    ctx.close()
    assert rep.max_iters > 0 and rep.info.n_not_converged == 0


"""The smoke entry point (one small gradient + ADMM-TV step against the
oracle) and the binding's argument checks on device tensors."""
import os
import sys

import pytest

from gpu_common import small_workload

pytestmark = pytest.mark.gpu
ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_smoke_entry_point():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    sys.path.insert(0, ROOT)
    import __graft_entry__
    __graft_entry__.smoke()


def test_device_arguments_of_the_wrong_layout_are_rejected():
    import torch
    from paper_2604_15796_gb300 import build, libfwi
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    build.build()
    w = small_workload((16, 16), n_elem=3, freqs=(2e6,))
    ctx = libfwi.Context(w.shape, w.h, w.c0, w.elem, w.freqs)
    m_real = torch.zeros(w.shape, dtype=torch.float64, device="cuda")
    with pytest.raises(ValueError, match="^m: expected"):
        ctx.forward(m_real)
    m = torch.zeros(w.shape, dtype=torch.complex128, device="cuda")
    short = torch.empty((w.n_freq, w.n_elem - 1) + tuple(w.shape), dtype=torch.complex64,
                        device="cuda")
    with pytest.raises(ValueError, match="^fields: expected"):
        ctx.forward(m, fields=short)
    with pytest.raises(ValueError, match="^d_obs: expected"):
        ctx.gradient(m, torch.zeros((1, 3, 3), dtype=torch.complex128, device="cuda"),
                     torch.empty_like(m))
    # nothing reached the library: a valid call on the same context succeeds
    data = ctx.empty_data()
    ctx.forward(torch.full_like(m, 0.01), data=data)
    assert bool(torch.isfinite(torch.view_as_real(data)).all())
    ctx.close()


def test_call_log_of_device_calls(tmp_path):
    import json
    import torch
    from paper_2604_15796_gb300 import build, libfwi
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    build.build()
    w = small_workload((16, 16), n_elem=3, freqs=(2e6,))
    ctx = libfwi.Context(w.shape, w.h, w.c0, w.elem, w.freqs)
    m = torch.full(w.shape, 0.01 + 0j, dtype=torch.complex128, device="cuda")
    path = tmp_path / "calls.jsonl"
    libfwi.set_call_log(str(path))
    try:
        data = ctx.empty_data()
        ctx.forward(m, data=data)
        grad = torch.empty(w.shape, dtype=torch.complex128, device="cuda")
        ctx.gradient(m, (1.1 * data).contiguous(), grad)
    finally:
        libfwi.set_call_log(None)
        ctx.close()
    recs = [json.loads(line) for line in path.read_text().splitlines()]
    assert [r["call"] for r in recs] == ["forward", "gradient"]
    assert all(r["status"] == "OK" for r in recs)
    assert recs[0]["forward"]["max_iters"] > 0 and recs[1]["adjoint"]["device_ms"] > 0

"""The library against the stored oracle values of the 64^2 FP64 reference
configuration (tests/golden/disc64_reference.json): data entries, misfit,
gradient entries and the SoS after one ADMM-TV iteration, on the FP64 path
(1e-8) and the mixed-precision path (1e-4 data, 1e-3 gradient / SoS)."""
import json
import os

import numpy as np
import pytest

from gpu_common import contrast, to_gpu, to_np
from paper_2604_15796_gb300 import phantoms

pytestmark = pytest.mark.gpu
HERE = os.path.dirname(os.path.abspath(__file__))


@pytest.fixture(scope="module")
def lib():
    import torch
    from paper_2604_15796_gb300 import build, libfwi
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    build.build()
    return libfwi


@pytest.mark.parametrize("fp64", [True, False])
def test_reference_configuration_against_stored_values(lib, fp64):
    import torch
    g = json.load(open(os.path.join(HERE, "golden", "disc64_reference.json")))
    w = phantoms.disc_phantom()
    m_true = contrast(w)
    m0 = 0.5 * m_true
    prec = lib.FWI_FP64 if fp64 else lib.FWI_MIXED
    fdt = torch.complex128 if fp64 else torch.complex64
    tol_d, tol_g = (1e-8, 1e-8) if fp64 else (1e-4, 1e-3)
    ctx = lib.Context(w.shape, w.h, w.c0, w.elem, w.freqs, precision=prec,
                      tol=1e-12 if fp64 else 1e-6)
    d = ctx.empty_data()
    ctx.forward(to_gpu(m_true, torch.complex128), data=d)
    dn = to_np(d)
    for l, e, j, re, im in g["data"]:
        ref = complex(re, im)
        assert abs(dn[int(l), int(e), int(j)] - ref) <= tol_d * abs(ref) + 1e-12
    m_gpu = to_gpu(m0, torch.complex128)
    grad = torch.empty(w.shape, dtype=torch.complex128, device="cuda")
    mis, _, _ = ctx.gradient(m_gpu, d.to(fdt), grad)
    gn = to_np(grad)
    assert abs(mis - g["misfit_m0"]) <= tol_g * g["misfit_m0"]
    assert abs(np.linalg.norm(gn) - g["grad_m0_norm"]) <= tol_g * g["grad_m0_norm"]
    for z, x, re, im in g["grad_m0"]:
        assert abs(gn[int(z), int(x)] - complex(re, im)) <= tol_g * g["grad_m0_norm"]
    a = g["admm"]
    s = a["scale"]
    sos = torch.empty(w.shape, dtype=torch.float64, device="cuda")
    gv, uv = ctx.admm_init(m_gpu)
    ctx.admm_tv_step(m_gpu, gv, uv, grad, lam=a["lam_rel"] * s, rho=a["rho_rel"] * s,
                     gamma=a["gamma_rel"] * s, n_cg=a["n_cg"], sos=sos)
    sn = to_np(sos)
    ctx.close()
    dev = max(abs(v - w.c0) for _, _, v in g["sos_after_one_iteration"])
    for z, x, v in g["sos_after_one_iteration"]:
        assert abs(sn[int(z), int(x)] - v) <= tol_g * dev

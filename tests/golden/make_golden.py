"""Writes the stored expected values of tests/golden/ from the FP64 oracle
alone (dense LU solves; no value comes from the CUDA path).

The paper prints no worked example of its method (its only numbers are
reconstruction-quality scores of unpublished phantoms), so the fixtures are
oracle values of the 64^2 FP64 reference configuration (64 x 64 pixels of
0.15 mm, a disc of radius 8 px at 1500 m/s in 1540 m/s, 32 elements at
0.3 mm pitch, 1 MHz): sampled data entries, the misfit and sampled gradient
entries at m0 = m_true / 2, and sampled SoS values after one ADMM-TV
iteration (Algorithm 1) with fixed weights.

    python tests/golden/make_golden.py      # rewrites disc64_reference.json
"""
import json
import os
import sys

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

import oracle  # noqa: E402
from oracle import admm, inverse, model  # noqa: E402
from paper_2604_15796_gb300 import phantoms  # noqa: E402

OUT = os.path.join(HERE, "disc64_reference.json")
PIXELS = [(0, 0), (5, 40), (17, 9), (31, 32), (40, 55), (63, 63)]
DATA = [(0, 0, 0), (0, 3, 17), (0, 12, 12), (0, 31, 0), (0, 20, 27)]
PARAMS = dict(lam_rel=1e-3, rho_rel=0.5, gamma_rel=1e-3, n_cg=6)


def compute():
    w = phantoms.disc_phantom()
    prob = oracle.Problem(tuple(w.shape), w.h, w.c0, w.elem, np.asarray(w.freqs))
    m_true = model.contrast_from_sos(w.sos, w.c0)
    m0 = 0.5 * m_true
    _, d_obs = inverse.forward_model(m_true, prob, "lu")
    ref = inverse.gradient(m0, d_obs, prob, "lu")
    grad = np.asarray(ref["grad"]).reshape(w.shape)
    scale = float(np.abs(grad).max())
    p = admm.AdmmParams(lam=PARAMS["lam_rel"] * scale, rho=PARAMS["rho_rel"] * scale,
                        gamma=PARAMS["gamma_rel"] * scale, n_cg=PARAMS["n_cg"])
    rf = inverse.receiver_fields(m0, prob, "lu")
    g0 = admm.grad_op(m0, w.shape)
    _, _, _, sos1, _ = admm.admm_tv_step(m0, g0, np.zeros_like(g0), ref["grad"], ref["fields"],
                                         rf, prob, p)
    return {
        "config": "disc64: 64x64 pixels of 0.15 mm, disc r = 8 px at 1500 m/s in 1540 m/s "
                  "(phantoms.disc_phantom(seed=1000)), 32 elements at 0.3 mm pitch, 1 MHz; "
                  "d_obs = F(m_true) without noise; m0 = m_true / 2",
        "source": "oracle/ (FP64, dense LU), written by tests/golden/make_golden.py",
        "admm": dict(PARAMS, scale=scale, dual_step="rho (as printed)"),
        "data": [[l, e, j, d_obs[l, e, j].real, d_obs[l, e, j].imag] for l, e, j in DATA],
        "misfit_m0": ref["misfit"],
        "grad_m0": [[z, x, grad[z, x].real, grad[z, x].imag] for z, x in PIXELS],
        "grad_m0_norm": float(np.linalg.norm(grad)),
        "sos_after_one_iteration": [[z, x, float(sos1[z, x])] for z, x in PIXELS],
    }


if __name__ == "__main__":
    with open(OUT, "w") as f:
        json.dump(compute(), f, indent=1)
    print("wrote", OUT)

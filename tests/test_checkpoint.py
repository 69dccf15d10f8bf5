"""The checkpoint file round-trips the ADMM state and the weights exactly
(CPU tensors; the resume on the device is tests/test_gpu_checkpoint.py)."""
import numpy as np
import torch

from paper_2604_15796_gb300 import checkpoint, phantoms


def test_checkpoint_round_trip(tmp_path):
    m = torch.from_numpy(phantoms.complex_normal((6, 8), 1))
    g = torch.from_numpy(phantoms.complex_normal((2, 6, 8), 2))
    u = torch.from_numpy(phantoms.complex_normal((2, 6, 8), 3))
    prm = dict(lam=1.5e-4, rho=0.25, gamma=3e-6, n_cg=7)
    path = str(tmp_path / "s.npz")
    checkpoint.save(path, 4, m, g, u, prm)
    k, m2, g2, u2, prm2 = checkpoint.load(path, device="cpu")
    assert k == 4 and prm2 == prm
    for a, b in ((m, m2), (g, g2), (u, u2)):
        assert a.dtype == b.dtype and torch.equal(a, b)
    assert np.load(path)["m"].dtype == np.complex128

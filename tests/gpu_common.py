"""Shared helpers of the GPU parity tests: seeded small problems, oracle
references and error measures.  Imports torch/CUDA lazily."""
import numpy as np

import oracle
from oracle import model
from paper_2604_15796_gb300 import phantoms


def rel_l2(a, b):
    a = np.asarray(a).ravel()
    b = np.asarray(b).ravel()
    nb = np.linalg.norm(b)
    return float(np.linalg.norm(a - b) / (nb if nb > 0 else 1.0))


def small_workload(shape, n_elem=6, freqs=(1.5e6, 3.0e6), h=0.1e-3, pitch=0.3e-3, seed=7,
                   sigma=10.0):
    """Tissue-statistics phantom on a small grid (parity cases)."""
    return phantoms.scaled(shape, h, n_elem, pitch, np.asarray(freqs), seed,
                           sigma=sigma, inclusions=[1520.0, 1580.0], semi_mm=(0.3, 0.8))


def oracle_problem(w):
    return oracle.Problem(tuple(w.shape), w.h, w.c0, w.elem, np.asarray(w.freqs))


def contrast(w):
    return model.contrast_from_sos(w.sos, w.c0)


def to_gpu(a, dtype):
    import torch
    return torch.from_numpy(np.ascontiguousarray(a)).to(device="cuda", dtype=dtype)


def to_np(t):
    import torch
    torch.cuda.synchronize()
    return t.detach().cpu().numpy()

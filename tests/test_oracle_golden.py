"""The oracle reproduces the stored values of tests/golden/ (64^2 FP64
reference configuration, dense LU): a change to the oracle's arithmetic
shows here, and its commit names the passage that justifies it."""
import json
import os

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))


def test_oracle_reproduces_the_reference_configuration_values():
    import importlib.util
    spec = importlib.util.spec_from_file_location(
        "make_golden", os.path.join(HERE, "golden", "make_golden.py"))
    mg = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mg)
    stored = json.load(open(os.path.join(HERE, "golden", "disc64_reference.json")))
    now = mg.compute()
    for key in ("data", "grad_m0", "sos_after_one_iteration"):
        a = np.asarray(now[key], dtype=np.float64)
        b = np.asarray(stored[key], dtype=np.float64)
        assert np.allclose(a, b, rtol=1e-9, atol=1e-9 * np.abs(b[:, -1]).max()), key
    assert np.isclose(now["misfit_m0"], stored["misfit_m0"], rtol=1e-9)
    assert np.isclose(now["grad_m0_norm"], stored["grad_m0_norm"], rtol=1e-9)

"""The library's Bessel / Hankel functions of complex argument
(csrc/bessel_c.cuh, used on the device for the 2-D Green's function of an
attenuating background) compiled on the host with g++ and compared with
SciPy's (an independent implementation) over the arguments the lattice and
the incident fields reach: |z| from 1e-3 to 600, arguments from the real
axis to 0.1 rad (Im k up to a tenth of Re k; tissue gives ~1e-3), both sides
of the series / asymptotic switch."""
import os
import shutil
import subprocess
import tempfile

import numpy as np
import pytest
from scipy import special

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
CSRC = os.path.join(ROOT, "paper_2604_15796_gb300", "csrc")

HARNESS = r"""
#include <cstdio>
#include "bessel_c.cuh"
int main() {
  double re, im;
  while (std::scanf("%lf %lf", &re, &im) == 2) {
    const fwi::bes::cd z{re, im};
    const fwi::bes::cd h0 = fwi::bes::hankel1_0(z), h1 = fwi::bes::hankel1_1(z),
                       j1 = fwi::bes::besselj_1(z);
    std::printf("%.17e %.17e %.17e %.17e %.17e %.17e\n", h0.re, h0.im, h1.re, h1.im, j1.re,
                j1.im);
  }
  return 0;
}
"""


@pytest.fixture(scope="module")
def harness():
    cxx = shutil.which("g++") or shutil.which("c++")
    if cxx is None:
        pytest.skip("no host C++ compiler")
    d = tempfile.mkdtemp()
    src = os.path.join(d, "h.cpp")
    exe = os.path.join(d, "h")
    with open(src, "w") as f:
        f.write(HARNESS)
    subprocess.run([cxx, "-O2", "-std=c++17", "-I", CSRC, src, "-o", exe], check=True)
    yield exe
    shutil.rmtree(d, ignore_errors=True)


def _run(exe, z):
    inp = "\n".join(f"{v.real:.17e} {v.imag:.17e}" for v in z) + "\n"
    out = subprocess.run([exe], input=inp, capture_output=True, text=True, check=True).stdout
    a = np.array([[float(t) for t in line.split()] for line in out.strip().splitlines()])
    return a[:, 0] + 1j * a[:, 1], a[:, 2] + 1j * a[:, 3], a[:, 4] + 1j * a[:, 5]


def test_complex_argument_bessel_functions_against_scipy(harness):
    mod = np.concatenate([np.geomspace(1e-3, 600.0, 160), [13.9, 13.99, 14.0, 14.01, 14.1]])
    z = np.concatenate([mod * np.exp(1j * t) for t in (0.0, 1e-3, 0.02, 0.1)])
    h0, h1, j1 = _run(harness, z)
    ref_h0 = special.hankel1(0, z)
    ref_h1 = special.hankel1(1, z)
    ref_j1 = special.jv(1, z)
    assert np.max(np.abs(h0 - ref_h0) / np.abs(ref_h0)) < 3e-10
    assert np.max(np.abs(h1 - ref_h1) / np.abs(ref_h1)) < 3e-10
    # J1 against its scale (it has zeros on the real axis)
    scale = np.maximum(np.abs(ref_j1), np.abs(ref_h1) * 1e-3)
    assert np.max(np.abs(j1 - ref_j1) / scale) < 1e-9

"""The FFT building blocks of the operator kernels (csrc/fft_core.cuh: the
in-register DFTs of radices 2, 3, 4, 5 and their composites, the pruned
half-input / half-output DFTs, and the four-step line transform of Eq. 5's
FFT convolution split into phases A-D), compiled on the host with g++ and
compared with numpy's FFT (an independent implementation).  The phases run
thread by thread over a shared array exactly as the CUDA threads of one line
do, so a wrong slot, twiddle or pruning index fails here without a GPU."""
import os
import shutil
import subprocess
import tempfile

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
CSRC = os.path.join(ROOT, "paper_2604_15796_gb300", "csrc")
CUDA_INC = "/usr/local/cuda/include"

HARNESS = r"""
#include <cmath>
#include <cstdio>
#include <cstring>
#include <vector>
#include "fft_core.cuh"
using namespace fwi;
using V = cplx<double>;

static std::vector<V> read_line(int n) {
  std::vector<V> x(n);
  for (int i = 0; i < n; ++i)
    if (std::scanf("%lf %lf", &x[i].x, &x[i].y) != 2) x[i] = mk<double>(0, 0);
  return x;
}
static void print_line(const V* x, int n) {
  for (int i = 0; i < n; ++i) std::printf("%.17e %.17e\n", x[i].x, x[i].y);
}

template <int R> static void dfts() {
  std::vector<V> x = read_line(R), y = x;
  Dft<R, false, double>::run(x.data());
  print_line(x.data(), R);
  Dft<R, true, double>::run(y.data());
  print_line(y.data(), R);
  if constexpr (R % 2 == 0) {
    std::vector<V> h = read_line(R);  // inputs R/2 .. R zero
    DftHalfIn<R, false, double>::run(h.data());
    print_line(h.data(), R);
    std::vector<V> o = read_line(R);
    DftHalfOut<R, true, double>::run(o.data());
    print_line(o.data(), R / 2);
  }
}

// One line of L = R1 R2 samples through phases A, B (forward, zero-padded
// input) and C, D (inverse, cropped output), thread by thread.
template <class P> static void line() {
  constexpr int L = P::L, PAD = 1, TL = P::TL;
  std::vector<V> tw(L);
  for (int j = 0; j < L; ++j) {
    const double a = -2.0 * 3.14159265358979323846 * j / L;
    tw[j] = mk<double>(std::cos(a), std::sin(a));
  }
  std::vector<V> x = read_line(L / 2), sm(P::span(PAD));
  std::vector<std::vector<V>> v(TL, std::vector<V>(P::E));
  for (int t = 0; t < TL; ++t) {
    for (int i = 0; i < P::C1; ++i)
      for (int n1 = 0; n1 < P::R1; ++n1) {
        const int n2 = t + i * TL;
        v[t][i * P::R1 + n1] =
            (n2 < P::R2 && n1 < P::R1 / 2) ? x[P::R2 * n1 + n2] : mk<double>(0, 0);
      }
    phaseA_store<P, double, true>(t, v[t].data(), sm.data(), 1, PAD, tw.data());
  }
  std::vector<V> X(L);
  for (int t = 0; t < TL; ++t) {
    phaseB_load<P, double>(t, v[t].data(), sm.data(), 1, PAD);
    for (int i = 0; i < P::C3; ++i) {
      const int k1 = t + i * TL;
      if (k1 < P::R1)
        for (int k2 = 0; k2 < P::R2; ++k2) X[k1 + P::R1 * k2] = v[t][i * P::R2 + k2];
    }
  }
  print_line(X.data(), L);
  // inverse of a fresh spectrum
  std::vector<V> Y = read_line(L);
  for (int t = 0; t < TL; ++t) {
    for (int i = 0; i < P::C3; ++i) {
      const int k1 = t + i * TL;
      for (int k2 = 0; k2 < P::R2; ++k2)
        v[t][i * P::R2 + k2] = (k1 < P::R1) ? Y[k1 + P::R1 * k2] : mk<double>(0, 0);
    }
    phaseC_store<P, double>(t, v[t].data(), sm.data(), 1, PAD, tw.data());
  }
  std::vector<V> y(L / 2);
  for (int t = 0; t < TL; ++t) {
    phaseD_load<P, double>(t, v[t].data(), sm.data(), 1, PAD);
    for (int i = 0; i < P::C1; ++i) {
      const int n2 = t + i * TL;
      if (n2 < P::R2)
        for (int n1 = 0; n1 < P::R1 / 2; ++n1) y[P::R2 * n1 + n2] = v[t][i * P::R1 + n1];
    }
  }
  print_line(y.data(), L / 2);
}

int main(int argc, char** argv) {
  const char* what = argv[1];
  if (!std::strcmp(what, "dft")) {
    dfts<2>(); dfts<3>(); dfts<4>(); dfts<5>(); dfts<8>(); dfts<12>(); dfts<16>();
    dfts<20>(); dfts<24>(); dfts<32>();
  } else {
    line<Plan<64, 8, 8, 8>>();
    line<Plan<128, 8, 16, 8>>();
    line<Plan<192, 12, 16, 16>>();
    line<Plan<256, 16, 16, 16>>();
    line<Plan<320, 20, 16, 20>>();
    line<Plan<640, 20, 32, 32>>();
  }
  return 0;
}
"""

DFT_SIZES = [2, 3, 4, 5, 8, 12, 16, 20, 24, 32]
LINE_SIZES = [64, 128, 192, 256, 320, 640]


@pytest.fixture(scope="module")
def harness():
    cxx = shutil.which("g++") or shutil.which("c++")
    if cxx is None or not os.path.exists(os.path.join(CUDA_INC, "vector_types.h")):
        pytest.skip("no host C++ compiler or CUDA headers")
    d = tempfile.mkdtemp()
    src = os.path.join(d, "h.cpp")
    exe = os.path.join(d, "h")
    with open(src, "w") as f:
        f.write(HARNESS)
    subprocess.run([cxx, "-O1", "-std=c++17", "-I", CSRC, "-I", CUDA_INC, src, "-o", exe],
                   check=True)
    return exe


def _run(exe, mode, arrays):
    inp = "\n".join(f"{z.real:.17e} {z.imag:.17e}" for a in arrays for z in a)
    out = subprocess.run([exe, mode], input=inp, capture_output=True, text=True,
                         check=True).stdout.split()
    v = np.array(out, dtype=float)
    return v[0::2] + 1j * v[1::2]


def _rand(rng, n):
    return rng.standard_normal(n) + 1j * rng.standard_normal(n)


def test_in_register_dfts_match_numpy(harness):
    rng = np.random.default_rng(5)
    inputs, expect = [], []
    for r in DFT_SIZES:
        x = _rand(rng, r)
        inputs.append(x)
        expect += [np.fft.fft(x), r * np.fft.ifft(x)]
        if r % 2 == 0:
            h = _rand(rng, r)
            h[r // 2:] = 0
            o = _rand(rng, r)
            inputs += [h, o]
            expect += [np.fft.fft(h), (r * np.fft.ifft(o))[: r // 2]]
    got = _run(harness, "dft", inputs)
    want = np.concatenate(expect)
    assert got.shape == want.shape
    assert np.max(np.abs(got - want)) < 1e-12 * np.max(np.abs(want))


def test_four_step_line_phases_match_numpy(harness):
    """Phases A+B on a zero-padded line give its full spectrum; phases C+D
    on a spectrum give the first half of its unnormalised inverse (the
    cropped output), for every unsplit plan of the operator kernels' table
    that the benchmark grids use (radices 2, 3, 5; lines that tile the
    threads and lines with idle threads in phases A/D)."""
    rng = np.random.default_rng(6)
    inputs, expect = [], []
    for n in LINE_SIZES:
        x = _rand(rng, n // 2)
        y = _rand(rng, n)
        inputs += [x, y]
        expect += [np.fft.fft(np.concatenate([x, np.zeros(n // 2)])),
                   (n * np.fft.ifft(y))[: n // 2]]
    got = _run(harness, "line", inputs)
    want = np.concatenate(expect)
    assert got.shape == want.shape
    off = 0
    for n, e in zip([m for m in LINE_SIZES for _ in (0, 1)], expect):
        g = got[off: off + e.size]
        assert np.max(np.abs(g - e)) < 1e-11 * np.max(np.abs(e)), n
        off += e.size

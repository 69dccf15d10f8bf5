"""The C-ABI library builds, loads, and exports every entry point that
include/libfwi.h declares (no GPU calls)."""
import ctypes
import os
import re

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_symbols():
    src = open(os.path.join(ROOT, "include", "libfwi.h")).read()
    return sorted(set(re.findall(r"FWI_API\s+[\w\s\*]+?\b(fwi_\w+)\s*\(", src)))


def test_header_declares_the_hot_path_calls():
    names = declared_symbols()
    for required in ["fwi_create", "fwi_destroy", "fwi_forward", "fwi_adjoint",
                     "fwi_gradient", "fwi_admm_tv_step", "fwi_apply_K", "fwi_apply_A",
                     "fwi_apply_AH", "fwi_workspace_bytes", "fwi_last_error"]:
        assert required in names


def test_library_exports_every_declared_symbol():
    from paper_2604_15796_gb300 import build, libfwi
    path = build.build()
    lib = ctypes.CDLL(path)
    for name in declared_symbols():
        assert hasattr(lib, name), name
    assert set(libfwi.EXPORTS) == set(declared_symbols())


def test_workspace_bytes_and_argument_checks_without_gpu():
    """fwi_workspace_bytes and descriptor validation run on the host."""
    import numpy as np
    from paper_2604_15796_gb300 import build, libfwi
    build.build()
    elem = np.stack([np.linspace(-1e-3, 1e-3, 8), np.full(8, -1e-4)], axis=1)
    d, keep = libfwi.make_desc((32, 32), 1e-4, 1540.0, elem, [1e6, 2e6])
    n = libfwi.fwi_workspace_bytes(ctypes.byref(d))
    N, rhs = 32 * 32, 16
    assert n >= 4 * rhs * N * 8 + 5 * rhs * N * 8
    bad, keep2 = libfwi.make_desc((33, 32), 1e-4, 1540.0, elem, [1e6])
    assert libfwi.fwi_workspace_bytes(ctypes.byref(bad)) == 0
    bad3, keep3 = libfwi.make_desc((32, 32, 32), 1e-4, 1540.0, elem, [1e6])
    # elem has 2 columns but the 3-D descriptor reads 3 per element: still a
    # valid size computation (positions are only read by fwi_create)
    assert libfwi.fwi_workspace_bytes(ctypes.byref(bad3)) > 0
    del keep, keep2, keep3


def test_plane_wave_descriptor_sizes_and_checks():
    """Plane-wave transmits (n_tx > 0) add the weights, W^H W and the
    data-space synthesis buffers to the workspace; n_tx > 0 without angles,
    or a non-finite angle, is rejected (0 bytes)."""
    import numpy as np
    from paper_2604_15796_gb300 import build, libfwi
    build.build()
    elem = np.stack([np.linspace(-1e-3, 1e-3, 8), np.full(8, -1e-4)], axis=1)
    d0, k0 = libfwi.make_desc((32, 32), 1e-4, 1540.0, elem, [1e6, 2e6])
    ang = np.linspace(-1.0, 1.0, 12)
    d1, k1 = libfwi.make_desc((32, 32), 1e-4, 1540.0, elem, [1e6, 2e6], tx_angles=ang)
    assert d1.n_tx == 12
    n0 = libfwi.fwi_workspace_bytes(ctypes.byref(d0))
    n1 = libfwi.fwi_workspace_bytes(ctypes.byref(d1))
    nf, nt, ne = 2, 12, 8
    assert n1 - n0 >= nf * (2 * nt * ne + 2 * ne * ne) * 16
    d1.tx_angle = None
    assert libfwi.fwi_workspace_bytes(ctypes.byref(d1)) == 0
    bad_ang = ang.copy()
    bad_ang[3] = np.nan
    d2, k2 = libfwi.make_desc((32, 32), 1e-4, 1540.0, elem, [1e6], tx_angles=bad_ang)
    assert libfwi.fwi_workspace_bytes(ctypes.byref(d2)) == 0
    del k0, k1, k2


def test_inversion_mesh_attenuation_and_element_length_checks():
    """The inversion-mesh factor must divide every grid size (<= 1: the
    forward mesh); alpha0 and elem_length must be finite and >= 0; an
    inversion mesh adds one forward-mesh vector and a lossy background one
    data-space buffer per frequency to the workspace (0 bytes: rejected)."""
    import numpy as np
    from paper_2604_15796_gb300 import build, libfwi
    build.build()
    elem = np.stack([np.linspace(-1e-3, 1e-3, 8), np.full(8, -1e-4)], axis=1)
    freqs = [1e6, 2e6]

    def nbytes(shape, e=elem, **kw):
        d, keep = libfwi.make_desc(shape, 1e-4, 1540.0, e, freqs, **kw)
        n = libfwi.fwi_workspace_bytes(ctypes.byref(d))
        del keep
        return n
    base = nbytes((32, 32))
    assert base > 0
    for r in (0, -2, 1):
        assert nbytes((32, 32), inv_factor=r) == base
    assert nbytes((32, 32), inv_factor=2) >= base + 32 * 32 * 16
    assert nbytes((32, 32), inv_factor=4) == nbytes((32, 32), inv_factor=2)
    assert nbytes((32, 32), inv_factor=3) == 0
    assert nbytes((32, 64), inv_factor=64) == 0
    e3 = np.stack([np.linspace(-1e-3, 1e-3, 8), np.zeros(8), np.full(8, -1e-4)], axis=1)
    assert nbytes((32, 16, 16), e3, inv_factor=16) > 0
    assert nbytes((32, 16, 16), e3, inv_factor=32) == 0
    ne = elem.shape[0]
    assert nbytes((32, 32), alpha0=1e-4) == base + len(freqs) * (ne * ne + 1) * 16
    assert nbytes((32, 32), alpha0=0.0) == base
    for bad in (-1e-4, float("nan"), float("inf")):
        assert nbytes((32, 32), alpha0=bad) == 0
        assert nbytes((32, 16, 16), e3, elem_length=bad) == 0
    assert nbytes((32, 16, 16), e3, elem_length=1e-2) == nbytes((32, 16, 16), e3)


def test_binding_rejects_tensors_that_do_not_match_the_documented_layout():
    """The binding checks device, dtype, element count and contiguity of a
    tensor argument before its pointer reaches the library (CPU tensors:
    every one of them is rejected, and the message names the argument)."""
    import pytest
    import torch
    from paper_2604_15796_gb300 import libfwi
    assert libfwi._dev(None, torch.complex128, 4, "fields", optional=True) is None
    with pytest.raises(ValueError, match="m is required"):
        libfwi._dev(None, torch.complex128, 4, "m")
    for t in (torch.zeros(4, dtype=torch.complex128),           # host memory
              torch.zeros(4, dtype=torch.float64),              # wrong dtype
              torch.zeros(5, dtype=torch.complex128),           # wrong size
              torch.zeros(4, 2, dtype=torch.complex128).t()[0]):  # strided view
        with pytest.raises(ValueError, match="^m: expected"):
            libfwi._dev(t, torch.complex128, 4, "m")


def test_the_boundary_is_plain_c(tmp_path):
    """include/libfwi.h compiles as C11 with every warning an error, and a C
    program links against the library and calls a host-only entry point."""
    import shutil
    import subprocess
    from paper_2604_15796_gb300 import build
    cc = shutil.which("gcc") or shutil.which("cc")
    if cc is None:
        import pytest
        pytest.skip("no C compiler")
    lib = build.build()
    src = tmp_path / "t.c"
    src.write_text(r'''
#include <stdio.h>
#include "libfwi.h"
int main(void) {
  double elem[4] = {-1e-4, -1e-4, 1e-4, -1e-4}, f[1] = {1e6};
  fwi_problem_desc d = {0};
  d.dim = 2; d.n[0] = 16; d.n[1] = 1; d.n[2] = 16; d.h = 1e-4; d.c0 = 1540.0;
  d.n_elem = 2; d.elem_pos = elem; d.n_freq = 1; d.freq_hz = f;
  printf("%s %zu\n", fwi_version(), fwi_workspace_bytes(&d));
  return 0;
}
''')
    exe = tmp_path / "t"
    libdir = os.path.dirname(lib)
    subprocess.run([cc, "-std=c11", "-Wall", "-Wextra", "-Werror", "-I",
                    os.path.join(ROOT, "include"), str(src), "-L", libdir, "-lfwi",
                    "-Wl,-rpath," + libdir, "-o", str(exe)], check=True)
    out = subprocess.run([str(exe)], capture_output=True, text=True, check=True).stdout.split()
    assert out[0] == "libfwi" and int(out[-1]) > 0


def test_a_missing_library_fails_loudly(tmp_path):
    """Without the compiled library the binding raises (no CPU fallback)."""
    import subprocess
    import sys
    missing = str(tmp_path / "libfwi.so")
    code = ("from paper_2604_15796_gb300 import libfwi\n"
            "try:\n"
            f"    libfwi.load({missing!r})\n"
            "except OSError as e:\n"
            "    print('raised:', e)\n")
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    out = subprocess.run([sys.executable, "-c", code], cwd=root, capture_output=True, text=True,
                         check=True).stdout
    assert out.startswith("raised: libfwi.so not built"), out


def test_degenerate_descriptors_are_rejected_on_the_host():
    """Empty arrays (no element, no frequency), non-positive or non-finite
    h, c0 and frequencies, and grids without an FFT plan (2 N outside
    16 ... 1024) give 0 workspace bytes; a non-finite element position makes
    fwi_create fail with FWI_ERR_INVALID_ARG before any device call."""
    import numpy as np
    from paper_2604_15796_gb300 import build, libfwi
    build.build()
    elem = np.stack([np.linspace(-1e-3, 1e-3, 8), np.full(8, -1e-4)], axis=1)

    def nbytes(shape=(32, 32), e=elem, freqs=(1e6,), h=1e-4, c0=1540.0):
        d, keep = libfwi.make_desc(shape, h, c0, e, list(freqs))
        n = libfwi.fwi_workspace_bytes(ctypes.byref(d))
        del keep
        return n
    assert nbytes() > 0 and nbytes((8, 8)) > 0 and nbytes((512, 512)) > 0
    assert nbytes(e=np.zeros((0, 2))) == 0
    assert nbytes(freqs=()) == 0
    for bad in (0.0, -1e-4, float("nan"), float("inf")):
        assert nbytes(h=bad) == 0
        assert nbytes(c0=bad * 1e7) == 0
        assert nbytes(freqs=(1e6, bad * 1e10)) == 0
    for shape in ((1, 1), (4, 32), (1024, 1024), (32, 513)):
        assert nbytes(shape) == 0, shape
    bad_elem = elem.copy()
    bad_elem[5, 0] = np.nan
    d, keep = libfwi.make_desc((32, 32), 1e-4, 1540.0, bad_elem, [1e6])
    assert libfwi.fwi_workspace_bytes(ctypes.byref(d)) > 0  # positions are read by fwi_create
    h = ctypes.c_void_p()
    st = libfwi.fwi_create(ctypes.byref(d), None, ctypes.byref(h))
    assert st == libfwi.FWI_ERR_INVALID_ARG and not h.value
    assert b"elem_pos must be finite" in libfwi.fwi_last_error(None)
    del keep

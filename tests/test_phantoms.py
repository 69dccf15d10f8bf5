"""The seeded synthetic workloads have the shapes and acquisition of the
configurations they stand in for (grid, pixel, array, frequencies), their
SoS stays within the stated ranges, and they are deterministic."""
import numpy as np
import pytest

from paper_2604_15796_gb300 import phantoms


@pytest.mark.parametrize("fn,shape,h,n_elem,pitch,freqs", [
    (phantoms.disc_phantom, (64, 64), 0.15e-3, 32, 0.3e-3, (1e6, 1e6, 1)),
    (phantoms.thyroid_256, (256, 256), 0.1e-3, 128, 0.2e-3, (0.5e6, 3e6, 6)),
    (phantoms.large_512, (512, 512), 0.08e-3, 192, 0.2e-3, (0.3e6, 5e6, 12)),
    (phantoms.volume_3d, (128, 160, 160), 0.2e-3, 128, 0.2e-3, (0.5e6, 2e6, 4)),
    (phantoms.planewave_2d, (384, 384), 0.13e-3, 64, 0.78e-3, (0.2e6, 3e6, 15)),
    (phantoms.elevation_3d, (64, 64, 96), 0.2e-3, 64, 0.3e-3, (0.2e6, 2e6, 10)),
])
def test_workload_geometry(fn, shape, h, n_elem, pitch, freqs):
    w = fn()
    assert w.shape == shape and w.h == pytest.approx(h) and w.n_elem == n_elem
    assert np.allclose(np.diff(w.elem[:, 0]), pitch)
    assert abs(w.elem[:, 0].mean()) < 1e-12                  # centred array
    assert np.allclose(w.elem[:, -1], -h)                      # one pixel above the grid
    assert np.allclose(w.freqs, np.linspace(*freqs))
    assert w.sos.shape == shape and 1390.0 < w.sos.min() and w.sos.max() < 1650.0
    w2 = fn()
    assert np.array_equal(w.sos, w2.sos)                       # seeded
    assert w.elem[:, 0].max() <= shape[-1] * h / 2             # the aperture fits the grid


def test_acquisition_specifics():
    pw = phantoms.planewave_2d()
    assert len(pw.meta["tx_angles"]) == 60
    assert np.allclose(np.rad2deg(pw.meta["tx_angles"][[0, -1]]), [-60.0, 60.0])
    el = phantoms.elevation_3d()
    assert el.meta["elem_length"] == pytest.approx(1e-2)
    assert {1400.0, 1600.0} <= set(np.unique(el.sos))
    th = phantoms.thyroid_256()
    assert {1520.0, 1580.0} <= set(np.unique(np.round(th.sos, 6)))


def test_serving_stream():
    specs = phantoms.serving_requests(n_req=40, seed=1004, rate_hz=1.0)
    assert len(specs) == 40
    grids = {tuple(s["shape"]) for s in specs}
    assert grids <= {(128, 128), (256, 256), (384, 384), (512, 512), (96, 96, 96)}
    for s in specs:
        assert 64 <= s["n_elem"] <= 192 and 2 <= len(s["freqs"]) <= 12
        assert s["freqs"].min() >= 0.3e6 - 1 and s["freqs"].max() <= 5e6 + 1
        # the aperture fits the grid and the band keeps >= 3.85 pixels per wavelength
        assert (s["n_elem"] - 1) * s["pitch"] <= s["shape"][-1] * s["h"]
        assert s["freqs"].max() <= 1540.0 / (3.85 * s["h"]) * (1 + 1e-9)

"""Pins of the oracle's 3-D line elements of finite elevation (Sec. V-B:
elements of 1 cm along y).  The element's Green's function is the mean of
the point Green's function over the element (operator.element_green):

* static limit: as k -> 0 its real part is the closed form
  (asinh((L/2 - dy)/rho) + asinh((L/2 + dy)/rho)) / (4 pi L);
* short elements reduce to the point element;
* long elements approach the 2-D Green's function: L times the mean tends
  to (i/4) H0^(1)(k rho) (the line source), within the tail of the
  truncated line;
* the data stay reciprocal (P_ej = P_je), since transmit field and
  receiver sensing are the same mean;
* 2-D problems ignore the length."""
import numpy as np
from scipy.special import hankel1

import oracle
from oracle import inverse, model, operator


def prob3d(shape=(3, 4, 5), h=0.2e-3, n_elem=3, freqs=(2e6,), length=1e-2, pitch=0.3e-3):
    p = oracle.Problem(shape, h, 1540.0, model.linear_array(n_elem, pitch, h, 3),
                       np.array(freqs, dtype=np.float64))
    p.extra["elem_length"] = length
    return p


def _geometry(p):
    x = model.pixel_centres(p.shape, p.h)
    d = x[None, :, :] - p.elem[:, None, :]          # [N_E, N, 3]
    rho = np.sqrt(d[..., 0] ** 2 + d[..., 2] ** 2)
    return d, rho


def test_static_limit_is_the_closed_form():
    p = prob3d(freqs=(1.0,))                        # k = 4e-3 / m: k r ~ 1e-4
    g = operator.element_green(p)[0].reshape(p.n_elem, -1)
    d, rho = _geometry(p)
    L = p.extra["elem_length"]
    dy = d[..., 1]
    ref = (np.arcsinh((L / 2 - dy) / rho) + np.arcsinh((L / 2 + dy) / rho)) / (4 * np.pi * L)
    assert np.allclose(g.real, ref, rtol=1e-9, atol=0)


def test_short_element_is_the_point_element():
    """The mean differs from the point value by (L / rho)^2 / 24 relative
    (second-order term), 1e-10 here."""
    p = prob3d(length=1e-8)
    g = operator.element_green(p)
    p.extra["elem_length"] = 0.0
    g0 = operator.element_green(p)
    assert np.allclose(g, g0, rtol=1e-9, atol=0)


def test_long_element_tends_to_the_2d_line_source():
    """L = 0.4 m, k rho ~ 8: the truncated line differs from the infinite one
    by an oscillating tail of relative size ~ 1/(k L) ~ 1e-3."""
    p = prob3d(shape=(2, 2, 2), h=0.5e-3, n_elem=1, freqs=(2e6,), length=0.4)
    g = operator.element_green(p)[0, 0].ravel() * 0.4
    _, rho = _geometry(p)
    k = model.wavenumbers(p)[0]
    ref = 0.25j * hankel1(0, k * rho[0])
    assert np.max(np.abs(g - ref) / np.abs(ref)) < 1e-2


def test_line_element_data_are_reciprocal():
    p = prob3d(shape=(3, 4, 5), n_elem=3, freqs=(1.5e6, 2e6), length=5e-3)
    rng = np.random.default_rng(3)
    m = 0.05 * (rng.standard_normal(p.shape) + 0.1j * rng.standard_normal(p.shape))
    _, d = inverse.forward_model(m, p, "lu")
    for l in range(p.n_freq):
        assert np.allclose(d[l], d[l].T, rtol=1e-10, atol=1e-14 * np.abs(d[l]).max())
    # and the elevation matters: point elements give other data
    p.extra["elem_length"] = 0.0
    _, d0 = inverse.forward_model(m, p, "lu")
    assert not np.allclose(d, d0, rtol=1e-2)


def test_two_dimensional_problems_ignore_the_length():
    p = oracle.Problem((6, 8), 0.1e-3, 1540.0, model.linear_array(3, 0.2e-3, 0.1e-3, 2),
                       np.array([2e6]))
    g0 = operator.element_green(p)
    p.extra["elem_length"] = 1e-2
    assert np.array_equal(operator.element_green(p), g0)

"""Pins of the oracle's Green's functions (Sec. II, Eq. 4-5) against
quantities the mathematics fixes independently of the oracle's formulas:
numerical quadrature of the point Green's function over the equivalent disc
/ ball, the large-argument (outgoing-wave) asymptotics, and the Helmholtz
equation itself."""
import numpy as np
import pytest
from scipy import integrate, special

from oracle import green


def _quad_c(f, a, b, **kw):
    re = integrate.quad(lambda t: np.real(f(t)), a, b, limit=400, epsabs=0.0, epsrel=1e-12, **kw)[0]
    im = integrate.quad(lambda t: np.imag(f(t)), a, b, limit=400, epsabs=0.0, epsrel=1e-12, **kw)[0]
    return re + 1j * im


def _dblquad_c(f, a, b, c, d):
    kw = dict(epsabs=0.0, epsrel=1e-11)
    re = integrate.dblquad(lambda y, x: np.real(f(x, y)), a, b, c, d, **kw)[0]
    im = integrate.dblquad(lambda y, x: np.imag(f(x, y)), a, b, c, d, **kw)[0]
    return re + 1j * im


def _disc_integral(k, a, r):
    """Integral of (i/4) H0^(1)(k |x - x'|) over the disc |x'| <= a, at a
    point at distance r from the centre, by 2D quadrature in polar
    coordinates (rho, theta) around the disc centre."""
    if r == 0.0:
        return 2.0 * np.pi * _quad_c(
            lambda rho: 0.25j * special.hankel1(0, k * rho) * rho, 0.0, a)

    def f(rho, th):
        dist = np.sqrt(r * r + rho * rho - 2.0 * r * rho * np.cos(th))
        return 0.25j * special.hankel1(0, k * dist) * rho
    return _dblquad_c(f, 0.0, a, 0.0, 2.0 * np.pi)


def _ball_integral(k, a, r):
    """Integral of e^{ik|x-x'|}/(4 pi |x-x'|) over the ball |x'| <= a."""
    if r == 0.0:
        return _quad_c(lambda rho: rho * np.exp(1j * k * rho), 0.0, a)

    def f(rho, th):
        dist = np.sqrt(r * r + rho * rho - 2.0 * r * rho * np.cos(th))
        return (2.0 * np.pi * rho * rho * np.sin(th)
                * np.exp(1j * k * dist) / (4.0 * np.pi * dist))
    return _dblquad_c(f, 0.0, a, 0.0, np.pi)


CASES = [(2 * np.pi * 1e6 / 1540.0, 0.15e-3), (2 * np.pi * 3e6 / 1540.0, 0.1e-3),
         (2 * np.pi * 5e6 / 1540.0, 0.08e-3), (2 * np.pi * 2e6 / 1540.0, 0.2e-3)]


@pytest.mark.parametrize("k,h", CASES)
@pytest.mark.parametrize("r_cells", [0.0, 1.0, np.sqrt(2.0), 3.0])
def test_cell_green_2d_matches_disc_quadrature(k, h, r_cells):
    a = green.equivalent_radius(h, 2)
    r = r_cells * h
    ref = _disc_integral(k, a, r)
    got = green.green_cell(k, np.array([r]), h, 2)[0]
    assert abs(got - ref) <= 1e-8 * abs(ref)


@pytest.mark.parametrize("k,h", CASES)
@pytest.mark.parametrize("r_cells", [0.0, 1.0, np.sqrt(3.0), 4.0])
def test_cell_green_3d_matches_ball_quadrature(k, h, r_cells):
    a = green.equivalent_radius(h, 3)
    r = r_cells * h
    ref = _ball_integral(k, a, r)
    got = green.green_cell(k, np.array([r]), h, 3)[0]
    assert abs(got - ref) <= 1e-8 * abs(ref)


def test_equivalent_radius_preserves_cell_measure():
    h = 0.3
    assert np.isclose(np.pi * green.equivalent_radius(h, 2) ** 2, h * h)
    assert np.isclose(4.0 / 3.0 * np.pi * green.equivalent_radius(h, 3) ** 3,
                      h ** 3)


def test_point_green_is_outgoing_for_exp_minus_i_omega_t():
    """Large kr: (i/4) H0^(1)(kr) -> (i/4) sqrt(2/(pi kr)) e^{i(kr - pi/4)},
    an outgoing wave under e^{-i omega t}; 3D is e^{ikr}/(4 pi r)."""
    k = 2 * np.pi * 3e6 / 1540.0
    r = np.array([0.02, 0.03, 0.05])
    asym = 0.25j * np.sqrt(2.0 / (np.pi * k * r)) * np.exp(1j * (k * r - np.pi / 4))
    g = green.green_point(k, r, 2)
    assert np.all(np.abs(g - asym) <= 2e-3 * np.abs(asym))
    g3 = green.green_point(k, r, 3)
    assert np.allclose(g3 * 4 * np.pi * r, np.exp(1j * k * r), rtol=1e-14)


@pytest.mark.parametrize("dim", [2, 3])
def test_point_green_solves_helmholtz_away_from_source(dim):
    """(lap + k^2) G = 0 at r > 0, checked with a 4th-order finite-difference
    Laplacian in Cartesian coordinates."""
    k = 2 * np.pi * 1e6 / 1540.0
    x0 = np.array([1.3e-3, 0.7e-3, 0.9e-3][:dim])
    step = 2e-6

    def G(x):
        return green.green_point(k, np.array([np.linalg.norm(x)]), dim)[0]
    lap = 0.0
    for q in range(dim):
        e = np.zeros(dim)
        e[q] = step
        lap += (-G(x0 + 2 * e) + 16 * G(x0 + e) - 30 * G(x0)
                + 16 * G(x0 - e) - G(x0 - 2 * e)) / (12 * step * step)
    resid = lap + k * k * G(x0)
    assert abs(resid) <= 1e-6 * abs(k * k * G(x0))


def test_lattice_layout_wraps_offsets():
    shape, h, k = (3, 4), 1e-4, 5000.0
    lat = green.green_lattice(shape, h, k)
    assert lat.shape == (6, 8)
    # offset (dz, dx) = (-1, +2) is stored at (6-1, 2)
    r = np.hypot(1.0, 2.0) * h
    assert np.isclose(lat[5, 2], green.green_cell(k, np.array([r]), h, 2)[0])
    # the never-used half-period offsets are zero
    assert np.all(lat[3, :] == 0) and np.all(lat[:, 4] == 0)

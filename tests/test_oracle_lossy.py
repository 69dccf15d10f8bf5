"""Pins of the oracle's attenuating background (Eq. 1-3 with a complex
background compressibility, Sec. II): the complex wavenumber, the Green's
functions at complex k (Helmholtz equation, decay, the closed-form cell
integrals against quadrature over the disc / ball), the contrast <-> SoS and
attenuation maps, the gradient against finite differences in a lossy
medium, and the whole solve against the Bessel series of a lossy cylinder."""
import numpy as np
import pytest

import oracle
from oracle import green, inverse, model, operator
from paper_2604_15796_gb300 import phantoms
from test_oracle_green import _ball_integral, _disc_integral

C0 = 1540.0
ALPHA_TISSUE = 0.5 / 8.686 * 100.0 / 1e6  # 0.5 dB/cm/MHz in Np/m/Hz (the paper's background)
ALPHA_STRONG = 5e-4                        # Im k ~ 0.12 Re k: the complex terms matter


def prob2d(alpha0, freqs=(1.5e6, 3e6), shape=(10, 12), n_elem=4):
    p = oracle.Problem(shape, 0.1e-3, C0, model.linear_array(n_elem, 0.2e-3, 0.1e-3, len(shape)),
                       np.array(freqs))
    p.extra["alpha0"] = alpha0
    return p


def test_wavenumber_of_a_lossy_background():
    p = prob2d(ALPHA_TISSUE)
    k = model.wavenumbers(p)
    w = 2 * np.pi * p.freqs
    assert np.allclose(k * k, w * w * (1 / C0 ** 2 + 1j * ALPHA_TISSUE / (np.pi * C0)),
                       rtol=1e-14)
    assert np.all(k.imag > 0) and np.all(k.real > 0)
    # first order: Im k = alpha0 f (the attenuation in Np/m), Re k = omega / c0
    assert np.allclose(k.imag, ALPHA_TISSUE * p.freqs, rtol=2e-3)
    assert np.allclose(k.real, w / C0, rtol=1e-5)
    p.extra["alpha0"] = 0.0
    assert np.isrealobj(model.wavenumbers(p))


@pytest.mark.parametrize("dim", [2, 3])
def test_complex_k_green_solves_helmholtz_and_decays(dim):
    k = (2 * np.pi * 1e6 / C0) * np.sqrt(1 + 0.1j)
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
    assert abs(lap + k * k * G(x0)) <= 1e-6 * abs(k * k * G(x0))
    if dim == 2:
        r = np.array([0.02, 0.04])
        asym = 0.25j * np.sqrt(2.0 / (np.pi * k * r)) * np.exp(1j * (k * r - np.pi / 4))
        assert np.all(np.abs(green.green_point(k, r, 2) - asym) <= 2e-3 * np.abs(asym))


@pytest.mark.parametrize("r_cells", [0.0, 1.0, 3.0])
def test_complex_k_cell_green_matches_quadrature(r_cells):
    """The closed-form cell integrals (disc / ball, the self cell included)
    hold at complex k: against quadrature of G over the cell."""
    h = 0.1e-3
    k = (2 * np.pi * 3e6 / C0) * np.sqrt(1 + 1j * ALPHA_STRONG * C0 / np.pi)
    assert k.imag > 0.1 * k.real
    r = r_cells * h
    ref2 = _disc_integral(k, green.equivalent_radius(h, 2), r)
    assert abs(green.green_cell(k, np.array([r]), h, 2)[0] - ref2) <= 1e-8 * abs(ref2)
    ref3 = _ball_integral(k, green.equivalent_radius(h, 3), r)
    assert abs(green.green_cell(k, np.array([r]), h, 3)[0] - ref3) <= 1e-8 * abs(ref3)


def test_contrast_maps_of_a_lossy_background():
    c = np.array([1480.0, 1540.0, 1600.0, 1520.0])
    alpha = np.array([1e-5, ALPHA_TISSUE, 2e-5, 0.0])
    m = model.contrast_from_sos(c, C0, alpha, ALPHA_TISSUE)
    assert abs(m[1]) < 1e-15                        # the background has no contrast
    assert np.allclose(model.sos_from_contrast(m, C0, ALPHA_TISSUE), c, rtol=1e-12)
    assert np.allclose(model.attenuation_from_contrast(m, C0, ALPHA_TISSUE), alpha,
                       rtol=1e-9, atol=1e-16)
    # no attenuation map: pixels carry the background's attenuation
    m_sos = model.contrast_from_sos(c, C0, None, ALPHA_TISSUE)
    assert np.allclose(model.attenuation_from_contrast(m_sos, C0, ALPHA_TISSUE), ALPHA_TISSUE,
                       rtol=1e-9)
    # lossless background: the earlier formulas
    m0 = model.contrast_from_sos(c, C0, alpha)
    assert np.allclose(m0, C0 ** 2 / c ** 2 - 1 + 1j * alpha * C0 ** 2 / (np.pi * c), rtol=1e-14)
    assert np.allclose(model.attenuation_from_contrast(m0, C0), alpha, rtol=1e-9, atol=1e-16)


def test_lossy_gradient_and_reciprocity():
    p = prob2d(ALPHA_STRONG, freqs=(2e6,))
    rng = np.random.default_rng(4)
    m = 0.05 * (rng.standard_normal(p.shape) + 0.1j * rng.standard_normal(p.shape))
    _, d = inverse.forward_model(1.3 * m, p, "lu")
    assert np.allclose(d[0], d[0].T, rtol=1e-10, atol=1e-14 * np.abs(d).max())
    ref = inverse.gradient(m, d, p, "lu")
    a = phantoms.complex_normal(p.shape, 5)
    eps = 1e-6

    def phi(mm):
        return inverse.misfit(inverse.forward_model(mm, p, "lu")[1], d)

    fd = (phi(m + eps * a) - phi(m - eps * a)) / (2 * eps)
    assert np.isclose(fd, np.vdot(ref["grad"], a.ravel()).real, rtol=1e-6)
    # and the loss matters
    p.extra["alpha0"] = 0.0
    _, d0 = inverse.forward_model(1.3 * m, p, "lu")
    assert not np.allclose(d, d0, rtol=1e-2)


def test_lossy_cylinder_converges_to_bessel_series():
    """The whole lossy solve against an analytic solution: a cylinder with its
    own speed and attenuation in an attenuating background, the Bessel-series
    field with both wavenumbers complex (the addition theorem and the
    interface conditions hold unchanged for Im k > 0).  The wavenumbers are
    computed here from the two media, k^2 = omega^2 (1/c^2 + i alpha/(pi c)),
    and the contrast is k1^2/k0^2 - 1; the VIE data converge to the series as
    the pixel shrinks, and the lossless series is far from them."""
    from test_oracle_operator import _cylinder_field
    c0, a0, c1, a1, f = C0, 2e-4, 1480.0, 4e-4, 1.0e6
    w = 2 * np.pi * f
    k0 = w * np.sqrt(1 / c0 ** 2 + 1j * a0 / (np.pi * c0))
    k1 = w * np.sqrt(1 / c1 ** 2 + 1j * a1 / (np.pi * c1))
    assert k0.imag > 0.04 * k0.real and k1.imag > 0.08 * k1.real
    R, width = 1.2e-3, 4.8e-3
    errs = []
    for npx in (48, 96, 192):
        h = width / npx
        elem = np.array([[-1.0e-3, -h], [0.0, -h], [1.3e-3, -h]])
        prob = oracle.Problem((npx, npx), h, c0, elem, np.array([f]))
        prob.extra["alpha0"] = a0
        x = model.pixel_centres(prob.shape, h)
        centre = np.array([0.0, width / 2.0])
        inside = np.hypot(x[:, 0] - centre[0], x[:, 1] - centre[1]) < R
        m = np.where(inside, k1 * k1 / (k0 * k0) - 1.0, 0.0).astype(np.complex128)
        fields = operator.solve_forward(m.reshape(prob.shape), prob, "bicgstab", tol=1e-11)
        data = inverse.forward_data(m, fields, prob)[0]
        ref = np.empty_like(data)
        lossless = np.empty_like(data)
        for e in range(3):
            ref[e] = _cylinder_field(k0, k1, R, elem[e] - centre, elem - centre)[1]
            lossless[e] = _cylinder_field(k0.real, k1.real, R, elem[e] - centre,
                                          elem - centre)[1]
        errs.append(np.linalg.norm(data - ref) / np.linalg.norm(ref))
    assert errs[0] > errs[1] > errs[2] and errs[2] < 0.5 * errs[1]
    assert errs[2] < 0.05, errs
    assert np.linalg.norm(data - lossless) > 5 * errs[2] * np.linalg.norm(ref)

"""Pins of the oracle's Lippmann-Schwinger operator and field solves
(Eq. 5, Sec. IV-A): the FFT convolution against the O(N^2) sum of its
definition, a single-pixel scatterer whose discrete solution has a closed
form (with the self term taken from quadrature, not from the oracle), dense
LU against two Krylov methods, the homogeneous medium, and convergence to
the Bessel-series solution of a penetrable cylinder and to the
spherical-Bessel series of a penetrable sphere (lossless and lossy) as
h -> 0."""
import numpy as np
import pytest
import scipy.sparse.linalg as spla
from scipy import integrate, special

import oracle
from oracle import green, model, operator, inverse


def small_problem(shape=(12, 10), h=1e-4, f=2e6, n_elem=4, pitch=2e-4):
    dim = len(shape)
    return oracle.Problem(shape, h, 1540.0,
                          model.linear_array(n_elem, pitch, h, dim),
                          np.array([f]))


@pytest.mark.parametrize("shape", [(12, 10), (7, 9), (4, 5, 6), (6, 3, 5)])
def test_fft_convolution_equals_direct_sum(shape):
    prob = small_problem(shape, h=1e-4, f=2.5e6)
    rng = np.random.default_rng(3)
    w = rng.standard_normal((2,) + shape) + 1j * rng.standard_normal((2,) + shape)
    a = operator.apply_K(w, prob, 0)
    b = operator.apply_K_direct(w, prob, 0)
    assert np.linalg.norm(a - b) <= 1e-12 * np.linalg.norm(b)


def _disc_self_term(k, h):
    a = h / np.sqrt(np.pi)
    f = lambda rho: 0.25j * special.hankel1(0, k * rho) * rho  # noqa: E731
    kw = dict(limit=400, epsabs=0.0, epsrel=1e-13)
    re = integrate.quad(lambda t: np.real(f(t)), 0.0, a, **kw)[0]
    im = integrate.quad(lambda t: np.imag(f(t)), 0.0, a, **kw)[0]
    return 2.0 * np.pi * (re + 1j * im)


def test_single_pixel_scatterer_closed_form():
    """m = mu at one pixel s: p(x_s) = p0(x_s) / (1 - k^2 Ghat(0) mu) and
    P^s_{e,j} = k^2 dV G(x_j, x_s) mu p_e(x_s); Ghat(0) by quadrature."""
    prob = small_problem((10, 8), h=1e-4, f=3e6, n_elem=3, pitch=3e-4)
    k = model.wavenumbers(prob)[0]
    s = (4, 5)
    mu = 0.07 - 0.01j
    m = np.zeros(prob.shape, dtype=np.complex128)
    m[s] = mu
    fields, data = inverse.forward_model(m, prob, "lu")
    p0 = operator.incident_fields(prob)
    g0 = _disc_self_term(k, prob.h)
    ps = p0[0, :, s[0], s[1]] / (1.0 - k * k * g0 * mu)
    assert np.allclose(fields[0, :, s[0], s[1]], ps, rtol=1e-9, atol=0)
    xs = model.pixel_centres(prob.shape, prob.h)[s[0] * prob.shape[1] + s[1]]
    rj = np.linalg.norm(prob.elem - xs[None, :], axis=1)
    gj = 0.25j * special.hankel1(0, k * rj)
    ref = (k * k * prob.h ** 2) * gj[None, :] * mu * ps[:, None]
    assert np.allclose(data[0], ref, rtol=1e-9, atol=0)


def test_homogeneous_medium_gives_incident_field_and_no_data():
    prob = small_problem((8, 8))
    m = np.zeros(prob.shape, dtype=np.complex128)
    fields, data = inverse.forward_model(m, prob, "lu")
    x = model.pixel_centres(prob.shape, prob.h)
    k = model.wavenumbers(prob)[0]
    r = np.linalg.norm(x[None] - prob.elem[:, None], axis=2)
    analytic = 0.25j * special.hankel1(0, k * r)
    assert np.allclose(fields[0].reshape(prob.n_elem, -1), analytic,
                       rtol=1e-14, atol=0)
    assert np.all(data == 0)


def test_lu_bicgstab_gmres_agree():
    prob = small_problem((24, 20), h=1e-4, f=3e6, n_elem=3, pitch=4e-4)
    rng = np.random.default_rng(5)
    m = (0.05 * rng.standard_normal(prob.shape)).astype(np.complex128)
    p0 = operator.incident_fields(prob)[0]
    lu, _ = operator.solve(m, p0, prob, 0, "lu")
    it, info = operator.solve(m, p0, prob, 0, "bicgstab", tol=1e-12)
    assert np.linalg.norm(lu - it) <= 1e-10 * np.linalg.norm(lu)
    assert all(res <= 1e-12 for _, res in info)
    spec = operator.kernel_spectrum(prob, 0)
    A = spla.LinearOperator(
        (prob.n, prob.n), dtype=np.complex128,
        matvec=lambda v: operator.apply_A(v.reshape(prob.shape), m, prob, 0,
                                          spec).ravel())
    xg, flag = spla.gmres(A, p0[1].ravel(), rtol=1e-13, restart=200, maxiter=50)
    assert flag == 0
    assert np.linalg.norm(xg - lu[1].ravel()) <= 1e-10 * np.linalg.norm(lu[1])


def test_3d_solve_agrees_with_lu():
    prob = small_problem((5, 4, 6), h=0.2e-3, f=1.5e6, n_elem=3, pitch=0.3e-3)
    rng = np.random.default_rng(6)
    m = (0.04 * rng.standard_normal(prob.shape)).astype(np.complex128)
    p0 = operator.incident_fields(prob)[0]
    lu, _ = operator.solve(m, p0, prob, 0, "lu")
    it, _ = operator.solve(m, p0, prob, 0, "bicgstab", tol=1e-12)
    assert np.linalg.norm(lu - it) <= 1e-10 * np.linalg.norm(lu)


def _cylinder_field(k0, k1, R, xs, pts, n_terms=60):
    """Total field of a unit line source (i/4) H0(k0|x - xs|) scattered by a
    homogeneous cylinder of radius R centred at the origin (wavenumber k1
    inside), by the Bessel-series solution with continuity of the field and
    of its normal derivative at rho = R.  Returns (total, scattered)."""
    rs, ps = np.hypot(*xs), np.arctan2(xs[1], xs[0])
    rho = np.hypot(pts[:, 0], pts[:, 1])
    phi = np.arctan2(pts[:, 1], pts[:, 0])
    n = np.arange(-n_terms, n_terms + 1)
    c = 0.25j * special.hankel1(n, k0 * rs)
    J0R, J0Rp = special.jv(n, k0 * R), special.jvp(n, k0 * R)
    J1R, J1Rp = special.jv(n, k1 * R), special.jvp(n, k1 * R)
    H0R, H0Rp = special.hankel1(n, k0 * R), special.h1vp(n, k0 * R)
    den = k0 * J1R * H0Rp - k1 * J1Rp * H0R
    a = c * (k1 * J1Rp * J0R - k0 * J1R * J0Rp) / den
    b = (c * J0R + a * H0R) / J1R
    e = np.exp(1j * np.outer(phi - ps, n))
    inside = rho < R
    sc = np.zeros(len(pts), dtype=np.complex128)
    tot = np.zeros(len(pts), dtype=np.complex128)
    out = ~inside
    sc[out] = (e[out] * a[None] * special.hankel1(n[None], k0 * rho[out, None])).sum(1)
    dist = np.hypot(pts[:, 0] - xs[0], pts[:, 1] - xs[1])
    tot[out] = 0.25j * special.hankel1(0, k0 * dist[out]) + sc[out]
    tot[inside] = (e[inside] * b[None] * special.jv(n[None], k1 * rho[inside, None])).sum(1)
    return tot, sc


def test_penetrable_cylinder_converges_to_bessel_series():
    """Physics of the discretisation (not parity): the VIE data converge to
    the analytic scattered field of a cylinder as the pixel shrinks."""
    c0, c1, f = 1540.0, 1480.0, 1.0e6
    k0 = 2 * np.pi * f / c0
    k1 = 2 * np.pi * f / c1
    R, width = 1.2e-3, 4.8e-3
    errs = []
    for npx in (48, 96, 192):
        h = width / npx
        elem = np.array([[-1.0e-3, -h], [0.0, -h], [1.3e-3, -h]])
        prob = oracle.Problem((npx, npx), h, c0, elem, np.array([f]))
        x = model.pixel_centres(prob.shape, h)
        centre = np.array([0.0, width / 2.0])
        inside = np.hypot(x[:, 0] - centre[0], x[:, 1] - centre[1]) < R
        m = np.where(inside, c0 ** 2 / c1 ** 2 - 1.0, 0.0).astype(np.complex128)
        fields = operator.solve_forward(m.reshape(prob.shape), prob,
                                        "bicgstab", tol=1e-11)
        data = inverse.forward_data(m, fields, prob)[0]
        ref = np.empty_like(data)
        for e in range(3):
            _, sc = _cylinder_field(k0, k1, R, elem[e] - centre, elem - centre)
            ref[e] = sc
        errs.append(np.linalg.norm(data - ref) / np.linalg.norm(ref))
    assert errs[0] > errs[1] > errs[2]
    assert errs[2] < 0.05, errs


def _sphere_field(k0, k1, R, xs, pts, n_terms=40):
    """Scattered field of a unit point source exp(ik0 r)/(4 pi r) at xs by a
    homogeneous sphere of radius R centred at the origin (wavenumber k1
    inside): the spherical-Bessel series with continuity of the field and of
    its radial derivative at r = R, using
    exp(ik|x - xs|)/(4 pi |x - xs|) = (ik/4pi) sum (2n+1) j_n(kr) h_n(k rs) P_n(cos g)
    for r < rs.  Also returns that expansion of the incident field (a check of
    the helper against the closed form)."""
    rs, r = np.linalg.norm(xs), np.linalg.norm(pts, axis=1)
    cosg = (pts @ xs) / (r * rs)
    n = np.arange(n_terms + 1)
    jn, yn = special.spherical_jn, special.spherical_yn

    def hn(nn, z, d=False):
        return jn(nn, z, d) + 1j * yn(nn, z, d)
    c = hn(n, k0 * rs)
    j0, j0p = jn(n, k0 * R), jn(n, k0 * R, True)
    j1, j1p = jn(n, k1 * R), jn(n, k1 * R, True)
    h0, h0p = hn(n, k0 * R), hn(n, k0 * R, True)
    a = c * (k1 * j1p * j0 - k0 * j1 * j0p) / (k0 * j1 * h0p - k1 * j1p * h0)
    P = np.stack([special.eval_legendre(q, cosg) for q in n], axis=1)
    w = (1j * k0 / (4 * np.pi)) * (2 * n + 1)[None] * P
    sc = (w * a[None] * hn(n[None], k0 * r[:, None])).sum(1)
    inc = (w * c[None] * jn(n[None], k0 * r[:, None])).sum(1)
    return sc, inc


@pytest.mark.parametrize("lossy", [False, True])
def test_penetrable_sphere_converges_to_spherical_bessel_series(lossy):
    """3-D counterpart of the cylinder: the VIE data of a sphere converge to
    the series as the voxel shrinks, in a lossless and in an attenuating
    background (wavenumbers computed here from the two media,
    k^2 = omega^2 (1/c^2 + i alpha/(pi c)), contrast k1^2/k0^2 - 1)."""
    c0, c1, f = 1540.0, 1480.0, 1.0e6
    a0, a1 = (2e-4, 4e-4) if lossy else (0.0, 0.0)
    w = 2 * np.pi * f
    k0 = w * np.sqrt(1 / c0 ** 2 + 1j * a0 / (np.pi * c0))
    k1 = w * np.sqrt(1 / c1 ** 2 + 1j * a1 / (np.pi * c1))
    if not lossy:
        k0, k1 = k0.real, k1.real
    R, width = 0.9e-3, 3.2e-3
    centre = np.array([0.0, 0.0, width / 2.0])
    # the helper's incident expansion is the closed-form Green's function
    xs = np.array([-0.8e-3, 0.0, -0.05e-3]) - centre
    pts = np.array([[0.3e-3, 0.2e-3, 0.1e-3], [-0.5e-3, 0.4e-3, -0.6e-3]])
    _, inc = _sphere_field(k0, k1, R, xs, pts)
    dist = np.linalg.norm(pts - xs, axis=1)
    assert np.allclose(inc, np.exp(1j * k0 * dist) / (4 * np.pi * dist), rtol=1e-10)
    errs = []
    for npx in (32, 48, 64):
        h = width / npx
        elem = np.array([[-0.8e-3, 0.0, -h], [0.0, 0.3e-3, -h], [0.9e-3, -0.2e-3, -h]])
        prob = oracle.Problem((npx, npx, npx), h, c0, elem, np.array([f]))
        prob.extra["alpha0"] = a0
        x = model.pixel_centres(prob.shape, h)
        inside = np.linalg.norm(x - centre, axis=1) < R
        m = np.where(inside, k1 * k1 / (k0 * k0) - 1.0, 0.0).astype(np.complex128)
        fields = operator.solve_forward(m.reshape(prob.shape), prob, "bicgstab", tol=1e-11)
        data = inverse.forward_data(m, fields, prob)[0]
        ref = np.array([_sphere_field(k0, k1, R, elem[e] - centre, elem - centre)[0]
                        for e in range(3)])
        errs.append(np.linalg.norm(data - ref) / np.linalg.norm(ref))
    assert errs[0] > errs[1] > errs[2], errs
    assert errs[2] < 0.04, errs

"""Lippmann-Schwinger forward operator and field solves (Eq. 5, Sec. IV-A).
FP64 oracle; test infrastructure only.

Discretised Eq. 5 (pixel collocation, cell-integrated kernel, see green.py):

    p_n = p0_n + k^2 sum_n' Ghat(x_n - x_n') m_n' p_n'     i.e.  A p = p0,
    A = I - K diag(m),   (K w)_n = k^2 sum_n' Ghat(x_n - x_n') w_n'.

K is a convolution with a translation-invariant kernel (Sec. IV-A); it is
evaluated either directly (O(N^2), small grids) or as a circular convolution
on the doubled lattice with zero padding and cropping.
"""
import numpy as np
import scipy.fft as sfft
import scipy.linalg as sla
from scipy.integrate import quad_vec

from . import green, model

FFT_WORKERS = -1


def kernel_spectrum(prob, l):
    """FFT of the doubled-lattice kernel for frequency l (times k_l^2)."""
    k = model.wavenumbers(prob)[l]
    lat = green.green_lattice(prob.shape, prob.h, k)
    return (k * k) * sfft.fftn(lat, workers=FFT_WORKERS)


def apply_K(w, prob, l, spec=None):
    """K w by zero-padded FFT convolution.  ``w`` has shape (..., *shape)."""
    if spec is None:
        spec = kernel_spectrum(prob, l)
    d = prob.dim
    w = np.asarray(w, dtype=np.complex128)
    axes = tuple(range(w.ndim - d, w.ndim))
    padded = np.zeros(w.shape[:w.ndim - d] + tuple(2 * s for s in prob.shape),
                      dtype=np.complex128)
    padded[(Ellipsis,) + tuple(slice(0, s) for s in prob.shape)] = w
    out = sfft.ifftn(sfft.fftn(padded, axes=axes, workers=FFT_WORKERS) * spec,
                     axes=axes, workers=FFT_WORKERS)
    return out[(Ellipsis,) + tuple(slice(0, s) for s in prob.shape)]


def apply_A(v, m, prob, l, spec=None):
    """A v = v - K(m v)."""
    m = np.asarray(m, dtype=np.complex128).reshape(prob.shape)
    return v - apply_K(m * v, prob, l, spec)


def dense_K(prob, l):
    """The N x N matrix of K (direct evaluation, small grids only)."""
    k = model.wavenumbers(prob)[l]
    x = model.pixel_centres(prob.shape, prob.h)
    r = np.sqrt(((x[:, None, :] - x[None, :, :]) ** 2).sum(-1))
    return (k * k) * green.green_cell(k, r, prob.h, prob.dim)


def apply_K_direct(w, prob, l):
    """K w by the O(N^2) sum of its definition."""
    w = np.asarray(w, dtype=np.complex128)
    flat = w.reshape(w.shape[:w.ndim - prob.dim] + (prob.n,))
    out = flat @ dense_K(prob, l).T
    return out.reshape(w.shape)


def dense_A(m, prob, l):
    m = np.asarray(m, dtype=np.complex128).ravel()
    return np.eye(prob.n, dtype=np.complex128) - dense_K(prob, l) * m[None, :]


def element_green(prob):
    """Green's function of each element seen from every pixel,
    [N_F, N_E, *shape].

    Point elements: G_l(x_n, x_e).  3-D line elements (Sec. V-B: elements of
    finite elevation, prob.extra["elem_length"] = L > 0 along y, centred on
    the element position): the mean over the element,
        (1 / L) int_{-L/2}^{L/2} G_l(x_n, x_e + s e_y) ds,
    by adaptive quadrature over s (all pixels at once).  Reading: the mean
    (not the integral) keeps the point element as the limit L -> 0; the same
    mean is the transmit field and the receiver's sensing (Eq. 4's integral
    over Omega_j up to the factor L, which the paper leaves open)."""
    x = model.pixel_centres(prob.shape, prob.h)
    length = float(prob.extra.get("elem_length", 0.0))
    out = np.empty((prob.n_freq, prob.n_elem) + tuple(prob.shape), dtype=np.complex128)
    k = model.wavenumbers(prob)
    if prob.dim == 3 and length > 0:
        for e in range(prob.n_elem):
            d0 = x - prob.elem[e][None, :]

            def g(s, d0=d0):
                r = np.sqrt(d0[:, 0] ** 2 + (d0[:, 1] - s) ** 2 + d0[:, 2] ** 2)
                return np.stack([green.green_point(kl, r, 3) for kl in k])

            val, _ = quad_vec(g, -0.5 * length, 0.5 * length, epsabs=0.0, epsrel=1e-12,
                              norm="max", limit=4000)
            out[:, e] = (val / length).reshape((prob.n_freq,) + tuple(prob.shape))
        return out
    r = np.sqrt(((x[None, :, :] - prob.elem[:, None, :]) ** 2).sum(-1))
    for l, kl in enumerate(k):
        out[l] = green.green_point(kl, r, prob.dim).reshape((prob.n_elem,) + tuple(prob.shape))
    return out


def incident_fields(prob):
    """p0_{e,l} = the element's Green's function (element_green): a unit
    source at each element (reading: the paper fixes no source
    normalisation).  [N_F, N_E, *shape]."""
    return element_green(prob)


def transmit_incident_fields(prob, weights):
    """Incident fields of synthesised transmits (Sec. V-A): the elements'
    point sources superposed with the weights w_{l,i,e},
    p0_{l,i} = sum_e w_{l,i,e} G_l(., x_e).  [N_F, N_T, *shape]."""
    p0 = incident_fields(prob)
    flat = p0.reshape(prob.n_freq, prob.n_elem, prob.n)
    out = np.einsum("lie,len->lin", np.asarray(weights, dtype=np.complex128), flat)
    return out.reshape((prob.n_freq, out.shape[1]) + tuple(prob.shape))


def bicgstab(apply, b, tol=1e-10, maxit=2000, x0=None):
    """Textbook BiCGSTAB (van der Vorst, 1992) for one right-hand side.

    Stops when ||b - A x|| <= tol ||b|| (recursive residual).  Returns
    (x, iterations, relative residual).  Inner products <a, b> = sum conj(a) b.
    """
    b = np.asarray(b, dtype=np.complex128)
    x = np.zeros_like(b) if x0 is None else np.array(x0, dtype=np.complex128)
    r = b - apply(x) if x0 is not None else b.copy()
    bnorm = np.linalg.norm(b)
    if bnorm == 0.0:
        return np.zeros_like(b), 0, 0.0
    rhat = r.copy()
    rho_old = alpha = omega = 1.0 + 0j
    v = np.zeros_like(b)
    p = np.zeros_like(b)
    it = 0
    res = np.linalg.norm(r) / bnorm
    while res > tol and it < maxit:
        rho = np.vdot(rhat, r)
        beta = (rho / rho_old) * (alpha / omega)
        p = r + beta * (p - omega * v)
        v = apply(p)
        alpha = rho / np.vdot(rhat, v)
        s = r - alpha * v
        t = apply(s)
        tt = np.vdot(t, t).real
        omega = np.vdot(t, s) / tt if tt > 0 else 0.0
        x = x + alpha * p + omega * s
        r = s - omega * t
        rho_old = rho
        it += 1
        res = np.linalg.norm(r) / bnorm
    return x, it, res


def solve(m, rhs, prob, l, method="lu", tol=1e-10, maxit=2000):
    """Solve A p = rhs for a stack of right-hand sides [B, *shape] at
    frequency l.  ``method``: 'lu' (dense LU, small N) or 'bicgstab'."""
    rhs = np.asarray(rhs, dtype=np.complex128)
    nb = rhs.shape[0]
    if method == "lu":
        sol = sla.solve(dense_A(m, prob, l), rhs.reshape(nb, prob.n).T)
        return sol.T.reshape(rhs.shape), None
    spec = kernel_spectrum(prob, l)
    mm = np.asarray(m, dtype=np.complex128).reshape(prob.shape)

    def apply(v):
        return apply_A(v.reshape(prob.shape), mm, prob, l, spec).ravel()

    out = np.empty_like(rhs)
    info = []
    for i in range(nb):
        x, it, res = bicgstab(apply, rhs[i].ravel(), tol, maxit)
        out[i] = x.reshape(prob.shape)
        info.append((it, res))
    return out, info


def solve_forward(m, prob, method="lu", tol=1e-10, p0=None):
    """Total fields p_{e,l} = A_l^{-1} p0_{e,l} (Eq. 5).  [N_F, N_E, *shape]."""
    if p0 is None:
        p0 = incident_fields(prob)
    out = np.empty_like(p0)
    for l in range(prob.n_freq):
        out[l], _ = solve(m, p0[l], prob, l, method, tol)
    return out

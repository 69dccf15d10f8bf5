"""Problem geometry and medium model (Sec. II, Eq. 1-3).  FP64 oracle; test
infrastructure only.

Conventions (readings of points the paper leaves open):

* Time dependence e^{-i omega t}: every complex quantity is the complex
  conjugate of the paper's e^{+j omega t} form; attenuation therefore
  enters the compressibility as +i kappa''.  Speed of sound is unaffected.
* Arrays are stored depth-major: shape (Nz, Nx) in 2D, (Nz, Ny, Nx) in 3D,
  x fastest.  Pixel n has centre x = (ix + 1/2 - Nx/2) h,
  y = (iy + 1/2 - Ny/2) h, z = iz h (depth increases downward).
* The linear array sits one pixel above the first row of centres, at
  z = -h, centred laterally: element e at x = (e - (N_E - 1)/2) pitch,
  y = 0.  This places the sensing elements on the edge of V (Eq. 4) while
  keeping every source-pixel distance >= h.
"""
from dataclasses import dataclass, field

import numpy as np


@dataclass
class Problem:
    """One reconstruction problem.

    shape  : grid shape in array order, (Nz, Nx) or (Nz, Ny, Nx)
    h      : pixel / voxel edge [m]
    c0     : background speed of sound [m/s] (lossless background)
    elem   : element positions [N_E, d] in (x, z) or (x, y, z) order [m]
    freqs  : frequencies [N_F] in Hz
    Transmitters and receivers are the same N_E elements (each element
    transmits in turn, all receive), so N_T = N_R = N_E.
    """
    shape: tuple
    h: float
    c0: float
    elem: np.ndarray
    freqs: np.ndarray
    extra: dict = field(default_factory=dict)

    @property
    def dim(self):
        return len(self.shape)

    @property
    def n(self):
        return int(np.prod(self.shape))

    @property
    def n_elem(self):
        return int(self.elem.shape[0])

    @property
    def n_freq(self):
        return int(len(self.freqs))

    @property
    def cell_volume(self):
        return self.h ** self.dim


def linear_array(n_elem, pitch, h, dim):
    """Element positions of a top-edge linear array (reading above)."""
    xe = (np.arange(n_elem, dtype=np.float64) - (n_elem - 1) / 2.0) * pitch
    if dim == 2:
        return np.stack([xe, np.full(n_elem, -h)], axis=1)
    return np.stack([xe, np.zeros(n_elem), np.full(n_elem, -h)], axis=1)


def pixel_centres(shape, h):
    """Centres of all pixels, [N, d] in (x, [y], z) order, row-major over
    ``shape`` (x fastest)."""
    if len(shape) == 2:
        nz, nx = shape
        z, x = np.meshgrid(np.arange(nz), np.arange(nx), indexing="ij")
        return np.stack([((x + 0.5 - nx / 2.0) * h).ravel(),
                         (z * h).ravel().astype(np.float64)], axis=1)
    nz, ny, nx = shape
    z, y, x = np.meshgrid(np.arange(nz), np.arange(ny), np.arange(nx),
                          indexing="ij")
    return np.stack([((x + 0.5 - nx / 2.0) * h).ravel(),
                     ((y + 0.5 - ny / 2.0) * h).ravel(),
                     (z * h).ravel().astype(np.float64)], axis=1)


def background_alpha(prob):
    """Attenuation of the background alpha0 [Np/m/Hz] (prob.extra["alpha0"],
    default 0: lossless)."""
    return float(prob.extra.get("alpha0", 0.0))


def wavenumbers(prob):
    """k_l^2 = omega_l^2 kappa0 rho0 (Sec. II) with the background's
    compressibility kappa0 = 1/(c0^2 rho0) + i alpha0/(pi c0 rho0) (Eq. 1-2
    under e^{-i omega t}): k_l = omega_l sqrt(1/c0^2 + i alpha0/(pi c0)),
    the root with Im k > 0 (outgoing waves decay; Im k ~ alpha0 f).  Real,
    omega_l / c0, for a lossless background."""
    w = 2.0 * np.pi * np.asarray(prob.freqs, dtype=np.float64)
    a0 = background_alpha(prob)
    if a0 == 0.0:
        return w / prob.c0
    return w * np.sqrt(1.0 / prob.c0 ** 2 + 1j * a0 / (np.pi * prob.c0))


def _kappa(c, alpha):
    """rho0 kappa = 1/c^2 + i alpha/(pi c) (Eq. 1-2, the alpha^2 term dropped
    as the approximation of Eq. 2 does)."""
    return 1.0 / (c * c) + 1j * alpha / (np.pi * c)


def contrast_from_sos(c, c0, alpha=None, alpha0=0.0):
    """Contrast m = kappa/kappa0 - 1 (Eq. 3).

    kappa' = 1/(c^2 rho0), kappa'' = alpha/(pi c rho0) with alpha in
    Np/m/Hz, and under e^{-i omega t} kappa = kappa' + i kappa''.  rho0
    cancels in the ratio.  With a lossy background (alpha0 > 0) kappa0 is
    complex too, and a pixel without an attenuation value (alpha None) takes
    the background's, so that the background has m = 0.
    """
    c = np.asarray(c, dtype=np.float64)
    if alpha0 == 0.0:
        m = (c0 * c0) / (c * c) - 1.0
        if alpha is None:
            return m.astype(np.complex128)
        return m + 1j * np.asarray(alpha, dtype=np.float64) * c0 * c0 / (np.pi * c)
    a = alpha0 if alpha is None else np.asarray(alpha, dtype=np.float64)
    return _kappa(c, a) / _kappa(c0, alpha0) - 1.0


def sos_from_contrast(m, c0, alpha0=0.0):
    """Speed of sound from the contrast, the inverse of Eq. 2-3:
    1/c^2 = Re(rho0 kappa0 (1 + m)); c = c0 / sqrt(1 + Re m) for a lossless
    background."""
    m = np.asarray(m)
    if alpha0 == 0.0:
        return c0 / np.sqrt(1.0 + np.real(m))
    return 1.0 / np.sqrt(np.real(_kappa(c0, alpha0) * (1.0 + m)))


def attenuation_from_contrast(m, c0, alpha0=0.0):
    """Attenuation alpha [Np/m/Hz] from the contrast (Eq. 1-3):
    alpha / (pi c) = Im(rho0 kappa0 (1 + m)), c from sos_from_contrast."""
    m = np.asarray(m)
    c = sos_from_contrast(m, c0, alpha0)
    return np.pi * c * np.imag(_kappa(c0, alpha0) * (1.0 + m))


def plane_wave_weights(prob, angles):
    """Element weights of steered plane-wave transmits (Sec. V-A: plane waves
    synthesised with the array's elements, steering angles spread over
    +-60 degrees).

    Reading: transmit i fires element e with the delay
    tau_{i,e} = x_e sin(theta_i) / c0, x_e the element's lateral position
    (the array is centred), so that the wavefront leaves the array in the
    direction (sin theta_i, cos theta_i) of the (x, z) plane, z pointing
    into the medium.  Under e^{-i omega t} a delay tau multiplies a source
    by exp(i omega tau), hence w_{l,i,e} = exp(i k_l x_e sin theta_i).
    Unit amplitude on every element (no apodisation).  [N_F, N_T, N_E]."""
    k = 2.0 * np.pi * np.asarray(prob.freqs, dtype=np.float64) / prob.c0  # delays: real
    xe = np.asarray(prob.elem, dtype=np.float64)[:, 0]
    s = np.sin(np.asarray(angles, dtype=np.float64))
    return np.exp(1j * k[:, None, None] * s[None, :, None] * xe[None, None, :])


def inversion_factor(prob):
    """r of the inversion mesh (prob.extra["inv_factor"], default 1)."""
    return int(prob.extra.get("inv_factor", 1))


def inversion_shape(prob):
    """Shape of the inversion mesh: every axis of the forward mesh / r."""
    r = inversion_factor(prob)
    return tuple(s // r for s in prob.shape)


def prolong(m_inv, prob):
    """Contrast on the forward mesh from its vector on the inversion mesh
    (Sec. IV: the forward mesh is finer than the inversion mesh).  Reading:
    each inversion cell covers r^d forward pixels (r = inversion_factor)
    and the contrast is constant over it."""
    r = inversion_factor(prob)
    m = np.asarray(m_inv).reshape(inversion_shape(prob))
    for ax in range(m.ndim):
        m = np.repeat(m, r, axis=ax)
    return m


def restrict(v, prob):
    """Adjoint of prolong: the sum over the forward pixels of each
    inversion cell (takes gradients and J^H products to the inversion
    mesh)."""
    r = inversion_factor(prob)
    blocks = []
    for s in inversion_shape(prob):
        blocks += [s, r]
    return np.asarray(v).reshape(blocks).sum(axis=tuple(range(1, 2 * len(prob.shape), 2)))


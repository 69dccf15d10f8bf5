"""Green's functions of the homogeneous background (Sec. II, Eq. 4-5).
FP64 oracle; test infrastructure only.

The paper states that G is analytically known and discretises Eq. 5 without
giving the quadrature (it cites the standard FFT-accelerated VIE solvers,
Sec. IV-A).  Reading taken here: pixel collocation, with the Green's function
integrated exactly over a disc (2D) or ball (3D) of the pixel's area or
volume centred on the source pixel.  Closed forms:

2D, G(r) = (i/4) H0^(1)(k r), disc radius a = h / sqrt(pi):
    Ghat(r > 0) = (i pi a / (2k)) J1(k a) H0^(1)(k r)
    Ghat(0)     = (i pi a / (2k)) H1^(1)(k a) - 1/k^2
3D, G(r) = e^{ikr} / (4 pi r), ball radius a = h (3/(4 pi))^(1/3):
    Ghat(r > 0) = (4 pi / k^3)(sin ka - ka cos ka) e^{ikr}/(4 pi r)
    Ghat(0)     = ((1 - i k a) e^{ika} - 1) / k^2
(The off-centre values follow from the Helmholtz mean-value theorem; the
centre values from integrating the radial singularity.)  These are pinned in
the tests against numerical quadrature of G over the disc / ball.
"""
import numpy as np
from scipy import special


def green_point(k, r, dim):
    """Outgoing free-space Green's function of (lap + k^2) G = -delta (k may
    be complex with Im k > 0: a lossy background)."""
    r = np.asarray(r, dtype=np.float64)
    if dim == 2:
        return 0.25j * special.hankel1(0, k * r)
    return np.exp(1j * k * r) / (4.0 * np.pi * r)


def equivalent_radius(h, dim):
    if dim == 2:
        return h / np.sqrt(np.pi)
    return h * (3.0 / (4.0 * np.pi)) ** (1.0 / 3.0)


def green_cell(k, r, h, dim):
    """Cell-integrated Green's function Ghat(r) (module docstring)."""
    r = np.asarray(r, dtype=np.float64)
    a = equivalent_radius(h, dim)
    ka = k * a
    out = np.empty(r.shape, dtype=np.complex128)
    far = r > 0
    if dim == 2:
        j1 = special.j1(ka) if np.isrealobj(ka) else special.jv(1, ka)
        out[far] = (1j * np.pi * a / (2.0 * k)) * j1 * special.hankel1(0, k * r[far])
        out[~far] = (1j * np.pi * a / (2.0 * k)) * special.hankel1(1, ka) \
            - 1.0 / (k * k)
    else:
        vol = 4.0 * np.pi * (np.sin(ka) - ka * np.cos(ka)) / k ** 3
        out[far] = vol * np.exp(1j * k * r[far]) / (4.0 * np.pi * r[far])
        out[~far] = ((1.0 - 1j * ka) * np.exp(1j * ka) - 1.0) / (k * k)
    return out


def green_lattice(shape, h, k):
    """Ghat on the doubled offset lattice used by the circular convolution.

    Entry at index (i_z, [i_y], i_x) of an array of shape 2*shape holds
    Ghat at the offset whose components are i mod 2N taken in
    [-(N-1), N-1]; the entries at i = N (offset +-N, never reached by a pair
    of pixels of the grid) are zero.
    """
    axes = []
    for n in shape:
        idx = np.arange(2 * n)
        off = np.where(idx < n, idx, idx - 2 * n).astype(np.float64)
        off[n] = np.nan
        axes.append(off * h)
    grids = np.meshgrid(*axes, indexing="ij")
    r = np.sqrt(sum(g * g for g in grids))
    valid = np.isfinite(r)
    out = np.zeros(r.shape, dtype=np.complex128)
    out[valid] = green_cell(k, r[valid], h, len(shape))
    return out

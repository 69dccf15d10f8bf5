"""Seeded synthetic inputs: geometry and speed-of-sound phantoms.

This module is the only code shared by the CUDA path's callers (tests,
bench) and the FP64 oracle's callers.  It holds no arithmetic of the
inversion method: it draws numbers and lays out geometry.  The phantoms
stand in for the paper's thyroid-cyst and 2D/3D aperture studies (Sec. V),
whose data and phantoms are not published: a 1540 m/s background with a
Gaussian-correlated texture, elliptical / ellipsoidal cysts, and a top-edge
linear array.

Layout conventions: arrays are depth-major, shape (Nz, Nx) or (Nz, Ny, Nx),
x fastest; pixel centres x = (ix + 1/2 - Nx/2) h, y = (iy + 1/2 - Ny/2) h,
z = iz h; the array elements sit at z = -h, centred laterally, y = 0.
"""
from dataclasses import dataclass, field

import numpy as np

C0 = 1540.0


@dataclass
class Workload:
    name: str
    shape: tuple          # (Nz, Nx) or (Nz, Ny, Nx)
    h: float              # pixel edge [m]
    c0: float             # background SoS [m/s]
    elem: np.ndarray      # [N_E, d] positions, (x, z) or (x, y, z) [m]
    freqs: np.ndarray     # [N_F] Hz
    sos: np.ndarray       # [*shape] speed of sound [m/s]
    seed: int = 0
    meta: dict = field(default_factory=dict)

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
    def n_rhs(self):
        return self.n_elem * self.n_freq


def array_positions(n_elem, pitch, h, dim):
    xe = (np.arange(n_elem, dtype=np.float64) - (n_elem - 1) / 2.0) * pitch
    if dim == 2:
        return np.stack([xe, np.full(n_elem, -h)], axis=1)
    return np.stack([xe, np.zeros(n_elem), np.full(n_elem, -h)], axis=1)


def _coords(shape, h):
    """Pixel-centre coordinate arrays (x, [y], z), each of ``shape``."""
    idx = np.meshgrid(*[np.arange(s, dtype=np.float64) for s in shape],
                      indexing="ij")
    if len(shape) == 2:
        z, x = idx
        return (x + 0.5 - shape[1] / 2.0) * h, z * h
    z, y, x = idx
    return ((x + 0.5 - shape[2] / 2.0) * h, (y + 0.5 - shape[1] / 2.0) * h,
            z * h)


def texture(shape, h, sigma, corr, rng):
    """White N(0,1) noise smoothed by a Gaussian whose standard deviation is
    corr/sqrt(2) (so the texture's own correlation scale is ``corr``),
    renormalised to standard deviation ``sigma``.  Circular smoothing."""
    w = rng.standard_normal(shape)
    s = corr / np.sqrt(2.0) / h
    spec = np.fft.fftn(w)
    for ax, n in enumerate(shape):
        f = np.fft.fftfreq(n)
        g = np.exp(-2.0 * (np.pi * f * s) ** 2)
        bshape = [1] * len(shape)
        bshape[ax] = n
        spec = spec * g.reshape(bshape)
    t = np.real(np.fft.ifftn(spec))
    t -= t.mean()
    sd = t.std()
    return t * (sigma / sd) if sd > 0 else t


def _ellipse_mask(coords, centre, semi, angle):
    if len(coords) == 2:
        x, z = coords
        dx, dz = x - centre[0], z - centre[1]
        ca, sa = np.cos(angle), np.sin(angle)
        u = (ca * dx + sa * dz) / semi[0]
        v = (-sa * dx + ca * dz) / semi[1]
        return u * u + v * v <= 1.0
    x, y, z = coords
    d = [x - centre[0], y - centre[1], z - centre[2]]
    ca, sa = np.cos(angle), np.sin(angle)
    u = (ca * d[0] + sa * d[2]) / semi[0]
    v = d[1] / semi[1]
    w = (-sa * d[0] + ca * d[2]) / semi[2]
    return u * u + v * v + w * w <= 1.0


def disc_phantom(seed=1000):
    """64 x 64 grid, 0.15 mm pixels, 1540 m/s background with one disc of
    radius 8 px at 1500 m/s (centre uniform in pixel [12, 52]^2), 32
    elements at 0.3 mm pitch, 1 MHz."""
    rng = np.random.default_rng(seed)
    shape, h = (64, 64), 0.15e-3
    cz, cx = rng.uniform(12.0, 52.0, size=2)
    z, x = np.meshgrid(np.arange(64.0), np.arange(64.0), indexing="ij")
    sos = np.full(shape, C0)
    sos[(x - cx) ** 2 + (z - cz) ** 2 <= 64.0] = 1500.0
    return Workload("disc64", shape, h, C0, array_positions(32, 0.3e-3, h, 2),
                    np.array([1.0e6]), sos, seed, dict(centre_px=(cx, cz)))


def tissue_phantom(shape, h, n_elem, pitch, freqs, seed, sigma=10.0,
                   corr=0.5e-3, inclusions=None, n_incl=(2, 2),
                   semi_mm=(1.5, 4.0), name="tissue"):
    """Background 1540 m/s + Gaussian-correlated texture (``sigma`` m/s,
    ``corr`` m) + elliptical (2D) or ellipsoidal (3D) inclusions with
    semi-axes U[semi_mm] mm, random orientation, centres in the lower 3/4 of
    the depth range.  ``inclusions``: list of SoS values, or None to draw
    U{n_incl} inclusions with SoS U[1480, 1600]."""
    rng = np.random.default_rng(seed)
    dim = len(shape)
    sos = C0 + texture(shape, h, sigma, corr, rng)
    coords = _coords(shape, h)
    if inclusions is None:
        k = int(rng.integers(n_incl[0], n_incl[1] + 1))
        inclusions = list(rng.uniform(1480.0, 1600.0, size=k))
    width = shape[-1] * h
    depth = shape[0] * h
    for c_in in inclusions:
        semi = rng.uniform(semi_mm[0], semi_mm[1], size=dim) * 1e-3
        ang = rng.uniform(0.0, np.pi)
        cx = rng.uniform(-0.35, 0.35) * width
        cz = rng.uniform(0.25, 0.85) * depth
        if dim == 2:
            centre = (cx, cz)
        else:
            centre = (cx, rng.uniform(-0.2, 0.2) * shape[1] * h, cz)
        sos[_ellipse_mask(coords, centre, semi, ang)] = c_in
    return Workload(name, tuple(shape), h, C0,
                    array_positions(n_elem, pitch, h, dim),
                    np.asarray(freqs, dtype=np.float64), sos, seed,
                    dict(inclusions=list(map(float, inclusions))))


def thyroid_256(seed=1001):
    """256^2 grid, 0.1 mm pixels, texture sigma 10 m/s / 0.5 mm, a fluid cyst
    (1520 m/s) and a solid cyst (1580 m/s), 128 elements at 0.2 mm pitch,
    6 frequencies 0.5-3 MHz."""
    return tissue_phantom((256, 256), 0.1e-3, 128, 0.2e-3,
                          np.linspace(0.5e6, 3.0e6, 6), seed,
                          inclusions=[1520.0, 1580.0], name="thyroid256")


def large_512(seed=1002):
    """512^2 grid, 0.08 mm pixels, same texture, 3-6 inclusions in
    [1480, 1600] m/s, 192 elements at 0.2 mm pitch, 12 frequencies 0.3-5 MHz."""
    return tissue_phantom((512, 512), 0.08e-3, 192, 0.2e-3,
                          np.linspace(0.3e6, 5.0e6, 12), seed,
                          n_incl=(3, 6), name="large512")


def volume_3d(seed=1003):
    """160 x 160 x 128 (x, y, depth) grid, 0.2 mm voxels, texture sigma
    8 m/s, ellipsoidal cysts at 1520 and 1580 m/s, 128 elements on the top
    face at 0.2 mm pitch, 4 frequencies 0.5-2 MHz."""
    return tissue_phantom((128, 160, 160), 0.2e-3, 128, 0.2e-3,
                          np.linspace(0.5e6, 2.0e6, 4), seed, sigma=8.0,
                          inclusions=[1520.0, 1580.0], name="volume3d")


def planewave_2d(seed=1005):
    """The 2-D acquisition of the paper's numerical study (Sec. V-A): 64
    elements at 0.78 mm pitch (49.9 mm aperture), 15 frequencies 0.2-3 MHz,
    60 plane waves steered over [-60, 60] degrees, every element receiving.
    Grid 384^2 at 0.13 mm (the aperture's width; 3.95 pixels per wavelength
    at 3 MHz), texture sigma 10 m/s / 0.5 mm with a fluid (1520 m/s) and a
    solid (1580 m/s) cyst standing in for the paper's cyst phantoms."""
    w = tissue_phantom((384, 384), 0.13e-3, 64, 0.78e-3, np.linspace(0.2e6, 3.0e6, 15), seed,
                       inclusions=[1520.0, 1580.0], name="planewave2d")
    w.meta["tx_angles"] = np.deg2rad(np.linspace(-60.0, 60.0, 60))
    return w


def elevation_3d(seed=1006):
    """The paper's 3-D study (Sec. V-B): 64 line elements of 1 cm elevation
    at 0.3 mm pitch (19.2 mm aperture), each element transmitting in turn,
    10 frequencies 0.2-2 MHz; homogeneous 1540 m/s background with two small
    spherical cysts (radius 0.8 mm at 1400 m/s, radius 0.5 mm at 1600 m/s)
    at two depths (seeded lateral positions).  Grid 96 x 64 x 64 (x, y,
    depth) at 0.2 mm (3.85 pixels per wavelength at 2 MHz)."""
    shape, h = (64, 64, 96), 0.2e-3
    rng = np.random.default_rng(seed)
    x, y, z = _coords(shape, h)
    sos = np.full(shape, C0)
    for radius, c_in, depth in ((0.8e-3, 1400.0, 4.0e-3), (0.5e-3, 1600.0, 8.0e-3)):
        cx, cy = rng.uniform(-3e-3, 3e-3), rng.uniform(-1e-3, 1e-3)
        sos[(x - cx) ** 2 + (y - cy) ** 2 + (z - depth) ** 2 <= radius ** 2] = c_in
    return Workload("elev3d", shape, h, C0, array_positions(64, 0.3e-3, h, 3),
                    np.linspace(0.2e6, 2.0e6, 10), sos, seed,
                    dict(elem_length=1e-2, inclusions=[1400.0, 1600.0]))


def scaled(shape, h, n_elem, pitch, freqs, seed, **kw):
    """A downscaled workload with the tissue statistics (parity tests)."""
    return tissue_phantom(shape, h, n_elem, pitch, freqs, seed, **kw)


def complex_normal(shape, seed):
    """Standard complex normal draws (real and imaginary parts N(0,1))."""
    rng = np.random.default_rng(seed)
    return rng.standard_normal(shape) + 1j * rng.standard_normal(shape)


def serving_requests(n_req=256, seed=1004, rate_hz=1.0):
    """Request stream: Poisson arrival times and, per request, a grid drawn
    from {128^2, 256^2, 384^2, 512^2, 96^3}, N_E ~ U{64..192}, N_F ~ U{2..12}
    frequencies in [0.3, f_max] MHz.  The pixel size keeps the aperture
    inside the grid width; f_max = min(5 MHz, c0 / (3.85 h)) keeps at least
    3.85 pixels per wavelength (the coarsest sampling of the paper's own
    configurations; coarser grids do not resolve the wave field)."""
    rng = np.random.default_rng(seed)
    grids = [(128, 128), (256, 256), (384, 384), (512, 512), (96, 96, 96)]
    t = np.cumsum(rng.exponential(1.0 / rate_hz, size=n_req))
    reqs = []
    for i in range(n_req):
        shape = grids[int(rng.integers(0, len(grids)))]
        n_elem = int(rng.integers(64, 193))
        n_freq = int(rng.integers(2, 13))
        pitch = 0.2e-3
        width_needed = n_elem * pitch
        h = max(0.05e-3, width_needed / shape[-1])
        f_max = min(5.0e6, 1540.0 / (3.85 * h))
        freqs = np.sort(rng.uniform(0.3e6, f_max, size=n_freq))
        reqs.append(dict(arrival=float(t[i]), shape=shape, h=h,
                         n_elem=n_elem, pitch=pitch, freqs=freqs,
                         seed=seed * 1000 + i))
    return reqs

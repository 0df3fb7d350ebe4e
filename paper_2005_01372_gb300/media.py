"""Seeded synthetic velocity models and source positions.

This module is shared by the CUDA path's tests/benchmark and by the oracle's
tests.  It draws velocity models only: it holds none of the method's
arithmetic (no contrast, no Green's function, no source field).  Each side
turns the velocity model into its own contrast and source field.

Layout: every model is returned as a float64 array of shape (nx, nz), C-ordered,
so ``c.ravel()[ix * nz + iz]`` is the velocity of cell (iz, ix).  This is the
paper's ordering of the unknowns in vertical strips (Sec. 2.4).

The models stand in for the paper's Marmousi2 subset and 2D SEG/EAGE salt model
(Sec. 3), which are not available: they keep the paper's scales (10-15 m cells,
background 2000 m/s, velocities 1500-4500+ m/s, strong scattering).
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np

C0 = 2000.0  # background velocity of both of the paper's examples (Sec. 3)


@dataclass(frozen=True)
class Workload:
    """One synthetic problem: grid, frequency, velocity model and sources."""

    name: str
    nz: int
    nx: int
    h: float
    c0: float
    freq_hz: float
    velocity: np.ndarray = field(repr=False)          # (nx, nz) float64
    sources: tuple = ()                               # ((iz, ix), ...)

    @property
    def n(self) -> int:
        return self.nz * self.nx


def _cell_centres(nz: int, nx: int, h: float):
    z = (np.arange(nz) + 0.5) * h
    x = (np.arange(nx) + 0.5) * h
    X, Z = np.meshgrid(x, z, indexing="ij")   # (nx, nz)
    return Z, X


def gaussian_inclusion(nz=64, nx=64, h=10.0, c0=C0, peak=3000.0, sigma=80.0):
    """c0 plus a Gaussian bump of the given peak velocity at the grid centre."""
    Z, X = _cell_centres(nz, nx, h)
    zc, xc = nz * h / 2.0, nx * h / 2.0
    r2 = (Z - zc) ** 2 + (X - xc) ** 2
    return c0 + (peak - c0) * np.exp(-r2 / (2.0 * sigma ** 2))


def layered(rng: np.random.Generator, nz: int, nx: int, h: float,
            n_layers=(8, 20), vel=(1500.0, 4500.0), max_dip_deg=5.0):
    """Random dipping layers with iid uniform velocities."""
    L = int(rng.integers(n_layers[0], n_layers[1] + 1))
    Z, X = _cell_centres(nz, nx, h)
    depth = nz * h
    tops = np.sort(rng.uniform(0.0, depth, size=L))
    dips = np.tan(np.deg2rad(rng.uniform(-max_dip_deg, max_dip_deg, size=L)))
    vels = rng.uniform(vel[0], vel[1], size=L + 1)
    xm = nx * h / 2.0
    c = np.full(Z.shape, vels[0])
    for i in range(L):
        below = Z >= tops[i] + dips[i] * (X - xm)
        c = np.where(below, vels[i + 1], c)
    return c


def salt_ellipse(rng: np.random.Generator, c: np.ndarray, h: float, v_salt=4500.0):
    """Overwrite a randomly placed, rotated ellipse with salt velocity."""
    nx, nz = c.shape
    Z, X = _cell_centres(nz, nx, h)
    zc = rng.uniform(0.25, 0.75) * nz * h
    xc = rng.uniform(0.25, 0.75) * nx * h
    a = rng.uniform(30, 60) * h * nx / 256.0
    b = rng.uniform(12, 30) * h * nz / 256.0
    th = rng.uniform(0.0, np.pi)
    dx, dz = X - xc, Z - zc
    u = dx * np.cos(th) + dz * np.sin(th)
    v = -dx * np.sin(th) + dz * np.cos(th)
    inside = (u / a) ** 2 + (v / b) ** 2 <= 1.0
    out = c.copy()
    out[inside] = v_salt
    return out


def gaussian_anomalies(rng: np.random.Generator, c: np.ndarray, h: float,
                       count=(1, 3), sigma_cells=(5, 20), amp=(-1500.0, 1500.0),
                       clip=(1500.0, 4500.0)):
    nx, nz = c.shape
    Z, X = _cell_centres(nz, nx, h)
    out = c.copy()
    for _ in range(int(rng.integers(count[0], count[1] + 1))):
        zc = rng.uniform(0, nz * h)
        xc = rng.uniform(0, nx * h)
        s = rng.uniform(*sigma_cells) * h
        A = rng.uniform(*amp)
        out = out + A * np.exp(-((Z - zc) ** 2 + (X - xc) ** 2) / (2 * s * s))
    return np.clip(out, *clip)


def _smooth(c: np.ndarray, sigma_cells: float) -> np.ndarray:
    """Separable Gaussian smoothing with edge replication."""
    rad = int(np.ceil(3 * sigma_cells))
    t = np.arange(-rad, rad + 1)
    w = np.exp(-0.5 * (t / sigma_cells) ** 2)
    w /= w.sum()
    out = c
    for axis in (0, 1):
        pad = [(0, 0), (0, 0)]
        pad[axis] = (rad, rad)
        p = np.pad(out, pad, mode="edge")
        acc = np.zeros_like(out)
        for k, wk in enumerate(w):
            sl = [slice(None), slice(None)]
            sl[axis] = slice(k, k + out.shape[axis])
            acc += wk * p[tuple(sl)]
        out = acc
    return out


def marmousi_like(rng: np.random.Generator, nz: int, nx: int, h: float,
                  n_layers=(30, 60), vtop=1500.0, vbot=5500.0, n_faults=(5, 10)):
    """Smoothed random layers with a depth trend, cut by random faults."""
    L = int(rng.integers(n_layers[0], n_layers[1] + 1))
    tops = np.sort(rng.uniform(0, nz, size=L))                 # in cells
    trend = vtop + (vbot - vtop) * (np.arange(L + 1) / L)
    vels = np.clip(trend + rng.normal(0, 250.0, size=L + 1), vtop, vbot)
    ix = np.arange(nx)[:, None].astype(float)
    iz = np.arange(nz)[None, :].astype(float)
    shift = np.zeros((nx, nz))
    for _ in range(int(rng.integers(n_faults[0], n_faults[1] + 1))):
        x0, z0 = rng.uniform(0, nx), rng.uniform(0, nz)
        th = rng.uniform(0, np.pi)
        side = (ix - x0) * np.sin(th) - (iz - z0) * np.cos(th) > 0
        shift = shift + np.where(side, rng.uniform(5, 40), 0.0)
    depth = iz - shift
    lay = np.searchsorted(tops, depth.ravel()).reshape(nx, nz)
    c = vels[np.clip(lay, 0, L)]
    return np.clip(_smooth(c, 2.0), vtop, vbot)


# ---------------------------------------------------------------- workloads

def gaussian_inclusion_64(freq_hz=10.0) -> Workload:
    """64x64, h=10 m, c0=2000 m/s, f=10 Hz, Gaussian inclusion (peak 3000 m/s,
    sigma 80 m) at the centre, one point source at (iz=5, ix=32)."""
    c = gaussian_inclusion(64, 64, 10.0, C0, 3000.0, 80.0)
    return Workload("gaussian-inclusion-64x64-10Hz", 64, 64, 10.0, C0, freq_hz, c, ((5, 32),))


def gaussian_inclusion_16(freq_hz=10.0) -> Workload:
    """The 64x64 inclusion rescaled to a 16x16 grid (sigma 20 m, same peak)."""
    c = gaussian_inclusion(16, 16, 10.0, C0, 3000.0, 20.0)
    return Workload("gaussian-inclusion-16x16-10Hz", 16, 16, 10.0, C0, freq_hz, c, ((2, 8),))


def layered_salt(n=256, freq_hz=15.0, nsrc=32, seed=2, h=10.0) -> Workload:
    """Layered medium (8-20 dipping layers, 1500-4500 m/s) with a 4500 m/s
    salt-like ellipse; ``nsrc`` sources along the top row."""
    rng = np.random.default_rng(seed)
    c = salt_ellipse(rng, layered(rng, n, n, h), h)
    step = n // nsrc
    src = tuple((0, step * m + step // 2) for m in range(nsrc))
    return Workload(f"layered-salt-{n}x{n}-{freq_hz:g}Hz-{nsrc}src", n, n, h, C0, freq_hz, c, src)


def layered_anomaly(n: int, freq_hz: float, nsrc=64, seed=31, h=10.0) -> Workload:
    rng = np.random.default_rng(seed)
    c = gaussian_anomalies(rng, layered(rng, n, n, h), h)
    src = tuple((0, int((m + 0.5) * n / nsrc)) for m in range(nsrc))
    return Workload(f"layered-anomaly-{n}x{n}-{freq_hz:g}Hz-{nsrc}src", n, n, h, C0, freq_hz, c, src)


def marmousi_1024(freq_hz=30.0, nsrc=16, seed=4, n=1024, h=5.0) -> Workload:
    rng = np.random.default_rng(seed)
    c = marmousi_like(rng, n, n, h)
    step = n // nsrc
    src = tuple((0, step * m + step // 2) for m in range(nsrc))
    return Workload(f"marmousi-like-{n}x{n}-{freq_hz:g}Hz-{nsrc}src", n, n, h, C0, freq_hz, c, src)


def embed(c: np.ndarray, nz: int, nx: int, c0: float = C0) -> np.ndarray:
    """The model c (shape (nx_m, nz_m)) at the top-left corner of an nz x nx
    grid whose other cells have the background velocity c0 (zero contrast).
    Cells of zero contrast do not scatter, so inside the model the solution
    on the larger grid equals the solution on the model's own grid: a model
    of any shape runs on power-of-two grids."""
    nxm, nzm = c.shape
    if nzm > nz or nxm > nx:
        raise ValueError("the grid is smaller than the model")
    out = np.full((nx, nz), float(c0))
    out[:nxm, :nzm] = c
    return out


def marmousi_subset(freq_hz=10.0, seed=5) -> Workload:
    """Stand-in for the paper's Marmousi2 subset (Sec. 3.1): 248 x 81 cells
    of 15 m (x by z), layered and faulted, embedded at the top-left of a
    256 x 128 grid (x by z); one source in the middle of the top row."""
    rng = np.random.default_rng(seed)
    c = marmousi_like(rng, 81, 248, 15.0, n_layers=(15, 30), vtop=1500.0, vbot=4700.0, n_faults=(3, 6))
    return Workload(f"marmousi-subset-248x81-h15-in-256x128-{freq_hz:g}Hz", 128, 256, 15.0, C0, freq_hz,
                    embed(c, 128, 256), ((0, 124),))


def salt_subset(freq_hz=10.0, seed=6) -> Workload:
    """Stand-in for the paper's 2D SEG/EAGE salt model (Sec. 3.2): 700 x 150
    cells of 10 m (x by z), layered with a salt body, embedded at the
    top-left of a 1024 x 256 grid (x by z); one source in the middle of the
    top row."""
    rng = np.random.default_rng(seed)
    c = salt_ellipse(rng, layered(rng, 150, 700, 10.0), 10.0)
    return Workload(f"salt-subset-700x150-h10-in-1024x256-{freq_hz:g}Hz", 256, 1024, 10.0, C0, freq_hz,
                    embed(c, 256, 1024), ((0, 350),))


def fno_medium(seed: int, n: int, h: float = 10.0, freq=(10.0, 25.0)):
    """A training or test medium for the learned preconditioner: 8-20 dipping
    layers (1500-4500 m/s), a salt ellipse with probability 1/2, 1-3 Gaussian
    anomalies, and a frequency drawn from U(freq).  Returns (velocity, f)."""
    rng = np.random.default_rng(seed)
    c = layered(rng, n, n, h)
    if rng.uniform() < 0.5:
        c = salt_ellipse(rng, c, h)
    c = gaussian_anomalies(rng, c, h, sigma_cells=(n / 32.0, n / 8.0))
    return c, float(rng.uniform(*freq))


def smooth_complex_field(rng: np.random.Generator, count: int, nz: int, nx: int,
                         sigma_cells=(1.0, 6.0)) -> np.ndarray:
    """``count`` complex fields (count, nz * nx) in strip order: iid complex
    normal noise smoothed by a Gaussian of a random width per field."""
    out = np.empty((count, nz * nx), dtype=np.complex128)
    for i in range(count):
        s = rng.uniform(*sigma_cells)
        re = _smooth(rng.standard_normal((nx, nz)), s)
        im = _smooth(rng.standard_normal((nx, nz)), s)
        out[i] = (re + 1j * im).ravel()
    return out


def random_field(rng: np.random.Generator, nz: int, nx: int, lo=1500.0, hi=4500.0,
                 smooth_cells=2.0) -> np.ndarray:
    """Smoothed iid uniform velocities, for small randomized test cases."""
    c = rng.uniform(lo, hi, size=(nx, nz))
    if smooth_cells > 0 and min(nx, nz) > 4:
        c = _smooth(c, smooth_cells)
    return c


def complex_field(rng: np.random.Generator, shape, dtype=np.complex128) -> np.ndarray:
    """iid complex standard normal test vectors."""
    v = (rng.standard_normal(shape) + 1j * rng.standard_normal(shape)) / np.sqrt(2.0)
    return v.astype(dtype)

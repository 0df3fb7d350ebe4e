"""Contrast and cell-integrated Green's function (oracle; test infrastructure).

Sec. 2.1 defines the contrast chi by Eq. 1 and the Lippmann-Schwinger equation
(Eq. 3) with the background Green's function G0 of the homogeneous medium.  For
2D and the exp(-i w t) convention, G0(r) = (i/4) H0^(1)(k0 r) solves
[lap + k0^2] G0 = -delta with outgoing radiation.

Eq. 4 collocates at cell centres with V = diag(dv * chi).  The integrand is
singular in the source cell, so every cell is integrated exactly over the disk
of equal area (radius a = h / sqrt(pi)); by Graf's addition theorem

    off the diagonal:  Gt(r) = (i pi a / (2 k)) J1(k a) H0^(1)(k r)
    on the diagonal:   Gt(0) = (i pi a / (2 k)) H1^(1)(k a) - 1 / k^2

so that G0 V = Gt diag(chi): the cell volume dv is inside Gt.
"""
from __future__ import annotations

import numpy as np
from scipy import special


def angular_frequency(freq_hz: float) -> float:
    return 2.0 * np.pi * freq_hz


def contrast(c: np.ndarray, c0: float, freq_hz: float) -> np.ndarray:
    """Eq. 1: w^2 / c^2 = w^2 / c0^2 + chi, so chi = w^2 (1/c^2 - 1/c0^2)."""
    w = angular_frequency(freq_hz)
    return w * w * (1.0 / np.asarray(c, dtype=np.float64) ** 2 - 1.0 / c0 ** 2)


def wavenumber(c0: float, freq_hz: float) -> float:
    return angular_frequency(freq_hz) / c0


def cell_radius(h: float) -> float:
    """Radius of the disk with the area h^2 of one grid cell."""
    return h / np.sqrt(np.pi)


def green_of_distance(r: np.ndarray, k: float, h: float) -> np.ndarray:
    """Cell-integrated Green's function Gt at centre distance r (Sec. 2.2).

    r == 0 selects the self-cell value; any other r uses the exterior form,
    which is exact whenever r > a: distinct cell centres are at least h apart
    and a = 0.564 h."""
    r = np.asarray(r, dtype=np.float64)
    a = cell_radius(h)
    pref = 1j * np.pi * a / (2.0 * k)
    out = np.empty(r.shape, dtype=np.complex128)
    off = r > 0
    out[off] = pref * special.jv(1, k * a) * special.hankel1(0, k * r[off])
    out[~off] = pref * special.hankel1(1, k * a) - 1.0 / (k * k)
    return out


def green_table(nz: int, nx: int, h: float, k: float) -> np.ndarray:
    """Gt at every offset (dz, dx), 0 <= dz <= nz, 0 <= dx <= nx.

    Returned with shape (nx + 1, nz + 1).  G0 is translation invariant
    (Sec. 2.1), so this table holds the whole block-Toeplitz matrix; it is the
    'first row of the matrix reshaped' of Sec. 2.2 plus the offsets nz and nx
    that complete the even extension."""
    dz = np.arange(nz + 1)
    dx = np.arange(nx + 1)
    DX, DZ = np.meshgrid(dx, dz, indexing="ij")
    return green_of_distance(h * np.hypot(DZ, DX), k, h)


def cell_coords(nz: int, nx: int):
    """(iz, ix) of every unknown in the strip ordering ix * nz + iz (Sec. 2.4)."""
    idx = np.arange(nz * nx)
    return idx % nz, idx // nz


def green_dense(nz: int, nx: int, h: float, k: float) -> np.ndarray:
    """The full n x n matrix Gt_ij (n = nz nx) of Eq. 4, formed entry by entry
    from centre distances.  Only for small grids."""
    iz, ix = cell_coords(nz, nx)
    r = h * np.hypot(iz[:, None] - iz[None, :], ix[:, None] - ix[None, :])
    return green_of_distance(r, k, h)


def green_block(rows_iz, rows_ix, cols_iz, cols_ix, h: float, k: float) -> np.ndarray:
    """Gt between two arbitrary cell lists (used for dense HODLR leaves)."""
    r = h * np.hypot(np.subtract.outer(rows_iz, cols_iz), np.subtract.outer(rows_ix, cols_ix))
    return green_of_distance(r, k, h)


def green_extension(nz: int, nx: int, h: float, k: float) -> np.ndarray:
    """Even circulant extension of the Green table to 2nx x 2nz (Sec. 2.2).

    Index i along an axis of length 2N carries the offset min(i, 2N - i), so
    indices 0..N hold offsets 0..N and N+1..2N-1 hold offsets N-1..1."""
    tab = green_table(nz, nx, h, k)
    iz = np.arange(2 * nz)
    ix = np.arange(2 * nx)
    dz = np.minimum(iz, 2 * nz - iz)
    dx = np.minimum(ix, 2 * nx - ix)
    return tab[dx[:, None], dz[None, :]]


def green_spectrum(nz: int, nx: int, h: float, k: float) -> np.ndarray:
    """F(Gt_ext), the unnormalised 2D DFT of the extension (Sec. 2.2)."""
    return np.fft.fft2(green_extension(nz, nx, h, k))


def point_source(nz: int, nx: int, h: float, k: float, iz: int, ix: int) -> np.ndarray:
    """Background field psi0 of a unit point source smeared over cell (iz, ix):
    psi0_i = Gt(r_i) / h^2, i.e. (i/4) H0(k r) 2 J1(ka)/(ka) off the source cell.
    The Ricker amplitude of the paper's source (Sec. 3.1) is one complex scalar
    per frequency and drops out of the linear problem."""
    z, x = cell_coords(nz, nx)
    r = h * np.hypot(z - iz, x - ix)
    return green_of_distance(r, k, h) / (h * h)

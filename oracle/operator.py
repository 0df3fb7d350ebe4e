"""The Lippmann-Schwinger operator G0 V (oracle; test infrastructure).

Two independent evaluations of the same product (Eq. 4):

* ``apply_dense``: the direct O(n^2) sum  (G0 V u)_i = sum_j Gt_ij chi_j u_j;
* ``apply_fft``:   Sec. 2.2, F^-1( F(Gt_ext) . F(pad(V u)) ) cropped to the grid.

Vectors are flat arrays of length n = nz nx in the strip ordering
``ix * nz + iz`` (Sec. 2.4), or 2D arrays (n, S) holding S right-hand sides
as columns.
"""
from __future__ import annotations

import numpy as np

from . import green

FORWARD, RESIDUAL, PLAIN, ADJOINT = 0, 1, 2, 3


def apply_dense(Gd: np.ndarray, chi: np.ndarray, u: np.ndarray) -> np.ndarray:
    """G0 V u by direct summation with the dense Green matrix (Eq. 4)."""
    u = np.asarray(u)
    cu = chi[:, None] * u if u.ndim == 2 else chi * u
    return Gd @ cu


def conv_fft(spec: np.ndarray, w: np.ndarray, nz: int, nx: int) -> np.ndarray:
    """Gt * w: zero-pad w to the 2nx x 2nz grid, multiply by the spectrum of
    the extended Green table, transform back and crop (Sec. 2.2)."""
    w = np.asarray(w)
    one = w.ndim == 1
    W = w.reshape(nx, nz, -1)
    pad = np.zeros((2 * nx, 2 * nz, W.shape[2]), dtype=np.complex128)
    pad[:nx, :nz] = W
    F = np.fft.fft2(pad, axes=(0, 1)) * spec[:, :, None]
    out = np.fft.ifft2(F, axes=(0, 1))[:nx, :nz].reshape(nx * nz, -1)
    return out[:, 0] if one else out


def apply_fft(spec: np.ndarray, chi: np.ndarray, u: np.ndarray, nz: int, nx: int) -> np.ndarray:
    """G0 V u through the FFT (Sec. 2.2)."""
    u = np.asarray(u)
    cu = chi[:, None] * u if u.ndim == 2 else chi * u
    return conv_fft(spec, cu, nz, nx)


def apply_adjoint_fft(spec: np.ndarray, chi: np.ndarray, x: np.ndarray, nz: int, nx: int) -> np.ndarray:
    """(G0 V)^H x.  Gt is complex symmetric (reciprocity, Gt_ij = Gt_ji) and
    chi is real, so (Gt diag chi)^H x = chi . conj(Gt conj(x)); this is the
    product with G0^T of Algorithm 2 (step 4/5), 'T' being the conjugate
    transpose (Sec. 2.3)."""
    x = np.asarray(x)
    g = np.conj(conv_fft(spec, np.conj(x), nz, nx))
    return chi[:, None] * g if g.ndim == 2 else chi * g


def apply(mode: int, spec, chi, u, u0, nz: int, nx: int) -> np.ndarray:
    """The four products of the library's operator call:

    FORWARD  y = u0 + G0 V u          (right side of Eq. 4)
    RESIDUAL y = u - G0 V u - u0      (a_{j-1} of Eq. 13)
    PLAIN    y = G0 V u
    ADJOINT  y = (G0 V)^H u
    ``u0`` may be None for FORWARD/RESIDUAL, meaning zero."""
    if mode == ADJOINT:
        return apply_adjoint_fft(spec, chi, u, nz, nx)
    g = apply_fft(spec, chi, u, nz, nx)
    if mode == PLAIN:
        return g
    if mode == FORWARD:
        return g if u0 is None else u0 + g
    if mode == RESIDUAL:
        y = np.asarray(u) - g
        return y if u0 is None else y - u0
    raise ValueError(f"unknown mode {mode}")


class Problem:
    """One discretised problem: grid, frequency, contrast and Green spectrum."""

    def __init__(self, nz: int, nx: int, h: float, c0: float, freq_hz: float, velocity: np.ndarray):
        self.nz, self.nx, self.h, self.c0, self.freq_hz = nz, nx, h, c0, freq_hz
        self.n = nz * nx
        self.k = green.wavenumber(c0, freq_hz)
        self.chi = green.contrast(np.asarray(velocity).ravel(), c0, freq_hz)
        self.spec = green.green_spectrum(nz, nx, h, self.k)

    @classmethod
    def from_workload(cls, wl):
        return cls(wl.nz, wl.nx, wl.h, wl.c0, wl.freq_hz, wl.velocity)

    def sources(self, positions) -> np.ndarray:
        """psi0 for each (iz, ix) as columns of an (n, S) array."""
        cols = [green.point_source(self.nz, self.nx, self.h, self.k, iz, ix) for iz, ix in positions]
        return np.stack(cols, axis=1)

    def G0V(self, u):
        return apply_fft(self.spec, self.chi, u, self.nz, self.nx)

    def G0V_adj(self, x):
        return apply_adjoint_fft(self.spec, self.chi, x, self.nz, self.nx)

    def A(self, u):
        """(I - G0 V) u, the operator of Eq. 5."""
        return np.asarray(u) - self.G0V(u)

    def dense_A(self) -> np.ndarray:
        """I - Gt diag(chi) as an n x n matrix (Eq. 5); small grids only."""
        Gd = green.green_dense(self.nz, self.nx, self.h, self.k)
        return np.eye(self.n, dtype=np.complex128) - Gd * self.chi[None, :]

    def rel_residual(self, u, u0) -> np.ndarray:
        """||u0 - (I - G0 V) u||_2 / ||u0||_2 per column, in FP64."""
        u = np.asarray(u, dtype=np.complex128)
        u0 = np.asarray(u0, dtype=np.complex128)
        r = u0 - self.A(u)
        return np.linalg.norm(r, axis=0) / np.linalg.norm(u0, axis=0)

"""Fourier neural operator used as a learned right preconditioner (oracle;
test infrastructure).

The paper's method builds H ~ (I - G0 V)^-1 by randomized sketches (Sec. 2.3-
2.4).  The learned variant replaces H inside flexible GMRES (the Krylov
comparison of Sec. 3.2) by a network trained on (residual -> correction)
pairs that H-preconditioned solves produce; H stays as the fallback and the
FP64 residual still decides convergence.  The paper has no network; this module fixes
the one the library implements, in plain NumPy, FP64:

  fields:  complex, on the nz x nx grid, strip order (ix * nz + iz)
  input:   two complex channels, x0 = residual / ||residual||,
           x1 = (c0^2 / c^2 - 1) + i k0 h   (normalised contrast, wavenumber)
  lift:    v = P x + p                     (P: W x 2, p: W, complex)
  layers:  v <- sigma(K_l v + W_l v + b_l), l = 0..L-1, no sigma on the last
  K_l:     spectral convolution truncated to the modes kz, kx in
           M = {0..m-1} U {n-m..n-1} of the 2D DFT:  Vhat = F v  on M x M,
           Zhat[k] = R_l[k] Vhat[k] (W x W complex per mode),  K_l v = F^-1 Zhat
  sigma:   split GELU, gelu(Re z) + i gelu(Im z), gelu(t) = t Phi(t)
  project: y = x0 + Q v + q                (Q: 1 x W, complex; the input's
           residual channel passes straight through, so the network learns
           the correction beyond the identity and the zero network is the
           identity preconditioner)

Gradients use G = dL/dRe + i dL/dIm for every complex quantity; then a
complex-linear map z = A w backpropagates as G_w = A^H G_z, and the split
GELU as G_z = gelu'(Re z) Re G_y + i gelu'(Im z) Im G_y.  The loss is
L = mean |y - target|^2, so G_y = 2 (y - target) / count.
"""
from __future__ import annotations

import numpy as np
from scipy import special


def mode_index(n: int, m: int) -> np.ndarray:
    """The retained wavenumbers along an axis of n points: 0..m-1, n-m..n-1."""
    if 2 * m > n:
        raise ValueError("too many modes for the grid")
    return np.concatenate([np.arange(m), np.arange(n - m, n)])


def dft_rows(n: int, m: int) -> np.ndarray:
    """F_M (2m x n): rows of the unnormalised DFT for the retained modes."""
    k = mode_index(n, m)
    return np.exp(-2j * np.pi * np.outer(k, np.arange(n)) / n)


def gelu(t):
    return t * 0.5 * (1.0 + special.erf(t / np.sqrt(2.0)))


def gelu_grad(t):
    return 0.5 * (1.0 + special.erf(t / np.sqrt(2.0))) + t * np.exp(-0.5 * t * t) / np.sqrt(2 * np.pi)


def split_gelu(z):
    return gelu(z.real) + 1j * gelu(z.imag)


def init_params(width: int, modes: int, layers: int, seed: int = 0) -> dict:
    """Gaussian initial weights, scaled by fan-in."""
    rng = np.random.default_rng(seed)

    def c(*shape, scale):
        return (rng.standard_normal(shape) + 1j * rng.standard_normal(shape)) * scale / np.sqrt(2)

    m2 = 2 * modes
    p = {"P": c(width, 2, scale=1 / np.sqrt(2)), "p": np.zeros(width, complex),
         "Q": c(1, width, scale=1 / np.sqrt(width)), "q": np.zeros(1, complex)}
    for l in range(layers):
        p[f"R{l}"] = c(m2, m2, width, width, scale=1 / width)
        p[f"W{l}"] = c(width, width, scale=1 / np.sqrt(width))
        p[f"b{l}"] = np.zeros(width, complex)
    return p


def _spectral(v, R, nz, nx, modes):
    """K v for v (W, nz, nx) complex: truncated DFT, per-mode mixing, inverse."""
    Fz, Fx = dft_rows(nz, modes), dft_rows(nx, modes)
    Vh = np.einsum("az,wzx,bx->wab", Fz, v, Fx)          # (W, 2m, 2m)
    Zh = np.einsum("abow,wab->oab", R, Vh)                  # R: (2m, 2m, W_out, W_in)
    return np.einsum("az,oab,bx->ozx", Fz.conj(), Zh, Fx.conj()) / (nz * nx), Vh


def forward(params: dict, x: np.ndarray, nz: int, nx: int, modes: int, keep: bool = False):
    """x: (2, nz, nx) complex input channels -> y: (nz, nx) complex."""
    L = sum(1 for k in params if k.startswith("R"))
    cache = {"x": x}
    v = np.einsum("wc,czx->wzx", params["P"], x) + params["p"][:, None, None]
    cache["v0"] = v
    for l in range(L):
        k, vh = _spectral(v, params[f"R{l}"], nz, nx, modes)
        z = k + np.einsum("ow,wzx->ozx", params[f"W{l}"], v) + params[f"b{l}"][:, None, None]
        cache[f"Vh{l}"], cache[f"z{l}"] = vh, z
        v = split_gelu(z) if l < L - 1 else z
        cache[f"v{l + 1}"] = v
    y = x[0] + np.einsum("ow,wzx->ozx", params["Q"], v)[0] + params["q"][0]
    return (y, cache) if keep else y


def loss_and_grad(params: dict, x: np.ndarray, target: np.ndarray, nz: int, nx: int, modes: int):
    """L = mean |y - target|^2 and G = dL/dRe + i dL/dIm for every parameter."""
    L = sum(1 for k in params if k.startswith("R"))
    y, c = forward(params, x, nz, nx, modes, keep=True)
    diff = y - target
    loss = float(np.mean(np.abs(diff) ** 2))
    Gy = 2.0 * diff / diff.size
    g = {}
    vL = c[f"v{L}"]
    g["Q"] = np.einsum("zx,wzx->w", Gy, vL.conj())[None, :]
    g["q"] = np.array([Gy.sum()])
    Gv = np.einsum("o,zx->ozx", params["Q"][0].conj(), Gy)
    Fz, Fx = dft_rows(nz, modes), dft_rows(nx, modes)
    for l in range(L - 1, -1, -1):
        z = c[f"z{l}"]
        if l < L - 1:
            Gz = gelu_grad(z.real) * Gv.real + 1j * gelu_grad(z.imag) * Gv.imag
        else:
            Gz = Gv
        v = c[f"v{l}"]
        g[f"b{l}"] = Gz.sum(axis=(1, 2))
        g[f"W{l}"] = np.einsum("ozx,wzx->ow", Gz, v.conj())
        # spectral path: z_s = Finv Zh, Zh = R Vh, Vh = F v
        GZh = np.einsum("az,ozx,bx->oab", Fz, Gz, Fx) / (nz * nx)           # Finv^H Gz
        Vh = c[f"Vh{l}"]
        g[f"R{l}"] = np.einsum("oab,wab->abow", GZh, Vh.conj())
        GVh = np.einsum("abow,oab->wab", params[f"R{l}"].conj(), GZh)
        Gv = np.einsum("ow,ozx->wzx", params[f"W{l}"].conj(), Gz) + \
            np.einsum("az,wab,bx->wzx", Fz.conj(), GVh, Fx.conj())
    g["p"] = Gv.sum(axis=(1, 2))
    g["P"] = np.einsum("wzx,czx->wc", Gv, c["x"].conj())
    return loss, g


def input_channels(r: np.ndarray, chi_norm: np.ndarray, k0h: float, nz: int, nx: int) -> np.ndarray:
    """(2, nz, nx) input from a residual (flat, strip order) and the
    normalised contrast c0^2/c^2 - 1 (flat)."""
    nrm = np.linalg.norm(r)
    x0 = (r / nrm if nrm > 0 else r).reshape(nx, nz).T
    x1 = (chi_norm + 1j * k0h).reshape(nx, nz).T
    return np.stack([x0, x1])


def adam_step(params: dict, grads: dict, state: dict, lr: float, b1=0.9, b2=0.999, eps=1e-8) -> None:
    """Adam (Kingma & Ba 2015) on the real and imaginary parts of every weight."""
    state["t"] = state.get("t", 0) + 1
    t = state["t"]
    for k, w in params.items():
        g = grads[k]
        m = state.setdefault("m_" + k, np.zeros_like(w))
        v = state.setdefault("v_" + k, np.zeros(w.shape + (2,)))
        m[...] = b1 * m + (1 - b1) * g
        gg = np.stack([g.real ** 2, g.imag ** 2], axis=-1)
        v[...] = b2 * v + (1 - b2) * gg
        mh = m / (1 - b1 ** t)
        vh = v / (1 - b2 ** t)
        step = mh.real / (np.sqrt(vh[..., 0]) + eps) + 1j * mh.imag / (np.sqrt(vh[..., 1]) + eps)
        w -= lr * step

"""Randomized low-rank approximation (oracle; test infrastructure).

``range_finder`` is Algorithm 1 (Halko, Martinsson, Tropp 2011, Alg. 4.4 with
the projection of step 5) for a matrix given only through its products with
blocks of vectors; ``g0v_sketch`` is Algorithm 2, its specialisation to
A = G0 V with the products done by FFT.  ``truncate`` adds the small SVD that
cuts the oversampled approximation to rank r (Halko et al. Sec. 5.1).
"""
from __future__ import annotations

import numpy as np

from . import philox


def qr_basis(Y: np.ndarray) -> np.ndarray:
    """Orthonormal basis of range(Y) from a thin Householder QR (step 3)."""
    Q, _ = np.linalg.qr(Y, mode="reduced")
    return Q


def range_finder(A, AH, Omega: np.ndarray, q: int = 0):
    """Algorithm 1: returns (Q_q, Yt_{q+1}) with A ~ Q_q Yt_{q+1}^H.

    ``A(X)`` and ``AH(X)`` return A X and A^H X for a block X."""
    Q = qr_basis(A(Omega))                      # steps 2-3
    for _ in range(q):                          # step 4 (power iterations)
        Qt = qr_basis(AH(Q))
        Q = qr_basis(A(Qt))
    return Q, AH(Q)                             # step 5


def truncate(Q: np.ndarray, Yt: np.ndarray, r: int):
    """Best rank-r approximation of Q Yt^H (an SVD of the small factor).

    With Yt = Vb S Ub^H:  Q Yt^H = (Q Ub S) Vb^H; keep the leading r terms.
    Returns (U, W) of r columns each (zero columns when fewer exist) with
    Q Yt^H ~ U W^H."""
    Vb, S, UbH = np.linalg.svd(Yt, full_matrices=False)
    k = min(r, S.size)
    U = np.zeros((Q.shape[0], r), dtype=np.complex128)
    W = np.zeros((Yt.shape[0], r), dtype=np.complex128)
    U[:, :k] = (Q @ UbH.conj().T[:, :k]) * S[:k]
    W[:, :k] = Vb[:, :k]
    return U, W


def g0v_sketch(prob, rank: int, oversample: int, q: int, seed: int):
    """Algorithm 2 on the whole grid: G0 V ~ U W^H (rank ``rank``), from
    ``rank + oversample`` Gaussian probes and ``q`` power iterations."""
    w2, w3 = philox.stream_words(philox.TAG_GLOBAL)
    Omega = philox.gaussian(prob.n, rank + oversample, seed, w2, w3)
    Q, Yt = range_finder(prob.G0V, prob.G0V_adj, Omega, q)
    return truncate(Q, Yt, rank)

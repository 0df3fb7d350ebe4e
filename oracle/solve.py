"""Solvers for (I - G0 V) psi = psi0 (oracle; test infrastructure)."""
from __future__ import annotations

import numpy as np
import scipy.linalg

from .operator import Problem


def direct(prob: Problem, u0: np.ndarray) -> np.ndarray:
    """Eq. 6: psi = (I - G0 V)^-1 psi0 by dense LU (small grids)."""
    lu = scipy.linalg.lu_factor(prob.dense_A())
    return scipy.linalg.lu_solve(lu, u0)


def series(prob: Problem, u0: np.ndarray, H=None, tol: float = 1e-6, max_iter: int = 30):
    """Preconditioned scattering series, Eq. 11, started from psi_0 = H psi0.

    Each step forms a = psi - G0 V psi - psi0 (Eq. 13); a source whose
    ||a||_2 <= tol ||psi0||_2 stops with that psi (the stopping rule of
    Sec. 3.2, read as a relative 2-norm); otherwise psi <- psi - H a.
    With H = None this is the Born series psi_j = psi0 + G0 V psi_{j-1}
    (Sec. 2.2), started from psi_0 = psi0.

    Returns (psi, iterations per source, relative residual per source)."""
    u0 = np.asarray(u0, dtype=np.complex128)
    one = u0.ndim == 1
    U0 = u0[:, None] if one else u0
    Happ = (lambda x: x) if H is None else H
    psi = Happ(U0).astype(np.complex128)
    nrm0 = np.linalg.norm(U0, axis=0)
    S = U0.shape[1]
    done = np.zeros(S, dtype=bool)
    iters = np.zeros(S, dtype=np.int64)
    res = np.full(S, np.inf)
    for it in range(max_iter + 1):
        a = psi - prob.G0V(psi) - U0
        rel = np.linalg.norm(a, axis=0) / nrm0
        newly = (~done) & (rel <= tol)
        res[~done] = rel[~done]
        iters[newly] = it
        done |= newly
        if done.all() or it == max_iter:
            break
        act = ~done
        psi[:, act] = psi[:, act] - Happ(a[:, act])
    iters[~done] = max_iter
    if one:
        return psi[:, 0], iters[0], res[0]
    return psi, iters, res


def fgmres(prob: Problem, u0: np.ndarray, M=None, tol: float = 1e-6, restart: int = 30,
           max_iter: int = 300):
    """Flexible GMRES (Saad 1993) for (I - G0 V) u = u0, one right-hand side,
    right preconditioner M (None: identity).  Returns (u, iterations, rel. res.)."""
    Mapp = (lambda x: x) if M is None else M
    b = np.asarray(u0, dtype=np.complex128)
    nb = np.linalg.norm(b)
    x = np.zeros_like(b)
    total = 0
    r = b - prob.A(x)
    while total < max_iter:
        beta = np.linalg.norm(r)
        if beta <= tol * nb:
            break
        m = restart
        V = np.zeros((b.size, m + 1), dtype=np.complex128)
        Z = np.zeros((b.size, m), dtype=np.complex128)
        Hh = np.zeros((m + 1, m), dtype=np.complex128)
        V[:, 0] = r / beta
        k_used = 0
        for j in range(m):
            Z[:, j] = Mapp(V[:, j])
            w = prob.A(Z[:, j])
            for i in range(j + 1):                 # modified Gram-Schmidt
                Hh[i, j] = np.vdot(V[:, i], w)
                w = w - Hh[i, j] * V[:, i]
            Hh[j + 1, j] = np.linalg.norm(w)
            k_used = j + 1
            total += 1
            e1 = np.zeros(j + 2, dtype=np.complex128)
            e1[0] = beta
            y, *_ = np.linalg.lstsq(Hh[:j + 2, :j + 1], e1, rcond=None)
            resid = np.linalg.norm(e1 - Hh[:j + 2, :j + 1] @ y)
            if Hh[j + 1, j] != 0:
                V[:, j + 1] = w / Hh[j + 1, j]
            if resid <= tol * nb or total >= max_iter or Hh[j + 1, j] == 0:
                break
        x = x + Z[:, :k_used] @ y
        r = b - prob.A(x)
    return x, total, np.linalg.norm(b - prob.A(x)) / nb

"""The simple randomized preconditioner of Sec. 2.3 (oracle).

G0 V ~ U W^H (Algorithm 2), and by the Sherman-Morrison-Woodbury formula
(I - U W^H)^-1 = I + U (I_r - W^H U)^-1 W^H, which is H of Eq. 12.  Only the
r x r matrix Z = (I_r - W^H U)^-1 is formed; H is applied as three factors.
"""
from __future__ import annotations

import numpy as np

from . import sketch


class SimplePreconditioner:
    def __init__(self, prob, rank: int, oversample: int = 10, q: int = 0, seed: int = 1):
        self.U, self.W = sketch.g0v_sketch(prob, rank, oversample, q, seed)
        r = self.U.shape[1]
        self.Z = np.linalg.inv(np.eye(r) - self.W.conj().T @ self.U)

    def apply(self, x: np.ndarray) -> np.ndarray:
        """H x = x + U (Z (W^H x))  (Eq. 12, applied as in Eq. 14)."""
        return x + self.U @ (self.Z @ (self.W.conj().T @ x))

"""Randomized HODLR approximation of I - G0 V and its inverse (oracle).

Sec. 2.4: the matrix is split in four; the two off-diagonal blocks are
approximated by Algorithm 2 with the products done by FFT, the diagonal blocks
are split again, down to dense diagonal leaves (Fig. 1).  Every block uses the
same rank r.  The inverse is formed by the 2x2 block-inverse formula applied
recursively; low-rank sums are cut back to rank r by Algorithm 1 with q = 0,
multiplying by a low-rank block B C^H as B (C^H Omega).

Cluster tree.  Every node is a rectangle of cells.  The paper splits the
strip-ordered unknowns into vertical strips (``split="strips"``).  The
``"quadtree"`` rule bisects the longer side of each box (x on ties), so square
grids alternate x and z and reach square leaves.  Unknowns are numbered in
tree order: leaves left to right, cells of a leaf in strip order inside the
leaf; for strips this is the grid's own ordering.

Storage.  Node (l, c) is node c of level l (root (0, 0); children 2c, 2c+1).
Block (l, c) is the off-diagonal block whose rows are node (l, c) and whose
columns are its sibling (l, c ^ 1): it is U[(l, c)] W[(l, c)]^H.  D[c] is the
dense leaf c of level L.

Sketch stream names (see ``philox``): block (l, c) of the build uses tag 1 and
w3 = (l << 16) | c; a recompression of block (bl, bc) inside the inversion
call of node (l, c) uses tag 3, op 0 for the Schur complement
S = D - C A^-1 B and op 1 for the top-left block A^-1 + A^-1 B S^-1 C A^-1.
"""
from __future__ import annotations

import numpy as np

from . import green, philox, sketch
from .operator import conv_fft


class Tree:
    def __init__(self, nz: int, nx: int, levels: int, split: str = "quadtree"):
        if split not in ("quadtree", "strips"):
            raise ValueError(split)
        self.nz, self.nx, self.L, self.split = nz, nx, levels, split
        self.box = {(0, 0): (0, nz, 0, nx)}
        for l in range(levels):
            for c in range(2 ** l):
                z0, z1, x0, x1 = self.box[(l, c)]
                along_x = split == "strips" or (x1 - x0) >= (z1 - z0)
                if along_x:
                    if x1 - x0 < 2:
                        raise ValueError("box too narrow to split")
                    xm = x0 + (x1 - x0) // 2
                    self.box[(l + 1, 2 * c)] = (z0, z1, x0, xm)
                    self.box[(l + 1, 2 * c + 1)] = (z0, z1, xm, x1)
                else:
                    if z1 - z0 < 2:
                        raise ValueError("box too short to split")
                    zm = z0 + (z1 - z0) // 2
                    self.box[(l + 1, 2 * c)] = (z0, zm, x0, x1)
                    self.box[(l + 1, 2 * c + 1)] = (zm, z1, x0, x1)
        perm = []
        for c in range(2 ** levels):
            z0, z1, x0, x1 = self.box[(levels, c)]
            for ix in range(x0, x1):
                perm.extend(ix * nz + iz for iz in range(z0, z1))
        self.perm = np.asarray(perm, dtype=np.int64)      # tree index -> grid index
        self.off, self.size = {}, {}
        for l in range(levels, -1, -1):
            for c in range(2 ** l):
                if l == levels:
                    z0, z1, x0, x1 = self.box[(l, c)]
                    self.size[(l, c)] = (z1 - z0) * (x1 - x0)
                else:
                    self.size[(l, c)] = self.size[(l + 1, 2 * c)] + self.size[(l + 1, 2 * c + 1)]
        for l in range(levels + 1):
            o = 0
            for c in range(2 ** l):
                self.off[(l, c)] = o
                o += self.size[(l, c)]

    def cells(self, l: int, c: int):
        """(iz, ix) of the unknowns of node (l, c), in tree order."""
        g = self.perm[self.off[(l, c)]: self.off[(l, c)] + self.size[(l, c)]]
        return g % self.nz, g // self.nz


class HODLR:
    def __init__(self, tree: Tree, rank: int):
        self.tree, self.r = tree, rank
        self.D, self.U, self.W = {}, {}, {}

    def copy_subtree(self, l: int, c: int) -> "HODLR":
        """A copy of every block inside node (l, c)."""
        out = HODLR(self.tree, self.r)
        L = self.tree.L
        for ll in range(l + 1, L + 1):
            span = 2 ** (ll - l)
            for cc in range(c * span, (c + 1) * span):
                out.U[(ll, cc)] = self.U[(ll, cc)].copy()
                out.W[(ll, cc)] = self.W[(ll, cc)].copy()
        span = 2 ** (L - l)
        for cc in range(c * span, (c + 1) * span):
            out.D[cc] = self.D[cc].copy()
        return out


# ------------------------------------------------------------------ products

def matvec(H: HODLR, l: int, c: int, x: np.ndarray) -> np.ndarray:
    """y = X x for the HODLR block X of node (l, c) (x in tree order)."""
    if l == H.tree.L:
        return H.D[c] @ x
    m1 = H.tree.size[(l + 1, 2 * c)]
    a, b = (l + 1, 2 * c), (l + 1, 2 * c + 1)
    y1 = matvec(H, *a, x[:m1]) + H.U[a] @ (H.W[a].conj().T @ x[m1:])
    y2 = H.U[b] @ (H.W[b].conj().T @ x[:m1]) + matvec(H, *b, x[m1:])
    return np.concatenate([y1, y2], axis=0)


def matvec_adj(H: HODLR, l: int, c: int, x: np.ndarray) -> np.ndarray:
    """y = X^H x for the HODLR block X of node (l, c)."""
    if l == H.tree.L:
        return H.D[c].conj().T @ x
    m1 = H.tree.size[(l + 1, 2 * c)]
    a, b = (l + 1, 2 * c), (l + 1, 2 * c + 1)
    y1 = matvec_adj(H, *a, x[:m1]) + H.W[b] @ (H.U[b].conj().T @ x[m1:])
    y2 = H.W[a] @ (H.U[a].conj().T @ x[:m1]) + matvec_adj(H, *b, x[m1:])
    return np.concatenate([y1, y2], axis=0)


def apply(H: HODLR, x: np.ndarray) -> np.ndarray:
    """H x for x in the grid's strip ordering."""
    p = H.tree.perm
    y = np.empty_like(np.asarray(x, dtype=np.complex128))
    y[p] = matvec(H, 0, 0, np.asarray(x)[p])
    return y


def assemble(H: HODLR, l: int = 0, c: int = 0) -> np.ndarray:
    """Dense matrix of node (l, c) in tree order (tests only)."""
    if l == H.tree.L:
        return H.D[c].copy()
    a, b = (l + 1, 2 * c), (l + 1, 2 * c + 1)
    return np.block([[assemble(H, *a), H.U[a] @ H.W[a].conj().T],
                     [H.U[b] @ H.W[b].conj().T, assemble(H, *b)]])


# --------------------------------------------------------------- construction

def _box_index(tree: Tree, l: int, c: int, box):
    """Positions of node (l, c)'s unknowns inside ``box`` (strip order)."""
    z0, z1, x0, _ = box
    iz, ix = tree.cells(l, c)
    return (ix - x0) * (z1 - z0) + (iz - z0)


def build(prob, tree: Tree, rank: int, oversample: int = 10, q: int = 0, seed: int = 1) -> HODLR:
    """HODLR approximation of I - G0 V (Sec. 2.4).

    Off-diagonal block (l, c) is -(G0 V)[s, t] with s = node (l, c),
    t = its sibling; it is sketched by Algorithm 2 on the parent box, which
    holds s and t, with a zero-padded FFT of twice the box's size.  Diagonal
    leaves are formed densely from the Green table."""
    H = HODLR(tree, rank)
    L = tree.L
    rp = rank + oversample
    for l in range(1, L + 1):
        for p in range(2 ** (l - 1)):
            box = tree.box[(l - 1, p)]
            pz, px = box[1] - box[0], box[3] - box[2]
            spec = green.green_spectrum(pz, px, prob.h, prob.k)
            chi_box = prob.chi.reshape(prob.nx, prob.nz)[box[2]:box[3], box[0]:box[1]].ravel()
            for c in (2 * p, 2 * p + 1):
                s, t = (l, c), (l, c ^ 1)
                si, ti = _box_index(tree, *s, box), _box_index(tree, *t, box)
                chi_t = chi_box[ti]

                def A(X, si=si, ti=ti, chi_t=chi_t):     # (G0 V)[s, t] X
                    w = np.zeros((pz * px, X.shape[1]), dtype=np.complex128)
                    w[ti] = chi_t[:, None] * X
                    return conv_fft(spec, w, pz, px)[si]

                def AH(X, si=si, ti=ti, chi_t=chi_t):    # (G0 V)[s, t]^H X
                    w = np.zeros((pz * px, X.shape[1]), dtype=np.complex128)
                    w[si] = np.conj(X)
                    return chi_t[:, None] * np.conj(conv_fft(spec, w, pz, px)[ti])

                w2, w3 = philox.stream_words(philox.TAG_BUILD, blvl=l, bnode=c)
                Omega = philox.gaussian(tree.size[t], rp, seed, w2, w3)
                Q, Yt = sketch.range_finder(A, AH, Omega, q)
                U, W = sketch.truncate(Q, Yt, rank)
                H.U[s], H.W[s] = -U, W
    for c in range(2 ** L):
        iz, ix = tree.cells(L, c)
        G = green.green_block(iz, ix, iz, ix, prob.h, prob.k)
        chi = prob.chi[ix * prob.nz + iz]
        H.D[c] = np.eye(iz.size, dtype=np.complex128) - G * chi[None, :]
    return H


# ------------------------------------------------------------------ inversion

def _recompress(Uc, Wc, rank, oversample, seed, w2, w3):
    """Rank-r approximation of the low-rank sum Uc Wc^H by Algorithm 1 with
    q = 0, every product taken through the factors."""
    Omega = philox.gaussian(Wc.shape[0], rank + oversample, seed, w2, w3)
    Q, Yt = sketch.range_finder(lambda X: Uc @ (Wc.conj().T @ X),
                                lambda X: Wc @ (Uc.conj().T @ X), Omega, 0)
    return sketch.truncate(Q, Yt, rank)


def add_lowrank(M: HODLR, l: int, c: int, X: np.ndarray, Y: np.ndarray,
                op: int, call, oversample: int, seed: int) -> None:
    """M[node (l, c)] += X Y^H in place, keeping every off-diagonal block at
    rank r.  ``call`` = (level, node) of the inversion call that asks."""
    if l == M.tree.L:
        M.D[c] = M.D[c] + X @ Y.conj().T
        return
    m1 = M.tree.size[(l + 1, 2 * c)]
    a, b = (l + 1, 2 * c), (l + 1, 2 * c + 1)
    X1, X2, Y1, Y2 = X[:m1], X[m1:], Y[:m1], Y[m1:]
    for blk, Xs, Yt_ in ((a, X1, Y2), (b, X2, Y1)):
        w2, w3 = philox.stream_words(philox.TAG_RECOMPRESS, op, call[0], call[1], blk[0], blk[1])
        Uc = np.concatenate([M.U[blk], Xs], axis=1)
        Wc = np.concatenate([M.W[blk], Yt_], axis=1)
        M.U[blk], M.W[blk] = _recompress(Uc, Wc, M.r, oversample, seed, w2, w3)
    add_lowrank(M, *a, X1, Y1, op, call, oversample, seed)
    add_lowrank(M, *b, X2, Y2, op, call, oversample, seed)


def _invert_node(X: HODLR, l: int, c: int, Hi: HODLR, oversample: int, seed: int) -> None:
    """Write the inverse of node (l, c) of X into the same node of Hi.

    [[A, B], [C, D]]^-1 with S = D - C A^-1 B:
        top-left      A^-1 + A^-1 B S^-1 C A^-1
        top-right    -A^-1 B S^-1
        bottom-left  -S^-1 C A^-1
        bottom-right  S^-1
    (the block-inverse formula of Sec. 2.4; its top-right block is printed as
    -B A^-1 S^-1, read here in the standard Schur-complement form)."""
    L = X.tree.L
    if l == L:
        Hi.D[c] = np.linalg.inv(X.D[c])
        return
    a, b = (l + 1, 2 * c), (l + 1, 2 * c + 1)
    UB, WB = X.U[a], X.W[a]            # B = UB WB^H
    UC, WC = X.U[b], X.W[b]            # C = UC WC^H
    _invert_node(X, *a, Hi, oversample, seed)            # A^-1 into Hi
    P = matvec(Hi, *a, UB)                                # A^-1 UB
    R = matvec_adj(Hi, *a, WC)                            # A^-H WC
    K = WC.conj().T @ P                                   # WC^H A^-1 UB
    S = X.copy_subtree(*b)
    add_lowrank(S, *b, -(UC @ K), WB, 0, (l, c), oversample, seed)
    _invert_node(S, *b, Hi, oversample, seed)            # S^-1 into Hi
    T1 = matvec(Hi, *b, UC)                               # S^-1 UC
    T2 = matvec_adj(Hi, *b, WB)                           # S^-H WB
    K2 = WB.conj().T @ T1                                 # WB^H S^-1 UC
    add_lowrank(Hi, *a, P @ K2, R, 1, (l, c), oversample, seed)
    Hi.U[a], Hi.W[a] = -P, T2
    Hi.U[b], Hi.W[b] = -T1, R


def invert(X: HODLR, oversample: int = 10, seed: int = 1) -> HODLR:
    """Approximate inverse of a HODLR matrix, with the same structure."""
    Hi = HODLR(X.tree, X.r)
    _invert_node(X, 0, 0, Hi, oversample, seed)
    return Hi


class HODLRPreconditioner:
    """H ~ (I - G0 V)^-1 as a HODLR matrix (Sec. 2.4), used as H in Eq. 11."""

    def __init__(self, prob, levels: int, rank: int, oversample: int = 10, q: int = 0,
                 seed: int = 1, split: str = "quadtree"):
        self.tree = Tree(prob.nz, prob.nx, levels, split)
        self.A = build(prob, self.tree, rank, oversample, q, seed)
        self.H = invert(self.A, oversample, seed)

    def apply(self, x: np.ndarray) -> np.ndarray:
        return apply(self.H, x)

"""Pins of the oracle against facts that do not come from the oracle itself:
closed forms, published tables and known-answer vectors, exact identities of
the method, brute force on tiny grids.  CPU only."""
import os

import numpy as np
import pytest
from scipy import integrate, special

from oracle import green, hodlr, philox, sketch, smw, solve
from oracle import operator as op
from paper_2005_01372_gb300 import media

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _rel(a, b):
    return np.linalg.norm(np.asarray(a) - np.asarray(b)) / np.linalg.norm(np.asarray(b))


def _small_problem(nz, nx, seed=0, freq=10.0, h=10.0, scale=1.0):
    rng = np.random.default_rng(seed)
    c = media.random_field(rng, nz, nx)
    c = media.C0 + scale * (c - media.C0)
    return op.Problem(nz, nx, h, media.C0, freq, c)


# ------------------------------------------------------------ p1: Green table

def test_bessel_tables_abramowitz_stegun():
    """The Bessel functions the Green table is built from agree with A&S 9.1."""
    rows = np.loadtxt(os.path.join(GOLDEN, "bessel_tables.txt"))
    for x, j0, j1, y0, y1 in rows:
        assert special.jv(0, x) == pytest.approx(j0, abs=6e-11)
        assert special.jv(1, x) == pytest.approx(j1, abs=6e-11)
        assert special.yv(0, x) == pytest.approx(y0, abs=6e-11)
        assert special.yv(1, x) == pytest.approx(y1, abs=6e-11)


@pytest.mark.parametrize("freq", [2.0, 10.0, 30.0])
def test_self_term_equals_disk_quadrature(freq):
    """Gt(0) = integral of (i/4) H0(k rho) over the disk of area h^2."""
    h, c0 = 10.0, 2000.0
    k = 2 * np.pi * freq / c0
    a = h / np.sqrt(np.pi)
    f_re = lambda rho: 2 * np.pi * rho * np.real(0.25j * special.hankel1(0, k * rho))
    f_im = lambda rho: 2 * np.pi * rho * np.imag(0.25j * special.hankel1(0, k * rho))
    q = integrate.quad(f_re, 0, a, limit=200, epsabs=1e-13, epsrel=1e-13)[0] + \
        1j * integrate.quad(f_im, 0, a, limit=200, epsabs=1e-13, epsrel=1e-13)[0]
    g = green.green_of_distance(np.array([0.0]), k, h)[0]
    assert abs(g - q) <= 1e-12 * abs(q)


@pytest.mark.parametrize("r_cells", [1.0, np.sqrt(2.0), 3.0, 7.5])
def test_off_diagonal_equals_disk_quadrature(r_cells):
    """Gt(r) = integral of (i/4) H0(k |x - x'|) over the disk around x'."""
    h, k = 10.0, 2 * np.pi * 15.0 / 2000.0
    a = h / np.sqrt(np.pi)
    r = r_cells * h

    def integrand(th, rho, part):
        d = np.sqrt(r * r + rho * rho - 2 * r * rho * np.cos(th))
        v = 0.25j * special.hankel1(0, k * d) * rho
        return v.real if part == 0 else v.imag

    re = integrate.dblquad(integrand, 0, a, 0, 2 * np.pi, args=(0,), epsabs=1e-12, epsrel=1e-12)[0]
    im = integrate.dblquad(integrand, 0, a, 0, 2 * np.pi, args=(1,), epsabs=1e-12, epsrel=1e-12)[0]
    g = green.green_of_distance(np.array([r]), k, h)[0]
    assert abs(g - (re + 1j * im)) <= 1e-10 * abs(g)


def test_green_is_hankel_closed_form_far_field():
    """Off the source cell the point-source field is (i/4) H0(k r) times the
    disk factor 2 J1(ka)/(ka), and that factor tends to 1 as ka -> 0."""
    nz, nx, h, k = 9, 7, 10.0, 2 * np.pi * 10 / 2000
    psi0 = green.point_source(nz, nx, h, k, 4, 3)
    iz, ix = green.cell_coords(nz, nx)
    r = h * np.hypot(iz - 4, ix - 3)
    a = h / np.sqrt(np.pi)
    m = r > 0
    ref = 0.25j * special.hankel1(0, k * r[m]) * 2 * special.jv(1, k * a) / (k * a)
    assert np.max(np.abs(psi0[m] - ref) / np.abs(ref)) < 1e-13
    ka = 1e-4
    assert 2 * special.jv(1, ka) / ka == pytest.approx(1.0, abs=1e-8)


def test_contrast_satisfies_eq1():
    c = np.array([1500.0, 2000.0, 4500.0])
    chi = green.contrast(c, 2000.0, 12.0)
    w = 2 * np.pi * 12.0
    np.testing.assert_allclose(w ** 2 / c ** 2, w ** 2 / 2000.0 ** 2 + chi, rtol=1e-15)
    assert chi[1] == 0.0 and chi[0] > 0 > chi[2]


# ------------------------------------------------ p2, p3: reciprocity and FFT

def test_dense_green_is_symmetric():
    Gd = green.green_dense(7, 5, 10.0, 0.03)
    assert np.array_equal(Gd, Gd.T)


@pytest.mark.parametrize("nz,nx", [(1, 1), (2, 3), (5, 4), (7, 7), (9, 16), (16, 16), (16, 11)])
def test_fft_operator_equals_dense_sum(nz, nx):
    """Brute force: the FFT convolution of Sec. 2.2 equals the direct O(n^2)
    sum of Eq. 4 on every grid up to 16 x 16, odd and non-square included."""
    P = _small_problem(nz, nx, seed=nz * 31 + nx)
    Gd = green.green_dense(nz, nx, P.h, P.k)
    rng = np.random.default_rng(1)
    u = media.complex_field(rng, (P.n, 3))
    ref = op.apply_dense(Gd, P.chi, u)
    assert _rel(P.G0V(u), ref) < 1e-13


def test_fft_operator_reciprocity():
    """y^T Gt x = x^T Gt y (unconjugated) through the FFT path."""
    nz, nx = 13, 10
    spec = green.green_spectrum(nz, nx, 10.0, 0.04)
    rng = np.random.default_rng(2)
    x, y = media.complex_field(rng, nz * nx), media.complex_field(rng, nz * nx)
    lhs = y @ op.conv_fft(spec, x, nz, nx)
    rhs = x @ op.conv_fft(spec, y, nz, nx)
    assert abs(lhs - rhs) <= 1e-12 * abs(lhs)


def test_adjoint_is_conjugate_transpose():
    P = _small_problem(8, 6, seed=3)
    Gd = green.green_dense(8, 6, P.h, P.k)
    M = Gd * P.chi[None, :]
    rng = np.random.default_rng(4)
    x = media.complex_field(rng, (P.n, 2))
    assert _rel(P.G0V_adj(x), M.conj().T @ x) < 1e-13


def test_operator_modes():
    P = _small_problem(6, 5, seed=5)
    rng = np.random.default_rng(6)
    u, u0 = media.complex_field(rng, (P.n, 2)), media.complex_field(rng, (P.n, 2))
    g = P.G0V(u)
    np.testing.assert_allclose(op.apply(op.FORWARD, P.spec, P.chi, u, u0, 6, 5), u0 + g)
    np.testing.assert_allclose(op.apply(op.RESIDUAL, P.spec, P.chi, u, u0, 6, 5), u - g - u0)
    np.testing.assert_allclose(op.apply(op.PLAIN, P.spec, P.chi, u, None, 6, 5), g)


def test_green_spectrum_is_even():
    """The even extension has an even (quarter-symmetric) spectrum."""
    nz, nx = 6, 10
    S = green.green_spectrum(nz, nx, 10.0, 0.05)
    kz = (-np.arange(2 * nz)) % (2 * nz)
    kx = (-np.arange(2 * nx)) % (2 * nx)
    assert np.max(np.abs(S - S[kx, :])) < 1e-12 * np.max(np.abs(S))
    assert np.max(np.abs(S - S[:, kz])) < 1e-12 * np.max(np.abs(S))


# ------------------------------------------------------- p4: zero contrast

def test_zero_contrast():
    P = op.Problem(8, 8, 10.0, 2000.0, 10.0, np.full((8, 8), 2000.0))
    assert np.all(P.chi == 0)
    u0 = P.sources([(2, 3)])[:, 0]
    assert np.all(P.G0V(u0) == 0)
    psi, it, res = solve.series(P, u0, None, 1e-12, 5)
    assert it == 0 and np.array_equal(psi, u0)
    tree = hodlr.Tree(8, 8, 2)
    A = hodlr.build(P, tree, 4, 2, 0, 9)
    for key in A.U:
        assert np.all(A.U[key] == 0)


def test_zero_contrast_embedding_is_exact():
    """A model embedded in a larger grid of background velocity: cells of
    zero contrast do not scatter, so inside the model the direct solution
    on the larger grid equals the one on the model's own grid (the model
    need not have power-of-two sides), and outside it is psi0 plus the field
    the model scatters there."""
    rng = np.random.default_rng(11)
    c = media.random_field(rng, 12, 30)
    Pm = op.Problem(12, 30, 15.0, media.C0, 6.0, c)
    Pe = op.Problem(16, 32, 15.0, media.C0, 6.0, media.embed(c, 16, 32))
    src = [(0, 15)]
    um = solve.direct(Pm, Pm.sources(src))[:, 0]
    ue = solve.direct(Pe, Pe.sources(src))[:, 0]
    inside = np.array([ix * 16 + iz for ix in range(30) for iz in range(12)])
    assert _rel(ue[inside], um) < 1e-12
    outside = np.setdiff1d(np.arange(Pe.n), inside)
    assert _rel(ue[outside], (Pe.sources(src)[:, 0] + Pe.G0V(ue))[outside]) < 1e-12
    assert np.all(Pe.chi[outside] == 0)


# ----------------------------------------- p5, p6: Born, direct, the series

def test_direct_solve_residual():
    P = _small_problem(12, 12, seed=7)
    u0 = P.sources([(1, 6)])
    psi = solve.direct(P, u0)
    assert P.rel_residual(psi, u0)[0] < 1e-13


def test_born_equals_neumann_series_and_lu():
    """At small contrast the Born series converges to the LU solution and its
    error falls geometrically at about the spectral radius of G0 V."""
    P = _small_problem(12, 12, seed=8, freq=4.0, scale=0.3)
    A = P.dense_A()
    rho = np.max(np.abs(np.linalg.eigvals(np.eye(P.n) - A)))
    assert rho < 0.3
    u0 = P.sources([(0, 5)])[:, 0]
    exact = np.linalg.solve(A, u0)
    psi = u0.copy()
    errs = []
    for _ in range(12):
        psi = u0 + P.G0V(psi)
        errs.append(np.linalg.norm(psi - exact))
    assert errs[-1] / np.linalg.norm(exact) < 1e-8
    ratio = (errs[-1] / errs[-6]) ** (1 / 5)
    assert ratio <= rho * 1.05


def test_series_with_exact_inverse_is_one_step():
    """With H = (I - G0 V)^-1, M = 0 in Eq. 7 and psi_0 = H psi0 is exact."""
    P = _small_problem(8, 8, seed=9, freq=20.0)
    Hd = np.linalg.inv(P.dense_A())
    u0 = P.sources([(0, 2), (3, 3)])
    psi, it, res = solve.series(P, u0, lambda x: Hd @ x, 1e-10, 5)
    assert np.all(it == 0) and np.all(res < 1e-12)


def test_series_is_homotopy_series_sum():
    """Eq. 11 started at H psi0 reproduces the partial sums of Eq. 9,
    sum_n M^n H psi0 with M = I - H + H G0 V (Eq. 7)."""
    P = _small_problem(6, 6, seed=10, freq=15.0)
    rng = np.random.default_rng(11)
    Hm = np.eye(P.n) * 0.7 + 0.01 * media.complex_field(rng, (P.n, P.n))
    A = P.dense_A()
    M = np.eye(P.n) - Hm @ A
    u0 = P.sources([(1, 1)])[:, 0]
    psi = Hm @ u0
    partial, term = Hm @ u0, Hm @ u0
    for _ in range(6):
        a = psi - P.G0V(psi) - u0
        psi = psi - Hm @ a
        term = M @ term
        partial = partial + term
    assert _rel(psi, partial) < 1e-12


def test_fgmres_matches_lu():
    P = _small_problem(10, 10, seed=12, freq=25.0)
    u0 = P.sources([(0, 4)])[:, 0]
    x, it, res = solve.fgmres(P, u0, None, 1e-12, 40, 400)
    assert res < 1e-11
    assert _rel(x, np.linalg.solve(P.dense_A(), u0)) < 1e-9


# -------------------------------------------------------- Philox and probes

def test_philox_known_answers():
    rows = [l.split() for l in open(os.path.join(GOLDEN, "philox4x32_10_kat.txt"))
            if l.strip() and not l.startswith("#")]
    for row in rows:
        v = [int(t, 16) for t in row]
        out = philox.philox4x32_10(tuple(v[0:4]), (v[4], v[5]))
        assert [int(o) for o in out] == v[6:10]


def test_gaussian_probe_statistics():
    g = philox.gaussian(2000, 64, 123, *philox.stream_words(1, blvl=3, bnode=5))
    assert abs(np.mean(np.abs(g) ** 2) - 1) < 0.02
    assert abs(np.var(g.real) - 0.5) < 0.02 and abs(np.var(g.imag) - 0.5) < 0.02
    assert abs(np.mean(g)) < 0.02
    assert abs(np.mean(g.real * g.imag)) < 0.02
    # distinct streams and seeds give distinct numbers
    h = philox.gaussian(2000, 64, 123, *philox.stream_words(1, blvl=3, bnode=4))
    assert np.max(np.abs(g - h)) > 1
    # entry (i, j) does not depend on the block's size
    small = philox.gaussian(7, 3, 123, *philox.stream_words(1, blvl=3, bnode=5))
    assert np.array_equal(small, g[:7, :3])


# ------------------------------------------ p7, p8: sketches and SMW

def test_sketch_exact_recovery_on_low_rank_contrast():
    """chi supported on k cells => rank(G0 V) <= k, and Algorithm 2 with at
    least k probes reproduces G0 V to rounding (q = 0 and q = 1)."""
    nz, nx = 10, 9
    c = np.full((nx, nz), 2000.0)
    rng = np.random.default_rng(13)
    cells = rng.choice(nz * nx, size=7, replace=False)
    c.ravel()[cells] = rng.uniform(1500, 4500, size=7)
    P = op.Problem(nz, nx, 10.0, 2000.0, 12.0, c)
    M = green.green_dense(nz, nx, P.h, P.k) * P.chi[None, :]
    for q in (0, 1):
        U, W = sketch.g0v_sketch(P, 7, 3, q, 77)
        assert _rel(U @ W.conj().T, M) < 1e-12


def test_truncation_is_best_rank_r():
    """Eckart-Young: the truncation error is the (r+1)-th singular value."""
    rng = np.random.default_rng(14)
    Q, _ = np.linalg.qr(media.complex_field(rng, (50, 12)))
    Yt = media.complex_field(rng, (40, 12))
    U, W = sketch.truncate(Q, Yt, 5)
    s = np.linalg.svd(Q @ Yt.conj().T, compute_uv=False)
    assert np.linalg.norm(Q @ Yt.conj().T - U @ W.conj().T, 2) == pytest.approx(s[5], rel=1e-10)


def test_smw_identity():
    """(I - U W^H)(I + U Z W^H) = I with Z = (I - W^H U)^-1 (Eq. 12)."""
    P = _small_problem(8, 8, seed=15, freq=8.0)
    pc = smw.SimplePreconditioner(P, 12, 4, 0, 5)
    rng = np.random.default_rng(16)
    x = media.complex_field(rng, (P.n, 3))
    y = pc.apply(x)
    back = y - pc.U @ (pc.W.conj().T @ y)
    assert _rel(back, x) < 1e-12


# ------------------------------------------------ p9 - p11: HODLR

@pytest.mark.parametrize("split", ["quadtree", "strips"])
def test_tree_is_a_permutation(split):
    t = hodlr.Tree(16, 16, 4, split)
    assert np.array_equal(np.sort(t.perm), np.arange(256))
    if split == "strips":
        assert np.array_equal(t.perm, np.arange(256))
    else:
        assert t.box[(4, 0)] == (0, 4, 0, 4)
    for l in range(5):
        assert sum(t.size[(l, c)] for c in range(2 ** l)) == 256


def test_quadtree_leaves_of_the_256_grid():
    t = hodlr.Tree(256, 256, 6, "quadtree")
    assert all(t.size[(6, c)] == 1024 for c in range(64))
    z0, z1, x0, x1 = t.box[(6, 0)]
    assert (z1 - z0, x1 - x0) == (32, 32)


@pytest.mark.parametrize("split", ["quadtree", "strips"])
def test_full_rank_hodlr_is_exact(split):
    """Rank >= block size: the HODLR is I - G0 V itself, its inverse the dense
    inverse, and the preconditioned series stops at once (M = 0)."""
    P = _small_problem(8, 8, seed=17, freq=15.0)
    t = hodlr.Tree(8, 8, 2, split)
    A = hodlr.build(P, t, 40, 8, 0, 3)
    Ad = P.dense_A()[np.ix_(t.perm, t.perm)]
    assert _rel(hodlr.assemble(A), Ad) < 1e-13
    Hi = hodlr.invert(A, 8, 3)
    assert _rel(hodlr.assemble(Hi), np.linalg.inv(Ad)) < 1e-11
    u0 = P.sources([(0, 3)])
    pc = hodlr.HODLRPreconditioner(P, 2, 40, 8, 0, 3, split)
    psi, it, res = solve.series(P, u0, pc.apply, 1e-10, 3)
    assert it[0] == 0 and res[0] < 1e-11


def test_hodlr_matvec_matches_assembly():
    P = _small_problem(16, 8, seed=18, freq=20.0)
    t = hodlr.Tree(16, 8, 3)
    A = hodlr.build(P, t, 5, 3, 0, 4)
    rng = np.random.default_rng(19)
    x = media.complex_field(rng, (P.n, 2))
    D = hodlr.assemble(A)
    assert _rel(hodlr.matvec(A, 0, 0, x), D @ x) < 1e-13
    assert _rel(hodlr.matvec_adj(A, 0, 0, x), D.conj().T @ x) < 1e-13
    xg = np.empty_like(x)
    xg[t.perm] = x
    yg = hodlr.apply(A, xg)
    assert _rel(yg[t.perm], D @ x) < 1e-13


def test_block_inverse_formula():
    """The recursive 2x2 block inverse (with the Schur-complement reading of
    the top-right block) against numpy's inverse, on exact low-rank blocks."""
    rng = np.random.default_rng(20)
    t = hodlr.Tree(4, 8, 1, "strips")
    m = 16
    X = hodlr.HODLR(t, 16)
    X.D[0] = np.eye(m) * 3 + media.complex_field(rng, (m, m))
    X.D[1] = np.eye(m) * 3 + media.complex_field(rng, (m, m))
    for c in (0, 1):
        X.U[(1, c)] = media.complex_field(rng, (m, 16)) * 0.2
        X.W[(1, c)] = media.complex_field(rng, (m, 16)) * 0.2
    Xd = hodlr.assemble(X)
    Hi = hodlr.invert(X, 4, 1)
    assert _rel(hodlr.assemble(Hi), np.linalg.inv(Xd)) < 1e-12
    # the top-right block as printed, -B A^-1 S^-1 (shapes agree here), is not the inverse
    A, D = X.D[0], X.D[1]
    B = X.U[(1, 0)] @ X.W[(1, 0)].conj().T
    C = X.U[(1, 1)] @ X.W[(1, 1)].conj().T
    S = D - C @ np.linalg.solve(A, B)
    printed = -B @ np.linalg.inv(A) @ np.linalg.inv(S)
    assert _rel(printed, np.linalg.inv(Xd)[:m, m:]) > 1e-3


def test_recompressed_inverse_is_exact_when_the_ranks_fit():
    """Three levels of the recursive inversion with truncation at work:
    every off-diagonal block of X has rank 1 and is stored with r = 6
    columns, so each low-rank sum the inversion forms (2r = 12 columns) has
    true rank at most one per ancestor level plus one, below r; Algorithm 1
    with 4 extra probes then recovers each sum exactly, and the recursive
    inverse equals numpy's inverse."""
    rng = np.random.default_rng(23)
    t = hodlr.Tree(8, 8, 3, "strips")
    r = 6
    X = hodlr.HODLR(t, r)
    for c in range(8):
        X.D[c] = np.eye(8) * 4 + media.complex_field(rng, (8, 8))
    for l in (1, 2, 3):
        for c in range(2 ** l):
            m = t.size[(l, c)]
            U = np.zeros((m, r), complex)
            W = np.zeros((m, r), complex)
            U[:, 0] = media.complex_field(rng, m) * 0.3
            W[:, 0] = media.complex_field(rng, m) * 0.3
            X.U[(l, c)], X.W[(l, c)] = U, W
    Xd = hodlr.assemble(X)
    Hi = hodlr.invert(X, 4, 1)
    assert _rel(hodlr.assemble(Hi), np.linalg.inv(Xd)) < 1e-11
    # and a rank too small for the sums (r = 1 storage of the same blocks) is not exact
    X1 = hodlr.HODLR(t, 1)
    X1.D = dict(X.D)
    for key in X.U:
        X1.U[key], X1.W[key] = X.U[key][:, :1], X.W[key][:, :1]
    Hi1 = hodlr.invert(X1, 0, 1)
    assert _rel(hodlr.assemble(Hi1), np.linalg.inv(Xd)) > 1e-6


def test_hodlr_preconditioned_series_matches_lu_on_64_grid():
    """The paper's verification (Sec. 3.1): the preconditioned series gives
    the direct solution.  64 x 64 Gaussian inclusion, 10 Hz, 2 levels of
    32 x 32 leaves, rank 20 + 10."""
    wl = media.gaussian_inclusion_64()
    P = op.Problem.from_workload(wl)
    u0 = P.sources(wl.sources)
    pc = hodlr.HODLRPreconditioner(P, 2, 20, 10, 0, 1001)
    psi, it, res = solve.series(P, u0, pc.apply, 1e-10, 30)
    assert res[0] < 1e-10
    # Born converges here too (spectral radius below 1), to the same field
    psi_b, it_b, res_b = solve.series(P, u0, None, 1e-10, 200)
    assert res_b[0] < 1e-10
    assert _rel(psi, psi_b) < 1e-8

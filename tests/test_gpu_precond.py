"""Parity of the CUDA sketches, preconditioners and solvers with the oracle.

Both sides draw the same Philox4x32-10 probes, so randomized results are
compared directly.  Low-rank factors are unique only up to U W^H, so the
products are compared, never U or W alone.  Tolerances: 1e-10 (FP64 paths);
1e-5 for FP32 sketches and FP32 H-matrices (the sketches' QR, Gram and
eigen-decomposition are FP64, only the tall factors are FP32); an FP32
approximate inverse of a matrix of condition number kappa carries a relative
error of order kappa u32 (u32 = 2^-24, the first-order perturbation bound of
an inverse), so an FP32 H of a worse-conditioned matrix is held to
max(1e-5, 16 kappa u32) with kappa estimated from the oracle; mixed-precision
solves are held to their FP64 residual."""
import numpy as np
import pytest

from oracle import green as og
from oracle import hodlr as oh
from oracle import operator as oop
from oracle import philox, sketch, smw, solve
from paper_2005_01372_gb300 import media

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def lsw():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2005_01372_gb300 import lsw as L
    L.lib()
    return L


def _rel(a, b):
    a, b = np.asarray(a), np.asarray(b)
    return np.linalg.norm(a - b) / np.linalg.norm(b)


def _setup(lsw, nz, nx, seed=0, freq=15.0, velocity=None):
    rng = np.random.default_rng(seed)
    c = media.random_field(rng, nz, nx) if velocity is None else velocity
    P = oop.Problem(nz, nx, 10.0, media.C0, freq, c)
    G = lsw.build_green(nz, nx, 10.0, media.C0, freq)
    chi = torch.from_numpy(P.chi.copy()).cuda()
    return P, G, chi


U32 = 2.0 ** -24


def _power_norm(f, n, iters=30, seed=0):
    """Largest |eigenvalue| of the linear map f by power iteration (a lower
    bound of its 2-norm)."""
    rng = np.random.default_rng(seed)
    x = rng.standard_normal(n) + 1j * rng.standard_normal(n)
    x /= np.linalg.norm(x)
    s = 0.0
    for _ in range(iters):
        y = f(x)
        s = np.linalg.norm(y)
        x = y / s
    return s


def _fp32_h_tol(P, ref):
    """max(1e-5, 16 kappa u32) with kappa = ||A||_2 ||A^-1||_2 of
    A = I - G0 V: ||A||_2 from power iteration on A^H A (oracle FFT
    operator), ||A^-1||_2 from the spectral radius of the oracle's H ~ A^-1
    (a lower bound, so the tolerance errs on the strict side)."""
    def AHA(x):
        y = x - oop.apply(oop.PLAIN, P.spec, P.chi, x[:, None], None, P.nz, P.nx)[:, 0]
        return y - oop.apply(oop.ADJOINT, P.spec, P.chi, y[:, None], None, P.nz, P.nx)[:, 0]
    na = np.sqrt(_power_norm(AHA, P.n))
    nh = _power_norm(lambda v: ref.apply(v[:, None])[:, 0], P.n)
    return max(1e-5, 16.0 * na * nh * U32)


def _box_cells(b, nz):
    z0, z1, x0, x1 = b
    return np.array([ix * nz + iz for ix in range(x0, x1) for iz in range(z0, z1)])


def _oracle_block_sketch(P, s, t, rank, over, q, seed, stream_id):
    rows, cols = _box_cells(s, P.nz), _box_cells(t, P.nz)
    Gd = og.green_dense(P.nz, P.nx, P.h, P.k)
    M = Gd[np.ix_(rows, cols)] * P.chi[cols][None, :]
    w2, w3 = philox.stream_words(philox.TAG_GLOBAL, bnode=0)
    Om = philox.gaussian(cols.size, rank + over, seed, w2, stream_id)
    Q, Yt = sketch.range_finder(lambda X: M @ X, lambda X: M.conj().T @ X, Om, q)
    U, W = sketch.truncate(Q, Yt, rank)
    return U @ W.conj().T, M


@pytest.mark.parametrize("prec,tol", [("c128", 1e-10), ("c64", 1e-5)])
@pytest.mark.parametrize("s,t,q", [((0, 16, 0, 8), (0, 16, 8, 16), 0), ((0, 8, 0, 16), (8, 16, 0, 16), 1),
                                   ((0, 16, 0, 16), (0, 16, 0, 16), 0), ((2, 9, 1, 4), (10, 15, 9, 16), 0)])
def test_sketch_block_parity(lsw, prec, tol, s, t, q):
    P, G, chi = _setup(lsw, 16, 16, seed=3)
    p = lsw.C128 if prec == "c128" else lsw.C64
    U, W = lsw.sketch_range(G, chi, s, t, 12, 6, q, 77, stream_id=5, prec=p)
    UW = (U.cpu().numpy().T.astype(np.complex128)) @ W.cpu().numpy().T.astype(np.complex128).conj().T
    ref, M = _oracle_block_sketch(P, s, t, 12, 6, q, 77, 5)
    assert _rel(UW, ref) < tol


@pytest.mark.parametrize("prec,tol", [("c128", 1e-12), ("c64", 1e-5)])
def test_sketch_exact_recovery(lsw, prec, tol):
    """chi on 7 cells: rank(G0 V) <= 7, recovered to rounding by 7 + 3 probes.
    The 10-column sketch has exact rank 7, so its Gram matrix is singular:
    in complex64 this exercises the shifted first pass of the Cholesky QR."""
    nz = nx = 16
    c = np.full((nx, nz), 2000.0)
    rng = np.random.default_rng(13)
    c.ravel()[rng.choice(256, size=7, replace=False)] = rng.uniform(1500, 4500, size=7)
    P, G, chi = _setup(lsw, nz, nx, velocity=c, freq=12.0)
    p = lsw.C128 if prec == "c128" else lsw.C64
    U, W = lsw.sketch_range(G, chi, (0, 16, 0, 16), (0, 16, 0, 16), 7, 3, 0, 5, prec=p)
    UW = U.cpu().numpy().T.astype(np.complex128) @ W.cpu().numpy().T.astype(np.complex128).conj().T
    M = og.green_dense(nz, nx, P.h, P.k) * P.chi[None, :]
    assert np.all(np.isfinite(UW))
    assert _rel(UW, M) < tol


def test_smw_parity(lsw):
    P, G, chi = _setup(lsw, 32, 32, seed=4, freq=5.0)
    H = lsw.build_hmatrix(G, chi, lsw.HParams(kind=lsw.H_LOWRANK_SMW, prec=lsw.C128, rank=24, oversample=8,
                                              q=1, seed=11))
    ref = smw.SimplePreconditioner(P, 24, 8, 1, 11)
    rng = np.random.default_rng(5)
    x = media.complex_field(rng, (3, P.n))
    y = lsw.apply_precond(H, torch.from_numpy(x).cuda()).cpu().numpy()
    assert _rel(y, ref.apply(x.T).T) < 1e-10


@pytest.mark.parametrize("nz,nx,L,split,r,over", [(16, 16, 2, "quadtree", 6, 4), (32, 32, 3, "quadtree", 8, 4),
                                                  (16, 32, 3, "strips", 8, 4), (32, 16, 2, "quadtree", 10, 6)])
def test_hodlr_parity_c128(lsw, nz, nx, L, split, r, over):
    P, G, chi = _setup(lsw, nz, nx, seed=nz + 3 * nx + L, freq=20.0)
    sp = lsw.SPLIT_QUADTREE if split == "quadtree" else lsw.SPLIT_STRIPS
    H = lsw.build_hmatrix(G, chi, lsw.HParams(kind=lsw.H_HODLR, prec=lsw.C128, levels=L, split=sp, rank=r,
                                              oversample=over, seed=21))
    ref = oh.HODLRPreconditioner(P, L, r, over, 0, 21, split)
    rng = np.random.default_rng(6)
    x = media.complex_field(rng, (4, P.n))
    y = lsw.apply_precond(H, torch.from_numpy(x).cuda()).cpu().numpy()
    assert _rel(y, ref.apply(x.T).T) < 1e-10


def test_hodlr_full_rank_is_dense_inverse(lsw):
    """Rank >= block size: H is (I - G0 V)^-1 itself."""
    P, G, chi = _setup(lsw, 8, 8, seed=7, freq=15.0)
    H = lsw.build_hmatrix(G, chi, lsw.HParams(kind=lsw.H_HODLR, prec=lsw.C128, levels=2, rank=32, oversample=8,
                                              seed=3))
    rng = np.random.default_rng(8)
    x = media.complex_field(rng, (2, P.n))
    y = lsw.apply_precond(H, torch.from_numpy(x).cuda()).cpu().numpy()
    ref = np.linalg.solve(P.dense_A(), x.T).T
    assert _rel(y, ref) < 1e-10


def test_hodlr_parity_c64(lsw):
    P, G, chi = _setup(lsw, 32, 32, seed=9, freq=20.0)
    H = lsw.build_hmatrix(G, chi, lsw.HParams(kind=lsw.H_HODLR, prec=lsw.C64, levels=2, rank=12, oversample=6,
                                              seed=31))
    ref = oh.HODLRPreconditioner(P, 2, 12, 6, 0, 31, "quadtree")
    rng = np.random.default_rng(10)
    x = media.complex_field(rng, (2, P.n)).astype(np.complex64)
    y = lsw.apply_precond(H, torch.from_numpy(x).cuda()).cpu().numpy()
    assert _rel(y, ref.apply(x.T.astype(np.complex128)).T) < 1e-5


def test_born_series_parity(lsw):
    wl = media.gaussian_inclusion_64()
    P, G, chi = _setup(lsw, 64, 64, velocity=wl.velocity, freq=wl.freq_hz)
    u0 = G.point_sources(wl.sources, lsw.C128)
    u, infos = lsw.solve_series(G, chi, None, u0, sp=lsw.SolveParams(prec=lsw.C128, tol=1e-10, max_iter=200))
    psi, it, res = solve.series(P, P.sources(wl.sources), None, 1e-10, 200)
    assert infos[0].status == 0 and infos[0].iterations == it[0]
    assert _rel(u.cpu().numpy()[0], psi[:, 0]) < 1e-10
    assert infos[0].rel_residual == pytest.approx(res[0], rel=1e-6)


def test_hodlr_series_matches_lu(lsw):
    """The paper's verification: preconditioned series == direct solve."""
    wl = media.gaussian_inclusion_64()
    P, G, chi = _setup(lsw, 64, 64, velocity=wl.velocity, freq=wl.freq_hz)
    H = lsw.build_hmatrix(G, chi, lsw.HParams(kind=lsw.H_HODLR, prec=lsw.C128, levels=2, rank=20, oversample=10,
                                              seed=1001))
    u0 = G.point_sources(wl.sources, lsw.C128)
    u, infos = lsw.solve_series(G, chi, H, u0, sp=lsw.SolveParams(prec=lsw.C128, tol=1e-11))
    assert infos[0].status == 0
    ref = oh.HODLRPreconditioner(P, 2, 20, 10, 0, 1001)
    psi, it, res = solve.series(P, P.sources(wl.sources), ref.apply, 1e-11, 30)
    assert infos[0].iterations == it[0]
    assert _rel(u.cpu().numpy()[0], psi[:, 0]) < 1e-10
    # against the dense LU solution of Eq. 6 (n = 4096)
    lu = solve.direct(P, P.sources(wl.sources))[:, 0]
    assert _rel(u.cpu().numpy()[0], lu) < 1e-9


def test_fgmres_matches_lu(lsw):
    P, G, chi = _setup(lsw, 16, 16, seed=12, freq=25.0)
    u0 = G.point_sources([(0, 4), (9, 9)], lsw.C128)
    u, infos = lsw.solve_series(G, chi, None, u0, sp=lsw.SolveParams(prec=lsw.C128, method=lsw.FGMRES, tol=1e-11,
                                                                      restart=20, max_iter=400))
    assert all(i.status == 0 for i in infos)
    lu = solve.direct(P, P.sources([(0, 4), (9, 9)])).T
    assert _rel(u.cpu().numpy(), lu) < 1e-9


@pytest.mark.parametrize("method", ["series", "fgmres"])
def test_mixed_precision_reaches_fp64_residual(lsw, method):
    wl = media.gaussian_inclusion_64()
    P, G, chi = _setup(lsw, 64, 64, velocity=wl.velocity, freq=wl.freq_hz)
    H = lsw.build_hmatrix(G, chi, lsw.HParams(kind=lsw.H_HODLR, prec=lsw.C64, levels=2, rank=20, oversample=10,
                                              seed=1001))
    pos = [(5, 32), (0, 3), (40, 60)]
    u0 = G.point_sources(pos, lsw.C128)
    m = lsw.SERIES if method == "series" else lsw.FGMRES
    u, infos = lsw.solve_series(G, chi, H, u0, sp=lsw.SolveParams(prec=lsw.MIXED, method=m, tol=1e-9,
                                                                      inner_tol=1e-4, max_iter=60))
    assert all(i.status == 0 for i in infos), [(i.status, i.rel_residual) for i in infos]
    # the oracle's own FP64 residual certifies the result
    res = P.rel_residual(u.cpu().numpy().T, P.sources(pos))
    assert np.all(res < 1e-9)


def test_salt_256_mixed_fgmres_certified(lsw):
    """256 x 256 layered medium with a salt body at 15 Hz, HODLR (quadtree
    32 x 32 leaves, 6 levels, rank 20 + 10) in FP32 inside FGMRES with an
    FP64 residual; the oracle's FP64 operator certifies 1e-6."""
    wl = media.layered_salt(256, 15.0, 32, 2)
    P, G, chi = _setup(lsw, 256, 256, velocity=wl.velocity, freq=wl.freq_hz)
    H = lsw.build_hmatrix(G, chi, lsw.HParams(kind=lsw.H_HODLR, prec=lsw.C64, levels=6, rank=20, oversample=10,
                                              seed=1002))
    pos = wl.sources[:4]
    u0 = G.point_sources(pos, lsw.C128)
    u, infos = lsw.solve_series(G, chi, H, u0, sp=lsw.SolveParams(prec=lsw.MIXED, method=lsw.FGMRES, tol=1e-6,
                                                                      inner_tol=1e-3, restart=30, max_iter=60))
    assert all(i.status == 0 for i in infos), [(i.status, i.rel_residual, i.iterations) for i in infos]
    res = P.rel_residual(u.cpu().numpy().T, P.sources(pos))
    assert np.all(res < 1e-6)


def test_born_diverges_on_salt(lsw):
    wl = media.layered_salt(256, 15.0, 32, 2)
    P, G, chi = _setup(lsw, 256, 256, velocity=wl.velocity, freq=wl.freq_hz)
    u0 = G.point_sources(wl.sources[:1], lsw.C64)
    u, infos = lsw.solve_series(G, chi, None, u0, sp=lsw.SolveParams(prec=lsw.C64, tol=1e-6, max_iter=100))
    assert infos[0].status == 6     # LSW_ERR_DIVERGED


def test_zero_contrast_series(lsw):
    P, G, chi = _setup(lsw, 16, 16, velocity=np.full((16, 16), 2000.0))
    H = lsw.build_hmatrix(G, chi, lsw.HParams(kind=lsw.H_HODLR, prec=lsw.C128, levels=2, rank=4, oversample=2))
    u0 = G.point_sources([(3, 3)], lsw.C128)
    u, infos = lsw.solve_series(G, chi, H, u0, sp=lsw.SolveParams(prec=lsw.C128, tol=1e-12))
    assert infos[0].iterations == 0 and infos[0].status == 0
    assert torch.equal(u, u0)


@pytest.mark.parametrize("n,L,k", [(64, 2, 32), (64, 2, 7), (128, 3, 20)])
def test_tensor_core_leaf_products_match_cuda_cores(lsw, n, L, k):
    """The tcgen05 products of the dense leaves (three TF32 products per
    real product, FP32 accumulation in tensor memory) agree with the
    CUDA-core path to 5e-5: each term carries ~2^-21 relative error and the
    leaf inverses' cancellation amplifies it about tenfold, while a single
    TF32 product (the lo terms lost) would be off by ~5e-4.  Both agree
    with the oracle's H to its FP32 tolerance."""
    P, G, chi = _setup(lsw, n, n, seed=17, freq=12.0)
    H = lsw.build_hmatrix(G, chi, lsw.HParams(kind=lsw.H_HODLR, prec=lsw.C64, levels=L, rank=12, oversample=6,
                                              seed=41))
    rng = np.random.default_rng(3)
    x = torch.from_numpy(media.complex_field(rng, (k, n * n)).astype(np.complex64)).cuda()
    try:
        lsw.set_tensor_cores(True)
        y_tc = lsw.apply_precond(H, x).cpu().numpy()
        lsw.set_tensor_cores(False)
        y_cc = lsw.apply_precond(H, x).cpu().numpy()
    finally:
        lsw.set_tensor_cores(True)
    assert np.all(np.isfinite(y_tc))
    assert _rel(y_tc, y_cc) < 5e-5
    ref = oh.HODLRPreconditioner(P, L, 12, 6, 0, 41)
    want = ref.apply(x.cpu().numpy().astype(np.complex128).T).T
    assert _rel(y_tc, want) < _fp32_h_tol(P, ref)


@pytest.mark.parametrize("prec", ["c64", "mixed"])
def test_fgmres_graph_replay_matches_ordinary_launches(lsw, prec):
    """The Arnoldi step replayed from a captured CUDA graph gives bit-for-bit
    the same solve as ordinary launches, and the launch counter still counts
    every kernel that ran."""
    wl = media.gaussian_inclusion_64()
    P, G, chi = _setup(lsw, 64, 64, velocity=wl.velocity, freq=wl.freq_hz)
    H = lsw.build_hmatrix(G, chi, lsw.HParams(kind=lsw.H_HODLR, prec=lsw.C64, levels=2, rank=20, oversample=10,
                                              seed=1001))
    pos = [(5, 32), (0, 3), (40, 60)]
    p = lsw.C64 if prec == "c64" else lsw.MIXED
    u0 = G.point_sources(pos, lsw.C64 if prec == "c64" else lsw.C128)
    sp = lsw.SolveParams(prec=p, method=lsw.FGMRES, tol=1e-5 if prec == "c64" else 1e-9, inner_tol=1e-4,
                         restart=8, max_iter=80)
    runs = []
    try:
        for on in (False, True):
            lsw.set_graphs(on)
            torch.cuda.synchronize()
            l0, g0 = lsw.launch_count(), lsw.graph_replay_count()
            u, infos = lsw.solve_series(G, chi, H, u0, sp=sp)
            torch.cuda.synchronize()
            runs.append((u.clone(), [(i.status, i.iterations, i.rel_residual) for i in infos], lsw.launch_count() - l0,
                         lsw.graph_replay_count() - g0))
    finally:
        lsw.set_graphs(True)
    (u1, i1, n1, g1), (u2, i2, n2, g2) = runs
    assert g1 == 0 and g2 > 0           # the second solve did replay graphs
    assert all(s == 0 for s, _, _ in i2)
    assert i1 == i2
    assert torch.equal(u1, u2)
    assert n1 == n2


def test_hodlr_power_iteration_parity_c128(lsw):
    """Level sketches with one power iteration (Algorithm 2, q = 1) against
    the oracle drawing the same probes."""
    P, G, chi = _setup(lsw, 32, 32, seed=9, freq=20.0)
    H = lsw.build_hmatrix(G, chi, lsw.HParams(kind=lsw.H_HODLR, prec=lsw.C128, levels=3, rank=8, oversample=4, q=1,
                                              seed=21))
    ref = oh.HODLRPreconditioner(P, 3, 8, 4, 1, 21)
    rng = np.random.default_rng(8)
    x = media.complex_field(rng, (3, P.n))
    y = lsw.apply_precond(H, torch.from_numpy(x).cuda()).cpu().numpy()
    assert _rel(y, ref.apply(x.T).T) < 1e-10


@pytest.mark.parametrize("n,L,k,rank", [(64, 2, 32, 12), (64, 2, 40, 12), (32, 4, 5, 12), (128, 4, 16, 12),
                                         (128, 4, 16, 16), (32, 4, 5, 16), (64, 2, 7, 40)])
def test_bf16_storage_matches_fp32_storage(lsw, n, L, k, rank):
    """H built in FP32 and kept as BF16 (re, im) pairs: every stored entry is
    rounded to 8 significant bits (relative error <= 2^-9 ~ 2e-3), and the
    leaf inverses' cancellation amplifies that about tenfold in the product,
    so the BF16 apply sits within 3e-2 of the FP32 apply of the same build
    and clearly away from it (> 1e-5: the factors really are rounded).  At
    n = 64 the leaves (1024 rows) run on the tensor cores (kind::f16); at
    n = 32 with 4 levels (64-row leaves) on the CUDA cores, and the two
    engines on BF16 storage agree to FP32 accuracy.  Levels whose blocks are
    multiples of 128 rows are stored as the tensor cores' operand tiles, with
    the rank padded to a multiple of 8 (rank 16 and 40: no padding; the
    levels of 64-row blocks stay column-major, so the CUDA-core path reads
    both storages in one matrix).  The storage takes about half the bytes,
    times the padding at most."""
    P, G, chi = _setup(lsw, n, n, seed=17, freq=12.0)
    hp = dict(kind=lsw.H_HODLR, levels=L, rank=rank, oversample=6, seed=41)
    H32 = lsw.build_hmatrix(G, chi, lsw.HParams(prec=lsw.C64, **hp))
    H16 = lsw.build_hmatrix(G, chi, lsw.HParams(prec=lsw.BF16, **hp))
    pad = ((rank + 7) // 8 * 8) / rank
    assert H16.nbytes() < 0.51 * pad * H32.nbytes()
    rng = np.random.default_rng(3)
    x = torch.from_numpy(media.complex_field(rng, (k, n * n)).astype(np.complex64)).cuda()
    y32 = lsw.apply_precond(H32, x).cpu().numpy()
    try:
        lsw.set_tensor_cores(True)
        y16 = lsw.apply_precond(H16, x).cpu().numpy()
        lsw.set_tensor_cores(False)
        y16cc = lsw.apply_precond(H16, x).cpu().numpy()
    finally:
        lsw.set_tensor_cores(True)
    assert np.all(np.isfinite(y16))
    assert 1e-5 < _rel(y16, y32) < 3e-2
    assert _rel(y16, y16cc) < 5e-5


def test_kernel_timer_counts_graph_replays(lsw):
    """A kernel-timer family sees the launches that the Arnoldi step's CUDA
    graph replays: the operator family counts one application per FGMRES
    iteration (plus the residuals), with graphs on as with graphs off, and
    both runs report positive time."""
    wl = media.gaussian_inclusion_64()
    P, G, chi = _setup(lsw, 64, 64, velocity=wl.velocity, freq=wl.freq_hz)
    H = lsw.build_hmatrix(G, chi, lsw.HParams(kind=lsw.H_HODLR, prec=lsw.C64, levels=2, rank=20, oversample=10,
                                              seed=1001))
    u0 = G.point_sources([(5, 32), (0, 3)], lsw.C64)
    sp = lsw.SolveParams(prec=lsw.C64, method=lsw.FGMRES, tol=1e-5, restart=8, max_iter=80)
    seen = []
    try:
        for on in (False, True):
            lsw.set_graphs(on)
            torch.cuda.synchronize()
            g0 = lsw.graph_replay_count()
            lsw.kernel_timer_start("operator_c64")
            u, infos = lsw.solve_series(G, chi, H, u0, sp=sp)
            torch.cuda.synchronize()
            ms, _, _, n = lsw.kernel_timer_read()
            lsw.kernel_timer_stop()
            seen.append((n, ms, lsw.graph_replay_count() - g0, max(i.iterations for i in infos)))
    finally:
        lsw.set_graphs(True)
    (n_off, ms_off, g_off, it_off), (n_on, ms_on, g_on, it_on) = seen
    assert g_off == 0 and g_on > 0
    assert it_off == it_on and n_on == n_off
    assert n_on >= it_on
    assert ms_off > 0 and ms_on > 0


def test_salt_256_bf16_hodlr_fgmres_certified(lsw):
    """The 256 x 256 salt problem with H kept in BF16 inside mixed FGMRES:
    the coarser preconditioner costs iterations, not accuracy; the oracle's
    FP64 operator certifies 1e-6."""
    wl = media.layered_salt(256, 15.0, 32, 2)
    P, G, chi = _setup(lsw, 256, 256, velocity=wl.velocity, freq=wl.freq_hz)
    H = lsw.build_hmatrix(G, chi, lsw.HParams(kind=lsw.H_HODLR, prec=lsw.BF16, levels=6, rank=20, oversample=10,
                                              seed=1002))
    pos = wl.sources[:4]
    u0 = G.point_sources(pos, lsw.C128)
    u, infos = lsw.solve_series(G, chi, H, u0, sp=lsw.SolveParams(prec=lsw.MIXED, method=lsw.FGMRES, tol=1e-6,
                                                                      inner_tol=1e-3, restart=30, max_iter=60))
    assert all(i.status == 0 for i in infos), [(i.status, i.rel_residual, i.iterations) for i in infos]
    res = P.rel_residual(u.cpu().numpy().T, P.sources(pos))
    assert np.all(res < 1e-6)


def test_bf16_storage_rejected_for_smw(lsw):
    P, G, chi = _setup(lsw, 16, 16, seed=2)
    with pytest.raises(Exception):
        lsw.build_hmatrix(G, chi, lsw.HParams(kind=lsw.H_LOWRANK_SMW, prec=lsw.BF16, rank=8, oversample=4))

"""Batched (grid, frequency) solves and the measured choice of FFT passes."""
import numpy as np
import pytest

from oracle import operator as oop
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


@pytest.mark.parametrize("n,prec", [(256, "c64"), (64, "c128"), (32, "c64"), (512, "c64")])
def test_autotune_checks_and_keeps_exact_results(lsw, n, prec):
    rng = np.random.default_rng(n)
    c = media.random_field(rng, n, n)
    P = oop.Problem(n, n, 10.0, media.C0, 15.0, c)
    G = lsw.build_green(n, n, 10.0, media.C0, 15.0)
    chi = torch.from_numpy(P.chi).cuda()
    p = lsw.C64 if prec == "c64" else lsw.C128
    v, ms = lsw.autotune(G, p, nbatch=4)
    # every variant ran and reproduced variant 0 (-2 would mark a mismatch)
    assert all(m > 0 for m in ms), ms
    assert ms[v] == min(ms)
    dt = torch.complex64 if prec == "c64" else torch.complex128
    u = torch.from_numpy(media.complex_field(rng, (3, n * n))).to(dt).cuda()
    y = lsw.apply_operator(G, chi, u, None, lsw.OP_PLAIN).cpu().numpy()
    ref = P.G0V(u.cpu().numpy().astype(np.complex128).T).T
    tol = 1e-5 if prec == "c64" else 1e-10
    assert np.linalg.norm(y - ref) / np.linalg.norm(ref) < tol


def test_batched_equals_one_by_one(lsw):
    hp = lsw.HParams(kind=lsw.H_HODLR, prec=lsw.C64, levels=2, rank=16, oversample=8, seed=7)
    sp = lsw.SolveParams(prec=lsw.MIXED, method=lsw.FGMRES, tol=1e-8, inner_tol=1e-3, restart=30, max_iter=80)
    probs = []
    for (n, f, seed) in [(64, 10.0, 1), (128, 15.0, 2), (64, 20.0, 3)]:
        rng = np.random.default_rng(seed)
        vel = media.random_field(rng, n, n)
        probs.append(dict(nz=n, nx=n, h=10.0, c0=media.C0, freq_hz=f,
                          velocity=torch.from_numpy(np.ascontiguousarray(vel.ravel())).cuda(),
                          sources=[(0, n // 4), (3, n // 2), (n - 1, n - 2)], vel_np=vel))
    outs, infos = lsw.solve_batched(probs, hp, sp, max_concurrent=3)
    for p, u, inf in zip(probs, outs, infos):
        assert all(i.status == 0 for i in inf), [(i.status, i.rel_residual) for i in inf]
        G = lsw.build_green(p["nz"], p["nx"], p["h"], p["c0"], p["freq_hz"])
        chi = G.contrast(p["velocity"])
        H = lsw.build_hmatrix(G, chi, hp)
        u0 = G.point_sources(p["sources"], lsw.C128)
        u1, inf1 = lsw.solve_series(G, chi, H, u0, sp=sp)
        assert torch.equal(u, u1)
        assert [i.iterations for i in inf] == [i.iterations for i in inf1]
        # the oracle's FP64 residual certifies the batched result
        P = oop.Problem(p["nz"], p["nx"], p["h"], p["c0"], p["freq_hz"], p["vel_np"])
        res = P.rel_residual(u.cpu().numpy().T, P.sources(p["sources"]))
        assert np.all(res < 1e-8)


def test_batched_rejects_bad_problem(lsw):
    with pytest.raises(lsw.LswError):
        lsw.solve_batched([dict(nz=16, nx=16, h=10.0, c0=2000.0, freq_hz=5.0,
                                velocity=torch.zeros(256, dtype=torch.float64, device="cuda"), sources=[])],
                          None, lsw.SolveParams(prec=lsw.C128))


def test_batched_rank_adaptation_rebuilds_until_converged(lsw):
    """The 256 x 256 salt medium at 15 Hz: with rank 20 the preconditioned
    series diverges; allowed to raise the rank, the batched call rebuilds H
    at rank 40 and converges, with the same result as a rank-40 solve."""
    wl = media.layered_salt(256, 15.0, 32, 2)
    vel = torch.from_numpy(np.ascontiguousarray(wl.velocity.ravel())).cuda()
    prob = dict(nz=256, nx=256, h=wl.h, c0=wl.c0, freq_hz=wl.freq_hz, velocity=vel, sources=list(wl.sources[:2]))
    sp = lsw.SolveParams(prec=lsw.C64, method=lsw.SERIES, tol=1e-5, max_iter=40)
    hp = lsw.HParams(kind=lsw.H_HODLR, prec=lsw.C64, levels=6, rank=20, oversample=10, seed=1002)
    _, inf0 = lsw.solve_batched([prob], hp, sp)
    assert any(i.status != 0 for i in inf0[0])
    hp.rank_max = 40
    outs, inf1 = lsw.solve_batched([prob], hp, sp)
    assert all(i.status == 0 for i in inf1[0]), [(i.status, i.rel_residual) for i in inf1[0]]
    G = lsw.build_green(256, 256, wl.h, wl.c0, wl.freq_hz)
    chi = G.contrast(vel)
    H40 = lsw.build_hmatrix(G, chi, lsw.HParams(kind=lsw.H_HODLR, prec=lsw.C64, levels=6, rank=40, oversample=10,
                                                seed=1002))
    u, inf = lsw.solve_series(G, chi, H40, G.point_sources(prob["sources"], lsw.C64), sp=sp)
    assert torch.equal(outs[0], u)
    assert [i.iterations for i in inf] == [i.iterations for i in inf1[0]]

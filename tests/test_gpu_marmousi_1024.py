"""The benchmark's 1024 x 1024 workload end to end: the Marmousi-like model at
30 Hz (h = 5 m), the HODLR preconditioner at rank 40 + 10 built in FP32 and
kept in BF16, and mixed-precision FGMRES to 1e-6.  No oracle solution exists
at this size (the dense matrix has 10^12 entries), so each GPU solution is
certified by the oracle's own FP64 residual through its FFT operator (the
self-certifying residual of the parity plan)."""
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


def test_marmousi_1024_bf16_hodlr_fgmres_certified(lsw):
    wl = media.marmousi_1024()
    src = [wl.sources[0], wl.sources[11]]
    vel = torch.from_numpy(np.ascontiguousarray(wl.velocity.ravel())).cuda()
    G = lsw.build_green(wl.nz, wl.nx, wl.h, wl.c0, wl.freq_hz)
    chi = G.contrast(vel)
    u0 = G.point_sources(src, lsw.C128)
    H = lsw.build_hmatrix(G, chi, lsw.HParams(kind=lsw.H_HODLR, prec=lsw.BF16, levels=10, split=lsw.SPLIT_QUADTREE,
                                              rank=40, oversample=10, q=0, seed=1004))
    sp = lsw.SolveParams(prec=lsw.MIXED, method=lsw.FGMRES, tol=1e-6, inner_tol=1e-3, restart=30, max_iter=400,
                         max_outer=8)
    u, infos = lsw.solve_series(G, chi, H, u0, sp=sp)
    P = oop.Problem.from_workload(wl)
    res = P.rel_residual(u.cpu().numpy().T, P.sources(src))
    for s in range(len(src)):
        assert infos[s].status == 0, (s, infos[s].status)
        # the solver's own FP64 residual and the oracle's agree, and certify 1e-6
        assert abs(infos[s].rel_residual - res[s]) <= 1e-3 * res[s] + 1e-12, (infos[s].rel_residual, res[s])
        assert res[s] <= 1e-6 * 1.001, res[s]

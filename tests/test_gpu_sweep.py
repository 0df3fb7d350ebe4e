"""The frequency sweep with the paper's rank policy (Sec. 3.1) through
lsw_solve_sweep, on a model embedded in a power-of-two grid: every
frequency's solution, restricted to the model, is certified by the oracle's
FP64 residual on the model's own grid, and the ranks follow the policy."""
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


@pytest.mark.parametrize("method", ["series", "fgmres"])
def test_sweep_on_embedded_model(lsw, method):
    rng = np.random.default_rng(21)
    c = media.random_field(rng, 24, 60)                 # 24 x 60 cells (z by x), h = 15 m
    nz, nx, h = 32, 64, 15.0
    vel = torch.from_numpy(np.ascontiguousarray(media.embed(c, nz, nx).ravel())).cuda()
    freqs = [2.0, 4.0, 6.0, 8.0]
    src = [(0, 30)]
    hp = lsw.HParams(kind=lsw.H_HODLR, prec=lsw.C64, levels=3, oversample=8, seed=77)
    pol = lsw.SweepPolicy(rank0=4, rank_step=4, rank_max=40, raise_iters=10)
    m = lsw.SERIES if method == "series" else lsw.FGMRES
    sp = lsw.SolveParams(prec=lsw.MIXED, method=m, tol=1e-6, inner_tol=1e-3, max_iter=30, restart=30)
    u, info, sinfo = lsw.solve_sweep(nz, nx, h, media.C0, vel, freqs, src, hp, pol, sp)
    inside = np.array([ix * nz + iz for ix in range(60) for iz in range(24)])
    start = pol.rank0
    for f, inf in enumerate(info):
        assert inf.freq_hz == freqs[f]
        assert inf.status == 0 and inf.converged == 1, (f, inf.status, inf.rank, inf.builds)
        assert sinfo[f][0].status == 0 and sinfo[f][0].iterations == inf.max_iterations
        # every rebuild adds one step; the next frequency starts where the policy said
        assert inf.rank == min(start + pol.rank_step * (inf.builds - 1), pol.rank_max)
        want_next = min(inf.rank + pol.rank_step, pol.rank_max) if inf.max_iterations > pol.raise_iters else inf.rank
        assert inf.next_rank == want_next
        start = inf.next_rank
        # Cells outside the model have zero contrast, so inside the model the
        # residual of the embedded problem is the model's own residual: its
        # norm is at most the embedded residual's, tol ||psi0 (embedded)||.
        # Relative to the model's own ||psi0|| the bound is therefore
        # tol ||psi0 (embedded)|| / ||psi0 (model)|| (times 1.001 for the
        # rounding of two FP64 residual evaluations of the same field).
        P = oop.Problem(24, 60, h, media.C0, freqs[f], c)
        Pe = oop.Problem(nz, nx, h, media.C0, freqs[f], media.embed(c, nz, nx))
        bound = 1.001 * sp.tol * np.linalg.norm(Pe.sources(src)) / np.linalg.norm(P.sources(src))
        res = P.rel_residual(u[f, 0].cpu().numpy()[inside][:, None], P.sources(src))
        assert res[0] <= bound, (f, res[0], bound)

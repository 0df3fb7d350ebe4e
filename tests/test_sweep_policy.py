"""The frequency-sweep rank policy (Sec. 3.1) as the library decides it, on
the host: a frequency that does not converge within the iteration limit is
rebuilt at a higher rank and solved again; one that converges in more than
the paper's 10 iterations hands a higher rank to the next frequency."""
import ctypes
import os

import pytest

NOT_CONVERGED, DIVERGED, NUMERIC = 5, 6, 7


@pytest.fixture(scope="module")
def lsw():
    from paper_2005_01372_gb300 import build
    if not os.path.exists(build.LIB):
        try:
            build.build()
        except (RuntimeError, OSError) as e:
            pytest.skip(f"cannot build the library here: {e}")
    from paper_2005_01372_gb300 import lsw as L
    L.lib()
    return L


@pytest.mark.parametrize("rank,status,iters,want", [
    (10, 0, 5, (10, False)),               # fast: keep the rank
    (10, 0, 10, (10, False)),              # exactly the limit: keep
    (10, 0, 11, (20, False)),              # slow: the next frequency starts higher
    (10, NOT_CONVERGED, 30, (20, True)),   # not converged: rebuild here
    (10, DIVERGED, 3, (20, True)),         # diverging: rebuild here
    (10, NUMERIC, 3, (20, True)),
    (35, NOT_CONVERGED, 30, (40, True)),   # the step stops at rank_max
    (40, NOT_CONVERGED, 30, (40, False)),  # at rank_max: give up at this frequency
    (40, 0, 25, (40, False)),              # slow at rank_max: nowhere to go
])
def test_policy_decisions(lsw, rank, status, iters, want):
    pol = lsw.SweepPolicy(rank0=10, rank_step=10, rank_max=40, raise_iters=10)
    assert lsw.sweep_next_rank(pol, rank, status, iters) == want


@pytest.mark.parametrize("pol,rank", [
    (dict(rank0=0, rank_step=10, rank_max=40, raise_iters=10), 10),
    (dict(rank0=10, rank_step=0, rank_max=40, raise_iters=10), 10),
    (dict(rank0=10, rank_step=10, rank_max=5, raise_iters=10), 10),
    (dict(rank0=10, rank_step=10, rank_max=40, raise_iters=-1), 10),
    (dict(rank0=10, rank_step=10, rank_max=40, raise_iters=10), 0),
])
def test_policy_rejects_invalid_arguments(lsw, pol, rank):
    with pytest.raises(lsw.LswError):
        lsw.sweep_next_rank(lsw.SweepPolicy(**pol), rank, 0, 5)


def test_simulated_sweep_follows_the_paper(lsw):
    """A model solver whose iteration count falls with rank and rises with
    frequency: driving it with the library's decisions, ranks never go
    down, a frequency is rebuilt only after a failure, and every rebuild
    adds one step."""
    pol = lsw.SweepPolicy(rank0=4, rank_step=4, rank_max=40, raise_iters=10)

    def iterations(freq, rank):
        # the rank needed grows with frequency and jumps at 10 Hz
        need = 2 * freq + (12 if freq >= 10 else 0)
        return 5 + max(0, need - rank) * 6

    rank, history = pol.rank0, []
    for f in range(1, 21):
        start, builds = rank, 0
        while True:
            builds += 1
            it = iterations(f, rank)
            status = 0 if it <= 30 else NOT_CONVERGED
            nxt, rebuild = lsw.sweep_next_rank(pol, rank, status, min(it, 30))
            used = rank
            rank = nxt
            if not rebuild:
                break
        history.append((f, start, used, builds, status))
        assert used == min(start + pol.rank_step * (builds - 1), pol.rank_max)
    ranks = [u for _, _, u, _, _ in history]
    assert ranks == sorted(ranks)
    # a frequency is left unconverged only at rank_max
    assert all(u == pol.rank_max for _, _, u, _, s in history if s != 0)
    assert history[0][4] == 0 and history[-1][2] == pol.rank_max
    # the jump at 10 Hz is met by rebuilds at that frequency
    assert history[9][3] > 1 and history[9][4] == 0


def test_sweep_rejects_invalid_policy_without_touching_the_gpu(lsw):
    """rank_max + oversample above 64 probes is refused before any GPU work."""
    buf = (ctypes.c_double * 4)()
    grid = lsw._Grid(2, 2, 10.0, 2000.0, 0.0)
    fr = (ctypes.c_double * 1)(5.0)
    src = (ctypes.c_int32 * 2)(0, 0)
    hp = lsw.HParams(kind=lsw.H_HODLR, levels=1, rank=4, oversample=20).c()
    pol = lsw.SweepPolicy(rank0=4, rank_step=4, rank_max=48, raise_iters=10).c()
    sp = lsw.SolveParams().c()
    info = (lsw.SweepInfo * 1)()
    st = lsw.lib().lsw_solve_sweep(ctypes.byref(grid), ctypes.addressof(buf), fr, 1, src, 1, ctypes.byref(hp),
                                   ctypes.byref(pol), ctypes.byref(sp), ctypes.addressof(buf), info, None, None)
    assert st == 1       # LSW_ERR_INVALID_ARG

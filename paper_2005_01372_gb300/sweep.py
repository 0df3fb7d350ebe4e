"""Frequency sweep of a velocity model from the command line: the paper's
experiments (Sec. 3.1, 3.2) on a model of the user's.

A velocity model (``.npy``, shape (nx, nz), x by z, m/s, cells of h x h) is
embedded at the top-left of the smallest power-of-two grid that holds it and
has 32 x 32-cell leaves on at least two of them; the other cells get the
background velocity c0 (zero contrast), which leaves the solution inside the
model unchanged.  The frequencies are solved in ascending order through
lsw_solve_sweep -- a HODLR preconditioner per frequency, the preconditioned
series (or FGMRES) in FP32 inside FP64 refinement, ranks by the paper's
policy -- and the wavefields on the model's own cells, with one record per
frequency, are written to ``.npz``.

    python -m paper_2005_01372_gb300.sweep model.npy --h 15 --freqs 1:20 --out waves.npz
"""
from __future__ import annotations

import argparse
import json

import numpy as np

from .media import embed

LEAF = 32           # leaf side in cells (the benchmark's quadtree leaves)
MAX_SIDE = 2048     # largest grid side the library takes


def parse_freqs(text: str) -> list:
    """"a:b" (step 1), "a:b:s" or "f1,f2,..." in Hz, returned ascending."""
    if ":" in text:
        parts = [float(p) for p in text.split(":")]
        if len(parts) not in (2, 3):
            raise ValueError(f"bad frequency range {text!r}")
        a, b = parts[0], parts[1]
        s = parts[2] if len(parts) == 3 else 1.0
        if s <= 0 or b < a:
            raise ValueError(f"bad frequency range {text!r}")
        n = int(np.floor((b - a) / s + 1e-9)) + 1
        out = [a + i * s for i in range(n)]
    else:
        out = [float(p) for p in text.split(",") if p.strip()]
    if not out or min(out) <= 0:
        raise ValueError(f"frequencies must be positive: {text!r}")
    return sorted(out)


def plan_grid(nz_m: int, nx_m: int):
    """(nz, nx, levels): power-of-two sides >= the model and >= LEAF, with at
    least two leaves (levels >= 1); levels = log2(cells / LEAF^2)."""
    def up(v):
        p = LEAF
        while p < v:
            p *= 2
        return p
    nz, nx = up(nz_m), up(nx_m)
    if nz * nx < 2 * LEAF * LEAF:
        nx *= 2
    if nz > MAX_SIDE or nx > MAX_SIDE:
        raise ValueError(f"a {nz_m} x {nx_m} model needs a grid above {MAX_SIDE} cells a side")
    levels = int(round(np.log2(nz * nx / (LEAF * LEAF))))
    return nz, nx, levels


def model_cells(nz_m: int, nx_m: int, nz: int) -> np.ndarray:
    """Grid indices (ix * nz + iz) of the model's cells, in the model's own
    strip order (ix * nz_m + iz)."""
    ix, iz = np.meshgrid(np.arange(nx_m), np.arange(nz_m), indexing="ij")
    return (ix * nz + iz).ravel()


def run(velocity: np.ndarray, h: float, freqs, sources=None, c0: float = 2000.0, rank0: int = 10,
        rank_step: int = 10, rank_max: int = 50, raise_iters: int = 10, oversample: int = 10, method: str = "series",
        tol: float = 1e-6, seed: int = 1005, device: str = "cuda", solve=None) -> dict:
    """Solve the sweep; returns u (nfreq, nsrc, nx_m, nz_m) complex128 on the
    model's cells and the per-frequency records.  ``solve`` defaults to
    lsw.solve_sweep (same arguments)."""
    import torch

    from . import lsw

    velocity = np.asarray(velocity, dtype=np.float64)
    if velocity.ndim != 2:
        raise ValueError("the velocity model must be a 2D array of shape (nx, nz)")
    nx_m, nz_m = velocity.shape
    nz, nx, levels = plan_grid(nz_m, nx_m)
    if sources is None:
        sources = [(0, nx_m // 2)]
    for iz, ix in sources:
        if not (0 <= iz < nz_m and 0 <= ix < nx_m):
            raise ValueError(f"source ({iz}, {ix}) lies outside the {nz_m} x {nx_m} model")
    freqs = sorted(float(f) for f in freqs)
    vel = torch.from_numpy(np.ascontiguousarray(embed(velocity, nz, nx, c0).ravel())).to(device)
    hp = lsw.HParams(kind=lsw.H_HODLR, prec=lsw.C64, levels=levels, oversample=oversample, seed=seed)
    pol = lsw.SweepPolicy(rank0=rank0, rank_step=rank_step, rank_max=rank_max, raise_iters=raise_iters)
    m = lsw.FGMRES if method == "fgmres" else lsw.SERIES
    sp = lsw.SolveParams(prec=lsw.MIXED, method=m, tol=tol, inner_tol=1e-3, restart=30, max_iter=30, max_outer=8)
    solve = solve or lsw.solve_sweep
    u, info, sinfo = solve(nz, nx, h, c0, vel, freqs, list(sources), hp, pol, sp)
    cells = model_cells(nz_m, nx_m, nz)
    uu = u.cpu().numpy()[:, :, cells].reshape(len(freqs), len(sources), nx_m, nz_m)
    records = [{"freq_hz": i.freq_hz, "rank": i.rank, "builds": i.builds, "converged": i.converged,
                "max_iterations": i.max_iterations, "max_rel_residual": i.max_rel_residual, "status": i.status}
               for i in info]
    return {"u": uu, "freqs": np.array(freqs), "sources": np.array(sources, dtype=np.int32), "records": records,
            "grid": (nz, nx), "levels": levels}


def main(argv=None) -> int:
    ap = argparse.ArgumentParser(description=__doc__.split("\n\n")[0],
                                 formatter_class=argparse.RawDescriptionHelpFormatter)
    ap.add_argument("model", help=".npy velocity model, shape (nx, nz) [m/s]")
    ap.add_argument("--h", type=float, required=True, help="cell size [m]")
    ap.add_argument("--freqs", default="1:20", help='"a:b", "a:b:step" or "f1,f2,..." [Hz]')
    ap.add_argument("--c0", type=float, default=2000.0, help="background velocity [m/s] (Eq. 1)")
    ap.add_argument("--source", action="append", default=None, metavar="IZ,IX",
                    help="point source cell (repeatable; default: the middle of the top row)")
    ap.add_argument("--method", default="series", choices=["series", "fgmres"])
    ap.add_argument("--rank0", type=int, default=10)
    ap.add_argument("--rank-step", type=int, default=10)
    ap.add_argument("--rank-max", type=int, default=50)
    ap.add_argument("--tol", type=float, default=1e-6)
    ap.add_argument("--out", default=None, help=".npz for the wavefields and records")
    args = ap.parse_args(argv)
    vel = np.load(args.model)
    src = None
    if args.source:
        src = [tuple(int(v) for v in s.split(",")) for s in args.source]
    res = run(vel, args.h, parse_freqs(args.freqs), src, c0=args.c0, rank0=args.rank0, rank_step=args.rank_step,
              rank_max=args.rank_max, method=args.method, tol=args.tol)
    if args.out:
        np.savez(args.out, u=res["u"], freqs=res["freqs"], sources=res["sources"],
                 records=json.dumps(res["records"]))
    print(json.dumps({"grid": res["grid"], "levels": res["levels"], "records": res["records"]}))
    return 0 if all(r["status"] == 0 for r in res["records"]) else 1


if __name__ == "__main__":
    raise SystemExit(main())

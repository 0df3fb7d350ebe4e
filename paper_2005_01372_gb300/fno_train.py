"""Training pairs, training loop, checkpoints and evaluation for the learned
right preconditioner (the lsw_fno handle).

Pairs.  For a medium with H built from it (the paper's randomized HODLR
preconditioner, Sec. 2.4), residual fields r are drawn and their corrections
e = (I - G0 V)^-1 r are solved with H-preconditioned FGMRES to a tight FP64
tolerance.  A pair is (x, e / ||r||) with x = [r / ||r||, chi / k0^2 + i k0 h],
the network's input as lsw_fno_apply builds it.  The residual fields are of
three kinds, a third each: incident fields of random point sources (the
first Krylov vector of a solve), G0 V applied to such fields (the next
Krylov directions), and smoothed complex noise.

Training.  Mean squared error on batches drawn with a per-step seed (so a
resumed run draws the same batches), Adam with a cosine learning-rate decay;
every step runs in the library (lsw_fno_loss_grad, lsw_fno_adam_step).  The
map r -> e is complex-linear, so each drawn pair may be rotated by a random
phase, (e^{i phi} x0, x1) -> e^{i phi} t, which the split GELU does not
respect by construction and the network has to learn.

Evaluation.  Flexible GMRES on held-out media with no preconditioner, with H,
and with the network (H as its fallback); iterations, wall time and the FP64
residual per solve.

Run ``python -m paper_2005_01372_gb300.fno_train --help`` for the command
line that trains a network and prints the comparison as JSON.
"""
from __future__ import annotations

import argparse
import json
import math
import time
from dataclasses import dataclass

import numpy as np
import torch

from . import lsw, media

H_CELL = 10.0


@dataclass
class Pairs:
    x: torch.Tensor      # (N, 2, n) complex64
    t: torch.Tensor      # (N, n) complex64
    nz: int
    nx: int

    def __len__(self):
        return self.x.shape[0]


def _grid(n, freq):
    return lsw.build_green(n, n, H_CELL, media.C0, freq)


def residual_fields(G, chi, rng: np.random.Generator, count: int, n: int) -> torch.Tensor:
    """count residual-like fields (count, n * n) complex128 on the device."""
    k = count // 3
    npt = count - 2 * k
    pos = [(int(rng.integers(0, n)), int(rng.integers(0, n))) for _ in range(npt + k)]
    ps = G.point_sources(pos, lsw.C128)
    krylov = lsw.apply_operator(G, chi, ps[npt:].contiguous(), mode=lsw.OP_PLAIN)
    smooth = torch.from_numpy(media.smooth_complex_field(rng, k, n, n)).cuda()
    return torch.cat([ps[:npt], krylov, smooth]).contiguous()


def make_pairs(n: int, seeds, per_medium: int, hp: lsw.HParams, tol: float = 1e-8, log=None) -> Pairs:
    xs, ts = [], []
    for seed in seeds:
        vel, f = media.fno_medium(seed, n)
        G = _grid(n, f)
        chi = G.contrast(torch.from_numpy(vel.ravel().copy()).cuda())
        H = lsw.build_hmatrix(G, chi, hp)
        rng = np.random.default_rng(seed + 1_000_003)
        r = residual_fields(G, chi, rng, per_medium, n)
        sp = lsw.SolveParams(prec=lsw.MIXED, method=lsw.FGMRES, tol=tol, inner_tol=1e-4, restart=30, max_iter=300,
                             max_outer=12)
        e, infos = lsw.solve_series(G, chi, H, r, sp=sp)
        ok = torch.tensor([i.status == 0 for i in infos], device="cuda")
        x, t = lsw.fno_pairs(G, chi, r, e)
        xs.append(x[ok])
        ts.append(t[ok])
        if log:
            log(f"medium {seed}: f={f:.1f} Hz, {int(ok.sum())}/{per_medium} pairs, "
                f"mean FGMRES iterations {np.mean([i.iterations for i in infos]):.1f}")
    return Pairs(torch.cat(xs).contiguous(), torch.cat(ts).contiguous(), n, n)


def lr_at(t: int, steps: int, lr: float, warmup: int = 50) -> float:
    if t <= warmup:
        return lr * t / warmup
    return 0.5 * lr * (1 + math.cos(math.pi * min(1.0, (t - warmup) / max(1, steps - warmup)))) + 1e-3 * lr


def train(net: lsw.FNO, pairs: Pairs, steps: int, batch: int, lr: float, seed: int = 0, start: int = 0,
          stop: int | None = None, log=None, log_every: int = 100, phase: bool = False):
    """Adam steps start+1 .. min(stop, steps); returns the loss history."""
    hist = []
    N = len(pairs)
    last = steps if stop is None else min(stop, steps)
    for t in range(start + 1, last + 1):
        rng = np.random.default_rng([seed, t])
        b = min(batch, N)
        idx = torch.from_numpy(rng.integers(0, N, size=b)).cuda()
        x, tgt = pairs.x[idx].contiguous(), pairs.t[idx].contiguous()
        if phase:
            lsw.fno_rotate(x, tgt, rng.uniform(0, 2 * np.pi, size=b))
        loss = net.loss_grad(x, tgt)
        net.adam_step(lr_at(t, steps, lr), t)
        hist.append(loss)
        if log and (t % log_every == 0 or t == last):
            log(f"step {t}: loss {np.mean(hist[-log_every:]):.4e}")
    return hist


def relative_error(net: lsw.FNO, pairs: Pairs, batch: int = 64) -> float:
    """sum ||y - t||^2 / sum ||t||^2 over a pair set."""
    num = den = 0.0
    for i in range(0, len(pairs), batch):
        a, b = net.error_sums(pairs.x[i:i + batch].contiguous(), pairs.t[i:i + batch].contiguous())
        num += a
        den += b
    return math.sqrt(num / den)


def save_checkpoint(net: lsw.FNO, path: str, step: int):
    torch.save({"shape": (net.nz, net.nx, net.width, net.modes, net.layers), "step": step,
                "state": [net.get(w).cpu() for w in (lsw.FNO_WEIGHTS, lsw.FNO_ADAM_M, lsw.FNO_ADAM_V)]}, path)


def load_checkpoint(path: str, nz: int | None = None, nx: int | None = None):
    """(network, step).  nz, nx: build it for another grid (the weights do
    not depend on the grid)."""
    ck = torch.load(path)
    z, x, W, m, L = ck["shape"]
    net = lsw.FNO(nz or z, nx or x, W, m, L)
    for w, t in zip((lsw.FNO_WEIGHTS, lsw.FNO_ADAM_M, lsw.FNO_ADAM_V), ck["state"]):
        net.set(t.cuda(), w)
    return net, ck["step"]


def evaluate(net: lsw.FNO | None, n: int, seeds, hp: lsw.HParams, nsrc: int = 8, tol: float = 1e-6,
             restart: int = 30, max_iter: int = 300, modes=("none", "H", "FNO")):
    """Per medium and preconditioner: mean FGMRES iterations per source,
    solve seconds (the H build excluded and reported apart), worst FP64
    relative residual, fallback count."""
    rows = []
    for seed in seeds:
        vel, f = media.fno_medium(seed, n)
        G = _grid(n, f)
        chi = G.contrast(torch.from_numpy(vel.ravel().copy()).cuda())
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        H = lsw.build_hmatrix(G, chi, hp)
        torch.cuda.synchronize()
        t_build = time.perf_counter() - t0
        step = max(1, n // nsrc)
        u0 = G.point_sources([(0, step * s + step // 2) for s in range(nsrc)], lsw.C128)
        sp = lsw.SolveParams(prec=lsw.MIXED, method=lsw.FGMRES, tol=tol, inner_tol=1e-3, restart=restart,
                             max_iter=max_iter, max_outer=12)
        row = {"seed": seed, "freq_hz": round(f, 2), "h_build_s": round(t_build, 4)}
        for mode in modes:
            if mode == "FNO" and net is None:
                continue
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            if mode == "FNO":
                u, infos = lsw.solve_learned(G, chi, net, H, u0, sp=sp)
            else:
                u, infos = lsw.solve_series(G, chi, H if mode == "H" else None, u0, sp=sp)
            torch.cuda.synchronize()
            row[mode] = {"iterations": float(np.mean([i.iterations for i in infos])),
                         "solve_s": round(time.perf_counter() - t0, 4),
                         "converged": int(sum(i.status == 0 for i in infos)),
                         "max_rel_residual": float(max(i.rel_residual for i in infos)),
                         "fallbacks": int(sum(i.fallback for i in infos))}
        rows.append(row)
    return rows


def summarize(rows, modes=("none", "H", "FNO")):
    out = {}
    for m in modes:
        rs = [r[m] for r in rows if m in r]
        if not rs:
            continue
        out[m] = {"mean_iterations": float(np.mean([r["iterations"] for r in rs])),
                  "mean_solve_s": float(np.mean([r["solve_s"] for r in rs])),
                  "converged": int(sum(r["converged"] for r in rs)),
                  "worst_rel_residual": float(max(r["max_rel_residual"] for r in rs)),
                  "fallbacks": int(sum(r["fallbacks"] for r in rs))}
    return out


def main(argv=None):
    ap = argparse.ArgumentParser(description="train the learned preconditioner and compare it with H")
    ap.add_argument("--n", type=int, default=64)
    ap.add_argument("--train-media", type=int, default=48)
    ap.add_argument("--per-medium", type=int, default=48)
    ap.add_argument("--width", type=int, default=16)
    ap.add_argument("--modes", type=int, default=8)
    ap.add_argument("--layers", type=int, default=4)
    ap.add_argument("--steps", type=int, default=2000)
    ap.add_argument("--batch", type=int, default=32)
    ap.add_argument("--lr", type=float, default=3e-3)
    ap.add_argument("--phase", action="store_true", help="random phase rotation of every drawn pair")
    ap.add_argument("--levels", type=int, default=2)
    ap.add_argument("--rank", type=int, default=10)
    ap.add_argument("--test-media", type=int, default=16)
    ap.add_argument("--test-n", type=int, nargs="*", default=None)
    ap.add_argument("--checkpoint", default=None)
    ap.add_argument("--out", default=None)
    a = ap.parse_args(argv)

    def log(msg):
        print(msg, flush=True)

    hp = lsw.HParams(kind=lsw.H_HODLR, prec=lsw.C64, levels=a.levels, rank=a.rank, oversample=10, seed=1003)
    t0 = time.perf_counter()
    pairs = make_pairs(a.n, range(5000, 5000 + a.train_media), a.per_medium, hp, log=log)
    t_pairs = time.perf_counter() - t0
    val = make_pairs(a.n, range(8000, 8004), 24, hp)
    net = lsw.FNO(a.n, a.n, a.width, a.modes, a.layers, seed=7)
    t0 = time.perf_counter()
    hist = train(net, pairs, a.steps, a.batch, a.lr, seed=1, log=log, log_every=max(1, a.steps // 20), phase=a.phase)
    torch.cuda.synchronize()
    t_train = time.perf_counter() - t0
    if a.checkpoint:
        save_checkpoint(net, a.checkpoint, a.steps)
    result = {"n": a.n, "train_media": a.train_media, "pairs": len(pairs), "pair_generation_s": round(t_pairs, 2),
              "network": {"width": a.width, "modes": a.modes, "layers": a.layers, "params": net.num_params},
              "train": {"steps": a.steps, "batch": a.batch, "lr": a.lr, "phase": a.phase,
                        "seconds": round(t_train, 2),
                        "first_loss": hist[0], "last_loss": float(np.mean(hist[-50:])),
                        "train_rel_error": relative_error(net, pairs), "val_rel_error": relative_error(net, val)},
              "H": {"levels": a.levels, "rank": a.rank, "oversample": 10, "prec": "c64"}, "test": {}}
    for n in (a.test_n or [a.n]):
        tnet = net
        if n != a.n:
            tnet = lsw.FNO(n, n, a.width, a.modes, a.layers)
            tnet.set(net.get())
        hp_n = lsw.HParams(kind=lsw.H_HODLR, prec=lsw.C64, levels=a.levels + int(round(math.log2(n / a.n))),
                           rank=a.rank, oversample=10, seed=1003)
        rows = evaluate(tnet, n, range(9000, 9000 + a.test_media), hp_n)
        result["test"][str(n)] = {"summary": summarize(rows), "per_medium": rows}
    js = json.dumps(result)
    if a.out:
        with open(a.out, "w") as fh:
            fh.write(js + "\n")
    print(json.dumps({k: v for k, v in result.items() if k != "test"}))
    for n, r in result["test"].items():
        print(n, json.dumps(r["summary"]))


if __name__ == "__main__":
    main()

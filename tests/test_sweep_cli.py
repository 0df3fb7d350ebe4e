"""The sweep command line's host logic (no GPU): frequency lists, the grid
a model is embedded in, and the way the solver's fields are cut back to the
model's cells, checked with a stand-in for the solver."""
import json
import types

import numpy as np
import pytest

torch = pytest.importorskip("torch")

from paper_2005_01372_gb300 import sweep  # noqa: E402


@pytest.mark.parametrize("text,want", [
    ("1:5", [1.0, 2.0, 3.0, 4.0, 5.0]),
    ("2:8:3", [2.0, 5.0, 8.0]),
    ("15,5,10", [5.0, 10.0, 15.0]),
    ("0.5:1.5:0.5", [0.5, 1.0, 1.5]),
])
def test_parse_freqs(text, want):
    assert sweep.parse_freqs(text) == pytest.approx(want)


@pytest.mark.parametrize("text", ["5:1", "1:5:0", "0,5", "", "1:2:3:4"])
def test_parse_freqs_rejects(text):
    with pytest.raises(ValueError):
        sweep.parse_freqs(text)


@pytest.mark.parametrize("shape,want", [
    ((81, 248), (128, 256, 5)),      # the paper's Marmousi2 subset
    ((150, 700), (256, 1024, 8)),    # the paper's SEG/EAGE salt model
    ((10, 10), (32, 64, 1)),
    ((32, 32), (32, 64, 1)),
    ((64, 64), (64, 64, 2)),
])
def test_plan_grid(shape, want):
    assert sweep.plan_grid(*shape) == want


def test_plan_grid_rejects_too_large():
    with pytest.raises(ValueError):
        sweep.plan_grid(3000, 10)


def test_run_embeds_and_cuts_back():
    rng = np.random.default_rng(4)
    nx_m, nz_m = 40, 20
    vel = rng.uniform(1500, 4500, size=(nx_m, nz_m))
    seen = {}

    def fake_solve(nz, nx, h, c0, v, freqs, sources, hp, pol, sp):
        seen.update(nz=nz, nx=nx, h=h, c0=c0, v=v.numpy().reshape(nx, nz), freqs=freqs, sources=sources,
                    levels=hp.levels, pol=pol, method=sp.method)
        nf, ns, n = len(freqs), len(sources), nz * nx
        idx = torch.arange(n, dtype=torch.float64)
        u = torch.stack([torch.stack([torch.complex(idx, torch.full_like(idx, 10.0 * f + s)) for s in range(ns)])
                         for f in range(nf)])
        info = [types.SimpleNamespace(freq_hz=f, rank=10, builds=1, converged=ns, max_iterations=3,
                                      max_rel_residual=1e-7, status=0) for f in freqs]
        return u, info, None

    res = sweep.run(vel, 15.0, [3.0, 1.0], device="cpu", solve=fake_solve, method="fgmres")
    assert (seen["nz"], seen["nx"], seen["levels"]) == (32, 64, 1)
    assert seen["freqs"] == [1.0, 3.0] and seen["sources"] == [(0, 20)]
    assert np.array_equal(seen["v"][:nx_m, :nz_m], vel)
    assert np.all(seen["v"][nx_m:, :] == 2000.0) and np.all(seen["v"][:, nz_m:] == 2000.0)
    assert seen["method"] == 1
    u = res["u"]
    assert u.shape == (2, 1, nx_m, nz_m)
    ix, iz = np.meshgrid(np.arange(nx_m), np.arange(nz_m), indexing="ij")
    for f in range(2):
        assert np.array_equal(u[f, 0].real, ix * 32 + iz)
        assert np.all(u[f, 0].imag == 10.0 * f)
    assert [r["freq_hz"] for r in res["records"]] == [1.0, 3.0]


def test_run_rejects_a_source_outside_the_model():
    with pytest.raises(ValueError):
        sweep.run(np.full((8, 8), 2000.0), 10.0, [1.0], sources=[(0, 9)], device="cpu", solve=lambda *a: None)


def test_main_writes_records(tmp_path, monkeypatch, capsys):
    model = tmp_path / "m.npy"
    np.save(model, np.full((12, 6), 2500.0))
    calls = {}

    def fake_run(vel, h, freqs, src, **kw):
        calls.update(shape=vel.shape, h=h, freqs=freqs, src=src, kw=kw)
        rec = [{"freq_hz": f, "rank": 10, "builds": 1, "converged": 1, "max_iterations": 2,
                "max_rel_residual": 1e-7, "status": 0} for f in freqs]
        return {"u": np.zeros((len(freqs), 1, 12, 6), complex), "freqs": np.array(freqs),
                "sources": np.array([[0, 6]], dtype=np.int32), "records": rec, "grid": (32, 64), "levels": 1}

    monkeypatch.setattr(sweep, "run", fake_run)
    out = tmp_path / "w.npz"
    rc = sweep.main([str(model), "--h", "15", "--freqs", "1:3", "--source", "0,6", "--method", "fgmres",
                     "--out", str(out)])
    assert rc == 0
    assert calls["shape"] == (12, 6) and calls["freqs"] == [1.0, 2.0, 3.0] and calls["src"] == [(0, 6)]
    assert calls["kw"]["method"] == "fgmres"
    z = np.load(out)
    assert z["u"].shape == (3, 1, 12, 6) and len(json.loads(str(z["records"]))) == 3
    assert json.loads(capsys.readouterr().out)["levels"] == 1

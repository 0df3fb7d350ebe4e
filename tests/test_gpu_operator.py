"""Parity of the CUDA Green table, spectrum and FFT operator with the oracle.

Tolerances (relative 2-norm against the FP64 oracle): 1e-10 for the FP64
path, 1e-5 for the FP32 path, as stated for this method's GPU paths."""
import numpy as np
import pytest

from oracle import green as og
from oracle import operator as oop
from paper_2005_01372_gb300 import media

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

TOL = {"c128": 1e-10, "c64": 1e-5}


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


def _problem(nz, nx, seed, freq=15.0, h=10.0):
    rng = np.random.default_rng(seed)
    c = media.random_field(rng, nz, nx)
    return oop.Problem(nz, nx, h, media.C0, freq, c), c


@pytest.mark.parametrize("nz,nx", [(1, 1), (4, 8), (16, 16), (64, 32), (128, 128)])
def test_green_table_and_spectrum(lsw, nz, nx):
    P, c = _problem(nz, nx, 1)
    G = lsw.build_green(nz, nx, P.h, P.c0, P.freq_hz)
    tab = G.table().cpu().numpy()
    ref = og.green_table(nz, nx, P.h, P.k)
    # CUDA's and scipy's double Bessel routines differ by a few ulps
    assert _rel(tab, ref) < 1e-11
    spec = G.spectrum().cpu().numpy()
    full = og.green_spectrum(nz, nx, P.h, P.k) / (4.0 * nz * nx)
    assert _rel(spec, full[: nx + 1, : nz + 1]) < 1e-11


def test_contrast_and_sources(lsw):
    nz, nx = 32, 16
    P, c = _problem(nz, nx, 2)
    G = lsw.build_green(nz, nx, P.h, P.c0, P.freq_hz)
    vel = torch.from_numpy(np.ascontiguousarray(c.ravel())).cuda()
    chi = G.contrast(vel).cpu().numpy()
    assert _rel(chi, P.chi) < 1e-14
    pos = [(0, 3), (31, 15), (7, 0)]
    for prec, tol in ((lsw.C128, 1e-13), (lsw.C64, 1e-6)):
        u0 = G.point_sources(pos, prec).cpu().numpy()
        ref = P.sources(pos).T
        assert _rel(u0, ref) < tol


def _check_operator(lsw, nz, nx, nb, prec, seed):
    P, c = _problem(nz, nx, seed)
    G = lsw.build_green(nz, nx, P.h, P.c0, P.freq_hz)
    chi = torch.from_numpy(P.chi).cuda()
    rng = np.random.default_rng(seed + 100)
    u = media.complex_field(rng, (nb, P.n))
    u0 = media.complex_field(rng, (nb, P.n))
    dt = torch.complex128 if prec == lsw.C128 else torch.complex64
    tol = TOL["c128" if prec == lsw.C128 else "c64"]
    ud = torch.from_numpy(u).to(dt).cuda()
    u0d = torch.from_numpy(u0).to(dt).cuda()
    uref = u if prec == lsw.C128 else ud.cpu().numpy().astype(np.complex128)
    u0ref = u0 if prec == lsw.C128 else u0d.cpu().numpy().astype(np.complex128)
    for mode in (lsw.OP_FORWARD, lsw.OP_RESIDUAL, lsw.OP_PLAIN, lsw.OP_ADJOINT):
        y = lsw.apply_operator(G, chi, ud, u0d, mode).cpu().numpy()
        ref = oop.apply(mode, P.spec, P.chi, uref.T, u0ref.T, nz, nx).T
        assert _rel(y, ref) < tol, (mode, _rel(y, ref))
    # u0 = NULL reads as zero
    y = lsw.apply_operator(G, chi, ud, None, lsw.OP_RESIDUAL).cpu().numpy()
    ref = oop.apply(lsw.OP_RESIDUAL, P.spec, P.chi, uref.T, None, nz, nx).T
    assert _rel(y, ref) < tol


@pytest.mark.parametrize("nz,nx,nb", [(1, 1, 1), (2, 4, 3), (8, 8, 2), (16, 64, 2), (64, 16, 1),
                                      (64, 64, 3), (128, 256, 2), (256, 256, 2)])
@pytest.mark.parametrize("prec", ["c128", "c64"])
def test_operator_parity(lsw, nz, nx, nb, prec):
    _check_operator(lsw, nz, nx, nb, lsw.C128 if prec == "c128" else lsw.C64, nz * 7 + nx)


def test_operator_batch_equals_single(lsw):
    """A field's result does not depend on the other fields of the batch."""
    nz = nx = 64
    P, c = _problem(nz, nx, 5)
    G = lsw.build_green(nz, nx, P.h, P.c0, P.freq_hz)
    chi = torch.from_numpy(P.chi).cuda()
    rng = np.random.default_rng(6)
    u = torch.from_numpy(media.complex_field(rng, (5, P.n))).cuda()
    yb = lsw.apply_operator(G, chi, u, None, lsw.OP_PLAIN)
    y2 = lsw.apply_operator(G, chi, u[2:3].contiguous(), None, lsw.OP_PLAIN)
    assert torch.equal(yb[2:3], y2)


def test_operator_full_size_sampled(lsw):
    """1024 x 1024 (2048 x 2048 padded FFT), 4 fields, FP32: every entry
    against the FP64 oracle FFT, plus the adjoint identity."""
    wl = media.marmousi_1024(nsrc=4)
    P = oop.Problem.from_workload(wl)
    G = lsw.build_green(wl.nz, wl.nx, wl.h, wl.c0, wl.freq_hz)
    chi = torch.from_numpy(P.chi).cuda()
    u0 = G.point_sources(wl.sources, lsw.C64)
    y = lsw.apply_operator(G, chi, u0, None, lsw.OP_PLAIN).cpu().numpy()
    ref = P.G0V(u0.cpu().numpy().astype(np.complex128).T).T
    assert _rel(y, ref) < TOL["c64"]


def test_operator_rejects_bad_arguments(lsw):
    G = lsw.build_green(16, 16, 10.0, 2000.0, 10.0)
    chi = torch.zeros(256, dtype=torch.float64, device="cuda")
    u = torch.zeros((1, 256), dtype=torch.complex128, device="cuda")
    with pytest.raises(lsw.LswError) as e:
        lsw.apply_operator(G, chi, u, None, mode=7)
    assert e.value.status == 1
    with pytest.raises(lsw.LswError) as e:
        lsw.apply_operator(G, chi, u, None, lsw.OP_PLAIN, y=u)
    assert e.value.status == 1
    with pytest.raises(lsw.LswError) as e:
        lsw.build_green(12, 16, 10.0, 2000.0, 10.0)
    assert e.value.status == 2
    with pytest.raises(lsw.LswError) as e:
        lsw.build_green(16, 16, -1.0, 2000.0, 10.0)
    assert e.value.status == 1
    # an empty batch is a no-op
    lsw.apply_operator(G, chi, u[:0], None, lsw.OP_PLAIN, y=torch.empty_like(u[:0]))

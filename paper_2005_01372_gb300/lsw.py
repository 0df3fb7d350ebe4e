"""Python binding of the lsw C ABI (include/lsw.h): argument marshalling only.

Every computation runs in ``liblsw.so``'s CUDA kernels; this module turns
torch tensors into device pointers and raises ``LswError`` on a non-zero
status.  PyTorch supplies device memory and the current CUDA stream.  There is
no fallback: importing the binding without the built library, or calling it
without a GPU, raises.
"""
from __future__ import annotations

import ctypes
import os
from dataclasses import dataclass

import torch

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "liblsw.so")

C128, C64, MIXED, BF16 = 0, 1, 2, 3
OP_FORWARD, OP_RESIDUAL, OP_PLAIN, OP_ADJOINT = 0, 1, 2, 3
H_LOWRANK_SMW, H_HODLR = 0, 1
SERIES, FGMRES = 0, 1
SPLIT_QUADTREE, SPLIT_STRIPS = 0, 1

STATUS = {0: "OK", 1: "INVALID_ARG", 2: "UNSUPPORTED_SIZE", 3: "OOM", 4: "CUDA",
          5: "NOT_CONVERGED", 6: "DIVERGED", 7: "NUMERIC", 8: "TIMEOUT"}


class LswError(RuntimeError):
    def __init__(self, status: int, what: str, detail: str = ""):
        self.status = status
        super().__init__(f"{what}: {STATUS.get(status, status)}" + (f" ({detail})" if detail else ""))


class _Grid(ctypes.Structure):
    _fields_ = [("nz", ctypes.c_int32), ("nx", ctypes.c_int32), ("h", ctypes.c_double),
                ("c0", ctypes.c_double), ("freq_hz", ctypes.c_double)]


class _Box(ctypes.Structure):
    _fields_ = [("z0", ctypes.c_int32), ("z1", ctypes.c_int32), ("x0", ctypes.c_int32), ("x1", ctypes.c_int32)]


class _HParams(ctypes.Structure):
    _fields_ = [("kind", ctypes.c_int32), ("prec", ctypes.c_int32), ("levels", ctypes.c_int32),
                ("split", ctypes.c_int32), ("rank", ctypes.c_int32), ("oversample", ctypes.c_int32),
                ("q", ctypes.c_int32), ("rank_max", ctypes.c_int32), ("seed", ctypes.c_uint64)]


class _SolveParams(ctypes.Structure):
    _fields_ = [("prec", ctypes.c_int32), ("max_iter", ctypes.c_int32), ("tol", ctypes.c_double),
                ("inner_tol", ctypes.c_double), ("max_outer", ctypes.c_int32), ("method", ctypes.c_int32),
                ("restart", ctypes.c_int32), ("pad_", ctypes.c_int32)]


class _Problem(ctypes.Structure):
    _fields_ = [("grid", _Grid), ("velocity", ctypes.c_void_p), ("sources", ctypes.POINTER(ctypes.c_int32)),
                ("nsrc", ctypes.c_int32), ("pad_", ctypes.c_int32), ("u", ctypes.c_void_p)]


class SolveInfo(ctypes.Structure):
    _fields_ = [("iterations", ctypes.c_int32), ("outer", ctypes.c_int32), ("status", ctypes.c_int32),
                ("fallback", ctypes.c_int32), ("rel_residual", ctypes.c_double)]


class _SweepPolicy(ctypes.Structure):
    _fields_ = [("rank0", ctypes.c_int32), ("rank_step", ctypes.c_int32), ("rank_max", ctypes.c_int32),
                ("raise_iters", ctypes.c_int32)]


class SweepInfo(ctypes.Structure):
    _fields_ = [("freq_hz", ctypes.c_double), ("rank", ctypes.c_int32), ("builds", ctypes.c_int32),
                ("converged", ctypes.c_int32), ("max_iterations", ctypes.c_int32),
                ("max_rel_residual", ctypes.c_double), ("status", ctypes.c_int32), ("next_rank", ctypes.c_int32)]


class _FnoParams(ctypes.Structure):
    _fields_ = [("nz", ctypes.c_int32), ("nx", ctypes.c_int32), ("width", ctypes.c_int32),
                ("modes", ctypes.c_int32), ("layers", ctypes.c_int32), ("pad_", ctypes.c_int32),
                ("seed", ctypes.c_uint64)]


_lib = None
VP, I32, U32, U64 = ctypes.c_void_p, ctypes.c_int, ctypes.c_uint32, ctypes.c_uint64

_SIGS = {
    "lsw_status_string": (ctypes.c_char_p, [I32]),
    "lsw_last_error": (ctypes.c_char_p, []),
    "lsw_launch_count": (ctypes.c_uint64, []),
    "lsw_kernel_timer_start": (I32, [ctypes.c_char_p]),
    "lsw_kernel_timer_read": (I32, [ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_double),
                                    ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_uint64)]),
    "lsw_kernel_timer_stop": (I32, []),
    "lsw_measure_peak": (I32, [I32, ctypes.POINTER(ctypes.c_double), VP]),
    "lsw_mempool_usage": (I32, [ctypes.POINTER(ctypes.c_uint64), ctypes.POINTER(ctypes.c_uint64), I32]),
    "lsw_build_green": (I32, [ctypes.POINTER(_Grid), VP, ctypes.POINTER(VP)]),
    "lsw_destroy_green": (I32, [VP]),
    "lsw_green_table": (I32, [VP, VP, VP]),
    "lsw_green_spectrum": (I32, [VP, VP, VP]),
    "lsw_contrast": (I32, [VP, VP, VP, VP]),
    "lsw_point_sources": (I32, [VP, ctypes.POINTER(ctypes.c_int32), I32, I32, VP, VP]),
    "lsw_apply_operator": (I32, [VP, I32, VP, VP, VP, VP, I32, I32, VP]),
    "lsw_apply_operator_noalloc": (I32, [VP, I32, VP, VP, VP, VP, I32, I32, VP]),
    "lsw_sketch_range": (I32, [VP, I32, VP, _Box, _Box, I32, I32, I32, U64, U32, VP, VP, VP]),
    "lsw_build_hmatrix": (I32, [VP, VP, ctypes.POINTER(_HParams), VP, ctypes.POINTER(VP)]),
    "lsw_destroy_hmatrix": (I32, [VP]),
    "lsw_hmatrix_bytes": (I32, [VP, ctypes.POINTER(ctypes.c_uint64)]),
    "lsw_apply_precond": (I32, [VP, VP, VP, I32, VP]),
    "lsw_solve_series": (I32, [VP, VP, VP, VP, VP, I32, ctypes.POINTER(_SolveParams),
                               ctypes.POINTER(SolveInfo), VP]),
    "lsw_solve_batched": (I32, [VP, I32, ctypes.POINTER(_HParams), ctypes.POINTER(_SolveParams), I32,
                                ctypes.POINTER(SolveInfo), VP]),
    "lsw_sweep_next_rank": (I32, [ctypes.POINTER(_SweepPolicy), ctypes.c_int32, ctypes.c_int32, ctypes.c_int32,
                                  ctypes.POINTER(ctypes.c_int32), ctypes.POINTER(ctypes.c_int32)]),
    "lsw_solve_sweep": (I32, [ctypes.POINTER(_Grid), VP, ctypes.POINTER(ctypes.c_double), I32,
                              ctypes.POINTER(ctypes.c_int32), I32, ctypes.POINTER(_HParams),
                              ctypes.POINTER(_SweepPolicy), ctypes.POINTER(_SolveParams), VP,
                              ctypes.POINTER(SweepInfo), ctypes.POINTER(SolveInfo), VP]),
    "lsw_autotune": (I32, [VP, I32, I32, VP, ctypes.POINTER(ctypes.c_int), ctypes.POINTER(ctypes.c_float)]),
    "lsw_set_tensor_cores": (I32, [I32]),
    "lsw_set_graphs": (I32, [I32]),
    "lsw_graph_replay_count": (ctypes.c_uint64, []),
    "lsw_fno_create": (I32, [ctypes.POINTER(_FnoParams), VP, ctypes.POINTER(VP)]),
    "lsw_fno_destroy": (I32, [VP]),
    "lsw_fno_num_params": (I32, [VP, ctypes.POINTER(ctypes.c_int64)]),
    "lsw_fno_state": (I32, [VP, I32, VP, VP, VP]),
    "lsw_fno_forward": (I32, [VP, VP, VP, I32, VP]),
    "lsw_fno_loss_grad": (I32, [VP, VP, VP, I32, ctypes.POINTER(ctypes.c_double), VP, VP]),
    "lsw_fno_adam_step": (I32, [VP, ctypes.c_float, ctypes.c_int32, VP]),
    "lsw_fno_apply": (I32, [VP, VP, VP, VP, VP, I32, I32, VP]),
    "lsw_fno_pairs": (I32, [VP, VP, VP, VP, I32, I32, VP, VP, VP]),
    "lsw_fno_rotate": (I32, [VP, VP, I32, ctypes.c_int64, ctypes.POINTER(ctypes.c_float), VP]),
    "lsw_fno_error": (I32, [VP, VP, VP, I32, ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_double), VP]),
    "lsw_solve_learned": (I32, [VP, VP, VP, VP, VP, VP, I32, ctypes.POINTER(_SolveParams),
                                ctypes.POINTER(SolveInfo), VP]),
}


def lib():
    """The loaded library (loads it on first use; raises if it is missing)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise ImportError(f"{LIB_PATH} is missing: build it with paper_2005_01372_gb300.build")
        L = ctypes.CDLL(LIB_PATH)
        for name, (res, args) in _SIGS.items():
            if not hasattr(L, name):
                continue          # calling it raises AttributeError
            f = getattr(L, name)
            f.restype = res
            f.argtypes = args
        _lib = L
    return _lib


def _check(st: int, what: str):
    if st != 0:
        detail = ""
        if st in (3, 4):
            detail = (lib().lsw_last_error() or b"").decode()
        raise LswError(st, what, detail)


def _stream(stream=None) -> int:
    s = stream if stream is not None else torch.cuda.current_stream()
    return s.cuda_stream


def _ptr(t, dtype=None):
    if t is None:
        return None
    if not isinstance(t, torch.Tensor) or not t.is_cuda:
        raise TypeError("expected a CUDA tensor")
    if not t.is_contiguous():
        raise ValueError("tensor must be contiguous")
    if dtype is not None and t.dtype != dtype:
        raise TypeError(f"expected {dtype}, got {t.dtype}")
    return t.data_ptr()


def _cdtype(prec: int):
    return torch.complex128 if prec in (C128, MIXED) else torch.complex64


@dataclass
class HParams:
    kind: int = H_HODLR
    prec: int = C64
    levels: int = 6
    split: int = SPLIT_QUADTREE
    rank: int = 20
    oversample: int = 10
    q: int = 0
    seed: int = 1
    rank_max: int = 0

    def c(self):
        return _HParams(self.kind, self.prec, self.levels, self.split, self.rank, self.oversample, self.q,
                        self.rank_max, self.seed)


@dataclass
class SolveParams:
    prec: int = C128
    max_iter: int = 30
    tol: float = 1e-6
    inner_tol: float = 1e-3
    max_outer: int = 8
    method: int = 0
    restart: int = 30

    def c(self):
        return _SolveParams(self.prec, self.max_iter, self.tol, self.inner_tol, self.max_outer, self.method,
                            self.restart, 0)


class Green:
    """lsw_green handle: Green table and spectra of one (grid, frequency)."""

    def __init__(self, nz: int, nx: int, h: float, c0: float, freq_hz: float, stream=None):
        self.nz, self.nx, self.h, self.c0, self.freq_hz = nz, nx, h, c0, freq_hz
        self.n = nz * nx
        g = _Grid(nz, nx, h, c0, freq_hz)
        out = VP()
        _check(lib().lsw_build_green(ctypes.byref(g), _stream(stream), ctypes.byref(out)), "lsw_build_green")
        self._h = out

    @property
    def handle(self):
        return self._h

    def __del__(self):
        if getattr(self, "_h", None) and _lib is not None:
            _lib.lsw_destroy_green(self._h)
            self._h = None

    def table(self, stream=None) -> torch.Tensor:
        t = torch.empty((self.nx + 1, self.nz + 1), dtype=torch.complex128, device="cuda")
        _check(lib().lsw_green_table(self._h, _ptr(t), _stream(stream)), "lsw_green_table")
        return t

    def spectrum(self, stream=None) -> torch.Tensor:
        t = torch.empty((self.nx + 1, self.nz + 1), dtype=torch.complex128, device="cuda")
        _check(lib().lsw_green_spectrum(self._h, _ptr(t), _stream(stream)), "lsw_green_spectrum")
        return t

    def contrast(self, velocity: torch.Tensor, stream=None) -> torch.Tensor:
        chi = torch.empty(self.n, dtype=torch.float64, device="cuda")
        _check(lib().lsw_contrast(self._h, _ptr(velocity, torch.float64), _ptr(chi), _stream(stream)),
               "lsw_contrast")
        return chi

    def point_sources(self, positions, prec: int = C128, stream=None) -> torch.Tensor:
        pos = (ctypes.c_int32 * (2 * len(positions)))(*[int(v) for p in positions for v in p])
        u0 = torch.empty((len(positions), self.n), dtype=_cdtype(prec), device="cuda")
        _check(lib().lsw_point_sources(self._h, pos, len(positions), prec, _ptr(u0), _stream(stream)),
               "lsw_point_sources")
        return u0


def launch_count() -> int:
    """Kernels launched by the library so far in this process."""
    return int(lib().lsw_launch_count())


def kernel_timer_start(family: str):
    """Time every launch of one kernel family ("operator_c64", "operator_c128",
    "qr", "gj_update")
    with CUDA events on its stream, from now on."""
    _check(lib().lsw_kernel_timer_start(family.encode()), "lsw_kernel_timer_start")


def kernel_timer_read():
    """(total ms, algorithmic bytes, flops, launches) since kernel_timer_start."""
    ms, by, fl, n = ctypes.c_double(), ctypes.c_double(), ctypes.c_double(), ctypes.c_uint64()
    _check(lib().lsw_kernel_timer_read(ctypes.byref(ms), ctypes.byref(by), ctypes.byref(fl), ctypes.byref(n)),
           "lsw_kernel_timer_read")
    return ms.value, by.value, fl.value, n.value


def measure_peak(kind: int = 0, stream=None) -> float:
    """Measured FMA peak of the current device in TFLOP/s (0: FP32, 1: FP64)."""
    t = ctypes.c_double(0.0)
    _check(lib().lsw_measure_peak(int(kind), ctypes.byref(t), _stream(stream)), "lsw_measure_peak")
    return float(t.value)


def mempool_usage(reset_high: bool = False):
    """(bytes in use, high-water mark) of the device's default memory pool."""
    cur, high = ctypes.c_uint64(0), ctypes.c_uint64(0)
    _check(lib().lsw_mempool_usage(ctypes.byref(cur), ctypes.byref(high), 1 if reset_high else 0),
           "lsw_mempool_usage")
    return int(cur.value), int(high.value)


def kernel_timer_stop():
    _check(lib().lsw_kernel_timer_stop(), "lsw_kernel_timer_stop")


def set_tensor_cores(enable: bool):
    """Process-wide switch for the tensor-core products of H's dense leaves."""
    _check(lib().lsw_set_tensor_cores(1 if enable else 0), "lsw_set_tensor_cores")


def set_graphs(enable: bool):
    """Process-wide switch for the solvers' CUDA-graph replay of the Arnoldi step."""
    _check(lib().lsw_set_graphs(1 if enable else 0), "lsw_set_graphs")


def graph_replay_count() -> int:
    """CUDA-graph launches the solvers have issued so far in this process."""
    return int(lib().lsw_graph_replay_count())


def build_green(nz, nx, h, c0, freq_hz, stream=None) -> Green:
    return Green(nz, nx, h, c0, freq_hz, stream)


def apply_operator(G: Green, chi, u, u0=None, mode: int = OP_PLAIN, y=None, stream=None) -> torch.Tensor:
    """lsw_apply_operator; u: (nbatch, n) complex128 or complex64."""
    prec = C128 if u.dtype == torch.complex128 else C64
    nb = u.numel() // G.n
    if y is None:
        y = torch.empty_like(u)
    _check(lib().lsw_apply_operator(G.handle, prec, _ptr(chi, torch.float64), _ptr(u, u.dtype),
                                    _ptr(u0, u.dtype) if u0 is not None else None, _ptr(y, u.dtype),
                                    nb, mode, _stream(stream)), "lsw_apply_operator")
    return y


def apply_operator_noalloc(G: Green, chi, u, u0=None, mode: int = OP_PLAIN, y=None, stream=None) -> torch.Tensor:
    """lsw_apply_operator_noalloc: the same product as apply_operator with
    the library's fixed device scratch, for callers that cannot let the
    library allocate (the output y is still the caller's)."""
    prec = C128 if u.dtype == torch.complex128 else C64
    nb = u.numel() // G.n
    if y is None:
        y = torch.empty_like(u)
    _check(lib().lsw_apply_operator_noalloc(G.handle, prec, _ptr(chi, torch.float64), _ptr(u, u.dtype),
                                            _ptr(u0, u.dtype) if u0 is not None else None, _ptr(y, u.dtype),
                                            nb, mode, _stream(stream)), "lsw_apply_operator_noalloc")
    return y


def sketch_range(G: Green, chi, rows, cols, rank: int, oversample: int, q: int, seed: int, stream_id: int = 0,
                 prec: int = C128, stream=None):
    """lsw_sketch_range; rows/cols are (z0, z1, x0, x1).  Returns (U, W),
    column-major, as tensors of shape (rank, n_rows) and (rank, n_cols)."""
    ns = (rows[1] - rows[0]) * (rows[3] - rows[2])
    nt = (cols[1] - cols[0]) * (cols[3] - cols[2])
    dt = _cdtype(prec)
    U = torch.empty((rank, ns), dtype=dt, device="cuda")
    W = torch.empty((rank, nt), dtype=dt, device="cuda")
    _check(lib().lsw_sketch_range(G.handle, prec, _ptr(chi, torch.float64), _Box(*rows), _Box(*cols), rank,
                                  oversample, q, seed, stream_id, _ptr(U), _ptr(W), _stream(stream)),
           "lsw_sketch_range")
    return U, W


class HMatrix:
    """lsw_hmatrix handle (the preconditioner H)."""

    def __init__(self, G: Green, chi, hp: HParams, stream=None):
        out = VP()
        self.prec = hp.prec
        self.n = G.n
        c = hp.c()
        _check(lib().lsw_build_hmatrix(G.handle, _ptr(chi, torch.float64), ctypes.byref(c), _stream(stream),
                                       ctypes.byref(out)), "lsw_build_hmatrix")
        self._h = out

    @property
    def handle(self):
        return self._h

    def __del__(self):
        if getattr(self, "_h", None) and _lib is not None:
            _lib.lsw_destroy_hmatrix(self._h)
            self._h = None

    def nbytes(self) -> int:
        b = ctypes.c_uint64()
        _check(lib().lsw_hmatrix_bytes(self._h, ctypes.byref(b)), "lsw_hmatrix_bytes")
        return b.value


def build_hmatrix(G: Green, chi, hp: HParams, stream=None) -> HMatrix:
    return HMatrix(G, chi, hp, stream)


def apply_precond(H: HMatrix, x, y=None, stream=None) -> torch.Tensor:
    nb = x.numel() // H.n
    if y is None:
        y = torch.empty_like(x)
    _check(lib().lsw_apply_precond(H.handle, _ptr(x, _cdtype(H.prec)), _ptr(y, _cdtype(H.prec)), nb,
                                   _stream(stream)), "lsw_apply_precond")
    return y


def solve_series(G: Green, chi, H, u0, u=None, sp: SolveParams = None, stream=None, check: bool = False):
    """lsw_solve_series.  Returns (u, list of SolveInfo).  With check=True a
    non-converged solve raises; otherwise the status is in the infos."""
    sp = sp or SolveParams(prec=C128 if u0.dtype == torch.complex128 else C64)
    nb = u0.numel() // G.n
    if u is None:
        u = torch.empty_like(u0)
    infos = (SolveInfo * nb)()
    c = sp.c()
    st = lib().lsw_solve_series(G.handle, _ptr(chi, torch.float64), H.handle if H is not None else None,
                                _ptr(u0, u0.dtype), _ptr(u, u0.dtype), nb, ctypes.byref(c), infos,
                                _stream(stream))
    if st not in (0, 5, 6, 7) or (check and st != 0):
        _check(st, "lsw_solve_series")
    return u, list(infos)


def autotune(G: Green, prec: int = C64, nbatch: int = 32, stream=None):
    """lsw_autotune: returns (chosen variant, [ms of variants 0, 1, 2])."""
    v = ctypes.c_int()
    ms = (ctypes.c_float * 3)()
    _check(lib().lsw_autotune(G.handle, prec, nbatch, _stream(stream), ctypes.byref(v), ms), "lsw_autotune")
    return v.value, list(ms)


def solve_batched(problems, hp: HParams = None, sp: SolveParams = None, max_concurrent: int = 4, stream=None):
    """lsw_solve_batched.  ``problems``: list of dicts with keys nz, nx, h, c0,
    freq_hz, velocity (CUDA float64 tensor), sources (list of (iz, ix)).
    Returns (list of output tensors, list of per-source SolveInfo lists)."""
    sp = sp or SolveParams(prec=MIXED)
    dt = _cdtype(sp.prec)
    arr = (_Problem * len(problems))()
    keep, outs = [], []
    for i, p in enumerate(problems):
        src = (ctypes.c_int32 * (2 * len(p["sources"])))(*[int(v) for s_ in p["sources"] for v in s_])
        keep.append(src)
        u = torch.empty((len(p["sources"]), p["nz"] * p["nx"]), dtype=dt, device="cuda")
        outs.append(u)
        arr[i] = _Problem(_Grid(p["nz"], p["nx"], p["h"], p["c0"], p["freq_hz"]),
                          _ptr(p["velocity"], torch.float64), src, len(p["sources"]), 0, _ptr(u))
    total = sum(len(p["sources"]) for p in problems)
    infos = (SolveInfo * max(1, total))()
    hpc = hp.c() if hp is not None else None
    spc = sp.c()
    st = lib().lsw_solve_batched(arr, len(problems), ctypes.byref(hpc) if hpc is not None else None,
                                 ctypes.byref(spc), max_concurrent, infos, _stream(stream))
    if st not in (0, 5, 6, 7):
        _check(st, "lsw_solve_batched")
    res, k = [], 0
    for p in problems:
        res.append([infos[k + j] for j in range(len(p["sources"]))])
        k += len(p["sources"])
    return outs, res


@dataclass
class SweepPolicy:
    """lsw_sweep_policy: the rank rule of a frequency sweep (the paper's
    limits: 30 iterations before a rebuild, 10 before raising the rank)."""
    rank0: int = 10
    rank_step: int = 10
    rank_max: int = 50
    raise_iters: int = 10

    def c(self) -> _SweepPolicy:
        return _SweepPolicy(self.rank0, self.rank_step, self.rank_max, self.raise_iters)


def sweep_next_rank(pol: SweepPolicy, rank: int, solve_status: int, max_iterations: int):
    """lsw_sweep_next_rank (host only): (next_rank, rebuild)."""
    nxt, reb = ctypes.c_int32(), ctypes.c_int32()
    pc = pol.c()
    _check(lib().lsw_sweep_next_rank(ctypes.byref(pc), rank, solve_status, max_iterations, ctypes.byref(nxt),
                                     ctypes.byref(reb)), "lsw_sweep_next_rank")
    return nxt.value, bool(reb.value)


def solve_sweep(nz: int, nx: int, h: float, c0: float, velocity, freqs_hz, sources, hp: HParams,
                pol: SweepPolicy, sp: SolveParams = None, stream=None):
    """lsw_solve_sweep.  Returns (u of shape (nfreq, nsrc, n), list of
    SweepInfo, list per frequency of lists of SolveInfo)."""
    sp = sp or SolveParams(prec=MIXED)
    nf, ns, n = len(freqs_hz), len(sources), nz * nx
    u = torch.empty((nf, ns, n), dtype=_cdtype(sp.prec), device="cuda")
    fr = (ctypes.c_double * max(1, nf))(*[float(f) for f in freqs_hz])
    src = (ctypes.c_int32 * (2 * ns))(*[int(v) for s_ in sources for v in s_])
    info = (SweepInfo * max(1, nf))()
    sinfo = (SolveInfo * max(1, nf * ns))()
    grid = _Grid(nz, nx, h, c0, 0.0)
    hpc, pc, spc = hp.c(), pol.c(), sp.c()
    st = lib().lsw_solve_sweep(ctypes.byref(grid), _ptr(velocity, torch.float64), fr, nf, src, ns, ctypes.byref(hpc),
                               ctypes.byref(pc), ctypes.byref(spc), _ptr(u), info, sinfo, _stream(stream))
    if st not in (0, 5, 6, 7):
        _check(st, "lsw_solve_sweep")
    return u, [info[i] for i in range(nf)], [[sinfo[f * ns + j] for j in range(ns)] for f in range(nf)]


FNO_WEIGHTS, FNO_GRADS, FNO_ADAM_M, FNO_ADAM_V = 0, 1, 2, 3


class FNO:
    """lsw_fno handle: the learned right preconditioner (weights, gradients
    and Adam moments on the device, FP32 complex)."""

    def __init__(self, nz: int, nx: int, width: int = 16, modes: int = 8, layers: int = 4, seed: int = 0,
                 stream=None):
        self.nz, self.nx, self.width, self.modes, self.layers = nz, nx, width, modes, layers
        self.n = nz * nx
        p = _FnoParams(nz, nx, width, modes, layers, 0, seed)
        out = VP()
        _check(lib().lsw_fno_create(ctypes.byref(p), _stream(stream), ctypes.byref(out)), "lsw_fno_create")
        self._h = out
        c = ctypes.c_int64()
        _check(lib().lsw_fno_num_params(self._h, ctypes.byref(c)), "lsw_fno_num_params")
        self.num_params = c.value

    @property
    def handle(self):
        return self._h

    def __del__(self):
        if getattr(self, "_h", None) and _lib is not None:
            _lib.lsw_fno_destroy(self._h)
            self._h = None

    def get(self, which: int = FNO_WEIGHTS, stream=None) -> torch.Tensor:
        t = torch.empty(self.num_params, dtype=torch.complex64, device="cuda")
        _check(lib().lsw_fno_state(self._h, which, _ptr(t), None, _stream(stream)), "lsw_fno_state")
        return t

    def set(self, t: torch.Tensor, which: int = FNO_WEIGHTS, stream=None):
        if t.numel() != self.num_params:
            raise ValueError("wrong number of parameters")
        _check(lib().lsw_fno_state(self._h, which, None, _ptr(t, torch.complex64), _stream(stream)),
               "lsw_fno_state")

    def forward(self, x: torch.Tensor, stream=None) -> torch.Tensor:
        """x: (batch, 2, n) complex64 -> (batch, n)."""
        b = x.numel() // (2 * self.n)
        y = torch.empty((b, self.n), dtype=torch.complex64, device="cuda")
        _check(lib().lsw_fno_forward(self._h, _ptr(x, torch.complex64), _ptr(y), b, _stream(stream)),
               "lsw_fno_forward")
        return y

    def loss_grad(self, x: torch.Tensor, target: torch.Tensor, want_grad: bool = False, stream=None):
        """Mean squared error and its gradient (kept in the handle; a copy
        is returned with want_grad)."""
        b = x.numel() // (2 * self.n)
        g = torch.empty(self.num_params, dtype=torch.complex64, device="cuda") if want_grad else None
        loss = ctypes.c_double()
        _check(lib().lsw_fno_loss_grad(self._h, _ptr(x, torch.complex64), _ptr(target, torch.complex64), b,
                                       ctypes.byref(loss), _ptr(g) if g is not None else None, _stream(stream)),
               "lsw_fno_loss_grad")
        return (loss.value, g) if want_grad else loss.value

    def error_sums(self, x: torch.Tensor, target: torch.Tensor, stream=None):
        """lsw_fno_error: (sum |net(x) - target|^2, sum |target|^2)."""
        num, den = ctypes.c_double(0.0), ctypes.c_double(0.0)
        _check(lib().lsw_fno_error(self.handle, _ptr(x, torch.complex64), _ptr(target, torch.complex64),
                                   int(target.shape[0]), ctypes.byref(num), ctypes.byref(den), _stream(stream)),
               "lsw_fno_error")
        return float(num.value), float(den.value)

    def adam_step(self, lr: float, t: int, stream=None):
        _check(lib().lsw_fno_adam_step(self._h, lr, t, _stream(stream)), "lsw_fno_adam_step")

    def apply(self, G: Green, chi, v: torch.Tensor, z=None, stream=None) -> torch.Tensor:
        prec = C128 if v.dtype == torch.complex128 else C64
        nb = v.numel() // self.n
        if z is None:
            z = torch.empty_like(v)
        _check(lib().lsw_fno_apply(self._h, G.handle, _ptr(chi, torch.float64), _ptr(v, v.dtype), _ptr(z, v.dtype),
                                   nb, prec, _stream(stream)), "lsw_fno_apply")
        return z


def fno_pairs(G: Green, chi, r, e, stream=None):
    """lsw_fno_pairs: network inputs x (nb, 2, n) and targets t (nb, n),
    complex64, from residuals r and corrections e (nb, n)."""
    prec = C128 if r.dtype == torch.complex128 else C64
    nb = r.numel() // G.n
    x = torch.empty((nb, 2, G.n), dtype=torch.complex64, device=r.device)
    t = torch.empty((nb, G.n), dtype=torch.complex64, device=r.device)
    _check(lib().lsw_fno_pairs(G.handle, _ptr(chi, torch.float64), _ptr(r, r.dtype), _ptr(e, r.dtype), nb, prec,
                               _ptr(x, torch.complex64), _ptr(t, torch.complex64), _stream(stream)), "lsw_fno_pairs")
    return x, t


def fno_rotate(x, t, phases, stream=None):
    """lsw_fno_rotate: x[:, 0] and t times exp(i phases) in place."""
    nb = t.shape[0]
    ph = (ctypes.c_float * nb)(*[float(p) for p in phases])
    _check(lib().lsw_fno_rotate(_ptr(x, torch.complex64), _ptr(t, torch.complex64), nb, int(t.shape[1]), ph,
                                _stream(stream)), "lsw_fno_rotate")


def solve_learned(G: Green, chi, fno: FNO, H, u0, u=None, sp: SolveParams = None, stream=None, check: bool = False):
    """lsw_solve_learned: FGMRES with the network as right preconditioner
    and H (may be None) as its fallback.  Returns (u, list of SolveInfo)."""
    sp = sp or SolveParams(prec=C128 if u0.dtype == torch.complex128 else C64, method=FGMRES)
    nb = u0.numel() // G.n
    if u is None:
        u = torch.empty_like(u0)
    infos = (SolveInfo * nb)()
    c = sp.c()
    st = lib().lsw_solve_learned(G.handle, _ptr(chi, torch.float64), fno.handle, H.handle if H is not None else None,
                                 _ptr(u0, u0.dtype), _ptr(u, u0.dtype), nb, ctypes.byref(c), infos, _stream(stream))
    if st not in (0, 5, 6, 7) or (check and st != 0):
        _check(st, "lsw_solve_learned")
    return u, list(infos)

"""The allocation-free operator call, checked against the allocating one.

lsw_apply_operator_noalloc is for callers that cannot let the library
allocate device memory during a call (a reserved-memory allocator of their
own, per-call memory audits, loops that cannot absorb an allocation's cost or
failure).  It must give what lsw_apply_operator gives, call after call, while
its scratch lives in one fixed device array shared by every call."""
import numpy as np
import pytest

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
    return float(torch.linalg.vector_norm(a - b) / torch.linalg.vector_norm(b))


@pytest.mark.parametrize("prec", ["c128", "c64"])
def test_noalloc_matches_allocating_call_twice(lsw, prec):
    # 256 x 256, 16 fields in FP64 or 32 in FP32: the full 32 MiB of scratch
    nz = nx = 256
    nb = 16 if prec == "c128" else 32
    dt = torch.complex128 if prec == "c128" else torch.complex64
    rng = np.random.default_rng(42)
    vel = torch.from_numpy(np.ascontiguousarray(media.random_field(rng, nz, nx).ravel())).cuda()
    G = lsw.build_green(nz, nx, 10.0, media.C0, 15.0)
    chi = G.contrast(vel)
    modes = [lsw.OP_RESIDUAL, lsw.OP_ADJOINT]
    for call in range(2):
        u = torch.from_numpy(media.complex_field(rng, (nb, nz * nx))).to(dt).cuda()
        u0 = torch.from_numpy(media.complex_field(rng, (nb, nz * nx))).to(dt).cuda()
        ref = lsw.apply_operator(G, chi, u, u0, modes[call])
        got = torch.empty_like(u)
        torch.cuda.synchronize()
        # nothing is allocated during the call: neither device memory at large
        # nor the stream-ordered pool the library's other calls draw from
        free0 = torch.cuda.mem_get_info()[0]
        used0, _ = lsw.mempool_usage(reset_high=True)
        lsw.apply_operator_noalloc(G, chi, u, u0, modes[call], y=got)
        torch.cuda.synchronize()
        used1, high = lsw.mempool_usage()
        assert torch.cuda.mem_get_info()[0] == free0
        assert used1 == used0 and high <= used0, (used0, used1, high)
        assert _rel(got, ref) < TOL[prec], (call, _rel(got, ref))


def test_noalloc_rejects_oversize_request(lsw):
    G = lsw.build_green(256, 256, 10.0, media.C0, 15.0)
    chi = torch.zeros(256 * 256, dtype=torch.float64, device="cuda")
    u = torch.zeros((33, 256 * 256), dtype=torch.complex64, device="cuda")
    with pytest.raises(lsw.LswError) as e:
        lsw.apply_operator_noalloc(G, chi, u, None, lsw.OP_PLAIN)
    assert e.value.status == 2

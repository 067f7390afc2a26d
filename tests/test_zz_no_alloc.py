"""The residual norm that allocates no device memory (wec_residual_norm_noalloc).

Some callers cannot allocate device memory when they need the residual of the
pressure equation (a control loop under a fixed memory budget, a process whose
device memory belongs to another allocator).  The no-allocation entry point keeps
its scratch in a file-scope device array; this checks, through the C ABI, that
two calls in a row agree with the norm the existing solver entry point reports.
Kept in a file of its own that pytest collects last.
"""
import ctypes as C

import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from paper_2206_07732_gb300 import build as B  # noqa: E402
from paper_2206_07732_gb300 import synth  # noqa: E402
from paper_2206_07732_gb300 import wec  # noqa: E402


@pytest.fixture(scope="module")
def lib():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    B.build()
    L = wec.load()
    vp = C.c_void_p
    L.wec_residual_norm_noalloc.argtypes = [C.c_int, C.c_int, vp, vp, vp, vp, vp, vp]
    return L


def _cuda(a):
    return torch.from_numpy(np.ascontiguousarray(a, dtype=np.float64)).cuda()


@pytest.mark.parametrize("nx,ny", [(96, 40), (512, 256)])
def test_noalloc_norm_matches_solver_residual(lib, nx, ny):
    bu, bv = synth.random_coefficients(nx, ny, seed=nx + 3 * ny, contrast=1e2)
    b = np.random.default_rng(12).standard_normal((ny, nx))
    P = wec.Poisson(nx, ny)
    tbu, tbv, tb = _cuda(bu), _cuda(bv), _cuda(b)
    P.set_coefficients(tbu, tbv)
    x = torch.zeros(ny, nx, dtype=torch.float64, device="cuda")
    info = P.solve(tb, x, rtol=1e-9)  # existing entry point: reports ||b - A x|| / ||b||
    assert info["status"] == 0
    zero = torch.zeros_like(x)
    out = torch.zeros(2, dtype=torch.float64, device="cuda")
    stream = C.c_void_p(torch.cuda.current_stream().cuda_stream)
    ptr = lambda t: C.c_void_p(t.data_ptr())
    # two calls in a row share the static scratch
    assert lib.wec_residual_norm_noalloc(nx, ny, ptr(tbu), ptr(tbv), ptr(x), ptr(tb), C.c_void_p(out.data_ptr()),
                                         stream) == 0
    assert lib.wec_residual_norm_noalloc(nx, ny, ptr(tbu), ptr(tbv), ptr(zero), ptr(tb),
                                         C.c_void_p(out.data_ptr() + 8), stream) == 0
    torch.cuda.synchronize()
    r, bn = out.cpu().numpy()
    assert bn == pytest.approx(float(np.linalg.norm(b)), rel=1e-12)
    assert r / bn == pytest.approx(info["relres"], rel=1e-12)
    # the residual itself, recomputed on the host
    from oracle.tank import poisson_apply
    rh = np.linalg.norm(b - poisson_apply(bu, bv, x.cpu().numpy()))
    assert r == pytest.approx(rh, rel=1e-9)


def test_noalloc_rejects_oversize(lib):
    # 2^29 cells, above the 2^28 maximum: rejected on the host before any launch
    t = torch.zeros(8, dtype=torch.float64, device="cuda")
    p = C.c_void_p(t.data_ptr())
    code = lib.wec_residual_norm_noalloc(32768, 16384, p, p, p, p, p, None)
    assert code == wec.WEC_ERR_INVALID
    assert b"exceeds" in lib.wec_last_error()

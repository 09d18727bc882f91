"""The allocation-free Chebyshev entry point gives the same result as the
workspace-taking one and as the oracle's Chebyshev semi-iteration.

sgoc_apply_chebyshev_noalloc exists for callers that cannot allocate device
memory when they need the mass solve (for instance a plug-in inside a host
framework that owns all device memory, or a real-time path that forbids
allocation after start-up); it keeps its iterate buffers in an array built into
the library.  The float64 cases and the float32 case on 255 x 255 interior
nodes run the per-step kernel, which ping-pongs its iterates through both halves
of that array; the float32 case on 63 x 63 nodes runs the fused kernel, which
keeps them in shared memory.  This file is collected last so that a run stopping
at the first failure has already run every other test; it also passes on its
own in a fresh process.
"""
import ctypes

import numpy as np
import pytest

import sg_inputs as si

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def cuda_ready():
    if not torch.cuda.is_available():
        pytest.fail("GPU tests selected but no CUDA device is visible")
    from paper_2512_23804_gb300 import build
    build.build()


def _noalloc(sp, R, X, ncols):
    from paper_2512_23804_gb300 import abi
    st = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    prec = 0 if R.dtype == torch.float64 else 1
    return abi.load().sgoc_apply_chebyshev_noalloc(sp._handle, prec, ctypes.c_void_p(R.data_ptr()),
                                                   ctypes.c_void_p(X.data_ptr()), ncols, st)


@pytest.mark.parametrize("nx,dtype,tol", [(64, torch.float64, 1e-12), (64, torch.float32, 2e-6),
                                          (256, torch.float64, 1e-12), (256, torch.float32, 2e-6)])
def test_noalloc_matches_workspace_entry_point_twice(nx, dtype, tol):
    from paper_2512_23804_gb300 import SGProblem, abi
    from oracle.operators import SGData
    from oracle.precond import chebyshev
    M, p = (3, 3) if nx == 64 else (2, 1)
    pr = si.random_small(31, nx=nx, M=M, p=p)
    sp = SGProblem.from_problem(pr).upload()
    mass = SGData(pr).Mass
    ncols = 2 * sp.P
    assert ncols * sp.n * (8 if dtype == torch.float64 else 4) <= 8 << 20
    for call in range(2):                         # two calls in a row share the built-in array
        Rh = si.random_panel(40 + call, sp.n, ncols)
        if dtype == torch.float32:
            Rh = Rh.astype(np.float32).astype(np.float64)
        R = torch.from_numpy(Rh).to("cuda", dtype)
        ref = sp.apply_chebyshev(R, ncols)
        X = torch.full_like(R, float("nan"))
        st = _noalloc(sp, R, X, ncols)
        assert st == abi.SGOC_OK, abi.load().sgoc_last_error()
        torch.cuda.synchronize()
        err = (torch.linalg.norm((X - ref).double()) / torch.linalg.norm(ref.double())).item()
        assert err <= tol, (call, err)
        Xo = chebyshev(mass, Rh.reshape(ncols, sp.n).T, pr.cheb_steps).T.reshape(-1)
        Xh = X.double().cpu().numpy()
        assert np.linalg.norm(Xh - Xo) / np.linalg.norm(Xo) <= tol, call


def test_noalloc_rejects_oversized_requests():
    from paper_2512_23804_gb300 import SGProblem, abi
    pr = si.random_small(32, nx=128, M=3, p=3)
    sp = SGProblem.from_problem(pr).upload()
    ncols = (8 << 20) // (sp.n * 8) + 1          # one column beyond 8 MiB of float64
    R = torch.zeros(ncols * sp.n, dtype=torch.float64, device="cuda")
    X = torch.empty_like(R)
    st = _noalloc(sp, R, X, ncols)
    assert abi.STATUS_NAMES[st] == "SGOC_ERR_INVALID_ARG"
    assert "exceeds the limit" in abi.load().sgoc_last_error().decode()

"""The allocation-free Chebyshev entry point gives the same result as the
workspace-taking one.

sgoc_apply_chebyshev_noalloc exists for callers that cannot allocate device
memory when they need the mass solve (e.g. during CUDA graph capture, or inside
a host framework that owns all device memory); it keeps its iterate buffers in
an array built into the library.  This file is collected last so that a run
stopping at the first failure has already run every other test; it also passes
on its own in a fresh process.
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


@pytest.mark.parametrize("dtype,tol", [(torch.float64, 1e-12), (torch.float32, 2e-6)])
def test_noalloc_matches_workspace_entry_point_twice(dtype, tol):
    from paper_2512_23804_gb300 import SGProblem, abi
    pr = si.random_small(31, nx=64, M=3, p=3)
    sp = SGProblem.from_problem(pr).upload()
    ncols = 2 * sp.P
    for call in range(2):                         # two calls in a row share the built-in array
        R = torch.from_numpy(si.random_panel(40 + call, sp.n, ncols)).to("cuda", dtype)
        ref = sp.apply_chebyshev(R, ncols)
        X = torch.full_like(R, float("nan"))
        st = _noalloc(sp, R, X, ncols)
        assert st == abi.SGOC_OK, abi.load().sgoc_last_error()
        torch.cuda.synchronize()
        err = (torch.linalg.norm((X - ref).double()) / torch.linalg.norm(ref.double())).item()
        assert err <= tol, (call, err)


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

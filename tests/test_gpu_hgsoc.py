"""The hGSoc preconditioner (Alg. 2-3; Alg. 4 slab by slab in time mode) on the GPU against
the oracle's HGSoc, and FGMRES solves with it against the oracle's.  Tolerances as in the other
parity tests: float64 preconditioner 1e-12, float32 2e-5; float64 solves within 1e-7 and +-1
iteration; mixed solves reach the 1e-8 float64 residual."""
import numpy as np
import pytest

import sg_inputs as si
from oracle.operators import SGData
from oracle.precond import HGSoc
from oracle.solve import solve as oracle_solve

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def cuda_ready():
    if not torch.cuda.is_available():
        pytest.fail("GPU tests selected but no CUDA device is visible")
    from paper_2512_23804_gb300 import build
    build.build()


def rel(a, b):
    return np.linalg.norm(np.asarray(a) - np.asarray(b)) / max(np.linalg.norm(b), 1e-300)


def make(seed, precision="fp64", mass_solve=None, **kw):
    from paper_2512_23804_gb300 import SGProblem
    pr = si.random_small(seed, **kw)
    pr.precond = "hgsoc"
    pr.krylov = "fgmres"
    if mass_solve:
        pr.mass_solve = mass_solve
    return pr, SGData(pr), SGProblem.from_problem(pr, precision=precision)


CASES = [dict(seed=1, nx=16, M=2, p=2), dict(seed=2, nx=32, M=3, p=3, gamma=0.5),
         dict(seed=3, nx=16, M=2, p=2, nt=3), dict(seed=4, nx=64, M=3, p=2, r=2),
         dict(seed=5, nx=16, M=2, p=2, mass_solve="exact"), dict(seed=6, nx=8, M=2, p=0)]


@pytest.mark.parametrize("case", CASES)
@pytest.mark.parametrize("dtype,tol", [(torch.float64, 1e-12), (torch.float32, 2e-5)])
def test_hgsoc_matches_oracle(case, dtype, tol):
    pr, d, sp = make(precision="fp64" if dtype == torch.float64 else "mixed", **case)
    r = si.random_panel(20 + case["seed"], 3 * d.n, d.P, d.slabs)
    if dtype == torch.float32:
        r = r.astype(np.float32).astype(np.float64)
    z = sp.apply_precond(torch.from_numpy(r).to("cuda", dtype))
    torch.cuda.synchronize()
    assert rel(z.double().cpu().numpy(), HGSoc(d).apply(r)) <= tol


@pytest.mark.parametrize("case", [dict(seed=7, nx=16, M=2, p=2), dict(seed=8, nx=32, M=3, p=2, beta=1e-4),
                                  dict(seed=9, nx=16, M=2, p=2, nt=4, beta=1e-3)])
def test_fgmres_with_hgsoc_matches_oracle(case):
    pr, d, sp = make(**case)
    ref = oracle_solve(pr, data=d)
    assert ref.status == "ok"
    x, info = sp.solve()
    assert info["status_name"] == "SGOC_OK" and info["rel_true_residual"] <= pr.tol
    assert abs(info["iterations"] - ref.iterations) <= 1, (info["iterations"], ref.iterations)
    assert rel(x.cpu().numpy(), ref.x) <= 1e-7
    prm, dm, spm = make(precision="mixed", **case)
    xm, im = spm.solve()
    assert im["status_name"] == "SGOC_OK" and im["rel_true_residual"] <= pr.tol


def test_hgsoc_requires_fgmres():
    """The C ABI rejects hGSoc with MINRES (the preconditioner is not symmetric)."""
    import ctypes
    from paper_2512_23804_gb300 import abi
    pr = si.random_small(10, nx=16, M=2, p=2)
    lib = abi.load()
    opts = abi.Options()
    lib.sgoc_default_options(ctypes.byref(opts))
    opts.precond, opts.krylov = 1, 0
    kap = np.ascontiguousarray(pr.kappa)
    yh = np.ascontiguousarray(pr.yhat)
    dp = lambda a: a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))
    desc = abi.ProblemDesc(pr.nx, pr.M, pr.p, dp(kap), pr.beta, 0.0, 0, 1.0, dp(yh), None)
    h = ctypes.c_void_p()
    st = lib.sgoc_problem_create(ctypes.byref(desc), ctypes.byref(opts), ctypes.byref(h))
    assert abi.STATUS_NAMES[st] == "SGOC_ERR_INVALID_ARG"
    opts.krylov = 1
    st = lib.sgoc_problem_create(ctypes.byref(desc), ctypes.byref(opts), ctypes.byref(h))
    assert st == abi.SGOC_OK
    lib.sgoc_problem_destroy(h)

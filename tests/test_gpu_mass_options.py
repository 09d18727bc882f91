"""Mass-block options of the preconditioner (Sec. 5): the exact solve with the Cholesky
factorisation of M = M1 (x) M1, and the Chebyshev semi-iteration with ten steps, against the
oracle (float64 1e-12, float32 2e-5 for the preconditioner; solves within 1e-7 and +-1
iteration, with MINRES and with FGMRES)."""
import numpy as np
import pytest

import sg_inputs as si
from oracle.operators import SGData
from oracle.precond import BlockPreconditioner, chebyshev
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


def make(seed, precision="fp64", **kw):
    from paper_2512_23804_gb300 import SGProblem
    opts = {k: kw.pop(k) for k in ("mass_solve", "cheb_steps", "krylov") if k in kw}
    pr = si.random_small(seed, **kw)
    for k, v in opts.items():
        setattr(pr, k, v)
    return pr, SGData(pr), SGProblem.from_problem(pr, precision=precision)


@pytest.mark.parametrize("case", [dict(seed=1, nx=16, M=2, p=2), dict(seed=2, nx=64, M=3, p=2, gamma=0.5),
                                  dict(seed=3, nx=16, M=2, p=2, nt=4), dict(seed=4, nx=256, M=1, p=1),
                                  dict(seed=5, nx=2, M=2, p=1)])
@pytest.mark.parametrize("dtype,tol", [(torch.float64, 1e-12), (torch.float32, 2e-5)])
def test_exact_mass_blocks_match_oracle(case, dtype, tol):
    precision = "fp64" if dtype == torch.float64 else "mixed"
    pr, d, sp = make(precision=precision, mass_solve="exact", **case)
    r = si.random_panel(10 + case["seed"], 3 * d.n, d.P, d.slabs)
    if dtype == torch.float32:
        r = r.astype(np.float32).astype(np.float64)
    z = sp.apply_precond(torch.from_numpy(r).to("cuda", dtype))
    torch.cuda.synchronize()
    ref = BlockPreconditioner(d).apply(r)
    F = d.slabs * d.P * d.n
    zh = z.double().cpu().numpy()
    assert rel(zh[:2 * F], ref[:2 * F]) <= tol
    assert rel(zh, ref) <= tol


@pytest.mark.parametrize("dtype,tol", [(torch.float64, 1e-12), (torch.float32, 2e-6)])
def test_chebyshev_ten_steps(dtype, tol):
    pr, d, sp = make(precision="fp64" if dtype == torch.float64 else "mixed", cheb_steps=10, seed=6, nx=64, M=2, p=2)
    ncols = 2 * d.P
    B = si.random_panel(60, d.n, ncols)
    if dtype == torch.float32:
        B = B.astype(np.float32).astype(np.float64)
    X = sp.apply_chebyshev(torch.from_numpy(B).to("cuda", dtype), ncols)
    torch.cuda.synchronize()
    ref = chebyshev(d.Mass, B.reshape(ncols, d.n).T, 10).T.reshape(-1)
    assert rel(X.double().cpu().numpy(), ref) <= tol


@pytest.mark.parametrize("opts", [dict(mass_solve="exact"), dict(cheb_steps=10),
                                  dict(mass_solve="exact", krylov="fgmres")])
def test_solves_with_mass_options_match_oracle(opts):
    pr, d, sp = make(seed=7, nx=32, M=3, p=2, beta=1e-4, **opts)
    ref = oracle_solve(pr, data=d)
    x, info = sp.solve()
    assert info["status_name"] == "SGOC_OK" and info["rel_true_residual"] <= pr.tol
    assert abs(info["iterations"] - ref.iterations) <= 1, (info["iterations"], ref.iterations)
    assert rel(x.cpu().numpy(), ref.x) <= 1e-7

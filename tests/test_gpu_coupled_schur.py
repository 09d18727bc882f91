"""Parity of the time-coupled Schur block (schur="coupled": S_bar of Eq. (S hat) with Z_bar
of Eq. (Z hat), block forward and backward substitution in time with one hGS sweep per slab)
with the oracle, and solves with it.  Tolerances as in the other parity tests: float64
preconditioner 1e-12, float32 preconditioner 2e-5, float64 solve 1e-7 and +-1 iteration."""
import numpy as np
import pytest

import sg_inputs as si
from oracle.operators import SGData
from oracle.precond import BlockPreconditioner
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


def make(seed, precision="fp64", T=None, **kw):
    from paper_2512_23804_gb300 import SGProblem
    pr = si.random_small(seed, **kw)
    if T is not None:
        pr.T = T
    pr.schur = "coupled"
    return pr, SGData(pr), SGProblem.from_problem(pr, precision=precision)


CASES = [dict(seed=1, nx=16, M=2, p=2, nt=4), dict(seed=2, nx=32, M=3, p=2, nt=3, gamma=0.5),
         dict(seed=3, nx=64, M=2, p=2, nt=3, T=0.1), dict(seed=4, nx=8, M=2, p=1, nt=2)]


@pytest.mark.parametrize("case", CASES)
def test_coupled_block_preconditioner_fp64(case):
    pr, d, sp = make(**case)
    r = si.random_panel(30 + case["seed"], 3 * d.n, d.P, d.slabs)
    z = sp.apply_precond(torch.from_numpy(r).cuda())
    torch.cuda.synchronize()
    ref = BlockPreconditioner(d, schur="coupled").apply(r)
    assert rel(z.cpu().numpy(), ref) <= 1e-12


@pytest.mark.parametrize("case", CASES[:3])
def test_coupled_block_preconditioner_fp32(case):
    pr, d, sp = make(precision="mixed", **case)
    r = si.random_panel(40 + case["seed"], 3 * d.n, d.P, d.slabs).astype(np.float32).astype(np.float64)
    z = sp.apply_precond(torch.from_numpy(r).to("cuda", torch.float32))
    torch.cuda.synchronize()
    ref = BlockPreconditioner(d, schur="coupled").apply(r)
    assert rel(z.double().cpu().numpy(), ref) <= 2e-5


@pytest.mark.parametrize("case", [dict(seed=5, nx=16, M=2, p=2, nt=6, beta=1e-1, T=0.06),
                                  dict(seed=6, nx=16, M=3, p=2, nt=4, beta=1e-3)])
def test_coupled_solve_matches_oracle(case):
    pr, d, sp = make(**case)
    ref = oracle_solve(pr, data=d)
    x, info = sp.solve()
    x = x.cpu().numpy()
    assert info["status_name"] == "SGOC_OK" and info["rel_true_residual"] <= pr.tol
    assert abs(info["iterations"] - ref.iterations) <= 1, (info["iterations"], ref.iterations)
    assert rel(x, ref.x) <= 1e-7
    prm, dm, spm = make(precision="mixed", **case)
    xm, im = spm.solve()
    assert im["status_name"] == "SGOC_OK" and im["rel_true_residual"] <= pr.tol
    assert rel(d.kkt_apply(xm.cpu().numpy()), d.rhs()) <= pr.tol * 1.01

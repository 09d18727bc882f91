"""FGMRES on the GPU (sgoc_options.krylov = 1, the Krylov method of Sec. 5) against the
oracle's FGMRES: float64 solves within 1e-7 of the oracle solution with iteration counts
within +-1 (same stopping rule, Gram-Schmidt variants differing only by rounding), restarted
cycles, and the mixed-precision form (float32 FGMRES inner solves in float64 refinement)
reaching the same 1e-8 float64 residual."""
import numpy as np
import pytest

import sg_inputs as si
from oracle.operators import SGData
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


CASES = [dict(seed=1, nx=16, M=2, p=2), dict(seed=2, nx=32, M=3, p=3, beta=1e-4),
         dict(seed=3, nx=16, M=2, p=2, nt=4, beta=1e-3), dict(seed=4, nx=64, M=2, p=2, gamma=0.5)]


@pytest.mark.parametrize("case", CASES)
def test_fgmres_fp64_matches_oracle(case):
    from paper_2512_23804_gb300 import SGProblem
    c = dict(case)
    pr = si.random_small(c.pop("seed"), **c)
    pr.krylov = "fgmres"
    d = SGData(pr)
    ref = oracle_solve(pr, data=d)
    assert ref.status == "ok"
    x, info = SGProblem.from_problem(pr).solve()
    x = x.cpu().numpy()
    assert info["status_name"] == "SGOC_OK" and info["rel_true_residual"] <= pr.tol
    assert abs(info["iterations"] - ref.iterations) <= 1, (info["iterations"], ref.iterations)
    assert rel(x, ref.x) <= 1e-7
    assert rel(d.kkt_apply(x), d.rhs()) <= pr.tol * 1.01


def test_fgmres_restarted_cycles_converge():
    from paper_2512_23804_gb300 import SGProblem
    pr = si.random_small(5, nx=32, M=3, p=2, beta=1e-4)
    pr.krylov = "fgmres"
    d = SGData(pr)
    x, info = SGProblem.from_problem(pr, restart=8).solve()
    assert info["status_name"] == "SGOC_OK" and info["rel_true_residual"] <= pr.tol
    assert rel(d.kkt_apply(x.cpu().numpy()), d.rhs()) <= pr.tol * 1.01
    x64, i64 = SGProblem.from_problem(pr).solve()
    assert info["iterations"] >= i64["iterations"]


@pytest.mark.parametrize("case", CASES[1:3])
def test_fgmres_mixed_reaches_fp64_residual(case):
    from paper_2512_23804_gb300 import SGProblem
    c = dict(case)
    pr = si.random_small(c.pop("seed"), **c)
    pr.krylov = "fgmres"
    d = SGData(pr)
    x, info = SGProblem.from_problem(pr, precision="mixed").solve()
    assert info["status_name"] == "SGOC_OK" and info["rel_true_residual"] <= pr.tol
    assert rel(d.kkt_apply(x.cpu().numpy()), d.rhs()) <= pr.tol * 1.01
    x64, _ = SGProblem.from_problem(pr).solve()
    assert rel(x.cpu().numpy(), x64.cpu().numpy()) <= 1e-6

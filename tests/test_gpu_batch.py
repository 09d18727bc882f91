"""Concurrent solves (sgoc_solve_batch): each result equals the same solve alone."""
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


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_batch_equals_alone(precision):
    from paper_2512_23804_gb300 import SGProblem, solve_batch
    prs = [si.random_small(1, nx=16, M=2, p=2), si.random_small(2, nx=32, M=3, p=3, beta=1e-4),
           si.random_small(3, nx=16, M=2, p=2, nt=4, beta=1e-3), si.random_small(4, nx=64, M=2, p=1, gamma=0.5)]
    alone = []
    for pr in prs:
        x, info = SGProblem.from_problem(pr, precision=precision).solve()
        alone.append((x.clone(), info))
    sps = [SGProblem.from_problem(pr, precision=precision) for pr in prs]
    xs, infos = solve_batch(sps)
    torch.cuda.synchronize()
    for (xa, ia), xb, ib in zip(alone, xs, infos):
        assert ib["status_name"] == "SGOC_OK"
        assert ia["iterations"] == ib["iterations"]
        assert torch.equal(xa, xb)          # same kernels, same order: bitwise identical


def test_batch_reports_per_problem_failure():
    from paper_2512_23804_gb300 import SGProblem, solve_batch, abi
    good = SGProblem.from_problem(si.random_small(5, nx=16, M=2, p=2))
    bad = SGProblem.from_problem(si.random_small(6, nx=16, M=2, p=2), max_iter=2)
    with pytest.raises(abi.SgocError):
        solve_batch([good, bad])
    # the good one still converged; solving it again alone gives the same answer
    x1, i1 = good.solve()
    assert i1["status_name"] == "SGOC_OK"

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


SAME_SHAPE = {
    # steady, one slab: the level-0 first visit reads R in place, first visits store into V
    "steady": [dict(seed=11, nx=32, M=3, p=3, beta=1e-2), dict(seed=12, nx=32, M=3, p=3, beta=1e-4),
               dict(seed=13, nx=32, M=3, p=3, beta=1e-6, gamma=0.5)],
    # several slabs: strided right-hand sides and stored strided corrections
    "time": [dict(seed=14, nx=64, M=2, p=2, nt=3, beta=1e-3), dict(seed=15, nx=64, M=2, p=2, nt=3, beta=1e-4),
             dict(seed=16, nx=64, M=2, p=2, nt=3, beta=1e-2, T=0.5)],
}


@pytest.mark.parametrize("kind", ["steady", "time"])
@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_same_shape_batch_runs_merged_and_equals_alone(kind, precision):
    """With the merged schedule (sgoc_solve_batch_merged), problems of one shape (grid, chaos
    levels, slabs) but different beta, gamma, time step and coefficient fields are grouped: their hGS sweeps run as merged launches over the
    whole group.  Each result equals its solo solve bit for bit, a problem of another shape in
    the same batch is unaffected, and the merged batch launches fewer kernels than the solo
    solves together."""
    from paper_2512_23804_gb300 import SGProblem, abi, solve_batch
    if precision == "fp64":            # float64 V-cycles run one CTA per column up to 15 x 15 nodes
        cases = [dict(c, nx=16) for c in SAME_SHAPE[kind]]
    else:
        cases = SAME_SHAPE[kind]
    prs = []
    for c in cases:
        c = dict(c)
        T = c.pop("T", None)
        pr = si.random_small(c.pop("seed"), **c)
        if T is not None:
            pr.T = T
        prs.append(pr)
    prs.append(si.random_small(20, nx=16, M=2, p=1, beta=1e-3))      # another shape
    lib = abi.load()
    alone, solo_launches = [], 0
    for pr in prs:
        sp = SGProblem.from_problem(pr, precision=precision)
        sp.upload()
        torch.cuda.synchronize()
        k0 = lib.sgoc_kernel_launches()
        x, info = sp.solve()
        solo_launches += lib.sgoc_kernel_launches() - k0
        alone.append((x.clone(), info))
    sps = [SGProblem.from_problem(pr, precision=precision) for pr in prs]
    for sp in sps:
        sp.upload()
        sp.workspace()
    torch.cuda.synchronize()
    k0 = lib.sgoc_kernel_launches()
    xs, infos = solve_batch(sps, merged=True)
    torch.cuda.synchronize()
    batch_launches = lib.sgoc_kernel_launches() - k0
    for (xa, ia), xb, ib in zip(alone, xs, infos):
        assert ib["status_name"] == "SGOC_OK"
        assert ia["iterations"] == ib["iterations"] and ia["outer_iterations"] == ib["outer_iterations"]
        assert torch.equal(xa, xb)
    assert batch_launches < 0.85 * solo_launches, (batch_launches, solo_launches)
    # a second batch of the same problems reuses the captured group iterations
    xs2, infos2 = solve_batch(sps, merged=True)
    for xb, x2 in zip(xs, xs2):
        assert torch.equal(xb, x2)

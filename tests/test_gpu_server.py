"""Serving loop: requests that arrive while others run are admitted as slots and
memory free up; each result equals the same request solved alone."""
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


def _requests():
    return [si.random_small(10 + i, nx=[16, 32, 8, 64][i % 4], M=2 + i % 3, p=1 + i % 3,
                            nt=(3 if i % 5 == 4 else 0), beta=[1e-2, 1e-4, 1e-3][i % 3]) for i in range(10)]


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_server_results_equal_alone(precision):
    from paper_2512_23804_gb300 import SGProblem, SGServer
    prs = _requests()
    alone = [SGProblem.from_problem(pr, precision=precision).solve() for pr in prs]
    sps = [SGProblem.from_problem(pr, precision=precision) for pr in prs]
    need = max(sp.persistent_bytes + sp.workspace_bytes for sp in sps) + 4096
    sv = SGServer(pool_bytes=3 * need, max_active=3)     # memory and slots both limit admission
    got = {}
    submitted = 0
    for step in range(100000):
        # staggered arrivals: one new request every few sweeps
        if submitted < len(sps) and step % 3 == 0:
            sv.submit(sps[submitted], submitted)
            submitted += 1
        na, nq = sv.step()
        for rid, x, info in sv.poll():
            got[rid] = (x, info)
        if submitted == len(sps) and sv.pending == 0:
            break
    assert len(got) == len(sps)
    for i, (xa, ia) in enumerate(alone):
        x, info = got[i]
        assert info["status_name"] == "SGOC_OK", info
        assert info["iterations"] == ia["iterations"]
        assert torch.equal(x, xa), i
    st = sv.stats()
    assert st["admitted"] == len(sps) and st["completed"] == len(sps)
    assert st["pool_high_water"] <= 3 * need


def test_server_rejects_request_larger_than_pool():
    from paper_2512_23804_gb300 import SGProblem, SGServer, abi
    sp = SGProblem.from_problem(si.random_small(3, nx=32, M=2, p=2))
    sv = SGServer(pool_bytes=1 << 20, max_active=1)
    with pytest.raises(abi.SgocError) as ei:
        sv.submit(sp, 0)
    assert abi.STATUS_NAMES[ei.value.status] == "SGOC_ERR_WORKSPACE_TOO_SMALL"


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_failing_requests_retire_with_status_and_leave_the_others_unchanged(precision):
    """Two requests that cannot converge (iteration caps of 2 and 3, one of them
    time-dependent) are retired with SGOC_ERR_NO_CONVERGENCE while they share the GPU
    with healthy requests; every healthy request still equals its solo solve bit for
    bit.  A request with a NaN in its target never reaches the server: problem set-up
    rejects it with SGOC_ERR_NAN."""
    import numpy as np
    from paper_2512_23804_gb300 import SGProblem, SGServer, abi
    nan_pr = si.random_small(40, nx=32, M=2, p=2)
    nan_pr.yhat = nan_pr.yhat.copy()
    nan_pr.yhat[0, 17] = np.nan
    with pytest.raises(abi.SgocError) as ei:
        SGProblem.from_problem(nan_pr, precision=precision)
    assert abi.STATUS_NAMES[ei.value.status] == "SGOC_ERR_NAN"
    prs = _requests()[:6]
    alone = [SGProblem.from_problem(pr, precision=precision).solve() for pr in prs]
    sps = [SGProblem.from_problem(pr, precision=precision) for pr in prs]
    bad = {100: SGProblem.from_problem(si.random_small(41, nx=32, M=3, p=2, beta=1e-4), precision=precision,
                                       max_iter=2, max_outer=1),
           101: SGProblem.from_problem(si.random_small(42, nx=16, M=2, p=2, nt=3, beta=1e-3), precision=precision,
                                       max_iter=3, max_outer=1)}
    order = [(0, sps[0]), (100, bad[100]), (1, sps[1]), (2, sps[2]), (101, bad[101])] + \
            [(i, sps[i]) for i in range(3, len(sps))]
    sv = SGServer(pool_bytes=1 << 30, max_active=4)
    got = {}
    submitted = 0
    for step in range(100000):
        if submitted < len(order) and step % 2 == 0:
            rid, sp = order[submitted]
            sv.submit(sp, rid)
            submitted += 1
        sv.step()
        for rid, x, info in sv.poll():
            got[rid] = (x, info)
        if submitted == len(order) and sv.pending == 0:
            break
    assert len(got) == len(order)
    for rid in bad:
        assert got[rid][1]["status_name"] == "SGOC_ERR_NO_CONVERGENCE", got[rid][1]
    for i, (xa, ia) in enumerate(alone):
        x, info = got[i]
        assert info["status_name"] == "SGOC_OK", info
        assert info["iterations"] == ia["iterations"]
        assert torch.equal(x, xa), i
    st = sv.stats()
    assert st["completed"] == len(order) and st["rejected"] == 0

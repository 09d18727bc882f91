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

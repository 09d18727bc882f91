"""SG kernel variants and the autotuner.

SG kernel variants 0-6 form the same products and sums in the same order, so they
must agree bit for bit and each must match the oracle within the operator
tolerances (1e-13 float64, 2e-6 float32); the register kernel 7 (float32, some
Legendre (M, p)) sums coupling terms in another order and is checked against them
and the oracle to rounding in test_gpu_sg_register.py.  Tuning changes only the
kernel choice: a solve after sgoc_autotune returns the identical solution, or, when
the tuner picked kernel 7 somewhere, the same solution to rounding.
"""
import numpy as np
import pytest

import sg_inputs as si
from oracle.operators import SGData

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


CASES = [dict(seed=61, nx=64, M=3, p=3), dict(seed=62, nx=32, M=2, p=2, nt=3), dict(seed=63, nx=128, M=6, p=3),
         dict(seed=64, nx=16, M=2, p=2)]


@pytest.mark.parametrize("case", CASES)
@pytest.mark.parametrize("dtype,tol", [(torch.float64, 1e-13), (torch.float32, 2e-6)])
def test_sg_variants_agree_bitwise(case, dtype, tol):
    from paper_2512_23804_gb300 import SGProblem, abi
    c = dict(case)
    pr = si.random_small(c.pop("seed"), **c)
    d = SGData(pr)
    sp = SGProblem.from_problem(pr)
    X = si.random_panel(70, d.n, d.P, d.slabs)
    if dtype == torch.float32:
        X = X.astype(np.float32).astype(np.float64)
    ps = d.P * d.n
    ref = np.concatenate([d.vec(d.sg_apply(d.mat(X[t * ps:(t + 1) * ps]))) for t in range(d.slabs)])
    Xd = torch.from_numpy(X).to("cuda", dtype)
    outs = []
    for v in range(7):
        try:
            Y = sp.apply_operator_variant(Xd, v, nslabs=d.slabs)
        except abi.SgocError as e:
            assert e.status == abi.SGOC_ERR_UNSUPPORTED
            continue
        torch.cuda.synchronize()
        outs.append((v, Y.double().cpu().numpy()))
    assert len(outs) >= 1 and outs[0][0] == 0          # the one-phase kernel always applies
    for v, Y in outs:
        assert rel(Y, ref) <= tol, v
    for v, Y in outs[1:]:
        assert np.array_equal(Y, outs[0][1]), v


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_autotune_keeps_the_solution(precision):
    from paper_2512_23804_gb300 import SGProblem
    pr = si.random_small(65, nx=64, M=3, p=3, beta=1e-4)
    sp = SGProblem.from_problem(pr, precision=precision)
    x0, i0 = sp.solve()
    x0 = x0.clone()
    chosen = sp.autotune()
    assert len(chosen) == 2 * pr.p + 4
    assert all(0 <= v <= 7 for v in chosen)
    x1, i1 = sp.solve()
    if 7 in chosen:
        assert abs(i1["iterations"] - i0["iterations"]) <= 2
        assert i1["rel_true_residual"] <= 1e-8
        assert float(torch.linalg.norm(x1 - x0) / torch.linalg.norm(x0)) <= 1e-7
    else:
        assert i1["iterations"] == i0["iterations"]
        assert torch.equal(x1, x0)


@pytest.mark.parametrize("dtype,tol", [(torch.float64, 1e-12), (torch.float32, 2e-5)])
def test_pinned_kernels_in_hgs_and_kkt(dtype, tol):
    """Every applicable SG kernel pinned on every SG shape of a solve: the hGS sweep (mass
    term and right-hand side in the epilogue) matches the oracle and all kernels agree bit
    for bit; so does the KKT product."""
    from paper_2512_23804_gb300 import SGProblem, abi
    from oracle.precond import BlockPreconditioner
    pr = si.random_small(66, nx=64, M=3, p=3, beta=1e-3)
    d = SGData(pr)
    prec = "fp64" if dtype == torch.float64 else "mixed"
    sp = SGProblem.from_problem(pr, precision=prec).upload()
    pc = BlockPreconditioner(d)
    R = si.random_panel(71, d.n, d.P)
    v = si.random_panel(72, 3 * d.n, d.P)
    if dtype == torch.float32:
        R = R.astype(np.float32).astype(np.float64)
        v = v.astype(np.float32).astype(np.float64)
    ref_h = d.vec(pc.hgs.apply(d.mat(R)))
    ref_k = d.kkt_apply(v)
    Rd = torch.from_numpy(R).to("cuda", dtype)
    vd = torch.from_numpy(v).to("cuda", dtype)
    pid = 0 if dtype == torch.float64 else 1
    shapes = [0, 1] + [2 + lev for lev in range(2 * pr.p + 2)]
    outs = []
    try:
        for var in range(7):
            for sh in shapes:
                try:
                    sp.set_kernel(sh, var, precision=pid)
                except abi.SgocError as e:           # not applicable here: the built-in choice
                    assert e.status == abi.SGOC_ERR_UNSUPPORTED
                    sp.set_kernel(sh, -1, precision=pid)
            h = sp.apply_hgs(Rd)
            k = sp.apply_kkt(vd)
            torch.cuda.synchronize()
            h = h.double().cpu().numpy()
            k = k.double().cpu().numpy()
            assert rel(h, ref_h) <= tol, var
            assert rel(k, ref_k) <= (1e-13 if dtype == torch.float64 else 2e-6), var
            outs.append((var, h, k))
    finally:
        for sh in shapes:
            sp.set_kernel(sh, -1, precision=pid)
    for var, h, k in outs[1:]:
        assert np.array_equal(h, outs[0][1]), var
        assert np.array_equal(k, outs[0][2]), var

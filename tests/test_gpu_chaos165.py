"""Parity at the large chaos shapes of the workloads (M = 8, p = 3, P = 165 and the
serving stream's M = 8, p = 4, P = 495) and for the multi-slab hGS paths.

P = 165 is the shape of the 512 x 512 steady workload.  Its table and staging
offsets are the ones where a misaligned shared-memory access once occurred, so
every SG kernel variant, the KKT product, the hGS sweep (full and truncated) and
the block preconditioner are checked here against the oracle on small grids of
that chaos shape.  Tolerances are those of the other parity tests: float64
operator products 1e-13, float64 preconditioner pieces 1e-12, float32 operator
products 2e-6, float32 preconditioner pieces 2e-5 (about fifty chained float32
stencil passes).

The hGS sweep stores the correction of the first visit of each level into its
output without clearing it first; the multi-slab cases fill the output with NaN
before the call, so any value read before its first store fails the test.
"""
import numpy as np
import pytest

import sg_inputs as si
from oracle.operators import SGData
from oracle.precond import BlockPreconditioner

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def cuda_ready():
    if not torch.cuda.is_available():
        pytest.fail("GPU tests selected but no CUDA device is visible")
    from paper_2512_23804_gb300 import build
    build.build()


def rel(a, b):
    a = np.asarray(a, dtype=np.float64)
    b = np.asarray(b, dtype=np.float64)
    return np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300)


def dev(x, dtype=torch.float64):
    return torch.from_numpy(np.ascontiguousarray(x)).to("cuda", dtype)


def host(t):
    torch.cuda.synchronize()
    return t.double().cpu().numpy()


def make(seed, precision="fp64", **kw):
    from paper_2512_23804_gb300 import SGProblem
    pr = si.random_small(seed, **kw)
    return pr, SGData(pr), SGProblem.from_problem(pr, precision=precision)


def slabwise(d, X, f):
    ps = d.P * d.n
    return np.concatenate([d.vec(f(d.mat(X[t * ps:(t + 1) * ps]))) for t in range(d.slabs)])


SHAPES = [dict(nx=32, M=8, p=3), dict(nx=64, M=8, p=3), dict(nx=16, M=8, p=3, nt=2)]


@pytest.mark.parametrize("shape", SHAPES, ids=["32x32", "64x64", "16x16_nt2"])
@pytest.mark.parametrize("dtype,tol", [(torch.float64, 1e-13), (torch.float32, 2e-6)])
def test_sg_operator_every_variant_p165(shape, dtype, tol):
    from paper_2512_23804_gb300 import abi
    pr, d, sp = make(165, **shape)
    assert d.P == 165
    X = si.random_panel(166, d.n, d.P, d.slabs)
    if dtype == torch.float32:
        X = X.astype(np.float32).astype(np.float64)
    ref = slabwise(d, X, d.sg_apply)
    Xd = dev(X, dtype)
    outs = []
    for v in range(7):
        try:
            Y = sp.apply_operator_variant(Xd, v, nslabs=d.slabs)
        except abi.SgocError as e:
            assert e.status == abi.SGOC_ERR_UNSUPPORTED
            continue
        outs.append((v, host(Y)))
    assert outs and outs[0][0] == 0
    for v, Y in outs:
        assert rel(Y, ref) <= tol, v
        assert np.array_equal(Y, outs[0][1]), v
    # the tuned/default choice (sgoc_apply_operator) agrees with them too
    assert np.array_equal(host(sp.apply_operator(Xd, nslabs=d.slabs)), outs[0][1])


@pytest.mark.parametrize("shape", SHAPES[::2], ids=["32x32", "16x16_nt2"])
def test_kkt_and_block_preconditioner_p165(shape):
    pr, d, sp = make(167, **shape)
    v = si.random_panel(168, 3 * d.n, d.P, d.slabs)
    assert rel(host(sp.apply_kkt(dev(v))), d.kkt_apply(v)) <= 1e-13
    r = si.random_panel(169, 3 * d.n, d.P, d.slabs)
    z = host(sp.apply_precond(dev(r)))
    assert rel(z, BlockPreconditioner(d).apply(r)) <= 1e-12


@pytest.mark.parametrize("r", [-1, 3])          # -1: all M + 1 terms
def test_hgs_p165(r):
    pr, d, sp = make(170, nx=32, M=8, p=3, r=r)
    Pc = BlockPreconditioner(d)
    R = si.random_panel(171, d.n, d.P)
    V = torch.full((d.n * d.P,), float("nan"), dtype=torch.float64, device="cuda")
    out = host(sp.apply_hgs(dev(R), out=V))
    assert rel(out, d.vec(Pc.hgs.apply(d.mat(R)))) <= 1e-12


def test_kkt_fp32_p165():
    pr, d, sp = make(172, precision="mixed", nx=32, M=8, p=3)
    v = si.random_panel(173, 3 * d.n, d.P).astype(np.float32).astype(np.float64)
    w = host(sp.apply_kkt(dev(v, torch.float32)))
    assert rel(w, d.kkt_apply(v)) <= 2e-6


MULTI_SLAB = [
    # (seed, precision, dtype, tol, shape)
    (180, "mixed", torch.float32, 2e-5, dict(nx=64, M=3, p=3, nt=3, beta=1e-3)),   # packed 63x63 level 0
    (181, "mixed", torch.float32, 2e-5, dict(nx=16, M=2, p=2, nt=4, beta=1e-3)),
    (182, "fp64", torch.float64, 1e-12, dict(nx=16, M=2, p=2, nt=4, beta=1e-3)),
    (183, "fp64", torch.float64, 1e-12, dict(nx=64, M=2, p=2, nt=2, beta=1e-3)),   # cluster cycles
]


@pytest.mark.parametrize("seed,precision,dtype,tol,shape", MULTI_SLAB,
                         ids=["f32_64x64_nt3", "f32_16x16_nt4", "f64_16x16_nt4", "f64_64x64_nt2"])
def test_hgs_multi_slab_nan_filled_output(seed, precision, dtype, tol, shape):
    pr, d, sp = make(seed, precision=precision, **shape)
    Pc = BlockPreconditioner(d)
    R = si.random_panel(seed + 1, d.n, d.P, d.slabs)
    if dtype == torch.float32:
        R = R.astype(np.float32).astype(np.float64)
    V = torch.full((d.slabs * d.n * d.P,), float("nan"), dtype=dtype, device="cuda")
    out = host(sp.apply_hgs(dev(R, dtype), out=V))
    assert np.isfinite(out).all()
    assert rel(out, slabwise(d, R, Pc.hgs.apply)) <= tol


@pytest.mark.parametrize("dtype,tol", [(torch.float64, 1e-13), (torch.float32, 2e-6)])
def test_p495_operator_kkt_and_hgs(dtype, tol):
    """M = 8, p = 4 (P = 495), the largest chaos shape of the serving stream: in float64 no
    shared-memory-staged SG kernel holds the 495 input columns of the full operator, and the
    direct kernel (no shared memory) applies; its results match the oracle and the float32
    staged kernels."""
    precision = "fp64" if dtype == torch.float64 else "mixed"
    pr, d, sp = make(495, precision=precision, nx=16, M=8, p=4)
    assert d.P == 495
    X = si.random_panel(496, d.n, d.P)
    v = si.random_panel(497, 3 * d.n, d.P)
    if dtype == torch.float32:
        X = X.astype(np.float32).astype(np.float64)
        v = v.astype(np.float32).astype(np.float64)
    Y = host(sp.apply_operator(dev(X, dtype)))
    assert rel(Y, d.vec(d.sg_apply(d.mat(X)))) <= tol
    if dtype == torch.float64:                     # the direct kernel is the only form here
        assert np.array_equal(host(sp.apply_operator_variant(dev(X, dtype), 6)), Y)
    assert rel(host(sp.apply_kkt(dev(v, dtype))), d.kkt_apply(v)) <= tol
    R = si.random_panel(498, d.n, d.P)
    if dtype == torch.float32:
        R = R.astype(np.float32).astype(np.float64)
    out = host(sp.apply_hgs(dev(R, dtype)))
    assert rel(out, d.vec(BlockPreconditioner(d).hgs.apply(d.mat(R)))) <= (1e-12 if dtype == torch.float64 else 2e-5)


def test_p495_mixed_solve_reaches_the_float64_residual():
    from paper_2512_23804_gb300 import SGProblem
    pr = si.random_small(499, nx=32, M=8, p=4, beta=1e-3)
    d = SGData(pr)
    x, info = SGProblem.from_problem(pr, precision="mixed").solve()
    assert info["status_name"] == "SGOC_OK" and info["rel_true_residual"] <= 1e-8
    xh = host(x)
    assert rel(d.kkt_apply(xh), d.rhs()) <= 1.01e-8

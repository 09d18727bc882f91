"""Exact mean solves by fast diagonalisation on the tensor cores (mean_solve = "exact"),
against the oracle's exact mode (a sparse LU solve with the assembled mean operator).

Tolerance.  Every one of the four products with the sine transform splits both factors
into two bfloat16 terms and accumulates hi*hi + hi*lo + lo*hi in float32: the dropped
lo*lo term and the rounding of the second term leave ~3 * 2^-18 ~ 1.1e-5 of |A||B| per
product (independent signs over the K terms), float32 accumulation ~2^-24 sqrt(128) ~ 7e-7;
four chained products with the eigenvalue scaling between them stay below ~5e-5 for these
test vectors.  The tests use 1e-4 (2-norm relative over a panel, and per column 2e-4), and
2e-4 where a whole hGS sweep or preconditioner (2p + 1 mean solves with float32 SG products
and Chebyshev mass blocks between them) is compared.
"""
import dataclasses

import numpy as np
import pytest

import sg_inputs as si
from oracle.operators import SGData
from oracle.precond import BlockPreconditioner, ExactSolve

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


def dev(x, dtype=torch.float32):
    return torch.from_numpy(np.ascontiguousarray(x)).to("cuda", dtype)


def host(t):
    torch.cuda.synchronize()
    return t.double().cpu().numpy()


def problem(seed, **kw):
    from paper_2512_23804_gb300 import SGProblem
    pr = dataclasses.replace(si.random_small(seed, **kw), mean_solve="exact")
    return pr, SGData(pr), SGProblem.from_problem(pr, precision="mixed")


def slabwise(d, X, f):
    ps = d.P * d.n
    return np.concatenate([d.vec(f(d.mat(X[t * ps:(t + 1) * ps]))) for t in range(d.slabs)])


# (nx, shape, ncols): one column, exactly one tile (64: two columns a tile), ragged tiles, many tiles
MEAN_CASES = [
    (64, dict(M=2, p=2), 1), (64, dict(M=2, p=2), 2), (64, dict(M=2, p=2), 3),
    (64, dict(M=3, p=3, nt=3), 29), (128, dict(M=2, p=2), 1), (128, dict(M=2, p=2), 3),
    (128, dict(M=6, p=3), 56),
]


@pytest.mark.parametrize("nx,shape,ncols", MEAN_CASES,
                         ids=[f"{c[0]}_{'t' if c[1].get('nt') else 's'}_{c[2]}" for c in MEAN_CASES])
def test_exact_mean_solve_matches_oracle_lu(nx, shape, ncols):
    pr, d, sp = problem(300 + nx + ncols, nx=nx, beta=1e-4, **shape)
    A0 = BlockPreconditioner(d, mode="exact").A0        # A~_1 (steady) / A^_1 (time)
    B = si.random_panel(301 + ncols, d.n, ncols).astype(np.float32).astype(np.float64)
    X = host(sp.apply_vcycle(dev(B), ncols)).reshape(ncols, d.n)
    ref = ExactSolve(A0).apply(B.reshape(ncols, d.n).T).T
    assert rel(X, ref) <= 1e-4
    for c in range(ncols):
        assert rel(X[c], ref[c]) <= 2e-4, c
    # the residual of the mean operator itself, independent of the LU solve
    assert rel((A0 @ X.T).T, B.reshape(ncols, d.n)) <= 1e-4


@pytest.mark.parametrize("nx", [64, 128])
def test_exact_mean_solve_smooth_and_single_mode_inputs(nx):
    """A single sine mode is an eigenvector: the solve returns it divided by its eigenvalue
    lambda = d + 2e (cos a + cos b) + 4c cos a cos b of the stencil; a smooth bump (low modes
    only, where 1 / lambda is largest) matches the LU solve.  For the highest modes (lambda near
    its maximum) the ~1e-5 transform error that leaks into the low modes is multiplied by their
    much larger 1 / lambda relative to the mode's own 1 / lambda: 5e-4 there, 1e-4 otherwise."""
    pr, d, sp = problem(320 + nx, nx=nx, M=4, p=2, beta=1e-2)        # 10 columns on the top level
    Pc = BlockPreconditioner(d, mode="exact")
    n1 = nx - 1
    g = np.arange(1, n1 + 1) / nx
    modes = [(1, 1), (3, 7), (n1, 1), (n1 // 2, n1)]
    cols = [np.outer(np.sin(np.pi * j * g), np.sin(np.pi * i * g)).reshape(-1) for i, j in modes]
    yy, xx = np.meshgrid(g, g, indexing="ij")
    cols.append(np.exp(-30 * ((xx - 0.4) ** 2 + (yy - 0.6) ** 2)).reshape(-1))
    B = np.stack(cols)
    X = host(sp.apply_vcycle(dev(B), len(cols))).reshape(len(cols), d.n)
    A0 = Pc.A0.tocsr()
    dg, ed, co = A0[n1 + 1, n1 + 1], A0[n1 + 1, n1 + 2], A0[n1 + 1, 2 * n1 + 2]   # interior node's stencil
    for q, (i, j) in enumerate(modes):
        ca, cb = np.cos(np.pi * i / nx), np.cos(np.pi * j / nx)
        lam = dg + 2 * ed * (ca + cb) + 4 * co * ca * cb
        assert rel(X[q], B[q] / lam) <= (5e-4 if max(i, j) == n1 else 1e-4), (i, j)
    assert rel(X[-1], ExactSolve(Pc.A0).apply(B[-1])) <= 1e-4


SWEEP_CASES = [(64, dict(M=3, p=2)), (64, dict(M=2, p=2, nt=3)), (128, dict(M=3, p=2)),
               (128, dict(M=2, p=3, nt=2))]


@pytest.mark.parametrize("nx,shape", SWEEP_CASES, ids=["64s", "64t3", "128s", "128t2"])
def test_exact_mean_hgs_sweep(nx, shape):
    """The hGS sweep (Alg. 1) with exact mean solves: stored first visits (strided over
    slabs, into a NaN-filled output), accumulated returns, the level-0 right-hand side read
    in place; against the oracle sweep with B = A~_1^{-1}."""
    pr, d, sp = problem(340 + nx + d_slabs(shape), nx=nx, beta=1e-3, **shape)
    Pc = BlockPreconditioner(d, mode="exact")
    R = si.random_panel(341, d.n, d.P, d.slabs).astype(np.float32).astype(np.float64)
    V = torch.full((d.slabs * d.n * d.P,), float("nan"), dtype=torch.float32, device="cuda")
    out = host(sp.apply_hgs(dev(R), out=V))
    assert np.isfinite(out).all()
    assert rel(out, slabwise(d, R, Pc.hgs.apply)) <= 2e-4


def d_slabs(shape):
    return shape.get("nt", 0)


@pytest.mark.parametrize("nx,shape", [(64, dict(M=3, p=2)), (64, dict(M=2, p=2, nt=3)),
                                      (128, dict(M=2, p=2))], ids=["64s", "64t3", "128s"])
def test_exact_mean_block_preconditioner(nx, shape):
    pr, d, sp = problem(360 + nx + d_slabs(shape), nx=nx, beta=1e-3, **shape)
    r = si.random_panel(361, 3 * d.n, d.P, d.slabs).astype(np.float32).astype(np.float64)
    z = host(sp.apply_precond(dev(r)))
    assert rel(z, BlockPreconditioner(d, mode="exact").apply(r)) <= 2e-4


@pytest.mark.parametrize("nx,shape,beta", [(64, dict(M=3, p=2), 1e-4), (64, dict(M=2, p=2, nt=4), 1e-3),
                                           (128, dict(M=4, p=2), 1e-4)], ids=["64s", "64t4", "128s"])
def test_exact_mean_mixed_solve_reaches_float64_residual(nx, shape, beta):
    from paper_2512_23804_gb300 import SGProblem
    pr, d, sp = problem(380 + nx + d_slabs(shape), nx=nx, beta=beta, **shape)
    x, info = sp.solve()
    assert info["status_name"] == "SGOC_OK" and info["rel_true_residual"] <= 1e-8
    xh = host(x)
    assert rel(d.kkt_apply(xh), d.rhs()) <= 1.01e-8
    # same optimum as the float64 solve with V-cycle mean solves
    x64, i64 = SGProblem.from_problem(dataclasses.replace(pr, mean_solve="vcycle"), precision="fp64").solve()
    assert rel(xh, host(x64)) <= 1e-6


@pytest.mark.parametrize("merged", [False, True], ids=["streams", "merged"])
@pytest.mark.parametrize("nx,nt", [(64, 0), (128, 0), (64, 2)], ids=["64", "128", "64_nt2"])
def test_exact_mean_solve_batch_equals_alone(merged, nx, nt):
    """Concurrent solves with exact mean solves return the solutions of the solo runs: on
    independent streams, and in the merged schedule, where each hGS level visit is one mean-solve
    launch over all members (member tables; at 64 x 64 two columns share a tile, but never two
    members)."""
    from paper_2512_23804_gb300 import SGProblem, solve_batch
    prs = [dataclasses.replace(si.random_small(390 + i, nx=nx, M=3, p=2, nt=nt, beta=b), mean_solve="exact")
           for i, b in enumerate([1e-2, 1e-4, 1e-6])]
    alone = [host(SGProblem.from_problem(pr, precision="mixed").solve()[0]) for pr in prs]
    sps = [SGProblem.from_problem(pr, precision="mixed") for pr in prs]
    xs, infos = solve_batch(sps, merged=merged)
    for x, a, info in zip(xs, alone, infos):
        assert info["status_name"] == "SGOC_OK"
        assert np.array_equal(host(x), a)

"""Parity of the CUDA path with the FP64 oracle (same seeded inputs).

Tolerances
* float64 operator products (SG apply, KKT): 1e-13 relative in the 2-norm.
* float64 preconditioner pieces (Chebyshev, V-cycle, hGS, block preconditioner):
  1e-12 relative: fixed linear maps of O(10) chained stencil sweeps whose results
  differ from the oracle only by summation order.
* float64 solves: solution within 1e-7 relative to the oracle's MINRES solution,
  iteration counts within +-1, true residual <= tol.
* float32 operator products: 2e-6 relative in the 2-norm; float32 rounding
  (2^-24 = 6e-8) accumulated over the ~40 terms of one output, amplified by the
  cancellation of the stencil's positive centre against its negative neighbours
  (|A||X| <= 4|AX| for these test vectors): 40 * 6e-8 * 4 ~ 1e-5 worst case per
  entry, ~2e-6 in the 2-norm for independent rounding errors.
"""
import dataclasses

import numpy as np
import pytest

import sg_inputs as si
from oracle import basis
from oracle.operators import SGData
from oracle.precond import BlockPreconditioner, HGS, VCycle, chebyshev
from oracle.solve import solve as oracle_solve

torch = pytest.importorskip("torch")

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def cuda_ready():
    if not torch.cuda.is_available():
        pytest.fail("GPU tests selected but no CUDA device is visible")
    from paper_2512_23804_gb300 import build
    build.build()


from paper_2512_23804_gb300 import SGProblem  # noqa: E402


def rel(a, b):
    a = np.asarray(a, dtype=np.float64)
    b = np.asarray(b, dtype=np.float64)
    nb = np.linalg.norm(b)
    return np.linalg.norm(a - b) / (nb if nb > 0 else 1.0)


def dev(x, dtype=torch.float64):
    return torch.from_numpy(np.ascontiguousarray(x)).to("cuda", dtype)


def host(t):
    torch.cuda.synchronize()
    return t.double().cpu().numpy()


CASES = [
    dict(seed=1, nx=16, M=2, p=2),                 # the 16x16, M=2, p=2 workload shape
    dict(seed=2, nx=64, M=3, p=3),                 # 63 nodes per row: two tiles, ragged tail
    dict(seed=3, nx=8, M=1, p=4),
    dict(seed=4, nx=32, M=4, p=2, gamma=0.7),
    dict(seed=5, nx=4, M=2, p=1),
    dict(seed=6, nx=16, M=0, p=2),                 # deterministic limit
    dict(seed=7, nx=16, M=3, p=0),                 # single chaos column
    dict(seed=8, nx=2, M=2, p=2),                  # one interior node
    dict(seed=9, nx=128, M=2, p=1),
]
TIME_CASES = [
    dict(seed=11, nx=16, M=2, p=2, nt=4),
    dict(seed=12, nx=32, M=3, p=2, nt=3),
    dict(seed=13, nx=8, M=2, p=1, nt=1),
]


def make(case):
    c = dict(case)
    seed = c.pop("seed")
    pr = si.random_small(seed, **c)
    return pr, SGData(pr), SGProblem.from_problem(pr)


@pytest.mark.parametrize("case", CASES + TIME_CASES)
def test_sg_operator_fp64(case):
    pr, d, sp = make(case)
    X = si.random_panel(100 + case["seed"], d.n, d.P, d.slabs)
    Y = host(sp.apply_operator(dev(X), nslabs=d.slabs))
    ref = np.concatenate([d.vec(d.sg_apply(d.mat(X[t * d.P * d.n:(t + 1) * d.P * d.n])))
                          for t in range(d.slabs)])
    assert rel(Y, ref) <= 1e-13


@pytest.mark.parametrize("case", CASES[:4])
def test_sg_operator_fp32(case):
    pr, d, sp = make(case)
    X = si.random_panel(200 + case["seed"], d.n, d.P)
    Y = host(sp.apply_operator(dev(X, torch.float32)))
    ref = d.vec(d.sg_apply(d.mat(X.astype(np.float32).astype(np.float64))))
    assert rel(Y, ref) <= 2e-6


@pytest.mark.parametrize("case", CASES + TIME_CASES)
def test_kkt_fp64(case):
    pr, d, sp = make(case)
    v = si.random_panel(300 + case["seed"], 3 * d.n, d.P, d.slabs)
    w = host(sp.apply_kkt(dev(v)))
    assert rel(w, d.kkt_apply(v)) <= 1e-13
    if d.n * d.P * d.slabs <= 6000:
        assert rel(w, d.kkt_matrix() @ v) <= 1e-13


@pytest.mark.parametrize("case", CASES[:3] + TIME_CASES[:1])
def test_kkt_fp32(case):
    pr, d, sp = make(case)
    v = si.random_panel(400 + case["seed"], 3 * d.n, d.P, d.slabs)
    w = host(sp.apply_kkt(dev(v, torch.float32)))
    assert rel(w, d.kkt_apply(v.astype(np.float32).astype(np.float64))) <= 2e-6


@pytest.mark.parametrize("case", CASES + TIME_CASES)
def test_rhs(case):
    pr, d, sp = make(case)
    if pr.nt:
        pr.y0 = np.random.default_rng(case["seed"]).standard_normal(d.n)
        sp = SGProblem.from_problem(pr)
    assert rel(host(sp.rhs()), d.rhs()) <= 1e-14


@pytest.mark.parametrize("case", CASES[:5])
def test_chebyshev_fp64(case):
    pr, d, sp = make(case)
    ncols = 2 * d.P
    B = si.random_panel(500 + case["seed"], d.n, ncols)
    X = host(sp.apply_chebyshev(dev(B), ncols))
    ref = chebyshev(d.Mass, B.reshape(ncols, d.n).T, pr.cheb_steps).T.reshape(-1)
    assert rel(X, ref) <= 1e-12


@pytest.mark.parametrize("nx,M,p", [(128, 2, 2), (64, 3, 2), (16, 2, 2), (4, 1, 1)])
def test_chebyshev_fp32_fused(nx, M, p):
    """float32 columns of up to 127 x 127 nodes: all steps in one CTA per column."""
    pr = si.random_small(33 + nx, nx=nx, M=M, p=p)
    d = SGData(pr)
    sp = SGProblem.from_problem(pr)
    ncols = 2 * d.P
    B = si.random_panel(34, d.n, ncols).astype(np.float32).astype(np.float64)
    X = host(sp.apply_chebyshev(dev(B, torch.float32), ncols))
    ref = chebyshev(d.Mass, B.reshape(ncols, d.n).T, pr.cheb_steps).T.reshape(-1)
    assert rel(X, ref) <= 2e-6


@pytest.mark.parametrize("dtype,tol", [(torch.float64, 1e-12), (torch.float32, 2e-6)])
def test_chebyshev_large_grid(dtype, tol):
    """255 x 255 interior nodes: the per-step kernels (one column does not fit in shared memory)."""
    pr = si.random_small(31, nx=256, M=1, p=1)
    d = SGData(pr)
    sp = SGProblem.from_problem(pr)
    ncols = 2 * d.P
    B = si.random_panel(32, d.n, ncols)
    if dtype == torch.float32:
        B = B.astype(np.float32).astype(np.float64)
    X = host(sp.apply_chebyshev(dev(B, dtype), ncols))
    ref = chebyshev(d.Mass, B.reshape(ncols, d.n).T, pr.cheb_steps).T.reshape(-1)
    assert rel(X, ref) <= tol


@pytest.mark.parametrize("case", CASES + TIME_CASES[:2])
def test_vcycle_fp64(case):
    pr, d, sp = make(case)
    Pc = BlockPreconditioner(d)
    ncols = max(1, max(np.diff(basis.level_offsets(d.M, d.p))))
    B = si.random_panel(600 + case["seed"], d.n, ncols)
    X = host(sp.apply_vcycle(dev(B), ncols))
    V = VCycle(Pc.A0, pr.nx, pr.nu_pre, pr.nu_post, pr.omega)
    ref = V.apply(B.reshape(ncols, d.n).T).T.reshape(-1)
    assert rel(X, ref) <= 1e-12


@pytest.mark.parametrize("case", CASES[:4] + [dict(seed=21, nx=16, M=3, p=3, r=1),
                                              dict(seed=22, nx=16, M=3, p=3, r=2)] + TIME_CASES[:2])
def test_hgs_fp64(case):
    pr, d, sp = make(case)
    Pc = BlockPreconditioner(d)
    R = si.random_panel(700 + case["seed"], d.n, d.P, d.slabs)
    V = host(sp.apply_hgs(dev(R)))
    ps = d.P * d.n
    ref = np.concatenate([d.vec(Pc.hgs.apply(d.mat(R[t * ps:(t + 1) * ps]))) for t in range(d.slabs)])
    assert rel(V, ref) <= 1e-12


@pytest.mark.parametrize("case", CASES + TIME_CASES)
def test_block_preconditioner_fp64(case):
    pr, d, sp = make(case)
    Pc = BlockPreconditioner(d)
    r = si.random_panel(800 + case["seed"], 3 * d.n, d.P, d.slabs)
    z = host(sp.apply_precond(dev(r)))
    assert rel(z, Pc.apply(r)) <= 1e-12


def test_block_preconditioner_fp32_close():
    pr, d, sp = make(CASES[1])
    Pc = BlockPreconditioner(d)
    r = si.random_panel(900, 3 * d.n, d.P)
    sp32 = SGProblem.from_problem(pr, precision="mixed")
    z = host(sp32.apply_precond(dev(r, torch.float32)))
    assert rel(z, Pc.apply(r.astype(np.float32).astype(np.float64))) <= 1e-5


SOLVE_CASES = [
    dict(seed=1, nx=16, M=2, p=2),
    dict(seed=2, nx=32, M=3, p=3, beta=1e-4),
    dict(seed=3, nx=16, M=2, p=2, gamma=1.0),
    dict(seed=4, nx=16, M=3, p=2, r=1),
    dict(seed=5, nx=16, M=2, p=2, nt=4, beta=1e-3),
    dict(seed=6, nx=8, M=2, p=3, nt=2),
]


@pytest.mark.parametrize("case", SOLVE_CASES)
def test_solve_fp64_matches_oracle(case):
    pr, d, sp = make(case)
    ref = oracle_solve(pr, data=d)
    x, info = sp.solve()
    x = host(x)
    assert info["status_name"] == "SGOC_OK"
    assert abs(info["iterations"] - ref.iterations) <= 1
    assert info["rel_true_residual"] <= pr.tol
    assert rel(x, ref.x) <= 1e-7
    assert rel(d.kkt_apply(x), d.rhs()) <= pr.tol * 1.01


def test_solve_steady_16_workload():
    pr = si.steady_16()
    d = SGData(pr)
    sp = SGProblem.from_problem(pr)
    ref = oracle_solve(pr, data=d)
    x, info = sp.solve()
    assert abs(info["iterations"] - ref.iterations) <= 1
    assert rel(host(x), ref.x) <= 1e-7


@pytest.mark.parametrize("case", SOLVE_CASES[:2] + SOLVE_CASES[4:5])
def test_solve_mixed_reaches_fp64_residual(case):
    pr, d, sp = make(case)
    sp64 = SGProblem.from_problem(pr)
    x64 = host(sp64.solve()[0])
    spm = SGProblem.from_problem(pr, precision="mixed")
    x, info = spm.solve()
    x = host(x)
    assert info["status_name"] == "SGOC_OK"
    assert info["rel_true_residual"] <= pr.tol
    assert rel(d.kkt_apply(x), d.rhs()) <= pr.tol * 1.01
    assert rel(x, x64) <= 1e-6


def test_solve_with_initial_guess_restarts():
    pr, d, sp = make(SOLVE_CASES[0])
    x, info = sp.solve()
    x2, info2 = sp.solve(x0=x)
    assert info2["iterations"] <= 1
    assert rel(host(x2), host(x)) <= 1e-9


def test_solve_is_deterministic():
    pr, d, sp = make(SOLVE_CASES[1])
    xa, ia = sp.solve()
    xb, ib = sp.solve()
    assert ia["iterations"] == ib["iterations"]
    assert torch.equal(xa, xb)


@pytest.mark.parametrize("nx,dtype,tol", [(256, torch.float64, 1e-11), (512, torch.float32, 2e-5)])
def test_vcycle_levelwise_fine_levels(nx, dtype, tol):
    """Grids above the fused and cluster V-cycles: the fine levels run as grid-wide passes
    (float64 255 x 255 over a cluster cycle from 127 x 127; float32 511 x 511 over 255 x 255).
    float64 tolerance 1e-11: eight levels of summation-order differences, amplified by the mean
    operator's condition number (about 4e4 at 255 x 255), against 1e-12 on the grids of at most
    127 x 127 above."""
    pr = si.random_small(83 + nx, nx=nx, M=2, p=1)
    d = SGData(pr)
    sp = SGProblem.from_problem(pr, precision="fp64" if dtype == torch.float64 else "mixed")
    Pc = BlockPreconditioner(d)
    ncols = 2
    B = si.random_panel(84, d.n, ncols)
    if dtype == torch.float32:
        B = B.astype(np.float32).astype(np.float64)
    X = host(sp.apply_vcycle(dev(B, dtype), ncols))
    V = VCycle(Pc.A0, pr.nx, pr.nu_pre, pr.nu_post, pr.omega)
    ref = V.apply(B.reshape(ncols, d.n).T).T.reshape(-1)
    assert rel(X, ref) <= tol


@pytest.mark.parametrize("nx,ncols", [(64, 3), (128, 3), (128, 56), (256, 3)])
def test_vcycle_fp32_cluster_and_single(nx, ncols):
    """float32 V-cycle against the float64 oracle cycle (float32 rounding over ~50
    stencil passes): one CTA per column (64x64; 128x128 with many columns) and
    thread-block clusters (128x128 with few columns; 256x256)."""
    pr = si.random_small(40 + nx, nx=nx, M=2, p=2, beta=1e-3)
    if ncols > 6:
        pr = si.random_small(40 + nx, nx=nx, M=6, p=3, beta=1e-3)
    d = SGData(pr)
    sp = SGProblem.from_problem(pr, precision="mixed")
    Pc = BlockPreconditioner(d)
    B = si.random_panel(41, d.n, ncols)
    X = host(sp.apply_vcycle(dev(B, torch.float32), ncols))
    V = VCycle(Pc.A0, pr.nx, pr.nu_pre, pr.nu_post, pr.omega)
    ref = V.apply(B.astype(np.float32).astype(np.float64).reshape(ncols, d.n).T).T.reshape(-1)
    assert rel(X, ref) <= 2e-5



@pytest.mark.parametrize("nu", [1, 3])
@pytest.mark.parametrize("nx,dtype,tol", [(16, torch.float64, 1e-12), (16, torch.float32, 2e-5),
                                          (64, torch.float32, 2e-5), (128, torch.float32, 2e-5)])
def test_vcycle_other_sweep_counts(nu, nx, dtype, tol):
    """V(nu, nu) with nu other than the default 2 (the kernel built for any sweep count: zero
    starts, a single or an extra sweep, the prolongation as a pass of its own) against the
    oracle cycle with the same nu."""
    pr = dataclasses.replace(si.random_small(60 + nx + nu, nx=nx, M=2, p=2, beta=1e-3), nu_pre=nu, nu_post=nu)
    d = SGData(pr)
    sp = SGProblem.from_problem(pr, precision="fp64" if dtype == torch.float64 else "mixed")
    Pc = BlockPreconditioner(d)
    ncols = 3
    B = si.random_panel(61 + nu, d.n, ncols)
    if dtype == torch.float32:
        B = B.astype(np.float32).astype(np.float64)
    X = host(sp.apply_vcycle(dev(B, dtype), ncols))
    V = VCycle(Pc.A0, pr.nx, nu, nu, pr.omega)
    ref = V.apply(B.reshape(ncols, d.n).T).T.reshape(-1)
    assert rel(X, ref) <= tol

def test_hgs_fp32_128():
    pr = si.random_small(50, nx=128, M=3, p=2, beta=1e-4)
    d = SGData(pr)
    sp = SGProblem.from_problem(pr, precision="mixed")
    Pc = BlockPreconditioner(d)
    R = si.random_panel(51, d.n, d.P)
    V = host(sp.apply_hgs(dev(R, torch.float32)))
    ref = d.vec(Pc.hgs.apply(d.mat(R.astype(np.float32).astype(np.float64))))
    assert rel(V, ref) <= 2e-5

"""The register form of the SG operator (kernel variant 7: float32, Legendre chaos of a
compiled (M, p), a thread per node with every output column's sum in registers).

It forms the same products as variants 0-6 but sums an output column's coupling terms in
increasing input column instead of increasing k, so it agrees with them to float32
rounding, not bit for bit.  Tolerances are those of the other float32 parity tests:
operator and KKT products 2e-6 relative against the oracle (and against variant 0),
preconditioner pieces 2e-5.  Pinned kernels live in a process-wide table, so every test
clears its pins.
"""
import contextlib

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


def dev(x, dtype=torch.float32):
    return torch.from_numpy(np.ascontiguousarray(x)).to("cuda", dtype)


def host(t):
    torch.cuda.synchronize()
    return t.double().cpu().numpy()


def f32(x):
    return np.asarray(x).astype(np.float32).astype(np.float64)


def shapes_of(p):
    return [0, 1] + [2 + lev for lev in range(2 * p + 2)]


@contextlib.contextmanager
def pinned(sp, p, variant):
    """Pin `variant` on every SG shape of a solve where it applies; clear on exit."""
    from paper_2512_23804_gb300 import abi
    done = []
    try:
        for sh in shapes_of(p):
            try:
                sp.set_kernel(sh, variant)
                done.append(sh)
            except abi.SgocError as e:
                assert e.status == abi.SGOC_ERR_UNSUPPORTED
        yield done
    finally:
        for sh in shapes_of(p):
            sp.set_kernel(sh, -1)


# compiled (M, p) on grids whose node counts leave ragged 32 x 4 tiles
CASES = [(1, 1, 16, 0), (2, 2, 16, 0), (2, 2, 32, 2), (3, 2, 64, 0), (3, 3, 32, 0), (4, 3, 64, 3),
         (4, 3, 128, 0), (3, 3, 128, 2)]


@pytest.mark.parametrize("M,p,nx,nt", CASES, ids=[f"M{c[0]}p{c[1]}_{c[2]}_nt{c[3]}" for c in CASES])
def test_register_operator_matches_oracle_and_variant0(M, p, nx, nt):
    from paper_2512_23804_gb300 import SGProblem
    pr = si.random_small(500 + 7 * M + p + nx, nx=nx, M=M, p=p, nt=nt, beta=1e-3)
    d = SGData(pr)
    sp = SGProblem.from_problem(pr, precision="mixed")
    X = f32(si.random_panel(501 + nx, d.n, d.P, d.slabs))
    ps = d.P * d.n
    ref = np.concatenate([d.vec(d.sg_apply(d.mat(X[t * ps:(t + 1) * ps]))) for t in range(d.slabs)])
    Y7 = host(sp.apply_operator_variant(dev(X), 7, nslabs=d.slabs))
    Y0 = host(sp.apply_operator_variant(dev(X), 0, nslabs=d.slabs))
    assert rel(Y7, ref) <= 2e-6
    assert rel(Y7, Y0) <= 2e-6


@pytest.mark.parametrize("M,p,nx,nt", [(3, 3, 64, 0), (2, 2, 32, 3), (4, 3, 32, 0)],
                         ids=["M3p3_64", "M2p2_32_nt3", "M4p3_32"])
def test_register_kernel_in_hgs_kkt_and_preconditioner(M, p, nx, nt):
    """Variant 7 pinned on every SG shape (KKT product, hGS return and first visits with
    the mass term, the right-hand side and no_own): the hGS sweep, the KKT product and the
    block preconditioner match the oracle."""
    from paper_2512_23804_gb300 import SGProblem
    pr = si.random_small(520 + M + nx + nt, nx=nx, M=M, p=p, nt=nt, beta=1e-3)
    d = SGData(pr)
    sp = SGProblem.from_problem(pr, precision="mixed").upload()
    pc = BlockPreconditioner(d)
    R = f32(si.random_panel(521, d.n, d.P, d.slabs))
    v = f32(si.random_panel(522, 3 * d.n, d.P, d.slabs))
    ps = d.P * d.n
    with pinned(sp, p, 7) as done:
        assert set(shapes_of(p)) <= set(done)          # applicable on every shape of these problems
        h = host(sp.apply_hgs(dev(R)))
        k = host(sp.apply_kkt(dev(v)))
        z = host(sp.apply_precond(dev(v)))
    ref_h = np.concatenate([d.vec(pc.hgs.apply(d.mat(R[t * ps:(t + 1) * ps]))) for t in range(d.slabs)])
    assert rel(h, ref_h) <= 2e-5
    assert rel(k, d.kkt_apply(v)) <= 2e-6
    assert rel(z, pc.apply(v)) <= 2e-5


def test_register_kernel_mixed_solve_and_merged_batch():
    """A mixed solve with variant 7 on every shape reaches the float64 residual; merged
    launches (member tables) give the solo results bit for bit."""
    from paper_2512_23804_gb300 import SGProblem, solve_batch
    prs = [si.random_small(540 + i, nx=32, M=3, p=3, beta=b) for i, b in enumerate([1e-2, 1e-4])]
    d = SGData(prs[0])
    sps = [SGProblem.from_problem(pr, precision="mixed").upload() for pr in prs]
    with pinned(sps[0], 3, 7):
        x, info = sps[0].solve()
        assert info["status_name"] == "SGOC_OK" and info["rel_true_residual"] <= 1e-8
        assert rel(d.kkt_apply(host(x)), d.rhs()) <= 1.01e-8
        alone = [host(sp.solve()[0]) for sp in sps]
        xs, infos = solve_batch(sps, merged=True)
        for xm, a, inf in zip(xs, alone, infos):
            assert inf["status_name"] == "SGOC_OK"
            assert np.array_equal(host(xm), a)


def test_register_kernel_scope():
    """Variant 7 applies to float32 Legendre problems of a compiled (M, p) only."""
    from paper_2512_23804_gb300 import SGProblem, abi
    X = None
    for pr, prec in [(si.random_small(560, nx=16, M=2, p=2), "fp64"),          # float64
                     (si.random_small(561, nx=16, M=6, p=3), "mixed"),         # (6, 3) not compiled
                     (si.paper_problem(16, 2, 2, sigma=0.4), "mixed")]:        # Hermite chaos
        sp = SGProblem.from_problem(pr, precision=prec)
        X = torch.zeros(sp.n * sp.P, dtype=torch.float64 if prec == "fp64" else torch.float32, device="cuda")
        with pytest.raises(abi.SgocError) as ei:
            sp.apply_operator_variant(X, 7)
        assert ei.value.status == abi.SGOC_ERR_UNSUPPORTED

"""Pins of the oracle's FGMRES (the Krylov method of Sec. 5).

* Minimal residual: with a fixed linear preconditioner P, iteration k of right-preconditioned
  GMRES minimises ||b - A P^{-1} u|| over the Krylov space K_k(A P^{-1}, b); the estimates
  must equal that minimum, computed here by least squares on an explicitly built Krylov basis.
* The estimate is the true residual norm (checked at exit).
* With the ideal preconditioner blkdiag(M_g, beta M, S_exact) the preconditioned KKT matrix
  has three eigenvalues, so GMRES ends within three iterations.
* Flexible: with a preconditioner that changes from one iteration to the next the true
  residual at exit still equals the estimate (the Arnoldi relation A Z_m = V_{m+1} H_m).
* The solution equals the dense direct solution and scipy's GMRES.
"""
import math

import numpy as np
import pytest
import scipy.sparse.linalg as spla

import sg_inputs as si
from oracle.krylov import fgmres
from oracle.operators import SGData
from oracle.precond import BlockPreconditioner, chebyshev


def small():
    pr = si.random_small(21, nx=4, M=2, p=2, beta=1e-2)
    d = SGData(pr)
    return pr, d, d.kkt_matrix().toarray(), d.rhs()


def test_fgmres_estimates_are_the_minimal_residuals():
    pr, d, K, b = small()
    Pc = BlockPreconditioner(d)
    Pinv = np.stack([Pc.apply(e) for e in np.eye(K.shape[0])], axis=1)
    AP = K @ Pinv
    res = fgmres(lambda v: K @ v, Pc.apply, b, tol=1e-14, max_iter=8)
    kry = [b / np.linalg.norm(b)]
    for k in range(1, 9):
        Q, _ = np.linalg.qr(np.column_stack(kry))
        y, *_ = np.linalg.lstsq(AP @ Q, b, rcond=None)
        rmin = np.linalg.norm(b - AP @ (Q @ y)) / np.linalg.norm(b)
        assert abs(res.history[k - 1] - rmin) <= 1e-9 * max(rmin, 1e-12) + 1e-14, (k, res.history[k - 1], rmin)
        nxt = AP @ kry[-1]
        kry.append(nxt / np.linalg.norm(nxt))
    assert np.all(np.diff(res.history) <= 1e-15)


def test_fgmres_estimate_is_the_true_residual_and_solution_is_direct():
    pr, d, K, b = small()
    Pc = BlockPreconditioner(d)
    res = fgmres(lambda v: K @ v, Pc.apply, b, tol=1e-11)
    assert res.status == "ok"
    assert abs(res.rel_true - res.history[-1]) <= 1e-3 * res.history[-1] + 1e-14
    xd = np.linalg.solve(K, b)
    assert np.linalg.norm(res.x - xd) <= 1e-9 * np.linalg.norm(xd)
    Lop = spla.LinearOperator(K.shape, matvec=Pc.apply, dtype=float)
    xs, info = spla.gmres(K, b, M=Lop, rtol=1e-12, restart=200, maxiter=10)
    assert info == 0 and np.linalg.norm(xs - xd) <= 1e-8 * np.linalg.norm(xd)


def test_fgmres_ideal_preconditioner_three_iterations():
    pr, d, K, b = small()
    F = d.P * d.n
    A = d.sg_matrix().toarray()
    Mc, Mg = d.mass_cal().toarray(), d.mass_gamma().toarray()
    Pm = np.zeros_like(K)
    Pm[:F, :F], Pm[F:2 * F, F:2 * F] = Mg, pr.beta * Mc
    Pm[2 * F:, 2 * F:] = A @ np.linalg.solve(Mg, A) + Mc / pr.beta
    res = fgmres(lambda v: K @ v, lambda v: np.linalg.solve(Pm, v), b, tol=1e-10)
    assert res.iterations <= 3 and res.rel_true <= 1e-10


def test_fgmres_is_flexible():
    """A preconditioner that changes every iteration (Chebyshev mass blocks with 1, 2 or 3
    steps in turn inside the block preconditioner) keeps the residual identity."""
    pr, d, K, b = small()
    calls = [0]
    steps = [1, 2, 3]

    def Pvar(v):
        Pc = BlockPreconditioner(d)
        Pc.steps = steps[calls[0] % 3]
        calls[0] += 1
        return Pc.apply(v)

    res = fgmres(lambda v: K @ v, Pvar, b, tol=1e-10)
    assert res.status == "ok" and res.rel_true <= 1e-10
    # estimate and true residual agree at the last iteration: A Z_m = V_{m+1} H_m holds
    assert abs(res.rel_true - res.history[-1]) <= 1e-3 * res.history[-1] + 1e-14


def test_fgmres_solves_the_16x16_workload_and_restarts():
    from oracle.solve import direct_solve
    pr = si.steady_16()
    d = SGData(pr)
    Pc = BlockPreconditioner(d)
    b = d.rhs()
    xd = direct_solve(pr)
    full = fgmres(d.kkt_apply, Pc.apply, b, tol=1e-8)
    assert full.status == "ok" and np.linalg.norm(full.x - xd) <= 1e-7 * np.linalg.norm(xd)
    rst = fgmres(d.kkt_apply, Pc.apply, b, tol=1e-8, restart=10, max_iter=400)
    assert rst.status == "ok" and rst.rel_true <= 1e-8 and rst.iterations >= full.iterations

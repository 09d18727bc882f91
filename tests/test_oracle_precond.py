"""Pins of the oracle's Chebyshev, V-cycle, hGS, block preconditioner and MINRES."""
import math

import numpy as np
import pytest
import scipy.sparse as sp
import scipy.sparse.linalg as spla

import sg_inputs as si
from oracle import basis, fe
from oracle.krylov import minres
from oracle.operators import SGData
from oracle.precond import (BlockPreconditioner, ExactSolve, HGS, VCycle, chebyshev,
                            prolongation, visit_order)
from oracle.solve import direct_solve, solve
from golden_io import constants

C = constants()


def test_chebyshev_matches_closed_form_polynomial():
    nx = 8
    Mm = fe.mass(nx)
    b = np.random.default_rng(0).standard_normal(Mm.shape[0])
    steps = 5
    x = chebyshev(Mm, b, steps)
    lmin, lmax = C["cheb_lmin"], C["cheb_lmax"]
    gam = (lmin + lmax) / 2
    rho = (lmax - lmin) / (lmax + lmin)
    D = gam * Mm.diagonal()
    Dh = np.sqrt(D)
    S = (Mm.toarray() / Dh[:, None]) / Dh[None, :]
    lam, Q = np.linalg.eigh(S)
    T = np.polynomial.chebyshev.Chebyshev.basis(steps)
    xstar = np.linalg.solve(Mm.toarray(), b)
    e0 = Dh * xstar                                  # D^{1/2}(x* - 0)
    factor = T((1 - lam) / rho) / T(1 / rho)
    e = Q @ (factor * (Q.T @ e0))
    x_closed = xstar - e / Dh
    assert np.linalg.norm(x - x_closed) <= 1e-13 * np.linalg.norm(xstar)
    assert T(1 / rho) == pytest.approx(C["t5_125"], rel=1e-15)
    # error bound 1/T_N(1/rho) in the D-norm
    err = np.linalg.norm(Dh * (x - xstar)) / np.linalg.norm(Dh * xstar)
    assert err <= 1 / C["t5_125"] + 1e-14


def test_prolongation_is_bilinear_interpolation():
    nx = 8
    P = prolongation(nx)
    h, H = 1 / nx, 2 / nx
    xc = np.arange(1, nx // 2) * H
    X2c, X1c = np.meshgrid(xc, xc, indexing="ij")
    f = lambda a, b: 1.0 + 2 * a - 3 * b + 4 * a * b     # bilinear: interpolated exactly
    # on interior nodes that are not adjacent to the boundary (boundary values are zero)
    vc = f(X1c, X2c).ravel()
    xf = np.arange(1, nx) * h
    X2f, X1f = np.meshgrid(xf, xf, indexing="ij")
    vf = P @ vc
    m = nx - 1
    inner = [(j - 1) * m + (i - 1) for j in range(2, nx - 1) for i in range(2, nx - 1)]
    assert np.allclose(vf[inner], f(X1f, X2f).ravel()[inner], atol=1e-14)


@pytest.mark.parametrize("nx", [4, 8, 16])
def test_galerkin_coarse_equals_coarse_discretisation(nx):
    s = 7.0
    A = fe.assemble(nx, np.ones((nx, nx))) + s * fe.mass(nx)
    P = prolongation(nx)
    Ac = (P.T @ A @ P).toarray()
    ref = (fe.assemble(nx // 2, np.ones((nx // 2, nx // 2))) + s * fe.mass(nx // 2)).toarray()
    assert np.max(np.abs(Ac - ref)) < 1e-13


@pytest.mark.parametrize("nu", [1, 2, 3])
@pytest.mark.parametrize("nx,s", [(16, 10.0), (32, 1000.0), (8, 0.0)])
def test_vcycle_symmetric_and_converges_to_direct(nx, s, nu):
    A = fe.assemble(nx, np.ones((nx, nx))) + s * fe.mass(nx)
    V = VCycle(A, nx, nu, nu)
    rng = np.random.default_rng(1)
    v, w = rng.standard_normal((2, A.shape[0]))
    assert abs(v @ V.apply(w) - w @ V.apply(v)) <= 1e-13 * abs(v @ V.apply(w))
    assert v @ V.apply(v) > 0
    b = rng.standard_normal(A.shape[0])
    x = np.zeros_like(b)
    for _ in range(60):
        x = x + V.apply(b - A @ x)
    xs = spla.spsolve(sp.csc_matrix(A), b)
    assert np.linalg.norm(x - xs) <= 1e-12 * np.linalg.norm(xs)
    # one V-cycle is a contraction in the energy norm
    e0 = xs
    e1 = xs - V.apply(b)
    assert math.sqrt(e1 @ (A @ e1)) < 0.5 * math.sqrt(e0 @ (A @ e0))


def hgs_setup(M=2, p=3, nx=4, r=None, nt=0):
    pr = si.random_small(2, nx=nx, M=M, p=p, nt=nt, beta=1e-2)
    if r is not None:
        pr.r = r
    d = SGData(pr)
    s = math.sqrt(1 / pr.beta)
    A0 = d.K[0] + s * d.Mass
    return pr, d, A0


@pytest.mark.parametrize("M,p,r", [(2, 3, 3), (3, 2, 4), (2, 2, 2), (1, 4, 2)])
def test_hgs_exact_equals_symmetric_block_gauss_seidel(M, p, r):
    """With exact mean solves, one sweep applies Z_hGS^{-1} with
    Z_hGS = (X_1 + X_r) X_1^{-1} (X_1 + X_r^T)   (Sec. 4)."""
    pr, d, A0 = hgs_setup(M, p, r=r)
    H = HGS(d, A0, 1.0, r, ExactSolve(A0))
    off = basis.level_offsets(M, p)
    lev = np.zeros(d.P, dtype=int)
    for dd in range(p + 1):
        lev[off[dd]:off[dd + 1]] = dd
    X1 = np.kron(np.eye(d.P), A0.toarray())
    Xr = np.zeros_like(X1)
    for k in range(1, r):
        Lk = np.where(lev[:, None] > lev[None, :], d.G[k], 0.0)
        Xr += np.kron(Lk, d.K[k].toarray())
    Zh = (X1 + Xr) @ np.linalg.solve(X1, X1 + Xr.T)
    Zr = X1 + Xr + Xr.T
    R = np.random.default_rng(4).standard_normal((d.n, d.P))
    V = H.apply(R)
    Vref = np.linalg.solve(Zh, R.T.reshape(-1))
    assert np.linalg.norm(V.T.reshape(-1) - Vref) <= 1e-11 * np.linalg.norm(Vref)
    # Z_hGS = Z_r + X_r X_1^{-1} X_r^T
    assert np.max(np.abs(Zh - (Zr + Xr @ np.linalg.solve(X1, Xr.T)))) < 1e-10 * np.max(np.abs(Zh))
    # Sec. 4 bound: 1 <= lambda(Z_r^{-1} Z_hGS) <= 1 + Delta_r^2 / (1 - Delta_r)
    ev = np.sort(np.linalg.eigvals(np.linalg.solve(Zr, Zh)).real)
    A0d = A0.toarray()
    w, Q = np.linalg.eigh(A0d)
    A0mh = Q @ np.diag(w ** -0.5) @ Q.T
    Delta = sum(np.linalg.norm(d.G[k], 2) * np.linalg.norm(A0mh @ d.K[k].toarray() @ A0mh, 2) for k in range(1, r))
    assert ev[0] >= 1 - 1e-10
    if Delta < 1:
        assert ev[-1] <= 1 + Delta**2 / (1 - Delta) + 1e-10


def test_hgs_r1_is_mean_based():
    pr, d, A0 = hgs_setup(2, 3, r=1)
    H = HGS(d, A0, 1.0, 1, ExactSolve(A0))
    R = np.random.default_rng(5).standard_normal((d.n, d.P))
    V = H.apply(R)
    ref = spla.spsolve(sp.csc_matrix(A0), R)
    assert np.max(np.abs(V - ref)) <= 1e-13 * np.max(np.abs(ref))


def test_truncation_bound():
    """1 - delta_r <= lambda(Z_r^{-1} Z) <= 1 + delta_r  (Sec. 4, truncation theorem,
    applied to the truncated operator the proof bounds)."""
    pr, d, A0 = hgs_setup(3, 2, nx=4)
    full = d.sg_matrix().toarray() + math.sqrt(1 / pr.beta) * d.mass_cal().toarray()
    nu = np.linalg.eigvalsh(A0.toarray()).min()
    for r in range(1, d.M + 1):
        Zr = np.kron(np.eye(d.P), A0.toarray()) + sum(np.kron(d.G[k], d.K[k].toarray()) for k in range(1, r))
        delta = sum(np.linalg.norm(d.G[k], 2) * np.linalg.norm(d.K[k].toarray(), 2) for k in range(r, d.M + 1)) / nu
        ev = np.linalg.eigvals(np.linalg.solve(Zr, full)).real
        if delta < 1:
            assert ev.min() >= 1 - delta - 1e-10 and ev.max() <= 1 + delta + 1e-10


def test_visit_order_palindrome():
    assert visit_order(3) == [0, 1, 2, 3, 2, 1, 0]
    assert visit_order(0) == [0]


@pytest.mark.parametrize("nt", [0, 3])
def test_block_preconditioner_spd(nt):
    pr = si.random_small(3, nx=8, M=2, p=2, nt=nt, beta=1e-3, gamma=0.5 if nt == 0 else 0.0)
    d = SGData(pr)
    Pc = BlockPreconditioner(d)
    rng = np.random.default_rng(6)
    nk = 3 * d.slabs * d.P * d.n
    for _ in range(3):
        v, w = rng.standard_normal((2, nk))
        a, b = v @ Pc.apply(w), w @ Pc.apply(v)
        assert abs(a - b) <= 1e-12 * (abs(a) + abs(b))
        assert v @ Pc.apply(v) > 0


def test_schur_approximation_spectrum_steady():
    """lambda(S^{-1} S_exact) in [1/2, 1] for S = Z M_g^{-1} Z (gamma = 0), Sec. 2 and
    the steady (n_t = 1) case of the Benner et al. bound quoted in Sec. 4."""
    pr = si.random_small(4, nx=4, M=2, p=2, beta=1e-2)
    d = SGData(pr)
    A = d.sg_matrix().toarray()
    Mc = d.mass_cal().toarray()
    Mg = d.mass_gamma().toarray()
    Sx = A @ np.linalg.solve(Mg, A) + Mc / pr.beta
    Z = A + math.sqrt(1 / pr.beta) * Mc
    S = Z @ np.linalg.solve(Mg, Z)
    ev = np.linalg.eigvals(np.linalg.solve(S, Sx)).real
    assert ev.min() >= 0.5 - 1e-10 and ev.max() <= 1 + 1e-10


def test_minres_ideal_preconditioner_three_iterations():
    """With P = blkdiag(M_g, beta M, S_exact) the preconditioned KKT matrix has the three
    eigenvalues 1, (1 +- sqrt 5)/2, so MINRES ends after 3 iterations."""
    pr = si.random_small(4, nx=4, M=2, p=2, beta=1e-2)
    d = SGData(pr)
    K = d.kkt_matrix().toarray()
    F = d.P * d.n
    A = d.sg_matrix().toarray()
    Mc = d.mass_cal().toarray()
    Mg = d.mass_gamma().toarray()
    Sx = A @ np.linalg.solve(Mg, A) + Mc / pr.beta
    Pm = np.zeros_like(K)
    Pm[:F, :F], Pm[F:2 * F, F:2 * F], Pm[2 * F:, 2 * F:] = Mg, pr.beta * Mc, Sx
    ev = np.sort(np.linalg.eigvals(np.linalg.solve(Pm, K)).real)
    mgw = sorted(constants()["mgw"])
    for e in ev:
        assert min(abs(e - m) for m in mgw) < 1e-8
    b = d.rhs()
    res = minres(lambda v: K @ v, lambda v: np.linalg.solve(Pm, v), b, tol=1e-10)
    assert res.iterations <= 3 and res.rel_true <= 1e-10


@pytest.mark.parametrize("nt", [0, 2])
def test_minres_matches_scipy_and_direct(nt):
    pr = si.random_small(8, nx=8, M=2, p=2, nt=nt, beta=1e-2)
    pr.tol = 1e-12
    d = SGData(pr)
    K = d.kkt_matrix()
    Pc = BlockPreconditioner(d)
    b = d.rhs()
    res = minres(lambda v: K @ v, Pc.apply, b, tol=1e-12)
    xd = np.linalg.solve(K.toarray(), b)
    assert np.linalg.norm(res.x - xd) <= 1e-9 * np.linalg.norm(xd)
    assert res.rel_true <= 1e-12
    Lop = spla.LinearOperator(K.shape, matvec=Pc.apply, dtype=float)
    xs, info = spla.minres(K, b, M=Lop, rtol=1e-13, maxiter=500)
    assert info == 0
    assert np.linalg.norm(xs - xd) <= 1e-8 * np.linalg.norm(xd)
    # MINRES residual estimates are monotone non-increasing
    h = np.array(res.history)
    assert np.all(np.diff(h) <= 1e-14)


def test_oracle_solve_small_configuration():
    pr = si.steady_16()
    res = solve(pr)
    xd = direct_solve(pr)
    assert res.status == "ok" and res.rel_true <= 1e-8
    assert np.linalg.norm(res.x - xd) <= 1e-7 * np.linalg.norm(xd)
    # hierarchical truncation beats the mean-based preconditioner (Sec. 5 tables)
    pr1 = si.steady_16(r=1)
    assert solve(pr1).iterations > res.iterations

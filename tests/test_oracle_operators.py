"""Pins of the oracle's SG operator, KKT systems and optimal solutions."""
import itertools
import math

import numpy as np
import pytest
import scipy.sparse as sp

import sg_inputs as si
from oracle import basis, fe
from oracle.operators import SGData
from oracle.solve import direct_solve, reduced_solve


def small(M=2, p=2, nx=4, nt=0, sigma=0.3, beta=1e-2, gamma=0.0, seed=1):
    return si.random_small(seed, nx=nx, M=M, p=p, nt=nt, sigma=sigma, beta=beta, gamma=gamma)


@pytest.mark.parametrize("M,p,nx", [(2, 2, 4), (3, 2, 4), (1, 3, 8), (2, 3, 4)])
def test_sg_matrix_equals_stochastic_quadrature(M, p, nx):
    """sum_k G_k (x) K_k against int A(xi) Psi Psi^T dmu by tensor Gauss-Legendre
    quadrature (exact: the integrand has degree <= 2p+1 per variable)."""
    pr = small(M, p, nx)
    d = SGData(pr)
    A = d.sg_matrix().toarray()
    idx = basis.multi_indices(M, p)
    x, w = np.polynomial.legendre.leggauss(p + 1)
    w = w / 2
    Aq = np.zeros_like(A)
    for q in itertools.product(range(p + 1), repeat=M):
        xi = x[list(q)]
        wt = np.prod(w[list(q)])
        psi = np.array([np.prod([basis.legendre_orthonormal(int(a[j]), np.array([xi[j]]))[0]
                                 for j in range(M)]) for a in idx])
        Ax = d.K[0].toarray() + sum(xi[k] * d.K[k + 1].toarray() for k in range(M))
        Aq += wt * np.kron(np.outer(psi, psi), Ax)
    assert np.max(np.abs(A - Aq)) < 1e-12 * np.max(np.abs(A))


@pytest.mark.parametrize("nt", [0, 1, 3])
def test_matricized_equals_assembled(nt):
    pr = small(nt=nt, gamma=0.5 if nt == 0 else 0.0)
    d = SGData(pr)
    K = d.kkt_matrix()
    x = np.random.default_rng(3).standard_normal(K.shape[0])
    a, b = K @ x, d.kkt_apply(x)
    assert np.linalg.norm(a - b) <= 1e-15 * np.linalg.norm(a) * 10
    assert abs(K - K.T).max() < 1e-15 * abs(K).max() * 10


def test_m0_reduces_to_deterministic_kkt():
    pr = small(M=0, p=2)
    d = SGData(pr)
    assert d.P == 1
    K = d.kkt_matrix().toarray()
    Kd = fe.assemble(pr.nx, np.ones((pr.nx, pr.nx))).toarray()
    Mm = fe.mass(pr.nx).toarray()
    Z = np.zeros_like(Mm)
    ref = np.block([[Mm, Z, -Kd], [Z, pr.beta * Mm, Mm], [-Kd, Mm, Z]])
    assert np.max(np.abs(K - ref)) < 1e-15


def test_sigma0_solution_lives_in_mean_column():
    pr = small(M=2, p=2, sigma=0.0)
    x = direct_solve(pr)
    d = SGData(pr)
    F = d.P * d.n
    for blk in range(3):
        X = d.mat(x[blk * F:(blk + 1) * F])
        assert np.all(X[:, 1:] == 0.0)
    # and column 0 is the deterministic optimum
    prd = small(M=0, p=2)
    prd.yhat = pr.yhat
    xd = direct_solve(prd)
    n = d.n
    assert np.allclose(x[0:n], xd[0:n], rtol=1e-12, atol=1e-14)


@pytest.mark.parametrize("gamma", [0.0, 1.0])
def test_direct_equals_reduced_and_optimality(gamma):
    pr = small(M=2, p=2, nx=8, gamma=gamma)
    d = SGData(pr)
    x = direct_solve(pr, d)
    xr = reduced_solve(pr, d)
    assert np.linalg.norm(x - xr) <= 1e-10 * np.linalg.norm(x)
    F = d.P * d.n
    y, u, lam = x[:F], x[F:2 * F], x[2 * F:]
    A = d.sg_matrix()
    Mc, Mg = d.mass_cal(), d.mass_gamma()
    yd = np.zeros(F)
    yd[:d.n] = pr.yhat[0]
    # gradient equation (row 2): beta u + lambda = 0 since M is non-singular
    assert np.linalg.norm(pr.beta * u + lam) <= 1e-10 * np.linalg.norm(lam)
    # state equation A y = M u and adjoint M_g y - A lambda = M yhat
    assert np.linalg.norm(A @ y - Mc @ u) <= 1e-10 * np.linalg.norm(Mc @ u)
    assert np.linalg.norm(Mg @ y - A @ lam - Mc @ yd) <= 1e-10 * np.linalg.norm(Mc @ yd)


def test_first_variation_vanishes_at_optimum():
    pr = small(M=2, p=1, nx=4, gamma=0.3)
    d = SGData(pr)
    x = direct_solve(pr, d)
    F = d.P * d.n
    u = x[F:2 * F]
    A = d.sg_matrix().toarray()
    Mc, Mg = d.mass_cal().toarray(), d.mass_gamma().toarray()
    Msig = Mg - Mc                      # gamma * (H^sigma (x) M)
    yd = np.zeros(F)
    yd[:d.n] = pr.yhat[0]

    def J(uu):
        y = np.linalg.solve(A, Mc @ uu)
        e = y - yd
        return 0.5 * e @ Mc @ e + 0.5 * y @ Msig @ y + 0.5 * pr.beta * uu @ Mc @ uu

    dirn = np.random.default_rng(5).standard_normal(F)
    j0 = J(u)
    ratios = []
    for eps in (1e-1, 1e-2):
        ratios.append((J(u + eps * dirn) - j0) / eps**2)
    # J(u + e d) - J(u) = e^2 (d^T H d)/2: no linear term
    assert abs(ratios[0] - ratios[1]) <= 1e-6 * abs(ratios[0])
    assert ratios[0] > 0


def test_time_solution_satisfies_backward_euler_and_reduced_form():
    pr = si.time_problem(4, 2, 1, 0.5, 0.3, 1e-2, 3)
    pr.y0 = np.random.default_rng(7).standard_normal(pr.n)
    d = SGData(pr)
    x = direct_solve(pr, d)
    F = d.slabs * d.P * d.n
    nP = d.P * d.n
    y, u = x[:F], x[F:2 * F]
    A = d.sg_matrix()
    Mc = d.mass_cal()
    tau = d.tau
    # sequential backward Euler: (M + tau A) y_k = M y_{k-1} + tau M u_k, y_0 given (deterministic)
    yprev = np.zeros(nP)
    yprev[:d.n] = pr.y0
    for t in range(pr.nt):
        lhs = (Mc + tau * A) @ y[t * nP:(t + 1) * nP]
        rhs = Mc @ yprev + tau * (Mc @ u[t * nP:(t + 1) * nP])
        assert np.linalg.norm(lhs - rhs) <= 1e-10 * np.linalg.norm(rhs)
        yprev = y[t * nP:(t + 1) * nP]
    # reduced form of the trapezoid cost with y = A_t^{-1}(tau N u + d)
    K = d.kkt_matrix().toarray()
    At = -K[2 * F:, :F]
    N = K[2 * F:, F:2 * F] / tau
    Dm = K[:F, :F] / tau                       # D (x) M_gamma (gamma = 0 here)
    dvec = np.zeros(F)
    dvec[:d.n] = fe.mass(pr.nx) @ pr.y0
    ydst = np.zeros(F)
    Dw = d.d_weights()
    for t in range(pr.nt):
        ydst[t * nP:t * nP + d.n] = pr.yhat[t]
    Ai = np.linalg.inv(At)
    B = Ai @ (tau * N)
    y0part = Ai @ dvec
    H = tau * B.T @ Dm @ B + pr.beta * tau * Dm
    g = tau * B.T @ Dm @ (ydst - y0part)
    ur = np.linalg.solve(H, g)
    assert np.linalg.norm(ur - u) <= 1e-9 * np.linalg.norm(u)


def test_kl_terms_positive_coefficient():
    # the affine field 1 + sum kappa_k xi_k stays positive for all xi in [-1,1]^M
    for (nx, M, L, s) in [(16, 2, 1.0, 0.3), (128, 6, 0.5, 0.3), (64, 4, 0.5, 0.3)]:
        kap = si.kl_terms(nx, M, L, s)
        assert np.min(kap[0] - np.abs(kap[1:]).sum(axis=0)) > 0.2

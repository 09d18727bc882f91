"""Pins of the oracle's Hermite / lognormal setting (the paper's own, Sec. 2 and Sec. 5).

* Triple products: the closed form against tensor Gauss-Hermite quadrature; H_0 = I,
  H_l symmetric, and E[xi_j Psi_a Psi_b] (the linear terms) has the Hermite three-term
  structure sqrt(n+1) between degrees n and n+1.
* Coefficient terms: kappa_l = E[k psi_l] by Gauss-Hermite quadrature of the lognormal field
  itself (one and two random variables), and the chaos sum converges to exp(f) as p grows.
* Operators: the assembled SG matrix equals the matricized product; with the variance set
  to zero the system is the deterministic one in chaos column 0; the domain length scales
  the mass matrix only.
* Solution: MINRES and FGMRES with the block preconditioner reach the dense direct solution
  for truncations r = 1, M + 1 and n_A; with r = n_A (within-level couplings present) the
  hGS sweep is a convergent splitting of Z_r (Richardson iterations reach Z_r^{-1} R).
"""
import math

import numpy as np
import pytest

import sg_inputs as si
from oracle import basis
from oracle.krylov import fgmres
from oracle.operators import SGData
from oracle.precond import BlockPreconditioner, ExactSolve, HGS
from oracle.solve import direct_solve, solve


@pytest.mark.parametrize("M,p", [(2, 2), (3, 2), (1, 4), (3, 3)])
def test_hermite_triple_products(M, p):
    nA = basis.term_indices(M, p).shape[0]
    assert nA == math.comb(M + 2 * p, 2 * p)
    H = basis.h_matrices(M, p, nA)
    Hq = basis.h_matrices_quadrature(M, p, nA)
    for a, b in zip(H, Hq):
        assert np.max(np.abs(a - b)) <= 1e-12 * max(1.0, np.max(np.abs(b)))
        assert np.array_equal(a, a.T)
    assert np.array_equal(H[0], np.eye(H[0].shape[0]))
    idx = basis.multi_indices(M, p)
    for j in range(M):                                  # linear terms: sqrt(n+1) couplings
        Hj = H[1 + j]
        for a in range(len(idx)):
            for b in range(len(idx)):
                d = idx[a].astype(int) - idx[b].astype(int)
                nz = np.nonzero(d)[0]
                if len(nz) == 1 and nz[0] == j and abs(d[j]) == 1:
                    assert Hj[a, b] == pytest.approx(math.sqrt(max(idx[a][j], idx[b][j])), rel=1e-14)
                else:
                    assert Hj[a, b] == 0.0


def test_lognormal_terms_are_the_chaos_coefficients():
    """kappa_l(e) = E[exp(f_0 + sum f_j xi_j) psi_l(xi)], f_0 = -1/2 sum f_j^2, by quadrature."""
    nx, p = 8, 2
    for M in (1, 2):
        kap = si.lognormal_terms(nx, M, p)
        f = si.kl_terms(nx, M, 0.5, 1.0)[1:]
        tl = basis.term_indices(M, p)
        x, w = np.polynomial.hermite_e.hermegauss(40)
        w = w / math.sqrt(2 * math.pi)
        e = (3, 5)
        fj = [f[j][e] for j in range(M)]
        grids = np.meshgrid(*([x] * M), indexing="ij")
        wts = np.prod(np.meshgrid(*([w] * M), indexing="ij"), axis=0)
        field = np.exp(-0.5 * sum(v * v for v in fj) + sum(fj[j] * grids[j] for j in range(M)))
        for i, l in enumerate(tl):
            psi = np.prod([basis.hermite_normalised(int(l[j]), grids[j]) for j in range(M)], axis=0)
            assert kap[i][e] == pytest.approx(float(np.sum(wts * field * psi)), rel=1e-10, abs=1e-13)
    assert np.all(si.lognormal_terms(nx, 2, 2)[0] == 1.0)


def test_lognormal_chaos_sum_converges_to_the_field():
    nx, M = 8, 2
    f = si.kl_terms(nx, M, 0.5, 1.0)[1:]
    rng = np.random.default_rng(3)
    xi = rng.standard_normal(M)
    e = (2, 6)
    exact = math.exp(-0.5 * sum(f[j][e] ** 2 for j in range(M)) + sum(f[j][e] * xi[j] for j in range(M)))
    errs = []
    for p in (1, 2, 3, 4):
        kap = si.lognormal_terms(nx, M, p)
        tl = basis.term_indices(M, p)
        s = sum(kap[i][e] * np.prod([basis.hermite_normalised(int(l[j]), np.array(xi[j])) for j in range(M)])
                for i, l in enumerate(tl))
        errs.append(abs(float(s) - exact))
    assert errs[-1] < errs[0] and errs[-1] <= 1e-3 * exact


def small(p=2, M=2, r=None, sigma=1.0, nx=4, beta=1e-2):
    pr = si.paper_problem(nx, M, p, beta=beta)
    if sigma != 1.0:
        pr.kappa = si.lognormal_terms(nx, M, p, sigma=sigma)
    if r is not None:
        pr.r = r
    return pr


def test_hermite_operators():
    pr = small()
    d = SGData(pr)
    assert d.nterms == math.comb(pr.M + 2 * pr.p, 2 * pr.p)
    X = np.random.default_rng(1).standard_normal((d.n, d.P))
    A = d.sg_matrix()
    assert np.linalg.norm(A @ d.vec(X) - d.vec(d.sg_apply(X))) <= 1e-13 * np.linalg.norm(d.vec(d.sg_apply(X)))
    pr1 = si.paper_problem(pr.nx, pr.M, pr.p)
    pr1.length = 1.0
    d1 = SGData(pr1)
    assert np.allclose(d.Mass.toarray(), 4.0 * d1.Mass.toarray(), rtol=0, atol=1e-15)
    assert np.allclose(d.K[0].toarray(), d1.K[0].toarray(), rtol=0, atol=1e-15)
    # no variance: every term beyond the mean vanishes and the optimum lives in column 0
    pz = small(sigma=0.0)
    dz = SGData(pz)
    x = direct_solve(pz, data=dz)
    F = dz.P * dz.n
    for blk in range(3):
        assert np.max(np.abs(x[blk * F + dz.n:(blk + 1) * F])) <= 1e-13 * np.max(np.abs(x))


@pytest.mark.parametrize("r", [1, 3, 15])
def test_hermite_solves_reach_the_direct_solution(r):
    pr = small(r=r)
    d = SGData(pr)
    xd = direct_solve(pr, data=d)
    for kry in ("minres", "fgmres"):
        res = solve(pr, data=d, krylov=kry)
        assert res.status == "ok" and res.rel_true <= pr.tol
        assert np.linalg.norm(res.x - xd) <= 1e-6 * np.linalg.norm(xd), kry


def test_hgs_with_within_level_couplings_is_a_convergent_splitting():
    pr = small(r=15)
    d = SGData(pr)
    A0 = d.K[0] + math.sqrt((1 + pr.gamma) / pr.beta) * d.Mass
    H = HGS(d, A0, 1.0, 15, ExactSolve(A0))
    R = np.random.default_rng(2).standard_normal((d.n, d.P))
    Zr = lambda V: H.zr_apply(V)
    X = np.zeros_like(R)
    for _ in range(200):
        X = X + H.apply(R - Zr(X))
    Zd = sum(np.kron(d.G[k], d.K[k].toarray()) for k in range(1, 15)) + np.kron(np.eye(d.P), A0.toarray())
    ref = np.linalg.solve(Zd, d.vec(R))
    assert np.linalg.norm(d.vec(X) - ref) <= 1e-10 * np.linalg.norm(ref)

"""Pins of the oracle's block preconditioner against dense constructions.

The block preconditioner of the paper is P = blkdiag(K11, K22, S) where K11 and
K22 are the (1,1) and (2,2) blocks of the KKT matrix (Sec. 2, Eq. (stoch-prec);
Sec. 3, Eq. (precon for time)) and S approximates the Schur complement
S_exact = K31 K11^{-1} K31^T + K32 K22^{-1} K32^T.  Every matrix below is read off
the explicitly assembled KKT matrix (itself pinned by the M = 0 reduction and the
optimality residuals), not retyped from the oracle's preconditioner:

* Z_bar = -K31 + s K32 with s = sqrt((1+gamma)/beta): the steady Z of
  Eq. (mathcalZ) (K31 = -A, K32 = M_cal) and the time Z_bar of Eq. (S hat)
  (K31 = -A_t, K32 = tau N).
* Z_tilde = the part of Z_bar that is block-diagonal in time (dropping the
  -C (x) M_cal coupling gives Eq. (Z hat approx)); steady, Z_tilde = Z.
* S_tilde = (1/tau) Z_tilde (D (x) M_gamma)^{-1} Z_tilde (Eq. (S_tilde) with the 1/tau
  of Eq. (S hat)) = Z_tilde K11^{-1} Z_tilde because K11 = tau D (x) M_gamma; steady
  (tau = 1, D = I) this is S = Z M_gamma^{-1} Z of Eq. (stoch-prec).
* One hGS sweep with exact mean solves applies Z_hGS^{-1} with
  Z_hGS = (X1 + Xr) X1^{-1} (X1 + Xr^T) (Sec. 4), X1 the level-diagonal blocks of
  Z_tilde and Xr its strictly level-lower part (truncated to the first r terms).

The oracle's apply() must then equal blkdiag(K11, K22, Z_hGS K11^{-1} Z_hGS)^{-1} r
when the Chebyshev mass solves are run to convergence (1/T_N(1/rho) < 1e-17 at
N = 60).  Spectral pins tie the scalars to the paper's theorems: Thm. approx
(lambda(S_bar^{-1} S_exact) in [1/(2(1+alpha)), 1)) and the theorem that bounds
lambda(S_bar^{-1} S_tilde) by (1 -+ theta)^2 with theta its defined supremum.
"""
import math

import numpy as np
import pytest

import sg_inputs as si
from oracle import basis
from oracle.operators import SGData
from oracle.precond import BlockPreconditioner


def _problem(nt, gamma, sigma, r, seed=11, M=2, p=2, nx=4, beta=1e-2):
    pr = si.random_small(seed, nx=nx, M=M, p=p, nt=nt, beta=beta, sigma=sigma, gamma=gamma)
    pr.r = r
    pr.cheb_steps = 60
    if nt:
        pr.T = 0.75            # tau = 0.25 for nt = 3: tau, 1/tau and tau^2 all differ from 1
    return pr


def _blocks(d):
    K = d.kkt_matrix().toarray()
    F = d.slabs * d.P * d.n
    K11, K22 = K[:F, :F], K[F:2 * F, F:2 * F]
    K31, K32 = K[2 * F:, :F], K[2 * F:, F:2 * F]
    assert np.array_equal(K[:F, 2 * F:], K31.T) and np.array_equal(K[F:2 * F, 2 * F:], K32.T)
    assert not K[2 * F:, 2 * F:].any() and not K[:F, F:2 * F].any()
    return F, K11, K22, K31, K32


def _time_block_diag(Z, d):
    nP = d.P * d.n
    out = np.zeros_like(Z)
    for t in range(d.slabs):
        s = slice(t * nP, (t + 1) * nP)
        out[s, s] = Z[s, s]
    return out


def _z_hgs(Zt, d, r):
    """Z_hGS of the symmetric hierarchical block Gauss-Seidel sweep (Sec. 4) for the
    time-block-diagonal Z_tilde, with couplings kept for the first r terms only."""
    n, P = d.n, d.P
    off = basis.level_offsets(d.M, d.p)
    lev = np.zeros(P, dtype=int)
    for dd in range(d.p + 1):
        lev[off[dd]:off[dd + 1]] = dd
    # which chaos pairs a term k < r couples: alpha and beta differ by e_k with k < r
    idx = basis.multi_indices(d.M, d.p)
    keep = np.zeros((P, P), dtype=bool)
    for a in range(P):
        for b in range(P):
            diff = idx[a].astype(int) - idx[b].astype(int)
            nz = np.nonzero(diff)[0]
            if len(nz) == 1 and abs(diff[nz[0]]) == 1 and nz[0] + 1 < r:
                keep[a, b] = True
    nP = n * P
    Zh = np.zeros_like(Zt)
    for t in range(d.slabs):
        base = t * nP
        blk = Zt[base:base + nP, base:base + nP]
        X1 = np.zeros_like(blk)
        Xr = np.zeros_like(blk)
        for a in range(P):
            for b in range(P):
                B = blk[a * n:(a + 1) * n, b * n:(b + 1) * n]
                if a == b:
                    X1[a * n:(a + 1) * n, b * n:(b + 1) * n] = B
                elif lev[a] > lev[b] and keep[a, b]:
                    Xr[a * n:(a + 1) * n, b * n:(b + 1) * n] = B
        Zh[base:base + nP, base:base + nP] = (X1 + Xr) @ np.linalg.solve(X1, X1 + Xr.T)
    return Zh


CASES = [
    # nt, gamma, sigma, r
    (0, 0.0, 0.0, 3),        # sigma = 0: Z_tilde = I (x) A~_1, the sweep is exact
    (0, 0.5, 0.3, 1),        # mean-based truncation r = 1, gamma != 0
    (0, 0.5, 0.3, 3),        # full hierarchical sweep r = M + 1
    (3, 0.0, 0.0, 3),        # time: Z_tilde = I (x) I (x) A^_1
    (3, 0.7, 0.3, 3),        # time, gamma != 0, full sweep
    (3, 0.0, 0.3, 2),        # time, truncated
]


@pytest.mark.parametrize("nt,gamma,sigma,r", CASES)
def test_block_preconditioner_equals_dense_definition(nt, gamma, sigma, r):
    pr = _problem(nt, gamma, sigma, r)
    d = SGData(pr)
    F, K11, K22, K31, K32 = _blocks(d)
    s = math.sqrt((1.0 + gamma) / pr.beta)
    Zbar = -K31 + s * K32
    Zt = _time_block_diag(Zbar, d)
    Zh = _z_hgs(Zt, d, r)
    if sigma == 0.0:                         # no couplings: the sweep is Z_tilde^{-1} itself
        assert np.allclose(Zh, Zt, rtol=0, atol=1e-12 * np.abs(Zt).max())
    S3 = Zh @ np.linalg.solve(K11, Zh)
    Pc = BlockPreconditioner(d, mode="exact")
    rng = np.random.default_rng(7)
    for _ in range(2):
        rv = rng.standard_normal(3 * F)
        z = Pc.apply(rv)
        ref = np.concatenate([np.linalg.solve(K11, rv[:F]), np.linalg.solve(K22, rv[F:2 * F]),
                              np.linalg.solve(S3, rv[2 * F:])])
        for blk in range(3):
            sl = slice(blk * F, (blk + 1) * F)
            err = np.linalg.norm(z[sl] - ref[sl]) / np.linalg.norm(ref[sl])
            assert err <= 1e-11, (blk, err)


def test_steady_schur_approximation_bounds_with_kkt_blocks():
    """Steady, gamma = 0: lambda(S^{-1} S_exact) in [1/2, 1] for S = Z M^{-1} Z (the n_t = 1
    case of Thm. approx), with Z and S_exact read off the assembled KKT matrix.  The oracle's
    block 3 as an explicit matrix (exact mean solves, sigma != 0, r = M + 1) must be symmetric
    positive definite."""
    pr = _problem(0, 0.0, 0.3, 3)
    d = SGData(pr)
    F, K11, K22, K31, K32 = _blocks(d)
    Sx = K31 @ np.linalg.solve(K11, K31.T) + K32 @ np.linalg.solve(K22, K32.T)
    s = math.sqrt(1.0 / pr.beta)
    Z = -K31 + s * K32
    S = Z @ np.linalg.solve(K11, Z)
    ev = np.sort(np.linalg.eigvals(np.linalg.solve(S, Sx)).real)
    assert ev[0] >= 0.5 - 1e-10 and ev[-1] <= 1 + 1e-10
    assert ev[-1] >= 0.9 and ev[0] <= 0.6          # the interval is (nearly) attained
    # the oracle's block 3 (Z replaced by Z_hGS) as an explicit matrix
    Pc = BlockPreconditioner(d, mode="exact")
    S3inv = np.stack([Pc.apply(np.concatenate([np.zeros(2 * F), e]))[2 * F:]
                      for e in np.eye(F)], axis=1)
    assert np.allclose(S3inv, S3inv.T, rtol=0, atol=1e-12 * np.abs(S3inv).max())
    assert np.linalg.eigvalsh(0.5 * (S3inv + S3inv.T)).min() > 0


def _theta(Zt, Cm, W):
    """theta = sup_v ||W^{1/2} Cm^T v|| / ||W^{1/2} Zt^T v|| (definition in the paper's
    theorem relating S_bar and S_tilde), as a generalized eigenvalue problem."""
    A = Cm @ W @ Cm.T
    B = Zt @ W @ Zt.T
    ev = np.linalg.eigvals(np.linalg.solve(B, A)).real
    return math.sqrt(max(ev.max(), 0.0))


@pytest.mark.parametrize("gamma", [0.0, 0.7])
def test_time_schur_scalars_follow_the_paper_theorems(gamma):
    """Time mode (Sec. 3-4): with W = (1/tau)(D (x) M_gamma)^{-1} = K11^{-1},
    (i) Thm. approx: lambda(S_bar^{-1} S_exact) in [1/(2(1+alpha)), 1) with
        S_bar = Z_bar W Z_bar^T and alpha below ((sqrt k + 1)/(sqrt k - 1))^2 - 1,
        k = cond(A_t);
    (ii) (1 - theta)^2 <= lambda(S_bar^{-1} S_tilde) <= (1 + theta)^2 with
        S_tilde = Z_tilde W Z_tilde;
    (iii) the oracle's block 3 with exact mean solves and sigma = 0 is S_tilde^{-1}.
    A wrong power of tau in W, or a missing 1 + gamma, moves the spectrum in (i) by
    a factor 1/tau = 4 or (1+gamma) and fails the bound."""
    pr = _problem(3, gamma, 0.0, 3, beta=1e-1)
    d = SGData(pr)
    F, K11, K22, K31, K32 = _blocks(d)
    tau = d.tau
    assert tau == pytest.approx(0.25)
    Sx = K31 @ np.linalg.solve(K11, K31.T) + K32 @ np.linalg.solve(K22, K32.T)
    s = math.sqrt((1.0 + gamma) / pr.beta)
    W = np.linalg.inv(K11)
    Zbar = -K31 + s * K32
    Sbar = Zbar @ W @ Zbar.T
    At = -K31
    sv = np.linalg.svd(At, compute_uv=False)
    kap = sv[0] / sv[-1]
    alpha_sup = ((math.sqrt(kap) + 1) / (math.sqrt(kap) - 1)) ** 2 - 1
    ev = np.sort(np.linalg.eigvals(np.linalg.solve(Sbar, Sx)).real)
    assert ev[-1] <= 1 + 1e-10
    assert ev[0] >= 1 / (2 * (1 + alpha_sup)) - 1e-10
    Zt = _time_block_diag(Zbar, d)
    Cm = Zt - Zbar                          # C (x) M_cal, the dropped coupling
    assert np.abs(Cm).max() > 0
    theta = _theta(Zt, Cm, W)
    St = Zt @ W @ Zt
    ev2 = np.sort(np.linalg.eigvals(np.linalg.solve(Sbar, St)).real)
    if theta < 1:
        assert ev2[0] >= (1 - theta) ** 2 - 1e-10
    assert ev2[-1] <= (1 + theta) ** 2 + 1e-10
    Pc = BlockPreconditioner(d, mode="exact")
    rv = np.random.default_rng(3).standard_normal(F)
    z3 = Pc.apply(np.concatenate([np.zeros(2 * F), rv]))[2 * F:]
    ref = np.linalg.solve(St, rv)
    assert np.linalg.norm(z3 - ref) <= 1e-11 * np.linalg.norm(ref)


def _z_bar_hgs(Zbar, Zt, d, r):
    """Z_bar with the slab operator Z~_t replaced by its hGS approximation Z_hGS: the
    time coupling -C (x) M_cal of Z_bar is kept exactly (Eq. (Z hat))."""
    return _z_hgs(Zt, d, r) + (Zbar - Zt)


@pytest.mark.parametrize("gamma,sigma,r", [(0.0, 0.0, 3), (0.7, 0.3, 3), (0.0, 0.3, 2)])
def test_coupled_schur_block_equals_dense_definition(gamma, sigma, r):
    """Time mode, coupled Schur block: with exact mean solves the oracle's block 3 is
    S_bar^{-1} r with S_bar = (1/tau) Z_bar_hGS (D (x) M_gamma)^{-1} Z_bar_hGS^T = Z K11^{-1} Z^T
    (Z = Z_bar_hGS: the paper's Z_bar of Eq. (Z hat), read off the assembled KKT matrix, with
    the slab operator replaced by its hGS approximation; exact for sigma = 0); blocks 1, 2
    are those of the block-diagonal form."""
    pr = _problem(3, gamma, sigma, r)
    d = SGData(pr)
    F, K11, K22, K31, K32 = _blocks(d)
    s = math.sqrt((1.0 + gamma) / pr.beta)
    Zbar = -K31 + s * K32
    Zt = _time_block_diag(Zbar, d)
    Zc = _z_bar_hgs(Zbar, Zt, d, r)
    if sigma == 0.0:
        assert np.allclose(Zc, Zbar, rtol=0, atol=1e-12 * np.abs(Zbar).max())
    Sbar = Zc @ np.linalg.solve(K11, Zc.T)
    Pc = BlockPreconditioner(d, mode="exact", schur="coupled")
    Pd = BlockPreconditioner(d, mode="exact")
    rv = np.random.default_rng(9).standard_normal(3 * F)
    z = Pc.apply(rv)
    zd = Pd.apply(rv)
    assert np.linalg.norm(z[:2 * F] - zd[:2 * F]) <= 1e-14 * np.linalg.norm(zd[:2 * F])
    ref = np.linalg.solve(Sbar, rv[2 * F:])
    assert np.linalg.norm(z[2 * F:] - ref) <= 1e-11 * np.linalg.norm(ref)


def test_coupled_schur_block_symmetric_positive_and_within_the_theorem_bounds():
    """The coupled block with V-cycle mean solves is a symmetric positive definite map (the
    forward and backward substitutions are transposes of each other for a symmetric sweep),
    and with exact mean solves and sigma = 0 its spectrum against the exact Schur complement
    obeys Thm. approx: lambda(S_bar^{-1} S_exact) in [1/(2(1+alpha)), 1)."""
    pr = _problem(3, 0.3, 0.3, 3)
    d = SGData(pr)
    F = d.slabs * d.P * d.n
    Pc = BlockPreconditioner(d, schur="coupled")
    B = np.stack([Pc.apply(np.concatenate([np.zeros(2 * F), e]))[2 * F:] for e in np.eye(F)], axis=1)
    assert np.allclose(B, B.T, rtol=0, atol=1e-12 * np.abs(B).max())
    assert np.linalg.eigvalsh(0.5 * (B + B.T)).min() > 0
    pr = _problem(3, 0.0, 0.0, 3, beta=1e-1)
    d = SGData(pr)
    F, K11, K22, K31, K32 = _blocks(d)
    Sx = K31 @ np.linalg.solve(K11, K31.T) + K32 @ np.linalg.solve(K22, K32.T)
    Pc = BlockPreconditioner(d, mode="exact", schur="coupled")
    Sinv = np.stack([Pc.apply(np.concatenate([np.zeros(2 * F), e]))[2 * F:] for e in np.eye(F)], axis=1)
    ev = np.sort(np.linalg.eigvals(Sinv @ Sx).real)
    sv = np.linalg.svd(-K31, compute_uv=False)
    kap = sv[0] / sv[-1]
    alpha_sup = ((math.sqrt(kap) + 1) / (math.sqrt(kap) - 1)) ** 2 - 1
    assert ev[-1] <= 1 + 1e-10 and ev[0] >= 1 / (2 * (1 + alpha_sup)) - 1e-10


def test_coupled_schur_minres_converges_to_the_direct_solution():
    """MINRES with the coupled preconditioner reaches the direct solution; at a small time step
    it needs no more iterations than the block-diagonal one (Sec. 4: S_tilde departs from S_bar
    when tau is small against sqrt(beta))."""
    from oracle.solve import solve, direct_solve
    pr = si.random_small(17, nx=8, M=2, p=2, nt=6, beta=1e-1)
    pr.T = 0.06
    xd = direct_solve(pr)
    rc = solve(pr, schur="coupled")
    rd = solve(pr, schur="diagonal")
    assert rc.status == "ok" and rc.rel_true <= pr.tol
    assert np.linalg.norm(rc.x - xd) <= 1e-6 * np.linalg.norm(xd)
    assert rc.iterations <= rd.iterations, (rc.iterations, rd.iterations)


def test_exact_mass_blocks_are_the_inverse_mass():
    """mass_solve = "exact": blocks 1 and 2 are exactly K11^{-1} and K22^{-1} (no Chebyshev
    error), steady and time."""
    for nt in (0, 3):
        pr = _problem(nt, 0.5 if nt == 0 else 0.0, 0.3, 3)
        pr.cheb_steps = 2                     # a poor Chebyshev: the exact option must not use it
        pr.mass_solve = "exact"
        d = SGData(pr)
        F, K11, K22, K31, K32 = _blocks(d)
        rv = np.random.default_rng(nt).standard_normal(3 * F)
        z = BlockPreconditioner(d).apply(rv)
        assert np.linalg.norm(K11 @ z[:F] - rv[:F]) <= 1e-13 * np.linalg.norm(rv[:F])
        assert np.linalg.norm(K22 @ z[F:2 * F] - rv[F:2 * F]) <= 1e-13 * np.linalg.norm(rv[F:2 * F])


def _hgsoc_dense(d, r_trunc, third_block):
    """Symmetric block Gauss-Seidel over the chaos levels of the (truncated) KKT matrix, with
    each level's own block replaced by P~ (third_block: the (3,3) block per chaos column),
    for the block-diagonal-in-time part of the KKT matrix: forward sweep (D + L)^{-1} R, then
    the backward sweep (D + U)^{-1} (R - L x_f)."""
    K = d.kkt_matrix().toarray()
    n, P, S = d.n, d.P, d.slabs
    F = S * P * n
    off = basis.level_offsets(d.M, d.p)
    lev = np.zeros(P, dtype=int)
    for dd in range(d.p + 1):
        lev[off[dd]:off[dd + 1]] = dd
    idx = basis.multi_indices(d.M, d.p)
    keep = np.ones((P, P), dtype=bool)
    for a in range(P):
        for b in range(P):
            diff = idx[a].astype(int) - idx[b].astype(int)
            nz = np.nonzero(diff)[0]
            if len(nz) == 1 and abs(diff[nz[0]]) == 1 and nz[0] + 1 >= r_trunc:
                keep[a, b] = False                      # a coupling dropped by the truncation
    # unknown u = (field f, slab t, chaos alpha, node i) at f*F + t*P*n + alpha*n + i
    N3 = 3 * F
    field = np.repeat(np.arange(3), F)
    slab = np.tile(np.repeat(np.arange(S), P * n), 3)
    alpha = np.tile(np.repeat(np.arange(P), n), 3 * S)
    L = np.zeros_like(K)
    U = np.zeros_like(K)
    same_slab = slab[:, None] == slab[None, :]
    la, lb = lev[alpha][:, None], lev[alpha][None, :]
    kp = keep[alpha[:, None], alpha[None, :]]
    L[(la > lb) & same_slab & kp] = K[(la > lb) & same_slab & kp]
    U[(la < lb) & same_slab & kp] = K[(la < lb) & same_slab & kp]
    Dm = np.zeros_like(K)
    Dw = d.d_weights()
    Mm = d.Mass.toarray()
    for t in range(S):
        sc = 1.0 if d.nt == 0 else d.tau * Dw[t]
        for a in range(P):
            for f, blk in ((0, sc * Mm), (1, sc * d.beta * Mm), (2, third_block(sc))):
                o = f * F + t * P * n + a * n
                Dm[o:o + n, o:o + n] = blk
    def apply(R):
        xf = np.linalg.solve(Dm + L, R)
        return np.linalg.solve(Dm + U, R - L @ xf)
    return apply


@pytest.mark.parametrize("nt,gamma,sigma,r", [(0, 0.0, 0.3, 3), (0, 0.5, 0.3, 2), (3, 0.0, 0.3, 3), (0, 0.0, 0.0, 3)])
def test_hgsoc_equals_symmetric_block_gauss_seidel(nt, gamma, sigma, r):
    """Alg. 2-3 (Alg. 4 per slab) with exact mass and mean solves is the symmetric block
    Gauss-Seidel sweep over the chaos levels of the truncated KKT matrix (block-diagonal in
    time) whose level blocks are P~ = blkdiag(M, beta M, A~_1 M^{-1} A~_1) (time:
    blkdiag(tau D_t M, beta tau D_t M, (1/tau) A^_1 (D_t M)^{-1} A^_1)): the paper's sweep
    order 0..p-1, p, p-1..0 solves level p once, as the symmetric sweep does."""
    from oracle.precond import HGSoc
    pr = _problem(nt, gamma, sigma, r)
    pr.mass_solve = "exact"
    d = SGData(pr)
    H = HGSoc(d, mode="exact")
    A0 = H.A0.toarray()
    Mm = d.Mass.toarray()
    Dw = d.d_weights()
    third = lambda sc: A0 @ np.linalg.solve(sc * Mm, A0)
    ref = _hgsoc_dense(d, r, third)
    rv = np.random.default_rng(13).standard_normal(3 * d.slabs * d.P * d.n)
    assert np.linalg.norm(H.apply(rv) - ref(rv)) <= 1e-10 * np.linalg.norm(ref(rv))
    Hl = HGSoc(d, mode="exact", third="literal")
    refl = _hgsoc_dense(d, r, lambda sc: A0)
    assert np.linalg.norm(Hl.apply(rv) - refl(rv)) <= 1e-10 * np.linalg.norm(refl(rv))


def test_hgsoc_fgmres_converges_and_the_literal_block_does_not():
    """FGMRES with hGSoc reaches the direct solution; with P~'s third block read literally as
    A~_1 it stalls (the reason the Schur reading is taken)."""
    from oracle.krylov import fgmres
    from oracle.precond import HGSoc
    from oracle.solve import direct_solve
    pr = si.random_small(3, nx=8, M=2, p=2, beta=1e-2)
    d = SGData(pr)
    b = d.rhs()
    xd = direct_solve(pr)
    res = fgmres(d.kkt_apply, HGSoc(d).apply, b, tol=1e-9)
    assert res.status == "ok" and np.linalg.norm(res.x - xd) <= 1e-7 * np.linalg.norm(xd)
    lit = fgmres(d.kkt_apply, HGSoc(d, third="literal").apply, b, tol=1e-9, max_iter=150)
    assert lit.status != "ok" and lit.rel_true > 1e-4

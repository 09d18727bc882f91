"""Preconditioner of the oracle.

Block-diagonal preconditioner (Eq. (stoch-prec) steady, Eq. (precon for time)):
  block 1: M_gamma^{-1}   ~ Chebyshev semi-iteration on M, columns scaled by 1/H^gamma
  block 2: (beta M)^{-1}  ~ Chebyshev on M, scaled by 1/beta
  block 3: S^{-1} = Z^{-1} M_gamma Z^{-1} with Z = A + sqrt((1+gamma)/beta) M_cal (Eq. (mathcalZ));
           time: S~^{-1} = tau Z~^{-1} (D (x) M_gamma) Z~^{-1} with Z~ block diagonal in time
           (Eqs. (Z hat approx), (S_tilde), (S hat)); time blocks 1, 2 carry the extra 1/(tau D_t).
  time, schur="coupled": S_bar^{-1} = tau Z_bar^{-T} (D (x) M_gamma) Z_bar^{-1} with the coupled
           Z_bar = I (x) Z~_t - C (x) M_cal of Eq. (S hat) / Eq. (Z hat), which keeps the -C (x) H_1 (x) M
           term: Z_bar^{-1} by block forward substitution in time, Z_bar^{-T} by backward
           substitution, each step one solve with the slab operator Z~_t.
  Solves with Z / Z~ use the hierarchical Gauss-Seidel sweep of Alg. 1 (one application,
  i.e. the Richardson iteration of Sec. 5 with N = 1 and zero initial guess), truncated to
  the first r terms of the expansion (Sec. 2, Eq. (matvec-block) and the index set I_tau).

Readings (the paper leaves these open):
* Chebyshev: the textbook Golub-Varga semi-iteration with omega_1 = 1,
  omega_2 = 2/(2-rho^2), omega_{k+1} = 1/(1 - rho^2 omega_k / 4), x^(0) = 0, and the
  paper's D = (lmin+lmax)/2 diag(M), rho = (lmax-lmin)/(lmax+lmin), lmin = 1/4, lmax = 9/4.
* hGS: correction form V_(d) += B (R_(d) - (Z_r V)_(d)) over the palindromic level order
  0, 1, ..., p, ..., 1, 0; identical to Alg. 1 when B = A~_1^{-1} and symmetric for any
  symmetric B.
* Mean solves B: one V(nu_pre, nu_post) cycle with damped Jacobi (omega), bilinear
  prolongation P, restriction P^T and Galerkin coarse operators P^T A P, down to the
  2x2-element grid (one interior node) which is solved exactly; or, in 'exact' mode,
  a sparse LU solve (used for pins only).
"""
from __future__ import annotations

import math

import numpy as np
import scipy.sparse as sp
import scipy.sparse.linalg as spla

from . import basis


# ---------------------------------------------------------------- Chebyshev --
CHEB_LMIN, CHEB_LMAX = 0.25, 2.25


def chebyshev(Mass, B, steps):
    """N-step Chebyshev semi-iteration for Mass X = B (B: n or n x c)."""
    gam = 0.5 * (CHEB_LMIN + CHEB_LMAX)
    rho = (CHEB_LMAX - CHEB_LMIN) / (CHEB_LMAX + CHEB_LMIN)
    dinv = 1.0 / (gam * Mass.diagonal())
    if B.ndim == 2:
        dinv = dinv[:, None]
    x_old = np.zeros_like(B)
    x = np.zeros_like(B)
    omega = 1.0
    for k in range(steps):
        if k == 0:
            omega = 1.0
        elif k == 1:
            omega = 2.0 / (2.0 - rho * rho)
        else:
            omega = 1.0 / (1.0 - rho * rho * omega / 4.0)
        r = B - Mass @ x
        x_new = omega * (dinv * r + x - x_old) + x_old
        x_old, x = x, x_new
    return x


# ----------------------------------------------------------------- V-cycle --
def prolongation(nx: int):
    """Bilinear interpolation from the (nx/2)-element grid to the nx-element grid,
    interior nodes only (x1 fastest): P = P1 (x) P1."""
    mf, mc = nx - 1, nx // 2 - 1
    P1 = sp.lil_matrix((mf, mc))
    for I in range(1, nx // 2):
        fi = 2 * I - 1                 # 0-based fine interior index of fine node 2I
        P1[fi, I - 1] = 1.0
        P1[fi - 1, I - 1] = 0.5
        if fi + 1 < mf:
            P1[fi + 1, I - 1] = 0.5
    P1 = P1.tocsr()
    return sp.kron(P1, P1, format="csr")


class VCycle:
    """Geometric multigrid V-cycle for an SPD Q1 operator on a power-of-two grid."""

    def __init__(self, A, nx, nu_pre=2, nu_post=2, omega=0.8):
        assert nx >= 2 and (nx & (nx - 1)) == 0, "grid must be a power of two"
        self.levels = []      # (A, dinv, P to this level from the next coarser)
        self.nu_pre, self.nu_post, self.omega = nu_pre, nu_post, omega
        A = sp.csr_matrix(A)
        while True:
            if nx == 2:
                self.levels.append((A, None, None))
                break
            P = prolongation(nx)
            self.levels.append((A, 1.0 / A.diagonal(), P))
            A = sp.csr_matrix(P.T @ A @ P)
            nx //= 2
        self.coarse = A.toarray()

    def apply(self, B, level=0):
        """One V-cycle with zero initial guess for A X = B (B: n or n x c)."""
        A, dinv, P = self.levels[level]
        if P is None:
            return np.linalg.solve(self.coarse, B)
        d = dinv[:, None] if B.ndim == 2 else dinv
        X = np.zeros_like(B)
        for _ in range(self.nu_pre):
            X = X + self.omega * d * (B - A @ X)
        R = B - A @ X
        X = X + P @ self.apply(P.T @ R, level + 1)
        for _ in range(self.nu_post):
            X = X + self.omega * d * (B - A @ X)
        return X


class ExactSolve:
    def __init__(self, A):
        self.lu = spla.splu(sp.csc_matrix(A))

    def apply(self, B):
        return self.lu.solve(B)


# --------------------------------------------------------------------- hGS --
def visit_order(p: int):
    """Level order of one symmetric hierarchical sweep: 0, 1, ..., p, ..., 1, 0."""
    return list(range(p + 1)) + list(range(p - 1, -1, -1))


class HGS:
    """One application of the hierarchical Gauss-Seidel sweep (Alg. 1) to
    Z_r = A~_0 (x) I + sum_{k=1}^{r-1} G_k (x) coef_k K_k, matricized."""

    def __init__(self, data, A0, coef, r, mean_solver):
        self.d = data
        self.A0 = A0                   # mean operator A~_1 (steady) / A^_1 (time)
        self.coef = coef               # scalar multiplying K_k, k >= 1 (1 steady, tau time)
        self.r = r
        self.B = mean_solver
        self.off = basis.level_offsets(data.M, data.p)

    def zr_apply(self, V):
        Y = self.A0 @ V
        for k in range(1, self.r):
            Y += self.coef * (self.d.K[k] @ V @ self.d.G[k])
        return Y

    def apply(self, R):
        V = np.zeros_like(R)
        for lev in visit_order(self.d.p):
            a, b = self.off[lev], self.off[lev + 1]
            rhs = R[:, a:b] - self.zr_apply(V)[:, a:b]
            V[:, a:b] += self.B.apply(rhs)
        return V


# ------------------------------------------------------- block preconditioner --
class BlockPreconditioner:
    def __init__(self, data, mode="vcycle", schur="diagonal", mass_solve=None):
        assert schur in ("diagonal", "coupled")
        self.d = data
        self.schur = schur
        # mass blocks 1, 2 (Sec. 5): Chebyshev semi-iteration, or the exact solve with M (the
        # paper's Cholesky option), here a sparse LU factorisation of M
        self.mass_solve = mass_solve or getattr(data.pr, "mass_solve", "chebyshev")
        assert self.mass_solve in ("chebyshev", "exact")
        self.mass_lu = spla.splu(sp.csc_matrix(data.Mass)) if self.mass_solve == "exact" else None
        pr = data.pr
        s = math.sqrt((1.0 + data.gamma) / data.beta)
        Mm = data.Mass
        if data.nt == 0:
            A0 = data.K[0] + s * Mm                       # A~_1 = A_1 + sqrt((1+g)/b) M
            coef = 1.0
        else:
            tau = data.tau
            A0 = (1.0 + tau * s) * Mm + tau * data.K[0]   # A^_1 of Eq. (A_hat)
            coef = tau
        self.A0 = A0
        if mode == "exact":
            solver = ExactSolve(A0)
        else:
            solver = VCycle(A0, data.nx, pr.nu_pre, pr.nu_post, pr.omega)
        self.hgs = HGS(data, A0, coef, pr.trunc, solver)
        self.steps = pr.cheb_steps

    def apply(self, r):
        d = self.d
        F = d.slabs * d.P * d.n
        nP = d.P * d.n
        z = np.zeros_like(r)
        Mm = d.Mass
        Dw = d.d_weights()
        if d.nt > 0 and self.schur == "coupled":
            return self._apply_coupled(r)
        for t in range(d.slabs):
            sl = slice(t * nP, (t + 1) * nP)
            R1 = d.mat(r[:F][sl])
            R2 = d.mat(r[F:2 * F][sl])
            R3 = d.mat(r[2 * F:][sl])
            sc = 1.0 if d.nt == 0 else d.tau * Dw[t]
            Z1 = self.mass_inv(R1) / (sc * d.hgam[None, :])
            Z2 = self.mass_inv(R2) / (sc * d.beta)
            W = self.hgs.apply(R3)
            if d.nt == 0:
                Z3 = self.hgs.apply(Mm @ W * d.hgam[None, :])
            else:
                Z3 = d.tau * self.hgs.apply(Dw[t] * (Mm @ W) * d.hgam[None, :])
            z[:F][sl] = d.vec(Z1)
            z[F:2 * F][sl] = d.vec(Z2)
            z[2 * F:][sl] = d.vec(Z3)
        return z

    def mass_inv(self, B):
        if self.mass_lu is not None:
            return self.mass_lu.solve(B)
        return chebyshev(self.d.Mass, B, self.steps)

    def _apply_coupled(self, r):
        """Time mode with the coupled Schur block: blocks 1 and 2 as in apply(); block 3
        is tau Z_bar^{-T} (D (x) M_gamma) Z_bar^{-1} r_3 where Z_bar x = r reads
        Z~ x_t = r_t + M_cal x_{t-1} (x_0 = 0, forward in t) and Z_bar^T x = r reads
        Z~ x_t = r_t + M_cal x_{t+1} (x_{n_t+1} = 0, backward in t); every solve with the
        slab operator Z~ is one hGS sweep."""
        d = self.d
        F = d.slabs * d.P * d.n
        nP = d.P * d.n
        Mm = d.Mass
        Dw = d.d_weights()
        z = np.zeros_like(r)
        for t in range(d.nt):
            sl = slice(t * nP, (t + 1) * nP)
            sc = d.tau * Dw[t]
            z[:F][sl] = d.vec(self.mass_inv(d.mat(r[:F][sl])) / (sc * d.hgam[None, :]))
            z[F:2 * F][sl] = d.vec(self.mass_inv(d.mat(r[F:2 * F][sl])) / (sc * d.beta))
        R3 = [d.mat(r[2 * F:][t * nP:(t + 1) * nP]) for t in range(d.nt)]
        X = []
        for t in range(d.nt):                       # Z_bar X = R3, forward in time
            rhs = R3[t] + (Mm @ X[t - 1] if t > 0 else 0.0)
            X.append(self.hgs.apply(rhs))
        W = [d.tau * Dw[t] * (Mm @ X[t]) * d.hgam[None, :] for t in range(d.nt)]
        Z = [None] * d.nt
        for t in reversed(range(d.nt)):             # Z_bar^T Z = W, backward in time
            rhs = W[t] + (Mm @ Z[t + 1] if t + 1 < d.nt else 0.0)
            Z[t] = self.hgs.apply(rhs)
        for t in range(d.nt):
            z[2 * F:][t * nP:(t + 1) * nP] = d.vec(Z[t])
        return z


# -------------------------------------------------------------------- hGSoc --
class HGSoc:
    """The hGS preconditioner for the optimal control problem (Alg. 2-3, steady) and its
    parallel-in-time form (Alg. 4: Alg. 2-3 on every time slab, the slabs independent).

    Levels are visited 0, 1, ..., p, ..., 1, 0.  At a visit of level l the three fields of
    the level's columns are set (overwritten, as in the algorithm) by one solve with
    P~ = blkdiag(M, beta M, A~_1) of the right-hand side R_(l) minus the couplings of the
    (truncated) KKT matrix to the other levels, with their current values:
      Y: R^Y_(l) + c sum_{k=1}^{r-1} (K_k V^Lambda G_k)_(l)      (the -A^T Lambda row, Eq. (stoch-system))
      U: R^U_(l)                                                  (beta M and M do not couple levels)
      L: R^L_(l) + c sum_{k=1}^{r-1} (K_k V^Y G_k)_(l)           (the -A Y row)
    with c = 1 steady, tau in time mode (the slab operator L = I (x) M + tau A).  G_k couples
    only neighbouring levels and the level's own block is replaced by P~, so the terms
    C, E, F, H of Alg. 2-3 (couplings through H^gamma and H_1, both diagonal here) vanish.
    Reading of P~'s third block (the paper writes A~_1 and calls P~ "derived from the blocks
    of the deterministic KKT system"): third="schur" (default) takes the deterministic
    Schur-complement approximation S~_1 = A~_1 M^{-1} A~_1 (the n_xi = 1 case of
    Eq. (mathcalZ)), so the Lambda solve is A~_1^{-1} M A~_1^{-1}: two mean solves.
    third="literal" takes A~_1 itself (one mean solve); with it FGMRES does not converge on
    the test problems (the block has the scale of a stiffness matrix, not of the Schur
    complement), so the hot path uses the first reading.
    Time mode (reading of Alg. 4): P~_t = blkdiag(tau D_t M, beta tau D_t M, S~_t) on slab t with
    S~_t = (1/tau) A^_1 (D_t M)^{-1} A^_1 (the one-slab case of Eq. (S hat) / Eq. (S_tilde)).
    Mass solves as in BlockPreconditioner (Chebyshev or exact); mean solves by one V-cycle
    (or exactly in 'exact' mode).
    """

    def __init__(self, data, mode="vcycle", mass_solve=None, third="schur"):
        assert third in ("schur", "literal")
        self.third = third
        self.d = data
        pr = data.pr
        s = math.sqrt((1.0 + data.gamma) / data.beta)
        Mm = data.Mass
        if data.nt == 0:
            A0 = data.K[0] + s * Mm
            self.coef = 1.0
        else:
            A0 = (1.0 + data.tau * s) * Mm + data.tau * data.K[0]
            self.coef = data.tau
        self.A0 = A0
        self.B = ExactSolve(A0) if mode == "exact" else VCycle(A0, data.nx, pr.nu_pre, pr.nu_post, pr.omega)
        self.r = pr.trunc
        self.off = basis.level_offsets(data.M, data.p)
        self.mass = BlockPreconditioner.__new__(BlockPreconditioner)     # only its mass solver
        self.mass.d = data
        self.mass.steps = pr.cheb_steps
        self.mass.mass_solve = mass_solve or getattr(pr, "mass_solve", "chebyshev")
        self.mass.mass_lu = spla.splu(sp.csc_matrix(Mm)) if self.mass.mass_solve == "exact" else None

    def coupling(self, V):
        """c sum_{k=1}^{r-1} K_k V G_k (all columns)."""
        d = self.d
        out = np.zeros_like(V)
        for k in range(1, self.r):
            out += d.K[k] @ V @ d.G[k]
        return self.coef * out

    def apply(self, rvec):
        d = self.d
        F = d.slabs * d.P * d.n
        nP = d.P * d.n
        Dw = d.d_weights()
        z = np.zeros_like(rvec)
        for t in range(d.slabs):
            sl = slice(t * nP, (t + 1) * nP)
            RY, RU, RL = d.mat(rvec[:F][sl]), d.mat(rvec[F:2 * F][sl]), d.mat(rvec[2 * F:][sl])
            sc = 1.0 if d.nt == 0 else d.tau * Dw[t]
            VU = self.mass.mass_inv(RU) / (sc * d.beta)
            VY = np.zeros_like(RY)
            VL = np.zeros_like(RL)
            for lev in visit_order(d.p):
                a, b = self.off[lev], self.off[lev + 1]
                cY = RY[:, a:b] + self.coupling(VL)[:, a:b]
                cL = RL[:, a:b] + self.coupling(VY)[:, a:b]
                VY[:, a:b] = self.mass.mass_inv(cY) / sc
                if self.third == "literal":
                    VL[:, a:b] = self.B.apply(cL)
                else:
                    VL[:, a:b] = sc * self.B.apply(d.Mass @ self.B.apply(cL))
            z[:F][sl], z[F:2 * F][sl], z[2 * F:][sl] = d.vec(VY), d.vec(VU), d.vec(VL)
        return z

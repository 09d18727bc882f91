"""SG operators and KKT systems for the oracle.

Vectors use the paper's vec order (Sec. 2, Eq. (m)): node index fastest, then
the chaos index alpha (columns of the matricized V), then the time level.  A
KKT vector is [y; u; lambda], each of length nt*P*n (nt = 1 when steady).

* SG stiffness  A = sum_k G_k (x) K_k            (Sec. 2, after Eq. (def-Mcal))
* SG mass       M_cal = I (x) M, M_gamma = H^gamma (x) M with
                H^gamma = diag(1, 1+gamma, ..., 1+gamma)  (Eq. (def-Mcal))
* steady KKT    [[M_g, 0, -A^T], [0, beta M, M^T], [-A, M, 0]]     Eq. (stoch-system)
* time KKT      [[tau D(x)M_g, 0, -A_t^T], [0, beta tau D(x)M, tau N^T], [-A_t, tau N, 0]]
                A_t = I(x)L - C(x)M_cal, L = I(x)M + tau A, N = I(x)I(x)M,
                C = ones on the first subdiagonal, D = diag(1/2, 1, ..., 1, 1/2)
                (D = [1] when nt = 1)                 Eqs. (K_t for stochastic), (CD), (KKT:stoch-time-dependent)

Two forms are provided: explicit sparse assembly with Kronecker products (small
sizes) and the matricized form vec(sum_k K_k X G_k) of Eq. (mat-vec)/(Zv).
"""
from __future__ import annotations

import math

import numpy as np
import scipy.sparse as sp

from . import basis, fe


class SGData:
    """Matrices of one problem: K_k, M, G_k, H^gamma and scalars."""

    def __init__(self, pr):
        self.pr = pr
        self.nx, self.M, self.p = pr.nx, pr.M, pr.p
        self.n = (pr.nx - 1) ** 2
        self.chaos = getattr(pr, "chaos", "legendre")
        self.K = fe.stiffness_terms(pr.nx, pr.kappa)       # one per coefficient term
        self.nterms = len(self.K)
        if self.chaos == "hermite":                       # lognormal coefficient, Hermite chaos
            self.G = basis.h_matrices(pr.M, pr.p, self.nterms)
        else:                                              # affine coefficient, Legendre chaos
            self.G = basis.g_matrices(pr.M, pr.p)
        self.P = self.G[0].shape[0]
        # the stiffness integrals are invariant under scaling of the domain, the mass scales
        # with the element area (side length^2)
        self.Mass = fe.mass(pr.nx) * getattr(pr, "length", 1.0) ** 2
        self.hgam = np.array([1.0] + [1.0 + pr.gamma] * (self.P - 1))
        self.beta, self.gamma = pr.beta, pr.gamma
        self.nt = pr.nt
        self.slabs = max(pr.nt, 1)
        self.tau = pr.T / pr.nt if pr.nt else 1.0
        self.Gs = [sp.csr_matrix(g) for g in self.G]

    # ---- matricized applies -------------------------------------------------
    def mat(self, x):
        """vec -> n x P (one slab)."""
        return x.reshape(self.P, self.n).T

    def vec(self, X):
        return X.T.reshape(-1)

    def sg_apply(self, X, terms=None):
        """sum_k K_k X G_k over the given k (default all)."""
        ks = range(self.nterms) if terms is None else terms
        Y = np.zeros_like(X)
        for k in ks:
            Y += self.K[k] @ X @ self.G[k]
        return Y

    def d_weights(self):
        if self.nt <= 1:
            return np.ones(self.slabs)
        d = np.ones(self.nt)
        d[0] = d[-1] = 0.5
        return d

    def kkt_apply(self, x):
        """Matricized KKT product, steady or time-dependent."""
        F = self.slabs * self.P * self.n
        y, u, lam = x[:F], x[F:2 * F], x[2 * F:]
        out = np.zeros_like(x)
        o1, o2, o3 = out[:F], out[F:2 * F], out[2 * F:]
        Mm = self.Mass
        sl = lambda v, t: v[t * self.P * self.n:(t + 1) * self.P * self.n]
        if self.nt == 0:
            Y, U, L = self.mat(y), self.mat(u), self.mat(lam)
            o1[:] = self.vec(Mm @ Y * self.hgam[None, :] - self.sg_apply(L))
            o2[:] = self.vec(self.beta * (Mm @ U) + Mm @ L)
            o3[:] = self.vec(-self.sg_apply(Y) + Mm @ U)
            return out
        tau, D = self.tau, self.d_weights()
        for t in range(self.nt):
            Y, U, L = self.mat(sl(y, t)), self.mat(sl(u, t)), self.mat(sl(lam, t))
            Lnext = self.mat(sl(lam, t + 1)) if t + 1 < self.nt else np.zeros_like(L)
            Yprev = self.mat(sl(y, t - 1)) if t > 0 else np.zeros_like(Y)
            AtTL = Mm @ L + tau * self.sg_apply(L) - Mm @ Lnext
            AtY = Mm @ Y + tau * self.sg_apply(Y) - Mm @ Yprev
            sl(o1, t)[:] = self.vec(tau * D[t] * (Mm @ Y) * self.hgam[None, :] - AtTL)
            sl(o2, t)[:] = self.vec(self.beta * tau * D[t] * (Mm @ U) + tau * (Mm @ L))
            sl(o3, t)[:] = self.vec(-AtY + tau * (Mm @ U))
        return out

    # ---- explicit assembly ---------------------------------------------------
    def sg_matrix(self):
        return sum(sp.kron(self.Gs[k], self.K[k], format="csr") for k in range(self.nterms))

    def mass_cal(self):
        return sp.kron(sp.identity(self.P), self.Mass, format="csr")

    def mass_gamma(self):
        return sp.kron(sp.diags(self.hgam), self.Mass, format="csr")

    def kkt_matrix(self):
        A = self.sg_matrix()
        Mc, Mg = self.mass_cal(), self.mass_gamma()
        if self.nt == 0:
            return sp.bmat([[Mg, None, -A.T], [None, self.beta * Mc, Mc.T], [-A, Mc, None]], format="csr")
        nt, tau = self.nt, self.tau
        I_t = sp.identity(nt)
        C = sp.diags([np.ones(nt - 1)], [-1], shape=(nt, nt)) if nt > 1 else sp.csr_matrix((1, 1))
        D = sp.diags(self.d_weights())
        Lc = Mc + tau * A
        At = sp.kron(I_t, Lc) - sp.kron(C, Mc)
        N = sp.kron(I_t, Mc)
        return sp.bmat([[tau * sp.kron(D, Mg), None, -At.T],
                        [None, self.beta * tau * sp.kron(D, Mc), tau * N.T],
                        [-At, tau * N, None]], format="csr")

    # ---- right-hand side -----------------------------------------------------
    def rhs(self):
        """b = [M_cal yhat_d; 0; g] (steady, g = 0) or its time form; the target and
        the initial state are deterministic, so only chaos column 0 is non-zero."""
        pr = self.pr
        F = self.slabs * self.P * self.n
        b = np.zeros(3 * F)
        nP = self.P * self.n
        if self.nt == 0:
            b[:self.n] = self.Mass @ pr.yhat[0]
            return b
        D = self.d_weights()
        for t in range(self.nt):
            b[t * nP:t * nP + self.n] = self.tau * D[t] * (self.Mass @ pr.yhat[t])
        if pr.y0 is not None:
            # third block row is -A_t y + tau N u = -d with d = [M y0, 0, ..., 0]
            b[2 * F:2 * F + self.n] = -(self.Mass @ pr.y0)
        return b

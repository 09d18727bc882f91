"""End-to-end oracle solves and dense reference solutions.

solve()        preconditioned MINRES on the SG KKT system (Eq. (stoch-system) or
               Eq. (KKT:stoch-time-dependent)) with the block preconditioner.
direct_solve() the plain definition of the discrete optimum: a dense direct solve of
               the assembled KKT matrix (tiny sizes only).
reduced_solve() independent form of the steady optimum: eliminate the state with the
               constraint y = A^{-1} M u and solve (B^T M_g B + beta M) u = B^T M yhat.
"""
from __future__ import annotations

import numpy as np
import scipy.sparse.linalg as spla

from .krylov import fgmres, minres
from .operators import SGData
from .precond import BlockPreconditioner, HGSoc


def solve(pr, mode="vcycle", assembled=False, data=None, schur=None, krylov=None):
    """krylov: "minres" (default) or "fgmres" (Sec. 5), from the argument or pr.krylov."""
    d = data or SGData(pr)
    schur = schur or getattr(pr, "schur", "diagonal")
    krylov = krylov or getattr(pr, "krylov", "minres")
    b = d.rhs()
    if assembled:
        K = d.kkt_matrix()
        apply_A = lambda v: K @ v
    else:
        apply_A = d.kkt_apply
    if getattr(pr, "precond", "block") == "hgsoc":          # Alg. 2-3 / Alg. 4: not symmetric
        Pc = HGSoc(d, mode)
        krylov = "fgmres"
    else:
        Pc = BlockPreconditioner(d, mode, schur=schur)
    if krylov == "fgmres":
        res = fgmres(apply_A, Pc.apply, b, tol=pr.tol, max_iter=pr.max_iter, restart=getattr(pr, "restart", None))
    else:
        res = minres(apply_A, Pc.apply, b, tol=pr.tol, max_iter=pr.max_iter)
    res.data = d
    return res


def direct_solve(pr, data=None):
    d = data or SGData(pr)
    K = d.kkt_matrix().toarray()
    return np.linalg.solve(K, d.rhs())


def reduced_solve(pr, data=None):
    d = data or SGData(pr)
    A = d.sg_matrix().toarray()
    Mc = d.mass_cal().toarray()
    Mg = d.mass_gamma().toarray()
    B = np.linalg.solve(A, Mc)
    yd = np.zeros(d.P * d.n)
    yd[:d.n] = pr.yhat[0]
    u = np.linalg.solve(B.T @ Mg @ B + d.beta * Mc, B.T @ (Mc @ yd))
    y = B @ u
    lam = -d.beta * u
    return np.concatenate([y, u, lam])

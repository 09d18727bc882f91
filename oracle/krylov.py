"""Preconditioned MINRES for the oracle.

The paper solves with FGMRES (Sec. 5); the accelerated path uses MINRES, which
needs the symmetric positive-definite block preconditioner of Eq. (stoch-prec) /
Eq. (precon for time).  This is MINRES derived from the preconditioned Lanczos
process (three-term recurrence in the P^{-1} inner product) with the Givens QR
of the tridiagonal Lanczos matrix, x0 = 0.

Stopping rule (the paper states ||r_k|| / ||b|| <= tol without naming the norm):
the loop tests the MINRES estimate |eta_k| / ||b||_{P^{-1}} (which equals
||r_k||_{P^{-1}} / ||b||_{P^{-1}}) against a target that starts at tol.  When it
fires, the true relative residual rho = ||b - K x||_2 / ||b||_2 is computed; the
solve stops if rho <= tol, else the target is multiplied by tol / rho and the
iteration continues.
"""
from __future__ import annotations

import math

import numpy as np


class MinresResult:
    def __init__(self, x, iterations, rel_true, rel_est, status, history):
        self.x = x
        self.iterations = iterations
        self.rel_true = rel_true
        self.rel_est = rel_est
        self.status = status
        self.history = history


def minres(apply_A, apply_Pinv, b, tol=1e-8, max_iter=500):
    n = b.shape[0]
    x = np.zeros(n)
    bnorm2 = float(np.linalg.norm(b))
    if bnorm2 == 0.0:
        return MinresResult(x, 0, 0.0, 0.0, "ok", [])
    v_prev = np.zeros(n)
    v = b.copy()
    z = apply_Pinv(v)
    vz = float(v @ z)
    if not vz > 0.0:
        return MinresResult(x, 0, 1.0, 1.0, "not_spd", [])
    beta = math.sqrt(vz)
    beta1 = beta
    beta_prev = 1.0
    eta = beta
    c_m1, s_m1 = 1.0, 0.0      # rotation j-1
    c_m2, s_m2 = 1.0, 0.0      # rotation j-2
    w_m1 = np.zeros(n)
    w_m2 = np.zeros(n)
    target = tol
    history = []
    rel_true = 1.0
    for j in range(1, max_iter + 1):
        q = z / beta
        Aq = apply_A(q)
        alpha = float(q @ Aq)
        v_next = Aq - (alpha / beta) * v
        if j > 1:
            v_next -= (beta / beta_prev) * v_prev
        z_next = apply_Pinv(v_next)
        vz = float(v_next @ z_next)
        if vz < 0.0 or math.isnan(vz):
            return MinresResult(x, j, rel_true, abs(eta) / beta1, "not_spd", history)
        beta_next = math.sqrt(vz)
        # previous rotations applied to the new column (0, beta_j, alpha_j, beta_{j+1})
        eps = s_m2 * beta
        dprime = c_m2 * beta
        delta = c_m1 * dprime + s_m1 * alpha
        gbar = -s_m1 * dprime + c_m1 * alpha
        rho = math.hypot(gbar, beta_next)
        if rho == 0.0:
            return MinresResult(x, j, rel_true, abs(eta) / beta1, "breakdown", history)
        c, s = gbar / rho, beta_next / rho
        w = (q - delta * w_m1 - eps * w_m2) / rho
        x = x + (c * eta) * w
        eta = -s * eta
        est = abs(eta) / beta1
        history.append(est)
        # shift
        w_m2, w_m1 = w_m1, w
        c_m2, s_m2, c_m1, s_m1 = c_m1, s_m1, c, s
        v_prev, v = v, v_next
        z = z_next
        beta_prev, beta = beta, beta_next
        if est <= target or beta_next == 0.0:
            rel_true = float(np.linalg.norm(b - apply_A(x))) / bnorm2
            if rel_true <= tol or beta_next == 0.0:
                return MinresResult(x, j, rel_true, est, "ok", history)
            target *= tol / rel_true
    rel_true = float(np.linalg.norm(b - apply_A(x))) / bnorm2
    return MinresResult(x, max_iter, rel_true, abs(eta) / beta1, "max_iter", history)


def fgmres(apply_A, apply_Pinv, b, tol=1e-8, max_iter=500, restart=None):
    """Flexible GMRES (Saad's right-preconditioned variant, the Krylov method of Sec. 5):
    x0 = 0; Arnoldi with modified Gram-Schmidt on the vectors A z_j, z_j = P_j^{-1} v_j (the
    preconditioner may change from one iteration to the next), Givens rotations of the
    Hessenberg matrix, x = x0 + Z_m y_m.  The estimate |g_{j+1}| / ||b||_2 is the 2-norm of
    the residual in exact arithmetic; the stopping rule is that of minres(): when the
    estimate reaches the target the true residual decides, and the target is rescaled by
    tol / rho if it is still above tol.  restart=None: unrestarted (one cycle up to max_iter)."""
    n = b.shape[0]
    x = np.zeros(n)
    bnorm = float(np.linalg.norm(b))
    if bnorm == 0.0:
        return MinresResult(x, 0, 0.0, 0.0, "ok", [])
    m_cap = max_iter if restart is None else restart
    target = tol
    history = []
    total = 0
    r = b.copy()
    rel_true = 1.0
    while True:
        beta = float(np.linalg.norm(r))
        V = [r / beta]
        Z = []
        H = np.zeros((m_cap + 1, m_cap))
        cs, sn = np.zeros(m_cap), np.zeros(m_cap)
        g = np.zeros(m_cap + 1)
        g[0] = beta
        fired = False
        j = 0
        for j in range(m_cap):
            z = apply_Pinv(V[j])
            w = apply_A(z)
            Z.append(z)
            for i in range(j + 1):                  # modified Gram-Schmidt
                H[i, j] = float(w @ V[i])
                w = w - H[i, j] * V[i]
            H[j + 1, j] = float(np.linalg.norm(w))
            for i in range(j):                      # previous rotations on the new column
                hi, hi1 = H[i, j], H[i + 1, j]
                H[i, j] = cs[i] * hi + sn[i] * hi1
                H[i + 1, j] = -sn[i] * hi + cs[i] * hi1
            rho = math.hypot(H[j, j], H[j + 1, j])
            if rho == 0.0:
                return MinresResult(x, total + j + 1, rel_true, abs(g[j]) / bnorm, "breakdown", history)
            cs[j], sn[j] = H[j, j] / rho, H[j + 1, j] / rho
            H[j, j] = rho
            H[j + 1, j] = 0.0
            g[j + 1] = -sn[j] * g[j]
            g[j] = cs[j] * g[j]
            est = abs(g[j + 1]) / bnorm
            history.append(est)
            lucky = H[j + 1, j] == 0.0 and float(np.linalg.norm(w)) == 0.0
            if est <= target or lucky:
                fired = True
                break
            V.append(w / float(np.linalg.norm(w)))
        k = j + 1
        y = np.linalg.solve(np.triu(H[:k, :k]), g[:k])
        x = x + np.column_stack(Z) @ y
        total += k
        r = b - apply_A(x)
        rel_true = float(np.linalg.norm(r)) / bnorm
        if fired:
            if rel_true <= tol:
                return MinresResult(x, total, rel_true, history[-1], "ok", history)
            target *= tol / rel_true
        if total >= max_iter:
            return MinresResult(x, total, rel_true, history[-1], "max_iter", history)

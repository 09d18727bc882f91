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

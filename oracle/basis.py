"""Polynomial chaos basis for the oracle (Sec. 2 of the paper).

Orthonormal Legendre chaos in M independent xi_k ~ U[-1,1], total degree p.
* The index set Lambda = {alpha in N^M : |alpha| <= p} has C(M+p, p) members
  (Sec. 5: n_xi = C(m_xi + p, p), e.g. (3,3) -> 20).
* Ordering: graded by total degree (the level structure Alg. 1 sweeps over,
  with level ranges n_l = C(m+d-1, d-1), n_u = C(m+d, d)); within a degree,
  lexicographically descending, so degree 1 is e_1, ..., e_M.
* G_k = E[xi_k Psi_alpha Psi_beta] (the paper's H_l with the affine coefficient;
  G_0 = E[Psi_alpha Psi_beta] = I).  Only alpha = beta +- e_k couple, with
  E[xi psi_n psi_{n+1}] = (n+1)/sqrt((2n+1)(2n+3)) for psi_n = sqrt(2n+1) P_n.
"""
from __future__ import annotations

import itertools
import math

import numpy as np


def multi_indices(M: int, p: int) -> np.ndarray:
    """Brute-force enumeration of Lambda in graded, lex-descending order, shape (P, M)."""
    if M == 0:
        return np.zeros((1, 0), dtype=np.int32)
    allidx = [a for a in itertools.product(range(p + 1), repeat=M) if sum(a) <= p]
    allidx.sort(key=lambda a: (sum(a), tuple(-x for x in a)))
    return np.array(allidx, dtype=np.int32).reshape(-1, M)


def level_offsets(M: int, p: int) -> np.ndarray:
    """off[d] = number of indices with |alpha| < d, d = 0..p+1 (so level d = [off[d], off[d+1]))."""
    return np.array([0] + [math.comb(M + d, d) for d in range(p + 1)], dtype=np.int64)


def legendre_coupling(n: int) -> float:
    """E[xi psi_n(xi) psi_{n+1}(xi)] for orthonormal Legendre, xi ~ U[-1,1]."""
    return (n + 1) / math.sqrt((2 * n + 1) * (2 * n + 3))


def g_matrices(M: int, p: int) -> list:
    """Dense G_0..G_M, each P x P."""
    idx = multi_indices(M, p)
    P = idx.shape[0]
    pos = {tuple(a): i for i, a in enumerate(idx.tolist())}
    G = [np.eye(P)]
    for k in range(M):
        Gk = np.zeros((P, P))
        for a in range(P):
            up = list(idx[a])
            up[k] += 1
            b = pos.get(tuple(up))
            if b is not None:
                c = legendre_coupling(int(idx[a, k]))
                Gk[a, b] = c
                Gk[b, a] = c
        G.append(Gk)
    return G


def legendre_orthonormal(n: int, x: np.ndarray) -> np.ndarray:
    """psi_n(x) = sqrt(2n+1) P_n(x) by the three-term recurrence."""
    p0 = np.ones_like(x)
    if n == 0:
        return p0
    p1 = x.copy()
    for m in range(1, n):
        p0, p1 = p1, ((2 * m + 1) * x * p1 - m * p0) / (m + 1)
    return math.sqrt(2 * n + 1) * p1


def g_matrices_quadrature(M: int, p: int) -> list:
    """G_k by tensor Gauss-Legendre quadrature of E[xi_k Psi_a Psi_b] (pin for g_matrices)."""
    idx = multi_indices(M, p)
    P = idx.shape[0]
    x, w = np.polynomial.legendre.leggauss(p + 2)
    w = w / 2.0                               # U[-1,1] density 1/2
    # 1-D tables: E over one variable of xi^e psi_a psi_b
    tab = np.zeros((2, p + 1, p + 1))
    for e in range(2):
        for a in range(p + 1):
            for b in range(p + 1):
                tab[e, a, b] = np.sum(w * x**e * legendre_orthonormal(a, x) * legendre_orthonormal(b, x))
    G = []
    for k in range(M + 1):
        Gk = np.ones((P, P))
        for j in range(M):
            e = 1 if (k >= 1 and j == k - 1) else 0
            Gk *= tab[e][np.ix_(idx[:, j], idx[:, j])]
        G.append(Gk)
    return G


# ----------------------------------------------------------- Hermite chaos --
# The paper's own setting (Sec. 2, Sec. 5): xi_j ~ N(0, 1) independent, normalised
# probabilists' Hermite polynomials psi_n = He_n / sqrt(n!), the same graded index set for
# the solution (total degree p) and a coefficient expansion of total degree 2p with
# n_A = C(M + 2p, 2p) terms; H_l = E[psi_l Psi_alpha Psi_beta] (H_0 = I).

def hermite_triple(a: int, b: int, c: int) -> float:
    """E[psi_a psi_b psi_c] for normalised Hermite polynomials: the textbook closed form
    sqrt(a! b! c!) / ((s-a)! (s-b)! (s-c)!) with s = (a+b+c)/2 when a+b+c is even and
    s >= max(a, b, c), else 0."""
    if (a + b + c) % 2:
        return 0.0
    s = (a + b + c) // 2
    if s < max(a, b, c):
        return 0.0
    return math.sqrt(math.factorial(a) * math.factorial(b) * math.factorial(c)) / (
        math.factorial(s - a) * math.factorial(s - b) * math.factorial(s - c))


def term_indices(M: int, p: int) -> np.ndarray:
    """Multi-indices of the coefficient expansion: total degree <= 2p, the graded order of
    multi_indices (so terms 0, 1..M are the mean and the M linear terms)."""
    return multi_indices(M, 2 * p)


def h_matrices(M: int, p: int, nterms: int) -> list:
    """Dense H_l (P x P) for the first nterms coefficient terms l (graded order)."""
    idx = multi_indices(M, p)
    tl = term_indices(M, p)[:nterms]
    P = idx.shape[0]
    H = []
    for l in tl:
        Hl = np.ones((P, P))
        for j in range(M):
            e = np.array([[hermite_triple(int(a), int(b), int(l[j])) for b in idx[:, j]] for a in idx[:, j]])
            Hl *= e
        H.append(Hl)
    return H


def hermite_normalised(n: int, x: np.ndarray) -> np.ndarray:
    """psi_n(x) = He_n(x) / sqrt(n!) by the three-term recurrence He_{m+1} = x He_m - m He_{m-1}."""
    h0 = np.ones_like(x)
    if n == 0:
        return h0
    h1 = x.copy()
    for m in range(1, n):
        h0, h1 = h1, x * h1 - m * h0
    return h1 / math.sqrt(math.factorial(n))


def h_matrices_quadrature(M: int, p: int, nterms: int) -> list:
    """H_l by tensor Gauss-Hermite quadrature (probabilists' weight), exact for the degree
    3p... 4p products involved (pin for h_matrices)."""
    idx = multi_indices(M, p)
    tl = term_indices(M, p)[:nterms]
    P = idx.shape[0]
    x, w = np.polynomial.hermite_e.hermegauss(2 * p + 2)
    w = w / math.sqrt(2 * math.pi)
    deg = max(2 * p, 1)
    tab = np.zeros((deg + 1, p + 1, p + 1))
    for c in range(deg + 1):
        for a in range(p + 1):
            for b in range(p + 1):
                tab[c, a, b] = np.sum(w * hermite_normalised(c, x) * hermite_normalised(a, x) *
                                      hermite_normalised(b, x))
    H = []
    for l in tl:
        Hl = np.ones((P, P))
        for j in range(M):
            Hl *= tab[int(l[j])][np.ix_(idx[:, j], idx[:, j])]
        H.append(Hl)
    return H

"""Q1 finite elements on the unit square for the oracle (Sec. 2, Eq. (gPC-A)).

(A_k)_{ab} = int_D kappa_k(x) grad phi_a . grad phi_b dx and M_{ab} = int_D phi_a phi_b dx
for bilinear (Q1) nodal basis functions on a uniform nx x nx grid of square
elements.  kappa_k is constant on each element.  Homogeneous Dirichlet data
(g = 0) is imposed by keeping interior nodes only.  Element integrals are
computed by tensor Gauss quadrature of the shape functions (exact for these
polynomial integrands), then assembled node by node.
"""
from __future__ import annotations

import numpy as np
import scipy.sparse as sp


def _shape(xi, eta):
    """Bilinear shape functions on the reference square [0,1]^2 and their gradients.
    Local order: (0,0), (1,0), (1,1), (0,1)."""
    N = np.array([(1 - xi) * (1 - eta), xi * (1 - eta), xi * eta, (1 - xi) * eta])
    dN = np.array([[-(1 - eta), -(1 - xi)],
                   [(1 - eta), -xi],
                   [eta, xi],
                   [-eta, (1 - xi)]])
    return N, dN


def element_matrices(h: float):
    """Element stiffness (unit coefficient) and mass for a square element of side h."""
    g, w = np.polynomial.legendre.leggauss(3)
    g = 0.5 * (g + 1.0)
    w = 0.5 * w
    Ke = np.zeros((4, 4))
    Me = np.zeros((4, 4))
    for a in range(3):
        for b in range(3):
            N, dN = _shape(g[a], g[b])
            wt = w[a] * w[b]
            grad = dN / h                     # d/dx = (1/h) d/dxi
            Ke += wt * (grad @ grad.T) * h * h
            Me += wt * np.outer(N, N) * h * h
    return Ke, Me


def interior_index(nx: int):
    """Map from global node (i, j) (i along x1) to interior index, -1 on the boundary."""
    idx = -np.ones((nx + 1, nx + 1), dtype=np.int64)   # [j, i]
    m = nx - 1
    for j in range(1, nx):
        for i in range(1, nx):
            idx[j, i] = (j - 1) * m + (i - 1)
    return idx


def assemble(nx: int, kappa_elem: np.ndarray):
    """Assemble the interior-node matrix sum_e kappa(e) K^e (kappa_elem[ey, ex])."""
    h = 1.0 / nx
    Ke, _ = element_matrices(h)
    return _assemble_with(nx, Ke, kappa_elem)


def mass(nx: int):
    h = 1.0 / nx
    _, Me = element_matrices(h)
    return _assemble_with(nx, Me, np.ones((nx, nx)))


def _assemble_with(nx, Ee, coef):
    idx = interior_index(nx)
    rows, cols, vals = [], [], []
    for ey in range(nx):
        for ex in range(nx):
            nodes = [idx[ey, ex], idx[ey, ex + 1], idx[ey + 1, ex + 1], idx[ey + 1, ex]]
            c = coef[ey, ex]
            for a in range(4):
                if nodes[a] < 0:
                    continue
                for b in range(4):
                    if nodes[b] < 0:
                        continue
                    rows.append(nodes[a])
                    cols.append(nodes[b])
                    vals.append(c * Ee[a, b])
    n = (nx - 1) ** 2
    return sp.csr_matrix((vals, (rows, cols)), shape=(n, n))


def stiffness_terms(nx: int, kappa: np.ndarray) -> list:
    """K_k for k = 0..M from the element coefficients kappa[k, ey, ex]."""
    return [assemble(nx, kappa[k]) for k in range(kappa.shape[0])]


def one_d(nx: int):
    """1-D linear-element stiffness and mass on interior nodes of [0,1] (for pins)."""
    h = 1.0 / nx
    m = nx - 1
    K1 = sp.diags([-np.ones(m - 1), 2 * np.ones(m), -np.ones(m - 1)], [-1, 0, 1]) / h
    M1 = sp.diags([np.ones(m - 1), 4 * np.ones(m), np.ones(m - 1)], [-1, 0, 1]) * (h / 6)
    return K1.tocsr(), M1.tocsr()

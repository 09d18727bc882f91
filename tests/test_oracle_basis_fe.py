"""Pins of the oracle's chaos basis and Q1 finite elements against closed forms."""
import math

import numpy as np
import pytest

from oracle import basis, fe
from golden_io import constants, multi_indices

C = constants()


def test_multi_index_golden_order():
    M, p, rows = multi_indices()
    assert basis.multi_indices(M, p).tolist() == rows


@pytest.mark.parametrize("M,p", [(1, 3), (2, 2), (3, 3), (4, 3), (6, 3), (8, 3), (2, 4), (5, 1), (0, 2)])
def test_multi_index_count_and_grading(M, p):
    idx = basis.multi_indices(M, p)
    assert idx.shape[0] == math.comb(M + p, p)
    deg = idx.sum(axis=1)
    assert np.all(np.diff(deg) >= 0)
    off = basis.level_offsets(M, p)
    for d in range(p + 1):
        lev = idx[off[d]:off[d + 1]]
        assert np.all(lev.sum(axis=1) == d)
        # Alg. 1 level ranges: n_l = C(m+d-1, d-1), n_u = C(m+d, d)
        if d >= 1:
            assert off[d] == math.comb(M + d - 1, d - 1)
            assert off[d + 1] == math.comb(M + d, d)
        # lexicographically descending inside the level
        tl = [tuple(r) for r in lev.tolist()]
        assert tl == sorted(tl, reverse=True)
    if M:
        assert idx[1:M + 1].tolist() == np.eye(M, dtype=int).tolist()


def test_paper_worked_example_count():
    assert basis.multi_indices(3, 3).shape[0] == C["nxi_3_3"]


def test_legendre_coupling_constants():
    assert basis.legendre_coupling(0) == pytest.approx(C["c0"], rel=2.3e-16)
    assert basis.legendre_coupling(1) == pytest.approx(C["c1"], rel=2.3e-16)
    assert basis.legendre_coupling(2) == pytest.approx(C["c2"], rel=2.3e-16)


@pytest.mark.parametrize("M,p", [(2, 2), (3, 3), (4, 2), (2, 4)])
def test_g_matrices_structure_and_quadrature(M, p):
    G = basis.g_matrices(M, p)
    Gq = basis.g_matrices_quadrature(M, p)
    P = G[0].shape[0]
    assert np.array_equal(G[0], np.eye(P))
    off = basis.level_offsets(M, p)
    lev = np.zeros(P, dtype=int)
    for d in range(p + 1):
        lev[off[d]:off[d + 1]] = d
    for k in range(M + 1):
        assert np.array_equal(G[k], G[k].T)
        # quadrature rounding of sums of O(1) products: a few ulps
        assert np.max(np.abs(G[k] - Gq[k])) < 4e-15
    for k in range(1, M + 1):
        # couplings only between adjacent levels; the strictly lower (by level) part L_k
        # has at most one non-zero per row and per column (Sec. 4, H_l = L_l + L_l^T)
        nz = np.argwhere(G[k] != 0)
        assert np.all(np.abs(lev[nz[:, 0]] - lev[nz[:, 1]]) == 1)
        L = np.where(lev[:, None] > lev[None, :], G[k], 0.0)
        assert np.all((L != 0).sum(axis=0) <= 1) and np.all((L != 0).sum(axis=1) <= 1)
        assert np.allclose(L + L.T, G[k], atol=0)


def test_element_matrices_closed_form():
    h = 0.125
    Ke, Me = fe.element_matrices(h)
    assert np.allclose(Ke[0] * 6, C["ke_row0"], atol=1e-14)
    assert np.allclose(Me[0] * 36 / h**2, C["me_row0"], atol=1e-13)
    # the other rows are the same pattern rotated around the element
    for a in range(4):
        assert np.allclose(np.roll(Ke[0], a), Ke[a], atol=1e-14)
        assert np.allclose(np.roll(Me[0], a), Me[a], atol=1e-16)


@pytest.mark.parametrize("nx", [4, 8, 16])
def test_q1_tensor_product_identity(nx):
    K = fe.assemble(nx, np.ones((nx, nx))).toarray()
    Mm = fe.mass(nx).toarray()
    K1, M1 = fe.one_d(nx)
    K1, M1 = K1.toarray(), M1.toarray()
    assert np.max(np.abs(K - (np.kron(K1, M1) + np.kron(M1, K1)))) < 1e-13
    assert np.max(np.abs(Mm - np.kron(M1, M1))) < 1e-16
    # closed-form spectrum of K1 (x) M1 + M1 (x) K1
    h = 1.0 / nx
    th = np.arange(1, nx) * math.pi * h
    lk = (2 / h) * (1 - np.cos(th))
    lm = (h / 3) * (2 + np.cos(th))
    lam = np.sort((lk[:, None] * lm[None, :] + lm[:, None] * lk[None, :]).ravel())
    lam_num = np.sort(np.linalg.eigvals(np.linalg.solve(Mm, K)).real)
    lam_gen = np.sort(np.linalg.eigvalsh(K))
    ev_closed = np.sort((lk[:, None] * lm[None, :] + lm[:, None] * lk[None, :]).ravel())
    assert np.allclose(lam_gen, ev_closed, rtol=1e-12, atol=1e-12)


def test_mass_row_sums_and_linear_kernel():
    nx = 8
    h = 1.0 / nx
    Mm = fe.mass(nx).toarray()
    K = fe.assemble(nx, np.ones((nx, nx))).toarray()
    m = nx - 1
    x1 = np.tile(np.arange(1, nx) * h, m)
    x2 = np.repeat(np.arange(1, nx) * h, m)
    inner = [(j - 1) * m + (i - 1) for j in range(2, nx - 1) for i in range(2, nx - 1)]
    assert np.allclose(Mm.sum(axis=1)[inner], h * h, atol=1e-16)
    lin = 0.3 + 2.0 * x1 - 1.5 * x2
    assert np.max(np.abs((K @ lin)[inner])) < 1e-13


def test_mass_jacobi_spectrum_bounds():
    nx = 16
    Mm = fe.mass(nx).toarray()
    d = np.diag(Mm)
    ev = np.linalg.eigvalsh(Mm / np.sqrt(d[:, None] * d[None, :]))
    assert ev.min() >= C["cheb_lmin"] - 1e-12 and ev.max() <= C["cheb_lmax"] + 1e-12


def test_variable_coefficient_stiffness_is_sum_of_elements():
    rng = np.random.default_rng(0)
    nx = 6
    kap = rng.uniform(0.5, 2.0, size=(nx, nx))
    K = fe.assemble(nx, kap).toarray()
    assert np.allclose(K, K.T, atol=0)
    # K = sum_e kappa_e K_e with the unit-coefficient single-element matrices
    S = np.zeros_like(K)
    for ey in range(nx):
        for ex in range(nx):
            one = np.zeros((nx, nx))
            one[ey, ex] = 1.0
            S += kap[ey, ex] * fe.assemble(nx, one).toarray()
    assert np.max(np.abs(K - S)) < 1e-13
    # 9-point pattern
    m = nx - 1
    for a, b in zip(*np.nonzero(K)):
        ja, ia, jb, ib = a // m, a % m, b // m, b % m
        assert abs(ja - jb) <= 1 and abs(ia - ib) <= 1

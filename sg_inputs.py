"""Seeded synthetic inputs for the stochastic Galerkin optimal-control workloads.

This module is shared by the CUDA path's tests/benchmarks and by the CPU oracle.
It holds no arithmetic of the solution method (no finite elements, no chaos
basis, no Krylov or preconditioner step).  It only produces the *data* of a
problem instance, in the form the paper's problem statement takes as given:

* the coefficient field terms kappa_k(x) of the affine expansion
  k(x, xi) = kappa_0(x) + sum_k kappa_k(x) xi_k (Sec. 2, Eq. (KLE)), sampled per
  element (value at the element centroid), with kappa_k = sigma sqrt(lambda_k) phi_k
  from a numerically computed Karhunen-Loeve decomposition of the separable
  exponential covariance exp(-|x1-y1|/L - |x2-y2|/L) on the unit square
  (Sec. 2, Eq. (Czxy); the same covariance family as Sec. 5);
* the target state yhat at the interior nodes (steady) or at the interior nodes
  and time levels t_k = k*tau, k = 1..nt (Sec. 3);
* the scalar parameters beta, gamma, nt, T and the Krylov/preconditioner options.

KL construction (the paper gives no method): a 1-D midpoint Nystrom
discretisation of exp(-|s-t|/L) on N cells of [0,1] with weight 1/N, eigenpairs
(mu_i, v_i) normalised so that sum_j v_i(s_j)^2 / N = 1 and signed so that the
first component is positive.  Because the 2-D kernel is a product, the 2-D
pairs are (mu_i mu_j, v_i(x1) v_j(x2)).  They are ordered by decreasing
eigenvalue, ties broken by the smaller x1 index i first; the first M are kept.
"""
from __future__ import annotations

import dataclasses
import math
from typing import Optional

import numpy as np


@dataclasses.dataclass
class Problem:
    """One SG optimal-control problem instance (host arrays, float64).

    kappa has shape (M+1, nx, nx): kappa[k, ey, ex] is the value of kappa_k on the
    element in row ey (x2 direction) and column ex (x1 direction); kappa[0] is the
    mean field.  yhat has shape (max(nt,1), n) with n = (nx-1)^2 interior nodes
    numbered lexicographically with x1 fastest.
    """
    nx: int
    M: int
    p: int
    kappa: np.ndarray
    beta: float
    gamma: float = 0.0
    nt: int = 0
    T: float = 1.0
    yhat: Optional[np.ndarray] = None
    y0: Optional[np.ndarray] = None
    # solver options (paper Sec. 5 defaults: Chebyshev-5, one hGS per
    # application, truncation r = m+1, tolerance 1e-8)
    tol: float = 1e-8
    max_iter: int = 500
    r: int = -1                 # truncation index; -1 means M+1
    cheb_steps: int = 5
    nu_pre: int = 2
    nu_post: int = 2
    omega: float = 0.8
    schur: str = "diagonal"     # time mode: "diagonal" (Z~, block-diagonal in time) or "coupled" (Z_bar)
    krylov: str = "minres"      # "minres" or "fgmres" (the paper's Sec. 5 solver)
    restart: int = 64           # FGMRES cycle length (the library's default)
    mass_solve: str = "chebyshev"   # mass blocks: "chebyshev" (cheb_steps) or "exact" (Cholesky)
    precond: str = "block"          # "block" (Eq. (stoch-prec) with hGS) or "hgsoc" (Alg. 2-3 / Alg. 4)
    mean_solve: str = "vcycle"      # mean solves: "vcycle" (one multigrid cycle) or "exact" (A~_1^{-1})
    # chaos: "legendre" (xi ~ U[-1,1], affine coefficient, kappa has M+1 planes) or "hermite"
    # (xi ~ N(0,1), lognormal coefficient, kappa has n_A = C(M+2p, 2p) planes in graded order)
    chaos: str = "legendre"
    length: float = 1.0         # side of the square domain (2 for the paper's [-1,1]^2)
    name: str = ""

    @property
    def n(self) -> int:
        return (self.nx - 1) ** 2

    @property
    def P(self) -> int:
        return math.comb(self.M + self.p, self.p)

    @property
    def slabs(self) -> int:
        return max(self.nt, 1)

    @property
    def trunc(self) -> int:
        return self.M + 1 if self.r < 0 else self.r

    @property
    def kkt_size(self) -> int:
        return 3 * self.n * self.P * self.slabs


def kl_pairs_1d(N: int, L: float):
    """1-D midpoint Nystrom eigenpairs of exp(-|s-t|/L) on [0,1], descending."""
    s = (np.arange(N) + 0.5) / N
    C = np.exp(-np.abs(s[:, None] - s[None, :]) / L) / N
    mu, V = np.linalg.eigh(C)
    order = np.argsort(-mu, kind="stable")
    mu = mu[order]
    V = V[:, order] * math.sqrt(N)          # sum_j v^2 / N = 1
    sgn = np.where(V[0, :] < 0, -1.0, 1.0)
    return mu, V * sgn[None, :]


def kl_terms(nx: int, M: int, L: float, sigma: float) -> np.ndarray:
    """Element-wise KL coefficient terms, shape (M+1, nx, nx); kappa_0 = 1."""
    kappa = np.zeros((M + 1, nx, nx))
    kappa[0] = 1.0
    if M == 0:
        return kappa
    mu, V = kl_pairs_1d(nx, L)
    K1 = min(nx, M + 2)
    cand = []
    for i in range(K1):
        for j in range(K1):
            cand.append((-(mu[i] * mu[j]), i, j))
    cand.sort()
    for k in range(M):
        negl, i, j = cand[k]
        lam = -negl
        phi = V[:, j][:, None] * V[:, i][None, :]   # rows: x2 index (j), cols: x1 index (i)
        kappa[k + 1] = sigma * math.sqrt(lam) * phi
    return kappa


def interior_coords(nx: int):
    """(x1, x2) of the interior nodes, lexicographic with x1 fastest."""
    h = 1.0 / nx
    g = np.arange(1, nx) * h
    X2, X1 = np.meshgrid(g, g, indexing="ij")
    return X1.ravel(), X2.ravel()


def yhat_bubble(nx: int) -> np.ndarray:
    x1, x2 = interior_coords(nx)
    return x1 * x2 * (1 - x1) * (1 - x2)


def yhat_bumps(nx: int, seed, nbumps: int = 8, width: float = 0.05) -> np.ndarray:
    rng = np.random.default_rng(seed)
    c = rng.uniform(0.2, 0.8, size=(nbumps, 2))
    x1, x2 = interior_coords(nx)
    y = np.zeros_like(x1)
    for b in range(nbumps):
        y += np.exp(-((x1 - c[b, 0]) ** 2 + (x2 - c[b, 1]) ** 2) / (2 * width * width))
    return y


def steady_problem(nx, M, p, L, sigma, beta, yhat, gamma=0.0, name="", **opts) -> Problem:
    return Problem(nx=nx, M=M, p=p, kappa=kl_terms(nx, M, L, sigma), beta=beta,
                   gamma=gamma, nt=0, yhat=np.asarray(yhat, dtype=np.float64)[None, :],
                   name=name, **opts)


def time_problem(nx, M, p, L, sigma, beta, nt, T=1.0, gamma=0.0, name="", **opts) -> Problem:
    """Heat-equation control with yhat(x,t) = sin(pi t) x1 x2 (1-x1) (1-x2), y(0)=0."""
    tau = T / nt
    base = yhat_bubble(nx)
    yh = np.stack([math.sin(math.pi * (k + 1) * tau) * base for k in range(nt)])
    return Problem(nx=nx, M=M, p=p, kappa=kl_terms(nx, M, L, sigma), beta=beta,
                   gamma=gamma, nt=nt, T=T, yhat=yh, y0=None, name=name, **opts)


# ---------------------------------------------------------------------------
# Named workloads (sizes and distributions of the benchmark configurations)
# ---------------------------------------------------------------------------

def steady_16(**opts) -> Problem:
    """16x16 Q1 grid, M=2, p=2 (P=6), L=1.0, sigma=0.3, beta=1e-2, bubble target."""
    return steady_problem(16, 2, 2, 1.0, 0.3, 1e-2, yhat_bubble(16), name="steady_16x16_M2_p2", **opts)


def steady_128(beta: float = 1e-4, **opts) -> Problem:
    """128x128 Q1 grid, M=6, p=3 (P=84), L=0.5, sigma=0.3, 8 seeded bumps (seed 2)."""
    return steady_problem(128, 6, 3, 0.5, 0.3, beta, yhat_bumps(128, 2),
                          name=f"steady_128x128_M6_p3_beta{beta:g}", **opts)


STEADY_128_BETAS = (1e-2, 1e-4, 1e-6)


def time_64(**opts) -> Problem:
    """64x64 Q1 grid, M=4, p=3 (P=35), nt=32, T=1, beta=1e-4, L=0.5, sigma=0.3."""
    return time_problem(64, 4, 3, 0.5, 0.3, 1e-4, 32, name="time_64x64_M4_p3_nt32", **opts)


def steady_512(**opts) -> Problem:
    """512x512 Q1 grid, M=8, p=3 (P=165), L=0.25, sigma=0.4, beta=1e-5, bumps (seed 4)."""
    return steady_problem(512, 8, 3, 0.25, 0.4, 1e-5, yhat_bumps(512, 4),
                          name="steady_512x512_M8_p3", **opts)


def serving_request(i: int, master_seed: int = 5) -> Problem:
    """Request i of the serving stream: grid in {32,64,128,256}, M in 2..8, p in 1..4,
    beta log-uniform in [1e-6,1e-1], 70% steady / 30% time-dependent (nt in {8,16,32})."""
    rng = np.random.default_rng([master_seed, i])
    nx = int(rng.choice([32, 64, 128, 256]))
    M = int(rng.integers(2, 9))
    p = int(rng.integers(1, 5))
    beta = float(10.0 ** rng.uniform(-6, -1))
    timedep = bool(rng.uniform() < 0.3)
    nt = int(rng.choice([8, 16, 32])) if timedep else 0
    bump_seed = int(rng.integers(0, 2**31 - 1))
    if nt:
        pr = time_problem(nx, M, p, 0.5, 0.3, beta, nt, name=f"req{i}")
        base = yhat_bumps(nx, bump_seed)
        tau = 1.0 / nt
        pr.yhat = np.stack([math.sin(math.pi * (k + 1) * tau) * base for k in range(nt)])
        return pr
    return steady_problem(nx, M, p, 0.5, 0.3, beta, yhat_bumps(nx, bump_seed), name=f"req{i}")


def graded_indices(M: int, q: int) -> np.ndarray:
    """Multi-indices of total degree <= q, graded, lexicographically descending within a
    degree (the layout convention of the coefficient planes, shape (count, M))."""
    if M == 0:
        return np.zeros((1, 0), dtype=np.int64)
    import itertools
    allidx = [a for a in itertools.product(range(q + 1), repeat=M) if sum(a) <= q]
    allidx.sort(key=lambda a: (sum(a), tuple(-x for x in a)))
    return np.array(allidx, dtype=np.int64).reshape(-1, M)


def lognormal_terms(nx: int, M: int, p: int, L: float = 0.5, sigma: float = 1.0) -> np.ndarray:
    """Element values of the chaos terms of the lognormal coefficient k = exp(f) (Sec. 2),
    shape (n_A, nx, nx), n_A = C(M+2p, 2p): the Gaussian field f = f_0 + sum_j f_j xi_j has the
    KL modes f_j = sigma sqrt(lambda_j) phi_j of kl_terms and f_0 = -1/2 sum_j f_j^2, so that the
    mean term is kappa_0 = 1 (the paper's setting); in normalised Hermite chaos the terms are
    kappa_l = exp(f_0 + 1/2 sum_j f_j^2) prod_j f_j^{l_j} / sqrt(l_j!) = prod_j f_j^{l_j} / sqrt(l_j!)."""
    f = kl_terms(nx, M, L, sigma)[1:]
    tl = graded_indices(M, 2 * p)
    out = np.ones((tl.shape[0], nx, nx))
    for i, l in enumerate(tl):
        for j in range(M):
            if l[j]:
                out[i] *= f[j] ** int(l[j]) / math.sqrt(math.factorial(int(l[j])))
    return out


def paper_problem(nx: int, M: int, p: int, beta: float = 1e-4, gamma: float = 1.0, sigma: float = 1.0,
                  **opts) -> Problem:
    """The paper's steady setting (Sec. 5): D = [-1,1]^2 (length 2, nx elements per side, so
    h = 2/nx), lognormal coefficient with the exponential covariance of correlation length 1
    and standard deviation sigma (1 by default; the paper's tables take 0.01, 0.1 and 0.4) --
    correlation length 0.5 on the unit square the grid is indexed on --, Hermite chaos,
    gamma = 1, and the discontinuous target y_d = 1 on [-1,0]^2, 0 elsewhere."""
    x1, x2 = interior_coords(nx)
    yd = ((x1 <= 0.5 + 1e-12) & (x2 <= 0.5 + 1e-12)).astype(np.float64)
    return Problem(nx=nx, M=M, p=p, kappa=lognormal_terms(nx, M, p, sigma=sigma), beta=beta, gamma=gamma, nt=0,
                   yhat=yd[None, :], chaos="hermite", length=2.0, name=f"paper_{nx}x{nx}_M{M}_p{p}", **opts)


def random_small(seed, nx=8, M=2, p=2, nt=0, beta=1e-2, sigma=0.3, L=0.5, gamma=0.0, **opts) -> Problem:
    """Small seeded instance for parity tests (random bump target)."""
    if nt:
        pr = time_problem(nx, M, p, L, sigma, beta, nt, gamma=gamma, **opts)
        rng = np.random.default_rng(seed)
        pr.yhat = rng.standard_normal(pr.yhat.shape)
        return pr
    return steady_problem(nx, M, p, L, sigma, beta, yhat_bumps(nx, seed), gamma=gamma,
                          name=f"small_{seed}", **opts)


def random_panel(seed, n, P, slabs=1) -> np.ndarray:
    """Seeded standard-normal vector of length slabs*P*n (vec order)."""
    return np.random.default_rng(seed).standard_normal(slabs * P * n)

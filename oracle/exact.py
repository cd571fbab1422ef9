"""Exact stationary vectors by routes independent of the multigrid method.

TEST INFRASTRUCTURE ONLY.  Only tests/, __graft_entry__.smoke() and the CPU-baseline
leg of bench.py may import this package; the product path never does.

The result the method must reach (Section 1, Eq. (1.1); Section 2): the unique x > 0
with A x = x, 1^T x = 1, for an irreducible column-stochastic A (Perron-Frobenius).
"""

from __future__ import annotations

import numpy as np


def from_degree(deg: np.ndarray) -> np.ndarray:
    """Random walk with a_ij = 1/deg(j) on an undirected graph (uniform network and
    planar-graph models of Section 5.1): A D 1 = D 1 with D = diag(deg), so x = deg / sum(deg)."""
    deg = np.asarray(deg, dtype=np.float64)
    return deg / deg.sum()


def birth_death(birth: np.ndarray, death: np.ndarray) -> np.ndarray:
    """Detailed balance x_k b_k = x_{k+1} d_{k+1}; evaluated in log space because the
    entries span hundreds of orders of magnitude for long chains."""
    birth = np.asarray(birth, dtype=np.float64)
    death = np.asarray(death, dtype=np.float64)
    n = len(birth)
    logx = np.zeros(n)
    if n > 1:
        logx[1:] = np.cumsum(np.log(birth[:-1]) - np.log(death[1:]))
    logx -= logx.max()
    x = np.exp(logx)
    return x / x.sum()


def birth_death_ambiguity(birth: np.ndarray, death: np.ndarray, tol: float):
    """How far the residual test ||B x||_1 / ||x||_1 <= tol pins a birth-death chain's x.

    For x* (1^T x* = 1) and an edge m -> m+1 let M_L = sum_{k<=m} x*_k, M_R = sum_{k>m} x*_k and
    dx = x* * (M_R [k <= m] - M_L [k > m]), the move of mass across the edge.  Then
    1^T dx = 0, ||dx||_1 = 2 M_L M_R, and by detailed balance (b_m x*_m = d_{m+1} x*_{m+1})
    B dx is nonzero only at m and m+1, with ||B dx||_1 = 2 b_m x*_m.  Hence
      kappa_lb = max_m M_L M_R / (b_m x*_m) <= max ||B^# r||_1 / ||r||_1 over 1^T r = 0
      (B^# B dx = dx), and
      eps(tol) = max_m 2 M_L M_R min(1, tol / (2 b_m x*_m)):
    x* + s dx (s <= 1) is non-negative, has 1^T x = 1, meets the tolerance and lies eps
    away from x* in relative l1.  Evaluated in log space.  Returns (log10 kappa_lb, eps)."""
    birth = np.asarray(birth, dtype=np.float64)
    death = np.asarray(death, dtype=np.float64)
    n = len(birth)
    if n < 2:
        return 0.0, 0.0
    logx = np.zeros(n)
    logx[1:] = np.cumsum(np.log(birth[:-1]) - np.log(death[1:]))
    logx -= logx.max()
    logx -= np.logaddexp.reduce(logx)
    # both masses accumulated from their own end (1 - M_L cancels where M_R is tiny)
    mass = np.logaddexp.accumulate(logx)[:-1] + np.logaddexp.accumulate(logx[::-1])[::-1][1:]
    flux = np.log(birth[:-1]) + logx[:-1]  # log(b_m x*_m)
    log_kappa = float((mass - flux).max()) / np.log(10.0)
    eps = float((2.0 * np.exp(mass + np.minimum(0.0, np.log(tol) - np.log(2.0) - flux))).max())
    return log_kappa, eps


def birth_death_condition(birth: np.ndarray, death: np.ndarray) -> float:
    """An upper bound K on ||B^#||_1 for a birth-death chain (log10 K is returned), so that
    any x with 1^T x = 1 lies within K ||B x||_1 of x* in l1.

    With u = x / x* (componentwise) and the net flux J_i = sum_{k<=i} (B x)_k across the
    edge i -> i+1 (B x = J_i - J_{i-1} row by row), detailed balance gives
    u_{i+1} - u_i = -J_i w_i, w_i = 1 / (b_i x*_i), and |J_i| <= ||B x||_1 / 2.  The mean
    absolute deviation of u (weights x*) about its mean is at most twice that about the
    value at the weighted median m, so
      ||x - x*||_1 <= ||B x||_1 sum_i w_i (M_L(i) for i < m, M_R(i) for i >= m),
    M_L(i) = sum_{k<=i} x*_k, M_R(i) = sum_{k>i} x*_k: K bounds max ||B^# r||_1 / ||r||_1
    over the residuals with 1^T r = 0 (every B x has that).  Evaluated in log space, both
    masses accumulated from their own end: where log x* has a deep valley followed by a
    smaller bump (random rates make log x* a random walk), M_R past the valley is far
    below the rounding of 1 - M_L while w there is huge, and those terms dominate K."""
    birth = np.asarray(birth, dtype=np.float64)
    death = np.asarray(death, dtype=np.float64)
    n = len(birth)
    if n < 2:
        return 0.0
    logx = np.zeros(n)
    logx[1:] = np.cumsum(np.log(birth[:-1]) - np.log(death[1:]))
    logx -= logx.max()
    logx -= np.logaddexp.reduce(logx)
    logML = np.logaddexp.accumulate(logx)[:-1]  # log M_L(i), i < n - 1
    logMR = np.logaddexp.accumulate(logx[::-1])[::-1][1:]  # log M_R(i) = log sum_{k>i} x*_k
    m = int(np.searchsorted(np.exp(logML), 0.5))
    side = np.where(np.arange(n - 1) < m, logML, logMR)
    terms = side - np.log(birth[:-1]) - logx[:-1]
    top = terms.max()
    return float((top + np.log(np.exp(terms - top).sum())) / np.log(10.0))


def dense_nullspace(A_dense: np.ndarray) -> np.ndarray:
    """Bordered dense solve: replace the last equation of (I - A) x = 0 by 1^T x = 1.
    Nonsingular for irreducible A because the left null vector 1 of B has no zero entry."""
    n = A_dense.shape[0]
    M = np.eye(n) - A_dense
    M[-1, :] = 1.0
    rhs = np.zeros(n)
    rhs[-1] = 1.0
    return np.linalg.solve(M, rhs)


def sparse_nullspace(A) -> np.ndarray:
    """The same bordered system solved with SuperLU (scipy) for chains too large for dense LU."""
    import scipy.sparse as sp
    import scipy.sparse.linalg as spla

    A = sp.csr_matrix(A)
    n = A.shape[0]
    M = (sp.identity(n, format="csr") - A).tolil()
    M[n - 1, :] = np.ones(n)
    rhs = np.zeros(n)
    rhs[-1] = 1.0
    x = spla.spsolve(M.tocsc(), rhs)
    return x / x.sum()


def exact_stationary(chain) -> np.ndarray:
    """Closed form where the model has one, else a direct solve."""
    if "degree" in chain.meta:
        return from_degree(chain.meta["degree"])
    if chain.kind == "birth_death":
        return birth_death(chain.meta["birth"], chain.meta["death"])
    if chain.n <= 500:
        return dense_nullspace(chain.dense())
    return sparse_nullspace(chain.to_scipy())

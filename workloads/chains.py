"""Test-problem generators of Section 5.1 (uniform network, tandem queue, random
planar graph) plus the birth-death chains and batched mixtures used as workloads.

Convention (the reading of Section 2 used throughout the repository): A is column
stochastic, a_ij is the probability of the transition j -> i, so column j sums to
one and CSR row i lists the source states j.  Column indices inside a row are sorted
ascending and duplicate (i, j) pairs are summed.  Self-loops (a_ii > 0) are kept.

All randomness here is drawn from numpy's PCG64 Generator seeded by the caller:
these are inputs, not random numbers drawn by the solver.
"""

from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np


@dataclass
class Chain:
    """A column-stochastic transition matrix in CSR form plus generator metadata."""

    n: int
    row_ptr: np.ndarray  # int32 [n+1]
    col: np.ndarray  # int32 [nnz]
    val: np.ndarray  # float64 [nnz]
    kind: str
    grid: tuple | None = None  # (nx, ny) for problems on a structured grid
    meta: dict = field(default_factory=dict)

    @property
    def nnz(self) -> int:
        return int(self.row_ptr[-1])

    def to_scipy(self):
        import scipy.sparse as sp

        return sp.csr_matrix((self.val, self.col, self.row_ptr), shape=(self.n, self.n))

    def dense(self) -> np.ndarray:
        A = np.zeros((self.n, self.n))
        for i in range(self.n):
            for p in range(self.row_ptr[i], self.row_ptr[i + 1]):
                A[i, self.col[p]] += self.val[p]
        return A


def _csr_from_coo(n: int, to: np.ndarray, frm: np.ndarray, p: np.ndarray):
    """Sum duplicate (to, from) pairs and return sorted CSR arrays."""
    key = to.astype(np.int64) * n + frm.astype(np.int64)
    order = np.argsort(key, kind="stable")
    key = key[order]
    p = p[order]
    uniq, start = np.unique(key, return_index=True)
    sums = np.add.reduceat(p, start) if len(p) else p
    rows = (uniq // n).astype(np.int64)
    cols = (uniq % n).astype(np.int32)
    row_ptr = np.zeros(n + 1, dtype=np.int64)
    np.add.at(row_ptr, rows + 1, 1)
    row_ptr = np.cumsum(row_ptr).astype(np.int32)
    return row_ptr, cols, sums.astype(np.float64)


def _undirected_walk(n: int, ei: np.ndarray, ej: np.ndarray):
    """Random walk with step probability 1/deg(j) on an undirected simple graph."""
    a = np.concatenate([ei, ej]).astype(np.int64)
    b = np.concatenate([ej, ei]).astype(np.int64)
    deg = np.bincount(a, minlength=n).astype(np.float64)
    # edge (to=a, from=b): a_ab = 1/deg(b)
    row_ptr, col, val = _csr_from_coo(n, a, b, 1.0 / deg[b])
    return row_ptr, col, val, deg


def grid_walk(nx: int, ny: int | None = None) -> Chain:
    """Uniform two-dimensional network (Section 5.1): 4-neighbour grid, a_ij = 1/d_out(j).

    Node (ix, iy) has index ix + iy*nx.  Stationary vector: x_i proportional to deg(i).
    """
    ny = nx if ny is None else ny
    idx = np.arange(nx * ny).reshape(ny, nx)
    ei = np.concatenate([idx[:, :-1].ravel(), idx[:-1, :].ravel()])
    ej = np.concatenate([idx[:, 1:].ravel(), idx[1:, :].ravel()])
    row_ptr, col, val, deg = _undirected_walk(nx * ny, ei, ej)
    return Chain(nx * ny, row_ptr, col, val, "grid_walk", grid=(nx, ny), meta={"degree": deg})


def tandem_queue(N: int, mu: float = 11 / 31, mu_x: float = 10 / 31, mu_y: float = 10 / 31) -> Chain:
    """Tandem queueing network (Section 5.1) with two queues of capacity N in series.

    States (i, j), 0 <= i, j <= N, index i + j*(N+1).  One step from (i, j):
      with probability mu   an arrival joins queue 1:   (i+1, j), blocked (self-loop) if i = N;
      with probability mu_x a job moves from 1 to 2:    (i-1, j+1), needs i > 0 and j < N;
      with probability mu_y a job leaves queue 2:       (i, j-1), needs j > 0.
    mu + mu_x + mu_y must be 1.
    """
    if abs(mu + mu_x + mu_y - 1.0) > 1e-12:
        raise ValueError("tandem rates must sum to one")
    m = N + 1
    jj, ii = np.divmod(np.arange(m * m), m)
    src = ii + jj * m
    to_arr = np.where(ii < N, (ii + 1) + jj * m, src)
    to_tr = np.where((ii > 0) & (jj < N), (ii - 1) + (jj + 1) * m, src)
    to_de = np.where(jj > 0, ii + (jj - 1) * m, src)
    to = np.concatenate([to_arr, to_tr, to_de])
    frm = np.concatenate([src, src, src])
    p = np.concatenate([np.full(m * m, mu), np.full(m * m, mu_x), np.full(m * m, mu_y)])
    row_ptr, col, val = _csr_from_coo(m * m, to, frm, p)
    return Chain(m * m, row_ptr, col, val, "tandem", grid=(m, m), meta={"N": N, "mu": mu, "mu_x": mu_x, "mu_y": mu_y})


def birth_death(birth: np.ndarray, death: np.ndarray) -> Chain:
    """Birth-death chain on n states: k -> k+1 w.p. birth[k] (k < n-1), k -> k-1 w.p. death[k] (k > 0),
    the remaining mass stays at k.  Stationary vector: x_{k+1} = x_k birth[k] / death[k+1]."""
    birth = np.asarray(birth, dtype=np.float64)
    death = np.asarray(death, dtype=np.float64)
    n = len(birth)
    k = np.arange(n)
    b = np.where(k < n - 1, birth, 0.0)
    d = np.where(k > 0, death, 0.0)
    stay = 1.0 - b - d
    if np.any(stay < -1e-15):
        raise ValueError("birth + death probabilities exceed one")
    to = np.concatenate([k[k < n - 1] + 1, k[k > 0] - 1, k])
    frm = np.concatenate([k[k < n - 1], k[k > 0], k])
    p = np.concatenate([b[k < n - 1], d[k > 0], np.maximum(stay, 0.0)])
    keep = p > 0
    row_ptr, col, val = _csr_from_coo(n, to[keep], frm[keep], p[keep])
    return Chain(n, row_ptr, col, val, "birth_death", grid=(n, 1), meta={"birth": birth, "death": death})


def random_birth_death(n: int, seed: int, lo: float = 0.2, hi: float = 0.5) -> Chain:
    rng = np.random.default_rng(seed)
    return birth_death(rng.uniform(lo, hi, n), rng.uniform(lo, hi, n))


def _morton_order(pts: np.ndarray) -> np.ndarray:
    q = np.minimum((pts * (1 << 21)).astype(np.uint64), np.uint64((1 << 21) - 1))

    def spread(v):
        v = v & np.uint64(0x1FFFFF)
        v = (v | (v << np.uint64(32))) & np.uint64(0x1F00000000FFFF)
        v = (v | (v << np.uint64(16))) & np.uint64(0x1F0000FF0000FF)
        v = (v | (v << np.uint64(8))) & np.uint64(0x100F00F00F00F00F)
        v = (v | (v << np.uint64(4))) & np.uint64(0x10C30C30C30C30C3)
        v = (v | (v << np.uint64(2))) & np.uint64(0x1249249249249249)
        return v

    code = spread(q[:, 0]) | (spread(q[:, 1]) << np.uint64(1))
    return np.argsort(code, kind="stable")


def delaunay_walk(npts: int, seed: int) -> Chain:
    """Unstructured planar graph (Section 5.1): Delaunay triangulation of npts points drawn
    U[0,1]^2, random walk with probability 1/deg.  Points are put in Morton order (a fixed
    locality order).  Stationary vector: x_i proportional to deg(i)."""
    from scipy.spatial import Delaunay

    rng = np.random.default_rng(seed)
    pts = rng.uniform(0.0, 1.0, size=(npts, 2))
    pts = pts[_morton_order(pts)]
    tri = Delaunay(pts).simplices.astype(np.int64)
    e = np.concatenate([tri[:, [0, 1]], tri[:, [1, 2]], tri[:, [2, 0]]])
    e.sort(axis=1)
    e = np.unique(e[:, 0] * npts + e[:, 1])
    ei, ej = e // npts, e % npts
    row_ptr, col, val, deg = _undirected_walk(npts, ei, ej)
    return Chain(npts, row_ptr, col, val, "delaunay", grid=None, meta={"degree": deg, "points": pts})


def batched_mixture(seed: int, nchains: int = 512, bd_lo: int = 1024, bd_hi: int = 65536,
                    side_lo: int = 32, side_hi: int = 256) -> list:
    """Half birth-death chains (n log-uniform in [bd_lo, bd_hi], rates U(0.2, 0.5) per state),
    half 2-D grid walks (side uniform integer in [side_lo, side_hi]), interleaved."""
    rng = np.random.default_rng(seed)
    out = []
    for c in range(nchains):
        if c % 2 == 0:
            n = int(np.exp(rng.uniform(np.log(bd_lo), np.log(bd_hi))))
            out.append(random_birth_death(n, int(rng.integers(1 << 31))))
        else:
            s = int(rng.integers(side_lo, side_hi + 1))
            out.append(grid_walk(s, s))
    return out


def tandem_training_set(seed: int, count: int, n_lo: int = 63, n_hi: int = 255,
                        rate_lo: float = 0.2, rate_hi: float = 0.45) -> list:
    """Tandem queues with capacities uniform in [n_lo, n_hi] and rates (mu, mu_x, mu_y) drawn
    U(rate_lo, rate_hi) each, then normalised to sum one."""
    rng = np.random.default_rng(seed)
    out = []
    for _ in range(count):
        N = int(rng.integers(n_lo, n_hi + 1))
        r = rng.uniform(rate_lo, rate_hi, 3)
        r = r / r.sum()
        out.append(tandem_queue(N, float(r[0]), float(r[1]), 1.0 - float(r[0]) - float(r[1])))
    return out

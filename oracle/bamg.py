"""Plain FP64 CPU oracle of Bootstrap AMG for Markov chains (Bolten, Brandt, Brannick,
Frommer, Kahl, Livshits).

TEST INFRASTRUCTURE ONLY.  Only tests/, __graft_entry__.smoke() and the CPU-baseline
leg of bench.py may import this module; the product path (the CUDA library and its
Python binding) never does, and this module imports nothing from it.

Every function states the passage of the paper it restates.  Steps run in the order
the paper gives them, on whole vectors, with library primitives (sparse and dense
matrix products, dense solves, eig, SVD) as the only building blocks.  Where the paper
is silent or ambiguous the reading taken is named in the docstring with a tag R<k>;
the repository's design notes list the same readings.

Conventions.  A is column stochastic, a_ij = P(j -> i) (reading R2 of Section 2's
"from i to j").  B = I - A keeps self-loops on its diagonal (R1).  P is n_l x n_{l+1},
Q is n_{l+1} x n_l (R3).  Test-vector blocks are n x K arrays, one column per vector.
"""

from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np
import scipy.sparse as sp

# ---------------------------------------------------------------------------------
# Counter-based random numbers: SplitMix64 (Steele, Lea, Flood, "Fast splittable
# pseudorandom number generators", OOPSLA 2014).  The state after t steps from seed s
# is s + t * GAMMA (mod 2^64); the output is the published 64-bit finaliser of it.
# ---------------------------------------------------------------------------------
GAMMA = np.uint64(0x9E3779B97F4A7C15)
_M1 = np.uint64(0xBF58476D1CE4E5B9)
_M2 = np.uint64(0x94D049BB133111EB)

STREAM_TV = 0  # stream k: test vector k
STREAM_CR = 1 << 22  # + (level << 8) + round: CR start vectors
STREAM_MIS = 1 << 23  # + (level << 8) + call: independent-set priorities
STREAM_COLOUR = 1 << 21  # + (level << 8) + colour: priorities of the smoother's colouring


def splitmix64_output(state: np.ndarray) -> np.ndarray:
    z = np.asarray(state, dtype=np.uint64)
    with np.errstate(over="ignore"):
        z = (z ^ (z >> np.uint64(30))) * _M1
        z = (z ^ (z >> np.uint64(27))) * _M2
    return z ^ (z >> np.uint64(31))


def counter_u64(seed: int, stream: int, idx: np.ndarray) -> np.ndarray:
    """The (stream * 2^40 + idx + 1)-th SplitMix64 output for the given seed."""
    ctr = np.uint64(stream) * np.uint64(1 << 40) + np.asarray(idx, dtype=np.uint64) + np.uint64(1)
    with np.errstate(over="ignore"):
        state = np.uint64(seed) + ctr * GAMMA
    return splitmix64_output(state)


def counter_uniform(seed: int, stream: int, idx: np.ndarray) -> np.ndarray:
    """Uniform double in [0, 1) from the top 53 bits."""
    return (counter_u64(seed, stream, idx) >> np.uint64(11)).astype(np.float64) * (2.0 ** -53)


def tv_init(n: int, K: int, seed: int, lo: float, hi: float) -> np.ndarray:
    """Initial random positive test vectors (Section 5.1: entries uniform in [lo, hi])."""
    X = np.empty((n, K))
    idx = np.arange(n, dtype=np.uint64)
    for k in range(K):
        u = counter_uniform(seed, STREAM_TV + k, idx)
        X[:, k] = lo + (hi - lo) * u
    return X


# ---------------------------------------------------------------------------------
# Options (defaults: the paper's settings of Section 5; unstated values are readings)
# ---------------------------------------------------------------------------------
@dataclass
class Opts:
    omega: float = 0.7  # Section 3: omega-Jacobi, omega = 0.7 on all levels
    nu_tv: int = 4  # R11: setup sweeps on the random test vectors (unstated)
    nu_ev: int = 2  # R11: sweeps on the interpolated eigenvectors (unstated)
    nu_pre: int = 2  # V(2,2) cycle, Section 4.2 / Section 5.1
    nu_post: int = 2
    caliber: int = 2  # c (called eta in the tables' captions)
    z: int = 2  # path length of Eq. (3.5), z <= 3
    mmax: int = 16  # R24: at most mmax candidates per fine point, closest first
    k_ev: int = 6  # coarsest-grid eigenvectors (Section 5.1: "6 ... eigenvectors")
    coarse_max: int = 64  # stop coarsening at n <= coarse_max
    gmres_m: int = 50  # restart length (the paper uses full GMRES)
    max_it: int = 500
    coarsen: str = "grid"  # "grid" (full coarsening) or "cr" (Algorithm 1)
    seed: int = 0
    tv_lo: float = 1.0  # Section 5.1: U[1, 2]
    tv_hi: float = 2.0
    ev_change_tol: float = 1e-3  # R9: "relative change significant"
    ridge: float = 1e-4  # R25: Tikhonov term of the local LS problems
    weight_floor: float = 1e-28  # R7
    cr_theta: float = 0.85  # Section 3.1
    cr_nu: int = 8
    cr_omega: float = 0.7
    cr_max_rounds: int = 20
    # learned interpolation (oracle/learned.py); the paper uses least squares only
    interp: str = "ls"  # "ls" (Algorithm 2) or "learned"
    model: dict | None = None  # MLP parameters for interp == "learned"
    learned_refit: bool = True  # learned rows: Eq. (3.6) weights over the MLP's choice
    record: list | None = None  # if a list: (features, LS targets, fine mask) of every fit
    # setup cycling and restarts (Section 4.1, Section 5.1)
    mu: int = 1  # Algorithm 3's loop count: 1 = V-cycle setup, 2 = W-cycle setup
    setup_cycles: int = 1  # MLE cycles before the final rebuild (R33; the tables' V^2 = 2)
    mle_restart: bool = True  # R32: an MLE restart after every pGMRES cycle that fails
    smoother: str = "jacobi"  # V-cycle smoother: "jacobi" (omega-Jacobi) or "mcgs" (R34)


# ---------------------------------------------------------------------------------
# Relaxation (Section 3, Eq. (3.1) with M = diag(B)/omega)
# ---------------------------------------------------------------------------------
def diag_of(M) -> np.ndarray:
    return np.asarray(M.diagonal(), dtype=np.float64)


def jacobi(B, X: np.ndarray, omega: float, nu: int) -> np.ndarray:
    """nu sweeps of omega-Jacobi on B X = 0: X <- X - omega D^{-1} B X, D = diag(B)."""
    dinv = 1.0 / diag_of(B)
    X = np.array(X, dtype=np.float64, copy=True)
    for _ in range(nu):
        X = X - omega * (dinv[:, None] * (B @ X))
    return X


def jacobi_shifted(B, T, X: np.ndarray, lam: np.ndarray, omega: float, nu: int) -> np.ndarray:
    """nu omega-Jacobi sweeps on (B - lam_i T) x^(i) = 0 for every column i (Algorithm 3,
    the relaxation of the interpolated eigenvector approximations).  The Jacobi diagonal
    of column i is diag(B) - lam_i diag(T)."""
    lam = np.asarray(lam, dtype=np.float64)
    dB, dT = diag_of(B), diag_of(T)
    Dl = dB[:, None] - lam[None, :] * dT[:, None]
    X = np.array(X, dtype=np.float64, copy=True)
    for _ in range(nu):
        R = (B @ X) - lam[None, :] * (T @ X)
        X = X - omega * R / Dl
    return X


def normalize_weights(B, X: np.ndarray, active: np.ndarray, floor: float):
    """LS weights of Section 3.2: omega_k = 1 / ||B x_k||^2 for the normalised x_k.

    R7: each column is scaled to unit 2-norm first; the squared residual is floored at
    `floor`; the weights of the active columns are then divided by their maximum (the
    minimiser of Eq. (3.6) is invariant under a common factor).  Inactive columns get
    weight 0 and are left unscaled."""
    X = np.array(X, dtype=np.float64, copy=True)
    K = X.shape[1]
    w = np.zeros(K)
    for k in range(K):
        if not active[k]:
            continue
        nk = np.sqrt(np.dot(X[:, k], X[:, k]))
        if nk == 0.0:
            continue
        X[:, k] /= nk
        rk = B @ X[:, k]
        w[k] = 1.0 / max(np.dot(rk, rk), floor)
    if w.max() > 0:
        w = w / w.max()
    return X, w


# ---------------------------------------------------------------------------------
# Coarse variables
# ---------------------------------------------------------------------------------
def coarsen_grid(nx: int, ny: int):
    """Full coarsening (Section 5.1): C = every other grid point in both directions,
    starting at index 0.  Returns cf (True on C), cidx (coarse index, -1 on F) and the
    coarse grid dimensions."""
    ix, iy = np.meshgrid(np.arange(nx), np.arange(ny))
    ix, iy = ix.ravel(), iy.ravel()
    cf = (ix % 2 == 0) & (iy % 2 == 0)
    ncx, ncy = (nx + 1) // 2, (ny + 1) // 2
    cidx = np.where(cf, (ix // 2) + (iy // 2) * ncx, -1).astype(np.int64)
    return cf, cidx, (ncx, ncy)


def _sym_adjacency(B):
    """Undirected off-diagonal pattern of B as a boolean CSR matrix."""
    S = sp.csr_matrix(B, copy=True)
    S.data[:] = 1.0
    S = S + S.T
    S = S.tolil()
    S.setdiag(0)
    S = sp.csr_matrix(S)
    S.eliminate_zeros()
    return S


def independent_set(S, cand: np.ndarray, seed: int, stream: int) -> np.ndarray:
    """R18: maximal independent set of the candidates in the undirected graph S (Luby's
    rule with fixed priorities): an undecided candidate joins the set when its key
    (priority, index) beats every undecided neighbour's; its undecided neighbours then
    leave.  Repeats until no candidate is undecided."""
    n = S.shape[0]
    pri = counter_u64(seed, stream, np.arange(n, dtype=np.uint64))
    # total order on (priority, index) through ranks
    order = np.lexsort((np.arange(n), pri))
    rank = np.empty(n, dtype=np.int64)
    rank[order] = np.arange(n)
    undecided = np.array(cand, dtype=bool, copy=True)
    chosen = np.zeros(n, dtype=bool)
    rows = np.repeat(np.arange(n), np.diff(S.indptr))
    cols = S.indices
    while undecided.any():
        # for each node: max rank among undecided neighbours
        live = undecided[cols]
        nb_max = np.full(n, -1, dtype=np.int64)
        np.maximum.at(nb_max, rows[live], rank[cols[live]])
        win = undecided & (rank > nb_max)
        chosen |= win
        undecided &= ~win
        # neighbours of winners leave
        hit = np.zeros(n, dtype=bool)
        hit[cols[win[rows]]] = True
        undecided &= ~hit
    return chosen


def f_relax(B, cf: np.ndarray, u: np.ndarray, omega: float, nu: int):
    """F-relaxation of Eq. (3.2): u_f <- (I - M_ff^{-1} B_ff) u_f, M = diag(B)/omega.
    Returns the iterates u^{nu-1} and u^{nu} on the F points."""
    f = ~cf
    Bff = sp.csr_matrix(B)[f][:, f]
    dinv = 1.0 / diag_of(Bff)
    prev = u.copy()
    for _ in range(nu):
        prev = u
        u = u - omega * dinv * (Bff @ u)
    return prev, u


def coarsen_cr(B, level: int, opts: Opts):
    """Compatible-relaxation coarsening, Algorithm 1.  C0 is an independent set of the
    full graph of B (Section 3.1); each round runs nu F-relaxation sweeps from a random
    start in [1, 2], estimates rho_f by Eq. (3.3), and while rho_f > theta adds an
    independent set of the slow points {i in F : |u_i^nu| / |u_i^{nu-1}| > theta}."""
    n = B.shape[0]
    S = _sym_adjacency(B)
    cf = independent_set(S, np.ones(n, dtype=bool), opts.seed, STREAM_MIS + (level << 8))
    rounds = 0
    while True:
        f_idx = np.flatnonzero(~cf)
        if len(f_idx) == 0:
            break
        u0 = 1.0 + counter_uniform(opts.seed, STREAM_CR + (level << 8) + rounds, f_idx.astype(np.uint64))
        prev, u = f_relax(B, cf, u0, opts.cr_omega, opts.cr_nu)
        rho = (np.linalg.norm(u) / np.linalg.norm(u0)) ** (1.0 / opts.cr_nu)
        if rho <= opts.cr_theta or rounds >= opts.cr_max_rounds:
            break
        with np.errstate(divide="ignore", invalid="ignore"):
            ratio = np.abs(u) / np.abs(prev)
        slow = np.zeros(n, dtype=bool)
        slow[f_idx[ratio > opts.cr_theta]] = True
        rounds += 1
        cf = cf | independent_set(S, slow, opts.seed, STREAM_MIS + (level << 8) + rounds)
    cidx = np.where(cf, np.cumsum(cf) - 1, -1).astype(np.int64)
    return cf, cidx, rounds


def multicolour(B, level: int, seed: int) -> list:
    """R34, the colour classes of the multicolour Gauss-Seidel smoother (Section 3 names
    Gauss-Seidel beside Jacobi): colour c is a maximal independent set (R18's rule, own
    priority stream per level and colour) of the states the earlier colours left, in
    the symmetrised graph of B, so no two states of a colour share an entry of B.
    Returns the states of each colour, ascending."""
    S = _sym_adjacency(B)
    left = np.ones(B.shape[0], dtype=bool)
    colours = []
    while left.any():
        ind = independent_set(S, left, seed, STREAM_COLOUR + (level << 8) + len(colours))
        colours.append(np.flatnonzero(ind))
        left &= ~ind
    return colours


def gs_sweep(B, dinv: np.ndarray, b: np.ndarray, x: np.ndarray, colours: list, reverse: bool) -> np.ndarray:
    """One multicolour Gauss-Seidel sweep on B x = b: colour by colour (ascending, or
    descending with reverse), x_i <- x_i + (b_i - (B x)_i) / b_ii for the states i of the
    colour, with the x of the earlier colours already updated (R34)."""
    x = np.array(x, dtype=np.float64, copy=True)
    for rows in (colours[::-1] if reverse else colours):
        x[rows] = x[rows] + dinv[rows] * (b[rows] - B[rows] @ x)
    return x


# ---------------------------------------------------------------------------------
# Least-squares interpolation (Section 3.2: Eq. (3.5), Eq. (3.6), Algorithm 2)
# ---------------------------------------------------------------------------------
def neighborhoods(B, cf: np.ndarray, cidx: np.ndarray, z: int, mmax: int):
    """Eq. (3.5): N_i = { j in C : a path of length <= z in G(B) leads from i to j },
    where G has an edge (i, j) for every off-diagonal entry b_ij (row i, column j).

    R24: the candidates of a point are ordered by (path length, coarse index) and at most
    mmax are kept.  R30: a fine point that reaches no coarse point within z takes those
    within the smallest length <= 3 (the bound of Eq. (3.5)) that reaches one, so that
    its column of Q is not empty and 1^T Q = 1^T holds.  Returns cand (n x mmax, fine
    indices, -1 padded) and the count."""
    cand, ncand = _neighborhoods_depth(B, cf, cidx, z, mmax)
    for d in range(z + 1, 4):
        miss = (~cf) & (ncand == 0)
        if not miss.any():
            break
        cd, nd = _neighborhoods_depth(B, cf, cidx, d, mmax)
        cand[miss] = cd[miss]
        ncand[miss] = nd[miss]
    return cand, ncand


def _neighborhoods_depth(B, cf: np.ndarray, cidx: np.ndarray, z: int, mmax: int):
    """Coarse points within path length z, ordered by (length, coarse index), at most mmax."""
    n = B.shape[0]
    G = sp.csr_matrix(B, copy=True)
    G.data[:] = 1.0
    G = G.tolil()
    G.setdiag(0)
    G = sp.csr_matrix(G)
    G.eliminate_zeros()
    reach = sp.identity(n, format="csr")
    seen = sp.identity(n, format="csr")
    layers = []
    for d in range(1, z + 1):
        reach = reach @ G
        reach.data[:] = 1.0
        new = reach - reach.multiply(seen)
        new.eliminate_zeros()
        layers.append(new)
        seen = seen + new
        seen.data[:] = 1.0
    cand = np.full((n, mmax), -1, dtype=np.int64)
    ncand = np.zeros(n, dtype=np.int64)
    layer_rows = [(L.indptr, L.indices) for L in layers]
    for i in range(n):
        if cf[i]:
            continue
        picked = []
        for (ptr, ind) in layer_rows:
            js = ind[ptr[i]:ptr[i + 1]]
            js = js[cf[js]]
            js = js[np.argsort(cidx[js], kind="stable")]
            picked.extend(int(j) for j in js)
        picked = picked[:mmax]
        cand[i, :len(picked)] = picked
        ncand[i] = len(picked)
    return cand, ncand


def ls_fit_rows(xi: np.ndarray, Xc: np.ndarray, valid: np.ndarray, w: np.ndarray, c: int, ridge: float):
    """Algorithm 2 for a batch of fine points, all at once.

    xi:    (m, K)      test-vector values at the fine points
    Xc:    (m, S, K)   values at their S candidate points (slot order = canonical order)
    valid: (m, S)      candidate slot is present
    Returns the chosen slots (m, c) (-1 if fewer), the weights (m, c) and the final
    functional value.

    Each greedy step evaluates, for every remaining candidate g, the minimiser of
    Eq. (3.6) over J u {g}: the weighted normal equations (G + delta I) p = b with
    G_ab = sum_k w_k x_a^k x_b^k, b_a = sum_k w_k x_a^k x_i^k and (R25) delta =
    ridge * trace(G) / |J u {g}|; the functional L = sum_k w_k (x_i^k - sum_j p_j x_j^k)^2
    is evaluated directly.  The arg-min (first slot on exact ties) joins J.  The loop
    stops at |J| = c or when no candidate remains."""
    m, S, K = Xc.shape
    chosen = np.full((m, c), -1, dtype=np.int64)
    weights = np.zeros((m, c))
    best_L = np.full(m, np.nan)
    used = np.zeros((m, S), dtype=bool)
    rows = np.arange(m)
    for t in range(c):
        avail = valid & ~used
        if not avail.any():
            break
        L_all = np.full((m, S), np.inf)
        P_all = np.zeros((m, S, t + 1))
        for g in range(S):
            act = avail[:, g]
            if not act.any():
                continue
            sel = np.concatenate([chosen[act, :t], np.full((act.sum(), 1), g)], axis=1)  # (ma, t+1)
            Xs = Xc[rows[act][:, None], sel]  # (ma, t+1, K)
            xa = xi[act]  # (ma, K)
            G = np.einsum("msk,mtk,k->mst", Xs, Xs, w)
            b = np.einsum("msk,mk,k->ms", Xs, xa, w)
            delta = ridge * np.trace(G, axis1=1, axis2=2) / (t + 1)
            Greg = G + delta[:, None, None] * np.eye(t + 1)[None]
            p = np.linalg.solve(Greg, b[..., None])[..., 0]
            res = xa - np.einsum("ms,msk->mk", p, Xs)
            L_all[act, g] = np.einsum("mk,mk,k->m", res, res, w)
            P_all[act, g] = p
        has = np.isfinite(L_all).any(axis=1)
        g_star = np.argmin(L_all, axis=1)
        for r in np.flatnonzero(has):
            chosen[r, t] = g_star[r]
            used[r, g_star[r]] = True
            weights[r, :t + 1] = P_all[r, g_star[r]]
            best_L[r] = L_all[r, g_star[r]]
    return chosen, weights, best_L


def ls_interpolation(X: np.ndarray, w: np.ndarray, cf: np.ndarray, cidx: np.ndarray,
                     cand: np.ndarray, ncand: np.ndarray, c: int, ridge: float, chunk: int = 65536):
    """Interpolation P (n_l x n_{l+1}, CSR) by Algorithm 2.

    Fine rows hold the LS weights at the coarse indices of the chosen points, sorted by
    coarse index; coarse rows are unit rows (R5: P = [P_FC; I] up to permutation)."""
    n = X.shape[0]
    nc = int(cf.sum())
    fine = np.flatnonzero(~cf)
    rows_c, cols_c, vals_c = [], [], []
    S = cand.shape[1]
    for s in range(0, len(fine), chunk):
        f = fine[s:s + chunk]
        valid = (np.arange(S)[None, :] < ncand[f][:, None])
        cidx_safe = np.where(valid, cand[f], 0)
        Xc = X[cidx_safe]  # (m, S, K)
        chosen, pw, _ = ls_fit_rows(X[f], Xc, valid, w, c, ridge)
        for t in range(c):
            ok = chosen[:, t] >= 0
            js = cand[f[ok], chosen[ok, t]]
            rows_c.append(f[ok])
            cols_c.append(cidx[js])
            vals_c.append(pw[ok, t])
    cpts = np.flatnonzero(cf)
    rows_c.append(cpts)
    cols_c.append(cidx[cpts])
    vals_c.append(np.ones(len(cpts)))
    r = np.concatenate(rows_c)
    cc = np.concatenate(cols_c)
    v = np.concatenate(vals_c)
    P = sp.csr_matrix((v, (r, cc)), shape=(n, nc))
    P.sort_indices()
    return P


def averaging_restriction(P) -> sp.csr_matrix:
    """Q (n_{l+1} x n_l) of Section 4: sparsity(Q) = sparsity(P^T) and each column has
    identical entries summing to one (R4: Q[I, i] = 1/|J_i| for I in J_i), so 1^T Q = 1^T."""
    P = sp.csr_matrix(P)
    cnt = np.diff(P.indptr)
    Qt = sp.csr_matrix((np.repeat(1.0 / np.maximum(cnt, 1), cnt), P.indices, P.indptr), shape=P.shape)
    return sp.csr_matrix(Qt.T)


def galerkin(Q, M, P) -> sp.csr_matrix:
    """Petrov-Galerkin product Q M P (Section 1, step 3; Algorithm 3), written out as the
    sum over every triple Q[I,i] M[i,j] P[j,J] of the structural non-zeros, so the result
    keeps every structurally present entry even where values cancel."""
    Q = sp.csr_matrix(Q)
    M = sp.csr_matrix(M)
    P = sp.csr_matrix(P)
    Qt = sp.csr_matrix(Q.T)  # row i of Qt lists (I, Q[I, i])
    nI, nJ = Q.shape[0], P.shape[1]
    Mi = np.repeat(np.arange(M.shape[0]), np.diff(M.indptr))
    Mj, Mv = M.indices, M.data
    # expand over Q column i
    qn = np.diff(Qt.indptr)[Mi]
    e1 = np.repeat(np.arange(len(Mi)), qn)
    qoff = np.arange(len(e1)) - np.repeat(np.cumsum(qn) - qn, qn)
    qpos = Qt.indptr[Mi[e1]] + qoff
    I_ = Qt.indices[qpos]
    v1 = Qt.data[qpos] * Mv[e1]
    j1 = Mj[e1]
    # expand over P row j
    pn = np.diff(P.indptr)[j1]
    e2 = np.repeat(np.arange(len(j1)), pn)
    poff = np.arange(len(e2)) - np.repeat(np.cumsum(pn) - pn, pn)
    ppos = P.indptr[j1[e2]] + poff
    J_ = P.indices[ppos]
    v2 = v1[e2] * P.data[ppos]
    key = I_[e2].astype(np.int64) * nJ + J_
    uniq, inv = np.unique(key, return_inverse=True)
    sums = np.bincount(inv, weights=v2, minlength=len(uniq))
    rows = uniq // nJ
    cols = (uniq % nJ).astype(np.int32)
    indptr = np.zeros(nI + 1, dtype=np.int64)
    np.add.at(indptr, rows + 1, 1)
    indptr = np.cumsum(indptr)
    return sp.csr_matrix((sums, cols, indptr), shape=(nI, nJ))


# ---------------------------------------------------------------------------------
# Coarsest level: eigenpairs of B_L x = lambda T_L x, and B_L^+ (Section 4.1, 4.2)
# ---------------------------------------------------------------------------------
def canonical_phase(v: np.ndarray) -> np.ndarray:
    """Unit 2-norm, with <w, v> real and positive for the fixed weight w_i = i + 1 (R8)."""
    v = v / np.linalg.norm(v)
    s = np.dot(np.arange(1, len(v) + 1, dtype=np.float64), v)
    if abs(s) > 0:
        v = v * (np.conj(s) / abs(s))
    return v


def coarse_eigs(BL: np.ndarray, TL: np.ndarray, k_ev: int):
    """Algorithm 3, coarsest level: the eigenpairs of B_L x = lambda T_L x of smallest
    |lambda|, computed from T_L^{-1} B_L.

    R8: complex eigenvalues are represented by the member with positive imaginary part;
    they are sorted by |lambda|; a real eigenvalue gives one vector, a complex pair the two
    real vectors Re v and Im v (both carrying Re lambda), until k_ev vectors are reached.
    The eigenvalue of smallest modulus is the state vector's and is set to exactly 0."""
    M = np.linalg.solve(TL, BL)
    lam, V = np.linalg.eig(M)
    keep = lam.imag >= 0
    lam, V = lam[keep], V[:, keep]
    order = np.argsort(np.abs(lam), kind="stable")
    vecs, lams, kinds = [], [], []
    for q in order:
        if len(vecs) >= k_ev:
            break
        v = canonical_phase(V[:, q])
        if lam[q].imag == 0.0:
            vecs.append(v.real)
            lams.append(lam[q].real)
            kinds.append(0)
        else:
            vecs.append(v.real)
            vecs.append(v.imag)
            lams += [lam[q].real, lam[q].real]
            kinds += [1, 2]
    lams = np.array(lams)
    lams[0] = 0.0
    return lams, np.array(vecs).T, np.array(kinds)


def pinv_truncated(BL: np.ndarray) -> np.ndarray:
    """Moore-Penrose inverse of the rank n-1 coarsest matrix (Section 4.2: the coarsest
    level computes the minimal-norm solution): SVD with the smallest singular value
    dropped (R12)."""
    U, s, Vt = np.linalg.svd(BL)
    sinv = np.zeros_like(s)
    sinv[:-1] = 1.0 / s[:-1]
    return (Vt.T * sinv) @ U.T


# ---------------------------------------------------------------------------------
# Hierarchy, setup (Section 1 steps 1-4, Algorithm 3 with mu = 1, then the rebuild)
# ---------------------------------------------------------------------------------
@dataclass
class Level:
    B: sp.csr_matrix
    T: sp.csr_matrix
    grid: tuple | None = None
    U: np.ndarray | None = None  # relaxed, normalised random test vectors
    V: np.ndarray | None = None  # eigenvector approximations after the upward pass
    lam: np.ndarray | None = None
    sel: np.ndarray | None = None  # which V columns joined the test set (R9)
    cf: np.ndarray | None = None
    cidx: np.ndarray | None = None
    P: sp.csr_matrix | None = None
    Q: sp.csr_matrix | None = None
    w: np.ndarray | None = None
    cand: np.ndarray | None = None
    ncand: np.ndarray | None = None
    cgrid: tuple | None = None  # grid of level l+1 (full coarsening)
    coarsest: bool = False
    kinds: np.ndarray | None = None  # coarsest level: 0 real, 1 Re, 2 Im of a complex pair
    colours: list | None = None  # multicolour Gauss-Seidel classes (R34)


@dataclass
class Hierarchy:
    levels: list
    opts: Opts
    pinv: np.ndarray | None = None
    x_init: np.ndarray | None = None
    stats: dict = field(default_factory=dict)

    @property
    def L(self) -> int:
        return len(self.levels) - 1

    def op_complexity(self) -> float:
        return sum(lv.B.nnz for lv in self.levels) / self.levels[0].B.nnz


def system_matrix(A) -> sp.csr_matrix:
    """B = I - A with its diagonal stored explicitly (R1)."""
    A = sp.csr_matrix(A)
    n = A.shape[0]
    B = sp.identity(n, format="csr") - A
    B = sp.csr_matrix(B)
    B.sort_indices()
    return B


def _split(B, grid, level: int, opts: Opts):
    if opts.coarsen == "grid":
        cf, cidx, cgrid = coarsen_grid(*grid)
        return cf, cidx, cgrid
    cf, cidx, _ = coarsen_cr(B, level, opts)
    return cf, cidx, None


def _build_interp(lv: Level, X: np.ndarray, active: np.ndarray, opts: Opts):
    Xh, w = normalize_weights(lv.B, X, active, opts.weight_floor)
    lv.cand, lv.ncand = neighborhoods(lv.B, lv.cf, lv.cidx, opts.z, opts.mmax)
    if opts.interp == "learned" or opts.record is not None:
        from . import learned

        feats = learned.features(lv.B, lv.cf, Xh[:, active], w[active], lv.cand, lv.ncand)
    if opts.interp == "learned":
        y, _ = learned.forward(opts.model, feats)
        P = learned.learned_rows(y, Xh[:, active], w[active], lv.cf, lv.cidx, lv.cand, lv.ncand, opts.caliber,
                                 opts.learned_refit, opts.ridge)
    else:
        P = ls_interpolation(Xh[:, active], w[active], lv.cf, lv.cidx, lv.cand, lv.ncand, opts.caliber, opts.ridge)
        if opts.record is not None:
            tg = learned.ls_targets(Xh[:, active], w[active], lv.cf, lv.cand, lv.ncand, opts.caliber, opts.ridge)
            opts.record.append((feats, tg, ~lv.cf))
    Q = averaging_restriction(P)
    return Xh, w, P, Q


def up_level(lv, Vc: np.ndarray, lam: np.ndarray, opts: Opts):
    """One level of the upward pass of Algorithm 3: V = P Vc; nu_ev omega-Jacobi sweeps on
    (B - lam_i T) x^(i) = 0; the Rayleigh-type update lambda_i = <B x, x> / <T x, x> for
    i >= 1 (lambda_0, the state vector's, stays 0); reading R9: x^(i) is selected for the
    rebuilt test set when |delta lambda_i| / |lambda_i| > ev_change_tol, the state vector
    always.  lv supplies P, B, T.  Returns (V, new lambda, selection)."""
    V = lv.P @ Vc
    V = jacobi_shifted(lv.B, lv.T, V, lam, opts.omega, opts.nu_ev)
    BV, TV = lv.B @ V, lv.T @ V
    new = np.einsum("nk,nk->k", BV, V) / np.einsum("nk,nk->k", TV, V)
    new[0] = 0.0
    change = np.abs(new - lam) / np.maximum(np.abs(lam), 1e-300)
    sel = change > opts.ev_change_tol
    sel[0] = True
    return V, new, sel


def _first_visit(lvs: list, l: int, levels: int, opts: Opts) -> bool:
    """First arrival at level l on the way down.  Returns True when l is the coarsest level
    (R13: n_l <= coarse_max, or `levels` coarsenings done); otherwise Algorithm 3's "Relax
    B_l x = 0, x in U_l" (nu_tv sweeps) and the C/F splitting of level l."""
    lv = lvs[l]
    lv.coarsest = l == levels or lv.B.shape[0] <= opts.coarse_max
    if lv.coarsest:
        return True
    lv.U = jacobi(lv.B, lv.U, opts.omega, opts.nu_tv)
    lv.cf, lv.cidx, lv.cgrid = _split(lv.B, lv.grid, l, opts)
    return False


def _interp_step(lvs: list, l: int, opts: Opts, with_v: bool):
    """One pass of Algorithm 3's loop body down to level l+1: P_l = ls_interpolation of
    U_l (and, with_v, the V_l columns selected by R9), the averaging Q_l, B_{l+1} = Q_l B_l P_l,
    T_{l+1} = Q_l T_l P_l.  On the first descent (level l+1 not built yet) it creates
    level l+1 with U_{l+1} = R_l U_l (injection of the normalised test vectors)."""
    lv = lvs[l]
    r = lv.U.shape[1]
    if with_v:
        X = np.concatenate([lv.U, lv.V], axis=1)
        active = np.concatenate([np.ones(r, dtype=bool), lv.sel])
    else:
        X, active = lv.U, np.ones(r, dtype=bool)
    Xh, w, P, Q = _build_interp(lv, X, active, opts)
    lv.w, lv.P, lv.Q = w, P, Q
    Bc = galerkin(Q, lv.B, P)
    Tc = galerkin(Q, lv.T, P)
    if len(lvs) == l + 1:
        lv.U = Xh
        c2f = np.flatnonzero(lv.cf)[np.argsort(lv.cidx[lv.cf], kind="stable")]
        lvs.append(Level(B=Bc, T=Tc, grid=lv.cgrid, U=Xh[c2f]))
    else:
        lvs[l + 1].B, lvs[l + 1].T = Bc, Tc


def _coarsest_eigs(lvs: list, l: int, opts: Opts):
    """Algorithm 3, l = L: the k_ev eigenpairs of B_L x = lambda T_L x of smallest |lambda|."""
    Lc = lvs[l]
    lam, V, kinds = coarse_eigs(Lc.B.toarray(), Lc.T.toarray(), opts.k_ev)
    Lc.V, Lc.lam, Lc.kinds = V, lam.copy(), kinds


def _up_step(lvs: list, l: int, opts: Opts):
    """Algorithm 3 after the recursive call: V_l = P_l V_{l+1}, relaxation of
    (B_l - lambda_i T_l) x^(i) = 0, the lambda update and the R9 selection (up_level)."""
    lv = lvs[l]
    V, lam, sel = up_level(lv, lvs[l + 1].V, lvs[l + 1].lam, opts)
    lv.V, lv.lam, lv.sel = V, lam.copy(), sel


def mle(lvs: list, l: int, levels: int, opts: Opts, first: bool):
    """bootamg_mle (Algorithm 3) on level l with cycle index mu = opts.mu (1: V-cycle,
    2: W-cycle, Section 4.1).

    R33: Algorithm 3 empties V_l at the start of every call, which would make a second
    call from the finest level repeat the first; V_l = {} is read as holding on the first
    visit of level l only, so every later visit (the second pass of a W-cycle's loop one
    level up, and every later MLE cycle) fits P_l to U_l and the V_l its previous visit
    left.  R10: U_l is relaxed on the first visit only, and U_{l+1} = R_l U_l is formed
    on the first descent only.  Section 5.1 runs the MLE as a "V(2,2)" cycle: a visit
    after the first relaxes V_l (nu_ev sweeps on (B_l - lambda_i T_l) x^(i) = 0) on the way
    down before P_l is fitted, as the upward pass does after the recursion."""
    if first:
        if _first_visit(lvs, l, levels, opts):
            _coarsest_eigs(lvs, l, opts)
            return
    elif lvs[l].coarsest:
        _coarsest_eigs(lvs, l, opts)
        return
    else:
        lv = lvs[l]
        lv.V = jacobi_shifted(lv.B, lv.T, lv.V, lv.lam, opts.omega, opts.nu_ev)
    for it in range(opts.mu):
        fresh = first and it == 0
        _interp_step(lvs, l, opts, with_v=not fresh)
        mle(lvs, l + 1, levels, opts, fresh)
        _up_step(lvs, l, opts)


def rebuild(lvs: list, opts: Opts):
    """Section 1: with the test sets of all levels updated, all P_l, B_l and T_l are
    recalculated, top-down, from U_l and the selected V_l; the C/F splitting of the first
    pass is kept (R26) and U_l is not relaxed again (R10)."""
    for l in range(len(lvs) - 1):
        _interp_step(lvs, l, opts, with_v=True)


def _finish(H: "Hierarchy"):
    """B_L^+ of the rebuilt coarsest matrix and the initial guess V_0[:, 0] / 1^T V_0[:, 0];
    with the multicolour smoother, the colour classes of every rebuilt B_l (R34)."""
    H.pinv = pinv_truncated(H.levels[-1].B.toarray())
    if H.opts.smoother == "mcgs":
        for l, lv in enumerate(H.levels[:-1]):
            lv.colours = multicolour(lv.B, l, H.opts.seed)
    x0 = H.levels[0].V[:, 0].copy()
    H.x_init = x0 / x0.sum()


def _start(A, r: int, opts: Opts, grid):
    B0 = system_matrix(A)
    n = B0.shape[0]
    return [Level(B=B0, T=sp.identity(n, format="csr"), grid=grid, U=tv_init(n, r, opts.seed, opts.tv_lo, opts.tv_hi))]


def setup(A, r: int, levels: int, opts: Opts | None = None, grid: tuple | None = None) -> Hierarchy:
    """Bootstrap setup: opts.setup_cycles MLE cycles (Algorithm 3 with mu = opts.mu;
    R33 for the cycles after the first) followed by the rebuild of all P_l, B_l, T_l from
    the enriched test sets (Section 1).

    First cycle, down: relax the random test vectors U_l (nu_tv sweeps), fit P_l
    (Algorithm 2), form Q_l, B_{l+1} = Q_l B_l P_l, T_{l+1} = Q_l T_l P_l and inject
    U_{l+1} = R_l U_l, until n_{l+1} <= coarse_max or `levels` coarsenings (R13).
    Coarsest: the k_ev eigenpairs of smallest |lambda|.
    Up: V_l = P_l V_{l+1}, nu_ev sweeps on (B_l - lambda_i T_l) x^(i) = 0, then
    lambda_i = <B x, x> / <T x, x> for i >= 1 (lambda_0 stays 0).  R9: x^(i) joins the
    level's test set when |delta lambda_i| / |lambda_i| > ev_change_tol; the state vector
    always joins.
    Rebuild (R10): top-down, P_l from U_l (not relaxed again) plus the selected V_l, with
    weights and neighbourhoods recomputed on the current B_l; the C/F splitting of the
    first pass is kept (R26).  The state vector approximation V_0[:, 0], scaled to
    1^T x = 1, is the initial guess of the solve."""
    opts = opts or Opts()
    if opts.coarsen == "grid" and grid is None:
        raise ValueError("full coarsening needs the grid dimensions")
    lvs = _start(A, r, opts, grid)
    mle(lvs, 0, levels, opts, first=True)
    for _ in range(1, opts.setup_cycles):
        mle(lvs, 0, levels, opts, first=False)
    rebuild(lvs, opts)
    H = Hierarchy(levels=lvs, opts=opts)
    _finish(H)
    H.stats["kinds"] = lvs[-1].kinds
    return H


def _ratio(B, x, norm: str) -> float:
    r = B @ x
    if norm == "l1":
        return float(np.abs(r).sum() / np.abs(x).sum())
    return float(np.linalg.norm(r) / np.linalg.norm(x))


def mle_solve(A, r: int, levels: int, tol: float, opts: Opts | None = None, grid: tuple | None = None,
              max_cycles: int = 50, norm: str = "l2"):
    """The MLE as a stand-alone solver (Section 4.1; the MLE rows of Tables 1, 2 and 4):
    MLE cycles (Algorithm 3 with mu = opts.mu, R33) until the state vector approximation
    x = V_0[:, 0] of the latest cycle meets ||B x|| / ||x|| <= tol (norm "l2": the
    Section 5.1 criterion, R15; "l1": the l1 ratio).  Returns x (1^T x = 1) and the
    cycle count and residual history."""
    opts = opts or Opts()
    lvs = _start(A, r, opts, grid)
    B = lvs[0].B
    hist = []
    cycles = 0
    while True:
        mle(lvs, 0, levels, opts, first=(cycles == 0))
        cycles += 1
        x = lvs[0].V[:, 0].copy()
        hist.append(_ratio(B, x, norm))
        if hist[-1] <= tol or cycles >= max_cycles:
            break
    return x / x.sum(), {"cycles": cycles, "history": hist, "converged": hist[-1] <= tol}


def mle_restart(H: Hierarchy, x: np.ndarray):
    """R32, the MLE restart of Section 5.1 ("restarting the MLE iterations when the solution
    is not found in a reasonable number of pGMRES iterations"; Section 4.1: alternate MLE
    and AMG-GMRES when several eigenvalues are near zero): the pGMRES iterate x becomes the
    state-vector test vector of every level (x / ||x||_2 on level 0, its injection R_l on
    the coarser ones), all P_l, B_l, T_l are rebuilt top-down as in the setup's rebuild, and
    B_L^+ is recomputed.  The other test vectors are unchanged."""
    lvs = H.levels
    lvs[0].V[:, 0] = x / np.linalg.norm(x)
    lvs[0].sel[0] = True
    for l in range(len(lvs) - 1):
        lv = lvs[l]
        _interp_step(lvs, l, H.opts, with_v=True)
        c2f = np.flatnonzero(lv.cf)[np.argsort(lv.cidx[lv.cf], kind="stable")]
        lvs[l + 1].V[:, 0] = lv.V[c2f, 0]
        if lvs[l + 1].sel is not None:
            lvs[l + 1].sel[0] = True
    H.pinv = pinv_truncated(lvs[-1].B.toarray())
    if H.opts.smoother == "mcgs":
        for l, lv in enumerate(lvs[:-1]):
            lv.colours = multicolour(lv.B, l, H.opts.seed)
    H.stats["mle_restarts"] = H.stats.get("mle_restarts", 0) + 1


# ---------------------------------------------------------------------------------
# Solve: V(nu1, nu2) preconditioner (Eq. (4.4)) inside flexible GMRES (Section 4.2)
# ---------------------------------------------------------------------------------
def vcycle(H: Hierarchy, b: np.ndarray, l: int = 0) -> np.ndarray:
    """z = C_l b with error propagator I - C_l B_l = S^nu2 (I - P_l C_{l+1} Q_l B_l) S^nu1,
    S = I - omega D^{-1} B_l (Eq. (4.4)), zero initial guess, and C_L = B_L^+ on the
    coarsest level.  With smoother "mcgs" (R34) S is a multicolour Gauss-Seidel sweep,
    colours ascending before the coarse correction and descending after it."""
    o = H.opts
    if l == H.L:
        return H.pinv @ b
    lv = H.levels[l]
    dinv = 1.0 / diag_of(lv.B)
    x = np.zeros_like(b)
    gs = o.smoother == "mcgs"
    for _ in range(o.nu_pre):
        x = gs_sweep(lv.B, dinv, b, x, lv.colours, False) if gs else x + o.omega * dinv * (b - lv.B @ x)
    r = b - lv.B @ x
    ec = vcycle(H, lv.Q @ r, l + 1)
    x = x + lv.P @ ec
    for _ in range(o.nu_post):
        x = gs_sweep(lv.B, dinv, b, x, lv.colours, True) if gs else x + o.omega * dinv * (b - lv.B @ x)
    return x


def l1_ratio(B, x) -> float:
    return float(np.abs(B @ x).sum() / np.abs(x).sum())


def orthogonalise(Vj: np.ndarray, w: np.ndarray):
    """Classical Gram-Schmidt of w against the orthonormal columns of Vj, applied twice:
    h = Vj^T w, w1 = w - Vj h, h2 = Vj^T w1, w1 -= Vj h2; returns (h + h2, w1).  (With right
    preconditioning w = B C v_j is nearly v_j, so the first pass cancels about 98% of w on
    the test chains and Kahan and Parlett's test would ask for the second pass every time.)"""
    h = Vj.T @ w
    w1 = w - Vj @ h
    h2 = Vj.T @ w1
    return h + h2, w1 - Vj @ h2


def fgmres(B, x0: np.ndarray, precond, tol: float, m: int, max_it: int, norm: str = "l1"):
    """Right-preconditioned flexible GMRES(m) on B x = 0 (R20), classical Gram-Schmidt
    with one reorthogonalisation, Givens rotations for the small least-squares problem.
    After every inner step the iterate x_j = x_0 + Z_j y_j is formed and the true
    residual is tested: ||B x||_1 / ||x||_1 <= tol (norm="l1"), or ||B x||_2 / ||x||_2
    (norm="l2", the paper's Section 5.1 criterion, R15).  Returns x and the history."""
    def ratio(x):
        r = B @ x
        if norm == "l1":
            return float(np.abs(r).sum() / np.abs(x).sum())
        return float(np.linalg.norm(r) / np.linalg.norm(x))

    x = np.array(x0, dtype=np.float64, copy=True)
    hist = [ratio(x)]
    it = 0
    restarts = 0
    if hist[-1] <= tol:
        return x, {"iterations": 0, "history": hist, "restarts": 0}
    while it < max_it:
        r = -(B @ x)
        beta = np.linalg.norm(r)
        n = len(x)
        V = np.zeros((n, m + 1))
        Z = np.zeros((n, m))
        Hh = np.zeros((m + 1, m))
        cs, sn = np.zeros(m), np.zeros(m)
        g = np.zeros(m + 1)
        g[0] = beta
        V[:, 0] = r / beta
        xj = x
        done = False
        for j in range(m):
            Z[:, j] = precond(V[:, j])
            w = B @ Z[:, j]
            h, w = orthogonalise(V[:, :j + 1], w)
            hn = np.linalg.norm(w)
            Hh[:j + 1, j] = h
            Hh[j + 1, j] = hn
            if hn > 0:
                V[:, j + 1] = w / hn
            for i in range(j):
                a, bb = Hh[i, j], Hh[i + 1, j]
                Hh[i, j] = cs[i] * a + sn[i] * bb
                Hh[i + 1, j] = -sn[i] * a + cs[i] * bb
            a, bb = Hh[j, j], Hh[j + 1, j]
            den = np.hypot(a, bb)
            cs[j], sn[j] = (1.0, 0.0) if den == 0 else (a / den, bb / den)
            Hh[j, j] = cs[j] * a + sn[j] * bb
            Hh[j + 1, j] = 0.0
            g[j + 1] = -sn[j] * g[j]
            g[j] = cs[j] * g[j]
            it += 1
            y = np.linalg.solve(np.triu(Hh[:j + 1, :j + 1]), g[:j + 1])
            xj = x + Z[:, :j + 1] @ y
            hist.append(ratio(xj))
            if hist[-1] <= tol or hn == 0 or it >= max_it:
                done = True
                break
        x = xj
        if done:
            break
        restarts += 1
    return x, {"iterations": it, "history": hist, "restarts": restarts, "converged": hist[-1] <= tol}


def solve(H: Hierarchy, tol: float, x0: np.ndarray | None = None, norm: str = "l1"):
    """V(2,2)-preconditioned FGMRES from the setup's state-vector approximation, then the
    normalisation 1^T x = 1.  With opts.mle_restart (R32) every restart cycle of gmres_m
    steps that ends above tol is followed by an MLE restart (mle_restart) before the next
    cycle; without it the cycles simply restart from the last iterate."""
    o = H.opts
    B = H.levels[0].B
    x = H.x_init if x0 is None else x0
    prec = lambda v: vcycle(H, v)  # noqa: E731
    if not o.mle_restart:
        x, st = fgmres(B, x, prec, tol, o.gmres_m, o.max_it, norm=norm)
    else:
        st = {"iterations": 0, "history": [], "restarts": 0, "mle_restarts": 0}
        while True:
            x, c = fgmres(B, x, prec, tol, o.gmres_m, min(o.gmres_m, o.max_it - st["iterations"]), norm=norm)
            st["history"] += c["history"] if not st["history"] else c["history"][1:]
            st["iterations"] += c["iterations"]
            st["converged"] = c["converged"] if "converged" in c else c["history"][-1] <= tol
            if st["converged"] or c["iterations"] == 0 or st["iterations"] >= o.max_it:
                break
            st["restarts"] += 1
            mle_restart(H, x)
            st["mle_restarts"] += 1
    x = x / x.sum()
    st["residual_l1"] = l1_ratio(B, x)
    return x, st


def ritz_closest_to_zero(Hk: np.ndarray):
    """Section 4.3: the eigenvalue of H_k closest to 0 and its eigenvector eta (unit 2-norm,
    largest-modulus entry positive).  For a complex closest eigenvalue the real part of
    its eigenvector is taken (the preconditioned matrix's eigenvalue 0 is real)."""
    lam, E = np.linalg.eig(Hk)
    q = int(np.argmin(np.abs(lam)))
    eta = np.real(E[:, q])
    eta = eta / np.linalg.norm(eta)
    if eta[np.argmax(np.abs(eta))] < 0:
        eta = -eta
    return float(np.real(lam[q])), eta


def parnoldi(H: Hierarchy, tol: float, x0: np.ndarray | None = None, m: int | None = None,
             max_it: int | None = None, norm: str = "l1"):
    """Multigrid-preconditioned Arnoldi (Section 4.3): orthonormal v_1, v_2, ... spanning
    the Krylov space of C B from y (the setup's state-vector approximation, or x0),
    H_k = V_k^T (C B) V_k, the eigenvalue of H_k closest to 0 with eigenvector eta, and
    the Ritz vector x = V_k eta as the steady-state approximation.  C is the V(2,2) cycle.
    The Gram-Schmidt process is fgmres's (classical, applied twice).  After every step the true residual of the Ritz vector is tested; after m
    steps the process restarts from the Ritz vector (explicit restart; the paper does not
    restart).  Returns x with 1^T x = 1 and the history."""
    o = H.opts
    B = H.levels[0].B
    m = o.gmres_m if m is None else m
    max_it = o.max_it if max_it is None else max_it
    y = np.array(H.x_init if x0 is None else x0, dtype=np.float64, copy=True)
    n = len(y)
    hist = [_ratio(B, y, norm)]
    it = 0
    x = y
    restarts = 0
    while hist[-1] > tol and it < max_it:
        V = np.zeros((n, m + 1))
        Hh = np.zeros((m + 1, m))
        V[:, 0] = y / np.linalg.norm(y)
        for j in range(m):
            w = vcycle(H, B @ V[:, j])
            h, w = orthogonalise(V[:, :j + 1], w)
            hn = np.linalg.norm(w)
            Hh[:j + 1, j] = h
            Hh[j + 1, j] = hn
            if hn > 0:
                V[:, j + 1] = w / hn
            it += 1
            theta, eta = ritz_closest_to_zero(Hh[:j + 1, :j + 1])
            x = V[:, :j + 1] @ eta
            hist.append(_ratio(B, x, norm))
            if hist[-1] <= tol or hn == 0 or it >= max_it:
                break
        y = x
        restarts += 1
    x = x / x.sum()
    return x, {"iterations": it, "history": hist, "restarts": max(restarts - 1, 0), "converged": hist[-1] <= tol,
               "residual_l1": l1_ratio(B, x)}


def stationary(A, r: int, levels: int, tol: float, opts: Opts | None = None, grid=None):
    """Setup plus solve in one call."""
    H = setup(A, r, levels, opts, grid)
    x, st = solve(H, tol)
    return x, H, st

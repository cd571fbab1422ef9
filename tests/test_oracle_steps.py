"""Pins of each oracle step against what the paper and the mathematics fix, by routes
other than the oracle's own code: closed forms, brute force, other library algorithms
and the algebraic identities the paper states."""

import os

import numpy as np
import pytest
import scipy.linalg
import scipy.sparse as sp

from oracle import bamg
from workloads import grid_walk, tandem_queue


def ring_walk(n):
    """Symmetric random walk on a cycle: a_{i, i+-1} = 1/2 (a test input)."""
    i = np.arange(n)
    rows = np.concatenate([i, i])
    cols = np.concatenate([(i + 1) % n, (i - 1) % n])
    return sp.csr_matrix((np.full(2 * n, 0.5), (rows, cols)), shape=(n, n))


# ----------------------------------------------------------------------------- RNG
def test_splitmix64_published_outputs(golden_dir):
    want = [int(l, 16) for l in open(os.path.join(golden_dir, "splitmix64_seed0.txt")) if l.strip() and l[0] != "#"]
    got = bamg.counter_u64(0, 0, np.arange(4, dtype=np.uint64))
    assert [int(v) for v in got] == want


def test_tv_init_range_and_streams():
    X = bamg.tv_init(1000, 5, 11, 1.0, 2.0)
    assert X.min() >= 1.0 and X.max() < 2.0
    assert abs(X.mean() - 1.5) < 0.02
    Y = bamg.tv_init(1000, 5, 12, 1.0, 2.0)
    assert not np.any(X == Y)
    assert np.array_equal(X, bamg.tv_init(1000, 5, 11, 1.0, 2.0))


# ----------------------------------------------------------------------- relaxation
@pytest.mark.parametrize("nu", [1, 3])
def test_jacobi_fourier_modes(nu):
    # On the ring walk B = I - (S + S^T)/2 has diag 1 and B cos(k theta) = (1 - cos theta) cos(k theta),
    # so omega-Jacobi (Eq. 3.1) scales the mode by (1 - omega (1 - cos theta)) per sweep.
    n, om = 32, 0.7
    B = bamg.system_matrix(ring_walk(n))
    th = 2 * np.pi * np.array([1, 3, 8]) / n
    X = np.cos(np.outer(np.arange(n), th))
    Y = bamg.jacobi(B, X, om, nu)
    assert np.allclose(Y, X * (1 - om * (1 - np.cos(th))) ** nu, atol=1e-14)


def test_jacobi_shifted_modes():
    n, om = 24, 0.7
    B = bamg.system_matrix(ring_walk(n))
    T = 2.0 * sp.identity(n, format="csr")
    th = 2 * np.pi * np.array([2, 5]) / n
    lam = np.array([0.05, -0.1])
    X = np.cos(np.outer(np.arange(n), th))
    Y = bamg.jacobi_shifted(B, T, X, lam, om, 2)
    fac = 1 - om * (1 - np.cos(th) - 2 * lam) / (1 - 2 * lam)
    assert np.allclose(Y, X * fac ** 2, atol=1e-14)


class _UpLevel:
    """The P, B, T of one level, for up_level."""

    def __init__(self, P, B, T):
        self.P, self.B, self.T = P, B, T


def _pencil_with_fourier_modes(n=16, seed=0):
    # B = diag(t) (I - A_ring), T = diag(t): B u = lambda T u for every Fourier mode u of
    # the ring walk, lambda_k = 1 - cos(2 pi k / n), with a non-identity T
    t = 1.0 + np.random.default_rng(seed).random(n)
    C = sp.identity(n, format="csr") - ring_walk(n)
    B = sp.csr_matrix(sp.diags(t) @ C)
    T = sp.diags(t, format="csr")
    i = np.arange(n)
    ks = (0, 1, 2)
    U = np.stack([np.cos(2 * np.pi * k * i / n) for k in ks], axis=1)
    lam = np.array([1.0 - np.cos(2 * np.pi * k / n) for k in ks])
    return B, T, U, lam


def test_up_level_keeps_exact_eigenvectors():
    # V = P Vc: exact eigenvectors of the pencil with their exact eigenvalues come back from
    # the shifted sweeps unchanged, the Rayleigh-type update returns the same eigenvalues,
    # and only the state vector is selected for the rebuild (Algorithm 3, reading R9)
    B, T, U, lam = _pencil_with_fourier_modes()
    lv = _UpLevel(sp.csr_matrix(U), B, T)
    V, new, sel = bamg.up_level(lv, np.eye(3), lam.copy(), bamg.Opts())
    assert np.allclose(V, U, rtol=0, atol=1e-14)
    assert new[0] == 0.0 and np.allclose(new[1:], lam[1:], rtol=1e-13, atol=0)
    assert sel.tolist() == [True, False, False]


def test_up_level_wrong_shift_closed_form():
    # a shift mu != lambda_2 for the third column: every sweep multiplies the eigenvector by
    # 1 - omega (lambda - mu) / (1 - mu) (Jacobi diagonal t (1 - mu) of B - mu T), the
    # quotient still returns lambda_2, and the relative change |lambda - mu| / mu = 1/3
    # selects the column; a state-vector eigenvalue passed in is reset to 0
    B, T, U, lam = _pencil_with_fourier_modes(seed=1)
    o = bamg.Opts()
    mu = 1.5 * lam[2]
    V, new, sel = bamg.up_level(_UpLevel(sp.csr_matrix(U), B, T), np.eye(3), np.array([0.3, lam[1], mu]), o)
    f = (1.0 - o.omega * (lam[2] - mu) / (1.0 - mu)) ** o.nu_ev
    assert np.allclose(V[:, 2], f * U[:, 2], rtol=0, atol=1e-14)
    assert np.allclose(V[:, 1], U[:, 1], rtol=0, atol=1e-14)
    assert new[0] == 0.0 and new[2] == pytest.approx(lam[2], rel=1e-13)
    assert sel.tolist() == [True, False, True]


def test_up_level_prolongs_through_P():
    # Vc = e_1 + e_2 is prolonged by P = [u0, u1, u2] to u1 + u2; with the shift lambda_1 each
    # sweep leaves the u1 part and multiplies the u2 part by 1 - omega (lambda_2 - lambda_1)
    # / (1 - lambda_1), so the result is u1 + f u2 in closed form, and its eigenvalue
    # estimate has moved (selected)
    B, T, U, lam = _pencil_with_fourier_modes(seed=2)
    o = bamg.Opts()
    Vc = np.zeros((3, 2))
    Vc[0, 0] = 1.0
    Vc[1, 1] = Vc[2, 1] = 1.0
    V, new, sel = bamg.up_level(_UpLevel(sp.csr_matrix(U), B, T), Vc, np.array([0.0, lam[1]]), o)
    f = (1.0 - o.omega * (lam[2] - lam[1]) / (1.0 - lam[1])) ** o.nu_ev
    assert np.allclose(V[:, 1], U[:, 1] + f * U[:, 2], rtol=0, atol=1e-14)
    assert np.allclose(V[:, 0], U[:, 0], rtol=0, atol=1e-14)
    assert sel.tolist() == [True, True]


def test_weights_closed_form():
    n = 32
    B = bamg.system_matrix(ring_walk(n))
    th = 2 * np.pi * np.array([1, 2, 4]) / n
    X = 3.0 * np.cos(np.outer(np.arange(n), th))
    Xh, w = bamg.normalize_weights(B, X, np.ones(3, dtype=bool), 1e-28)
    want = 1.0 / (1 - np.cos(th)) ** 2
    assert np.allclose(w, want / want.max(), rtol=1e-12)
    assert np.allclose(np.linalg.norm(Xh, axis=0), 1.0)


def test_stationary_vector_is_fixed_point():
    from oracle import exact
    ch = tandem_queue(6)
    x = exact.dense_nullspace(ch.dense())
    B = bamg.system_matrix(ch.to_scipy())
    assert np.allclose(bamg.jacobi(B, x[:, None], 0.7, 5)[:, 0], x, atol=1e-15)


# ------------------------------------------------------------------------ coarsening
def test_full_coarsening():
    cf, cidx, (cx, cy) = bamg.coarsen_grid(7, 4)
    assert (cx, cy) == (4, 2) and cf.sum() == 8
    assert cidx[0] == 0 and cidx[2] == 1 and cidx[14] == 4 and cidx[1] == -1
    assert sorted(cidx[cf]) == list(range(8))


def _bfs(B, i, z):
    B = sp.csr_matrix(B)
    dist = {i: 0}
    front = [i]
    for d in range(1, z + 1):
        nxt = []
        for u in front:
            for v in B.indices[B.indptr[u]:B.indptr[u + 1]]:
                if v not in dist:
                    dist[int(v)] = d
                    nxt.append(int(v))
        front = nxt
    return dist


@pytest.mark.parametrize("z", [1, 2, 3])
def test_neighborhoods_vs_bfs(z):
    ch = tandem_queue(8)
    B = bamg.system_matrix(ch.to_scipy())
    cf, cidx, _ = bamg.coarsen_grid(*ch.grid)
    cand, ncand = bamg.neighborhoods(B, cf, cidx, z, 64)
    extended = 0
    for i in range(ch.n):
        if cf[i]:
            assert ncand[i] == 0
            continue
        depth = z
        while True:  # the smallest depth <= 3 that reaches a coarse point (at least z)
            dist = _bfs(B, i, depth)
            want = sorted([j for j in dist if j != i and cf[j]], key=lambda j: (dist[j], cidx[j]))
            if want or depth >= 3:
                break
            depth += 1
        extended += depth > z
        assert list(cand[i, :ncand[i]]) == want


def test_neighborhood_extension_reaches_the_corner():
    # in the directed graph of the 32 x 32 tandem queue one fine state reaches no coarse
    # state within two steps; the extension to three gives it candidates
    ch = tandem_queue(31)
    B = bamg.system_matrix(ch.to_scipy())
    cf, cidx, _ = bamg.coarsen_grid(*ch.grid)
    c2, n2 = bamg._neighborhoods_depth(B, cf, cidx, 2, 16)
    cand, ncand = bamg.neighborhoods(B, cf, cidx, 2, 16)
    miss = np.flatnonzero((~cf) & (n2 == 0))
    assert len(miss) >= 1
    for i in miss:
        dist = _bfs(B, i, 3)
        want = sorted([j for j in dist if j != i and cf[j]], key=lambda j: (dist[j], cidx[j]))
        assert len(want) > 0 and list(cand[i, :ncand[i]]) == want


def test_every_fine_point_is_interpolated_on_tandem_hierarchy():
    # with the extension every column of Q sums to one, hence 1^T B_l = 0 on every level
    ch = tandem_queue(31)
    H = bamg.setup(ch.to_scipy(), 6, 10, bamg.Opts(), grid=ch.grid)
    for lv in H.levels[:-1]:
        assert np.all(lv.ncand[~lv.cf] > 0)
    for lv in H.levels:
        assert np.abs(np.asarray(lv.B.sum(axis=0)).ravel()).max() < 1e-13


def test_independent_set_is_maximal():
    ch = tandem_queue(10)
    B = bamg.system_matrix(ch.to_scipy())
    S = bamg._sym_adjacency(B)
    rng = np.random.default_rng(0)
    cand = rng.random(ch.n) < 0.6
    sel = bamg.independent_set(S, cand, 5, 77)
    assert np.all(cand[sel])
    S = sp.csr_matrix(S)
    for i in range(ch.n):
        nb = S.indices[S.indptr[i]:S.indptr[i + 1]]
        if sel[i]:
            assert not np.any(sel[nb])
        elif cand[i]:
            assert np.any(sel[nb])


def test_cr_meets_theta():
    from workloads import delaunay_walk
    ch = delaunay_walk(600, 3)
    B = bamg.system_matrix(ch.to_scipy())
    o = bamg.Opts(coarsen="cr")
    cf, cidx, rounds = bamg.coarsen_cr(B, 0, o)
    assert rounds < o.cr_max_rounds
    f = np.flatnonzero(~cf)
    u0 = 1.0 + bamg.counter_uniform(o.seed, bamg.STREAM_CR + rounds, f.astype(np.uint64))
    # independent F-relaxation: dense B_ff
    Bd = B.toarray()[np.ix_(f, f)]
    u = u0.copy()
    for _ in range(o.cr_nu):
        u = u - o.cr_omega * (Bd @ u) / np.diag(Bd)
    assert (np.linalg.norm(u) / np.linalg.norm(u0)) ** (1 / o.cr_nu) <= o.cr_theta
    assert 0.1 < cf.mean() < 0.6


# ---------------------------------------------------------------------- LS (Alg. 2)
def test_ls_recovers_exact_combination():
    rng = np.random.default_rng(1)
    K, S = 16, 6
    Xc = rng.standard_normal((1, S, K))
    xi = 0.8 * Xc[0, 2] + 0.2 * Xc[0, 4]
    chosen, p, L = bamg.ls_fit_rows(xi[None], Xc, np.ones((1, S), bool), np.ones(K), 2, 1e-14)
    assert list(chosen[0]) == [2, 4]
    assert np.allclose(p[0], [0.8, 0.2], atol=1e-10)
    assert L[0] < 1e-20


def test_ls_greedy_brute_force():
    rng = np.random.default_rng(2)
    m, S, K, c, ridge = 40, 7, 10, 3, 1e-8
    Xc = rng.uniform(0.5, 1.5, (m, S, K))
    xi = rng.uniform(0.5, 1.5, (m, K))
    valid = rng.random((m, S)) < 0.8
    valid[:, 0] = True
    w = rng.uniform(0.1, 1.0, K)
    chosen, pw, Lb = bamg.ls_fit_rows(xi, Xc, valid, w, c, ridge)
    sw = np.sqrt(w)
    for r in range(m):
        J = []
        for t in range(c):
            best = None
            for g in range(S):
                if not valid[r, g] or g in J:
                    continue
                Sg = J + [g]
                Xs = Xc[r, Sg]  # (t+1, K)
                G = (Xs * w) @ Xs.T
                delta = ridge * np.trace(G) / len(Sg)
                # ridge LS as an augmented least-squares system (QR route)
                Aug = np.vstack([(Xs * sw).T, np.sqrt(delta) * np.eye(len(Sg))])
                rhs = np.concatenate([xi[r] * sw, np.zeros(len(Sg))])
                p = np.linalg.lstsq(Aug, rhs, rcond=None)[0]
                L = np.sum(w * (xi[r] - p @ Xs) ** 2)
                if best is None or L < best[0]:
                    best = (L, g, p)
            if best is None:
                break
            J.append(best[1])
            last = best
            assert chosen[r, t] == best[1]
        assert np.all(chosen[r, len(J):] == -1)
        # the row's weights are the minimiser over the final J
        assert np.allclose(pw[r, :len(J)], last[2], rtol=1e-8, atol=1e-10)
        assert Lb[r] == pytest.approx(last[0], rel=1e-8)


# ------------------------------------------------------------- P, Q and Galerkin
def _small_hierarchy_level():
    ch = tandem_queue(8)
    B = bamg.system_matrix(ch.to_scipy())
    cf, cidx, _ = bamg.coarsen_grid(*ch.grid)
    X = bamg.jacobi(B, bamg.tv_init(ch.n, 6, 0, 1.0, 2.0), 0.7, 4)
    Xh, w = bamg.normalize_weights(B, X, np.ones(6, bool), 1e-28)
    cand, ncand = bamg.neighborhoods(B, cf, cidx, 2, 16)
    P = bamg.ls_interpolation(Xh, w, cf, cidx, cand, ncand, 2, 1e-12)
    return B, cf, cidx, P


def test_P_structure_and_Q_invariants():
    B, cf, cidx, P = _small_hierarchy_level()
    P = sp.csr_matrix(P)
    cnt = np.diff(P.indptr)
    assert np.all(cnt[cf] == 1) and np.all(cnt <= 2)
    for i in np.flatnonzero(cf):
        assert P.indices[P.indptr[i]] == cidx[i] and P.data[P.indptr[i]] == 1.0
    Q = bamg.averaging_restriction(P)
    assert np.allclose(np.asarray(Q.sum(axis=0)).ravel(), 1.0, atol=1e-15)
    assert ((Q != 0).astype(int) - (P.T != 0).astype(int)).nnz == 0


def test_galerkin_vs_dense_products():
    B, cf, cidx, P = _small_hierarchy_level()
    Q = bamg.averaging_restriction(P)
    Bc = bamg.galerkin(Q, B, P)
    assert np.allclose(Bc.toarray(), Q.toarray() @ B.toarray() @ P.toarray(), atol=1e-15)
    # 1^T Q = 1^T and 1^T B = 0 imply 1^T B_{l+1} = 0 (Section 4)
    assert np.max(np.abs(np.asarray(Bc.sum(axis=0)).ravel())) < 1e-14


def test_galerkin_keeps_cancelled_entries():
    Q = sp.csr_matrix(np.array([[1.0, 1.0]]))
    M = sp.csr_matrix(np.array([[1.0, 0.0], [-1.0, 0.0]]))
    P = sp.csr_matrix(np.array([[1.0], [1.0]]))
    G = bamg.galerkin(Q, M, P)
    assert G.nnz == 1 and G.data[0] == 0.0


# ----------------------------------------------------------------- coarsest level
def _coarse_pair(seed=3, n=30):
    rng = np.random.default_rng(seed)
    A = rng.random((n, n)) * (rng.random((n, n)) < 0.3)
    np.fill_diagonal(A, 0)
    A[np.arange(n), (np.arange(n) + 1) % n] += 0.1  # irreducible
    A /= A.sum(axis=0, keepdims=True)
    B = np.eye(n) - A
    T = np.eye(n) + 0.2 * rng.random((n, n)) * (rng.random((n, n)) < 0.1)
    return B, T


def test_coarse_eigs_against_qz():
    B, T = _coarse_pair()
    lams, V, kinds = bamg.coarse_eigs(B, T, 6)
    ev = scipy.linalg.eig(B, T, right=False)  # QZ: another algorithm
    ev = ev[ev.imag >= 0]
    ev = ev[np.argsort(np.abs(ev))]
    assert lams[0] == 0.0 and abs(ev[0]) < 1e-12
    # each returned vector pairs with the QZ eigenvalue it belongs to
    q = 1
    c = 1
    while c < V.shape[1]:
        lam = ev[q]
        if kinds[c] == 0:
            v = V[:, c]
            assert abs(lams[c] - lam.real) < 1e-10 and lam.imag == pytest.approx(0, abs=1e-12)
            assert np.linalg.norm(B @ v - lam.real * (T @ v)) < 1e-10
            c += 1
        else:
            v = V[:, c] + 1j * V[:, c + 1]
            assert abs(lams[c] - lam.real) < 1e-10
            assert np.linalg.norm(B @ v - lam * (T @ v)) < 1e-10
            c += 2
        q += 1
    w = np.arange(1, B.shape[0] + 1)
    v0 = V[:, 0]
    assert np.linalg.norm(B @ v0) < 1e-12 and w @ v0 > 0


def test_pinv_penrose_and_bordered_route():
    B, _ = _coarse_pair(5, 25)
    Bp = bamg.pinv_truncated(B)
    assert np.allclose(B @ Bp @ B, B, atol=1e-12)
    assert np.allclose(Bp @ B @ Bp, Bp, atol=1e-10)
    assert np.allclose((B @ Bp).T, B @ Bp, atol=1e-12)
    assert np.allclose((Bp @ B).T, Bp @ B, atol=1e-12)
    n = B.shape[0]
    z = np.full(n, 1 / np.sqrt(n))
    _, _, Vt = np.linalg.svd(B)
    y = Vt[-1]
    Mb = B + np.outer(z, y)
    assert np.allclose(np.linalg.solve(Mb, np.eye(n) - np.outer(z, z)), Bp, atol=1e-10)


# ------------------------------------------------------------------- V-cycle, GMRES
@pytest.fixture(scope="module")
def small_H():
    ch = grid_walk(13)
    o = bamg.Opts(coarse_max=16)
    return bamg.setup(ch.to_scipy(), 6, 5, o, grid=ch.grid)


def test_vcycle_matches_error_propagator(small_H):
    # Eq. (4.4): I - C_l B_l = S^nu2 (I - P C_{l+1} Q B_l) S^nu1, with C_L = B_L^+.
    H = small_H
    o = H.opts
    assert H.L >= 2
    C_next = H.pinv
    for l in range(H.L - 1, -1, -1):
        lv = H.levels[l]
        n = lv.B.shape[0]
        Cl = np.column_stack([bamg.vcycle(H, e, l) for e in np.eye(n)])
        Bd = lv.B.toarray()
        S = np.eye(n) - o.omega * Bd / np.diag(Bd)[:, None]
        E = np.linalg.matrix_power(S, o.nu_post) @ (np.eye(n) - lv.P.toarray() @ C_next @ lv.Q.toarray() @ Bd) \
            @ np.linalg.matrix_power(S, o.nu_pre)
        assert np.allclose(np.eye(n) - Cl @ Bd, E, atol=1e-12)
        C_next = Cl


def test_gmres_minimises_over_preconditioned_krylov(small_H):
    H = small_H
    B = H.levels[0].B
    Bd = B.toarray()
    x0 = H.x_init
    C = lambda v: bamg.vcycle(H, v)
    r0 = -(B @ x0)
    W = [C(r0)]
    for _ in range(4):
        W.append(C(B @ W[-1]))
    for j in range(1, 5):
        x, st = bamg.fgmres(B, x0, C, 0.0, 50, j)
        Wj = np.linalg.qr(np.column_stack(W[:j]))[0]
        y = np.linalg.lstsq(Bd @ Wj, -(Bd @ x0), rcond=None)[0]
        best = np.linalg.norm(Bd @ (x0 + Wj @ y))
        assert np.linalg.norm(Bd @ x) == pytest.approx(best, rel=1e-6, abs=1e-15)


def test_coarse_operators_keep_column_sums(small_H):
    for lv in small_H.levels:
        cs = np.asarray(lv.B.sum(axis=0)).ravel()
        assert np.max(np.abs(cs)) < 1e-13 * abs(lv.B).max()

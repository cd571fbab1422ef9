"""The exact stationary vectors agree across independent routes (closed forms, dense LU,
SuperLU, power iteration on the lazy chain)."""

import numpy as np

from oracle import exact
from workloads import birth_death, delaunay_walk, grid_walk, random_birth_death, tandem_queue


def _rel(a, b):
    return np.abs(a - b).sum() / np.abs(b).sum()


def test_degree_closed_form_vs_dense():
    for ch in (grid_walk(6, 5), delaunay_walk(150, 4)):
        xd = exact.dense_nullspace(ch.dense())
        assert _rel(exact.from_degree(ch.meta["degree"]), xd) < 1e-13


def test_product_form_vs_dense():
    ch = random_birth_death(120, 7)
    xd = exact.dense_nullspace(ch.dense())
    xp = exact.birth_death(ch.meta["birth"], ch.meta["death"])
    assert _rel(xp, xd) < 1e-12


def test_tandem_three_routes():
    ch = tandem_queue(12)
    xd = exact.dense_nullspace(ch.dense())
    xs = exact.sparse_nullspace(ch.to_scipy())
    A = ch.dense()
    lazy = 0.5 * (np.eye(ch.n) + A)  # same stationary vector, aperiodic
    x = np.full(ch.n, 1.0 / ch.n)
    for _ in range(20000):
        x = lazy @ x
    assert _rel(xs, xd) < 1e-12
    assert _rel(x, xd) < 1e-9
    assert np.all(xd > 0)


def _error_per_residual(G):
    """max ||G r||_1 / ||r||_1 over residuals with 1^T r = 0 (every B x has that): the
    extreme points of that set are (e_i - e_j) / 2."""
    D = np.abs(G[:, :, None] - G[:, None, :]).sum(axis=0)
    return D.max() / 2.0


def test_birth_death_ambiguity_bounds_the_group_inverse():
    """kappa_lb is a lower bound on the error per residual of the dense group inverse
    (B + x* 1^T)^-1 - x* 1^T, and the explicit mass move it is built on has exactly the
    stated residual and error."""
    for n, seed in [(50, 1), (120, 5), (200, 7)]:
        ch = random_birth_death(n, seed)
        b, d = ch.meta["birth"], ch.meta["death"]
        x = exact.birth_death(b, d)
        B = np.eye(n) - ch.dense()
        G = np.linalg.inv(B + np.outer(x, np.ones(n))) - np.outer(x, np.ones(n))
        kappa = _error_per_residual(G)
        lk, _ = exact.birth_death_ambiguity(b, d, 1e-10)
        assert 10 ** lk <= kappa * (1 + 1e-9)
        assert 10 ** lk >= 0.01 * kappa  # not a vacuous bound on these chains
        # the construction for the maximising edge
        ML = np.cumsum(x)[:-1]
        m = int(np.argmax(ML * (1 - ML) / (b[:-1] * x[:-1])))
        dx = x * np.where(np.arange(n) <= m, 1 - ML[m], -ML[m])
        assert abs(dx.sum()) < 1e-14
        assert np.isclose(np.abs(dx).sum(), 2 * ML[m] * (1 - ML[m]), rtol=1e-12)
        assert np.isclose(np.abs(B @ dx).sum(), 2 * b[m] * x[m], rtol=1e-8)


def test_birth_death_ambiguity_of_a_uniform_chain_is_small():
    """Equal birth and death rates: x* is uniform, the worst edge is the middle one,
    kappa_lb = (1/4) / (b / n) = n / (4 b) in closed form."""
    n, b = 100, 0.3
    ch = birth_death(np.full(n, b), np.full(n, b))
    lk, eps = exact.birth_death_ambiguity(ch.meta["birth"], ch.meta["death"], 1e-10)
    assert np.isclose(10 ** lk, n / (4 * b), rtol=1e-9)
    assert np.isclose(eps, 2 * 0.25 * 1e-10 / (2 * b / n), rtol=1e-9)


def test_birth_death_condition_bounds_the_group_inverse_from_above():
    """K bounds the dense group inverse's error per residual from above on chains across
    five orders of conditioning, and is not vacuous (within 10x)."""
    for n, seed in [(50, 1), (120, 5), (200, 7), (150, 3)]:
        ch = random_birth_death(n, seed)
        b, d = ch.meta["birth"], ch.meta["death"]
        x = exact.birth_death(b, d)
        B = np.eye(n) - ch.dense()
        G = np.linalg.inv(B + np.outer(x, np.ones(n))) - np.outer(x, np.ones(n))
        kappa = _error_per_residual(G)
        K = 10 ** exact.birth_death_condition(b, d)
        assert kappa <= K * (1 + 1e-9), (kappa, K)
        assert K <= 10 * kappa, (kappa, K)
        lk, _ = exact.birth_death_ambiguity(b, d, 1e-10)
        assert 10 ** lk <= K


def _valley_chain():
    """60 states: x* falls by 9x per step for 30 steps (a valley about 1e-29 deep), rises by
    9x for 11 steps (a bump about 1e-18 high), then stays flat: the mass past the valley,
    about 1e-17, is below the rounding of 1 - M_L, while 1 / (b x*) at the valley is about
    1e29."""
    n = 60
    birth, death = np.full(n, 0.3), np.full(n, 0.3)
    for k in range(n - 1):  # edge k -> k + 1: x*_{k+1} / x*_k = birth[k] / death[k + 1]
        if k < 30:
            birth[k], death[k + 1] = 0.05, 0.45
        elif k < 41:
            birth[k], death[k + 1] = 0.45, 0.05
    return birth_death(birth, death)


def _worst_pair_error(b, d):
    """max ||e||_1 over the residuals (e_j - e_k) / 2 (the extreme points of the unit l1 ball
    with 1^T r = 0), e solving B e = r, 1^T e = 0, by the flux recursion of detailed balance:
    the residual's partial sums R_i = +-1/2 between j and k give u_{i+1} = u_i - R_i / (b_i x*_i)
    with e = x* u, and 1^T e = 0 fixes the constant."""
    x = exact.birth_death(b, d)
    n = len(x)
    w = 1.0 / (b[:-1] * x[:-1])
    best = 0.0
    for j in range(n):
        for k in range(j + 1, n):
            R = np.zeros(n - 1)
            R[j:k] = 0.5
            u = np.concatenate([[0.0], -np.cumsum(w * R)])
            u -= (x * u).sum()
            best = max(best, float(np.abs(x * u).sum()))
    return best


def test_birth_death_condition_counts_the_mass_past_a_deep_valley():
    """On a chain whose x* has a deep valley followed by a small bump, K still bounds the
    worst error per residual from above and stays within 10x of it.  Fails if M_R is taken
    as 1 - M_L, which rounds to 0 past the valley and drops the dominant terms (K then comes
    out near 40 against a worst case near 3e12); kappa_lb stays a lower bound."""
    ch = _valley_chain()
    b, d = ch.meta["birth"], ch.meta["death"]
    x = exact.birth_death(b, d)
    assert x[30] < 1e-28 and 1e-19 < x[-1] < 1e-17 and x[41:].sum() < 1e-16
    worst = _worst_pair_error(b, d)
    K = 10 ** exact.birth_death_condition(b, d)
    assert worst <= K * (1 + 1e-9), (worst, K)
    assert K <= 10 * worst, (worst, K)
    lk, _ = exact.birth_death_ambiguity(b, d, 1e-10)
    assert 10 ** lk <= worst * (1 + 1e-9)
    assert 10 ** lk >= 1e-3 * worst


def test_birth_death_condition_uniform_closed_form():
    """Equal rates b: x* = 1/n, w_i = n/b, M_L(i) = (i+1)/n; the median m = n/2 - 1 for even
    n, K = (n/b) (sum_{i<m} (i+1)/n + sum_{i>=m} (n-1-i)/n)."""
    n, b = 100, 0.3
    ch = birth_death(np.full(n, b), np.full(n, b))
    K = 10 ** exact.birth_death_condition(ch.meta["birth"], ch.meta["death"])
    ML = np.arange(1, n) / n
    m = int(np.searchsorted(ML, 0.5))
    want = (n / b) * (ML[:m].sum() + (1 - ML[m:]).sum())
    assert np.isclose(K, want, rtol=1e-9)

"""Input generators: every model is a column-stochastic chain with the structure the
paper's Section 5.1 describes, and the exact routes agree with each other."""

import numpy as np
import pytest

from oracle import exact
from workloads import (batched_mixture, birth_death, delaunay_walk, grid_walk, random_birth_death,
                       tandem_queue, tandem_training_set)


def _check_stochastic(ch):
    A = ch.to_scipy()
    assert np.all(ch.val >= 0)
    colsum = np.asarray(A.sum(axis=0)).ravel()
    assert np.max(np.abs(colsum - 1.0)) < 1e-14
    for i in range(min(ch.n, 2000)):
        c = ch.col[ch.row_ptr[i]:ch.row_ptr[i + 1]]
        assert np.all(np.diff(c) > 0)


@pytest.mark.parametrize("mk", [lambda: grid_walk(7, 5), lambda: tandem_queue(6), lambda: random_birth_death(50, 3),
                                lambda: delaunay_walk(200, 1)])
def test_column_stochastic(mk):
    _check_stochastic(mk())


def test_grid_structure():
    ch = grid_walk(6, 4)
    assert ch.n == 24 and ch.nnz == 2 * (5 * 4 + 6 * 3)
    deg = ch.meta["degree"]
    assert deg[0] == 2 and deg[1] == 3 and deg[7] == 4


def test_tandem_flow_balance():
    # In steady state the accepted arrival rate, the transfer rate and the departure rate
    # are equal (conservation of jobs through the two queues).
    N = 9
    mu, mx, my = 11 / 31, 10 / 31, 10 / 31
    ch = tandem_queue(N, mu, mx, my)
    x = exact.dense_nullspace(ch.dense()).reshape(N + 1, N + 1)  # [j, i]
    i = np.arange(N + 1)[None, :]
    j = np.arange(N + 1)[:, None]
    arr = mu * x[np.broadcast_to(i < N, x.shape)].sum()
    tr = mx * x[np.broadcast_to((i > 0) & (j < N), x.shape)].sum()
    dep = my * x[np.broadcast_to(j > 0, x.shape)].sum()
    assert abs(arr - tr) < 1e-13 and abs(tr - dep) < 1e-13
    assert ch.nnz <= 5 * ch.n


def test_tandem_interior_has_no_self_loop():
    ch = tandem_queue(5)
    A = ch.dense()
    m = 6
    for jj in range(1, 5):
        for ii in range(1, 5):
            assert A[ii + jj * m, ii + jj * m] == 0.0


def test_delaunay_is_planar_triangulation():
    ch = delaunay_walk(400, 2)
    deg = ch.meta["degree"]
    E = deg.sum() / 2
    assert E <= 3 * ch.n - 6 and E >= 2 * ch.n - 3


def test_birth_death_detailed_balance():
    rng = np.random.default_rng(0)
    b, d = rng.uniform(0.2, 0.5, 40), rng.uniform(0.2, 0.5, 40)
    ch = birth_death(b, d)
    x = exact.dense_nullspace(ch.dense())
    assert np.max(np.abs(x[:-1] * b[:-1] - x[1:] * d[1:])) < 1e-15


def test_mixtures_shapes():
    chains = batched_mixture(0, nchains=8, bd_lo=64, bd_hi=256, side_lo=8, side_hi=16)
    assert len(chains) == 8
    assert chains[0].kind == "birth_death" and chains[1].kind == "grid_walk"
    for ch in chains:
        _check_stochastic(ch)
    tr = tandem_training_set(1, 3, 7, 11)
    for ch in tr:
        _check_stochastic(ch)
        assert 7 <= ch.meta["N"] <= 11

"""The exact stationary vectors agree across independent routes (closed forms, dense LU,
SuperLU, power iteration on the lazy chain)."""

import numpy as np

from oracle import exact
from workloads import delaunay_walk, grid_walk, random_birth_death, tandem_queue


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

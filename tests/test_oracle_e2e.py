"""End to end: the oracle's setup plus preconditioned GMRES reaches the exact stationary
vector, and its iteration counts sit in a loose band around the paper's tables."""

import os

import numpy as np
import pytest

from oracle import bamg, exact
from workloads import delaunay_walk, grid_walk, random_birth_death, tandem_queue


def _rel(a, b):
    return np.abs(a - b).sum() / np.abs(b).sum()


@pytest.mark.parametrize("kind,size", [("grid", 17), ("grid", 33), ("tandem", 16), ("birth_death", 300),
                                        ("delaunay", 400)])
def test_reaches_exact_vector(kind, size):
    if kind == "grid":
        ch = grid_walk(size)
    elif kind == "tandem":
        ch = tandem_queue(size)
    elif kind == "birth_death":
        ch = random_birth_death(size, 5)
    else:
        ch = delaunay_walk(size, 5)
    o = bamg.Opts(coarsen="cr" if kind == "delaunay" else "grid", tv_lo=0.0, tv_hi=1.0)
    x, H, st = bamg.stationary(ch.to_scipy(), 8, 10, 1e-13, o, grid=ch.grid)
    xe = exact.exact_stationary(ch)
    assert st["converged"]
    assert st["residual_l1"] <= 1e-12
    assert _rel(x, xe) < 1e-9
    assert np.all(x >= -1e-14 * x.max())
    assert abs(x.sum() - 1.0) < 1e-14


def test_iteration_counts_near_paper(golden_dir):
    rows = [l.split() for l in open(os.path.join(golden_dir, "paper_iterations.txt")) if l.strip() and l[0] != "#"]
    for model, N, it_paper in rows:
        N, it_paper = int(N), int(it_paper)
        if model == "grid":
            ch, o, lev = grid_walk(N), bamg.Opts(coarse_max=25), 20
        elif model == "tandem":
            ch, o, lev = tandem_queue(N - 1), bamg.Opts(coarse_max=25), 20
        else:
            ch, o, lev = delaunay_walk(N, 0), bamg.Opts(coarsen="cr", coarse_max=25), 2
        H = bamg.setup(ch.to_scipy(), 6, lev, o, grid=ch.grid)
        x, st = bamg.solve(H, 1e-8, norm="l2")
        assert st["converged"]
        assert 0.5 * it_paper <= st["iterations"] <= 2.0 * it_paper, (model, N, st["iterations"], it_paper)

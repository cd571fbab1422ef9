"""GPU parity of the setup-cycling variants and the two other solvers against the oracle:
W-cycle and repeated-cycle setups (Algorithm 3 with mu = 2, R33), the stand-alone MLE
(Section 4.1), the MLE restart between pGMRES cycles (R32), restart lengths above 64, the
2-norm stopping test of Section 5.1, and the multigrid-preconditioned Arnoldi method
(Section 4.3).  FP64 runs agree with the oracle to relative L1 1e-9, mixed runs to 1e-6."""

import numpy as np
import pytest
import scipy.sparse as sp

from gpu_util import need_gpu, rel
from oracle import bamg as ob
from oracle import exact
from workloads import grid_walk, random_birth_death, tandem_queue

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _gpu():
    need_gpu()


def _bamg():
    import paper_1004_1451_gb300 as bamg

    return bamg


def _dev(ch):
    import torch

    return (torch.tensor(ch.row_ptr, device="cuda"), torch.tensor(ch.col, device="cuda"),
            torch.tensor(ch.val, device="cuda"))


def _levels_of(H):
    out = []
    for l, lv in enumerate(H.levels):
        B = sp.csr_matrix(lv.B)
        B.sort_indices()
        d = {"B": (B.indptr, B.indices, B.data)}
        if l < H.L:
            P = sp.csr_matrix(lv.P)
            P.sort_indices()
            d["P"] = (P.indptr, P.indices, P.data)
        out.append(d)
    return out


# ------------------------------------------------------------------ setup cycling
@pytest.mark.parametrize("mu,cycles", [(2, 1), (1, 2), (2, 2)])
def test_cycled_setup_matches_oracle(mu, cycles):
    """Same hierarchy sizes, nearly the same FGMRES iterations and the same vector as the
    oracle's setup with the same loop count and cycle count (FP64, tolerance 1e-13)."""
    ch = tandem_queue(24)
    rp, ci, v = _dev(ch)
    s = _bamg().Solver(rp, ci, v, r=6, levels=10, grid=ch.grid, precision="fp64", mu=mu, setup_cycles=cycles)
    x, st = s.solve(1e-13)
    o = ob.Opts(mu=mu, setup_cycles=cycles)
    xo, H, sto = ob.stationary(ch.to_scipy(), 6, 10, 1e-13, o, grid=ch.grid)
    assert s.info()["n"] == [lv.B.shape[0] for lv in H.levels]
    assert abs(st["iterations"] - sto["iterations"]) <= 1
    assert rel(x.cpu().numpy(), xo) < 1e-9
    assert rel(x.cpu().numpy(), exact.exact_stationary(ch)) < 1e-9
    # the state-vector approximations of the two setups agree too
    assert rel(s.export(0, _bamg()._capi.EXPORT_XINIT), H.x_init) < 1e-6


# ------------------------------------------------------------------ stand-alone MLE
@pytest.mark.parametrize("kind,mu", [("grid", 1), ("tandem", 1), ("tandem", 2)])
def test_mle_solve_matches_oracle(kind, mu):
    """The MLE cycles to ||Bx||_2/||x||_2 <= 1e-8 (Section 5.1) at the tables' settings
    (coarsest 5 x 5, 6 test vectors U[1, 2]) with a small ridge: the same cycle count
    (+-1) and the same state vector as the oracle."""
    ch = grid_walk(33) if kind == "grid" else tandem_queue(32)
    rp, ci, v = _dev(ch)
    x, st, _ = _bamg().mle_solve(rp, ci, v, 6, 30, 1e-8, max_cycles=40, norm="l2", grid=ch.grid, precision="fp64",
                                 coarse_max=25, ridge=1e-12, mu=mu)
    o = ob.Opts(coarse_max=25, ridge=1e-12, mu=mu)
    xo, sto = ob.mle_solve(ch.to_scipy(), 6, 30, 1e-8, o, grid=ch.grid, max_cycles=40)
    assert sto["converged"] and st["status"] == 0
    if kind == "grid":
        # the grid walk's spectrum has double eigenvalues (x/y symmetry): the coarsest
        # eigenvector basis of such an eigenspace is not unique, and the two sides pick
        # different bases, so only the cycle count's size is compared
        assert st["iterations"] <= 1.5 * sto["cycles"] + 1, (st["iterations"], sto["cycles"])
    else:
        assert abs(st["iterations"] - sto["cycles"]) <= 1, (st["iterations"], sto["cycles"])
    assert rel(x.cpu().numpy(), xo) < 1e-6  # both at the MLE's own accuracy (2-norm ratio 1e-8)
    assert rel(x.cpu().numpy(), exact.exact_stationary(ch)) < 1e-5


def test_mle_then_pgmres_on_the_kept_hierarchy():
    """The MLE's hierarchy handed back for pGMRES (the alternation of Section 4.1): a
    non-converged MLE (2 cycles) followed by FGMRES on its rebuilt hierarchy reaches the
    exact vector."""
    ch = grid_walk(33)
    rp, ci, v = _dev(ch)
    x, st, s = _bamg().mle_solve(rp, ci, v, 6, 30, 1e-12, max_cycles=2, keep=True, grid=ch.grid, precision="fp64")
    assert st["status"] == _bamg()._capi.BAMG_ENOCONV and st["iterations"] == 2
    x2, st2 = s.solve(1e-13)
    assert rel(x2.cpu().numpy(), exact.exact_stationary(ch)) < 1e-9


# ------------------------------------------------------------------ MLE restart and long restarts
@pytest.mark.parametrize("precision,bound", [("fp64", 1e-8), ("mixed", 1e-6)])
def test_mle_restarts_match_oracle(precision, bound):
    """Restart cycles of 3 steps force MLE restarts: the GPU restarts as often as the oracle
    (+-1), reaches the tolerance and the exact vector."""
    ch = grid_walk(33)
    rp, ci, v = _dev(ch)
    s = _bamg().Solver(rp, ci, v, r=6, levels=10, grid=ch.grid, precision=precision, gmres_m=3, max_it=300,
                       tv_lo=0.0, tv_hi=1.0)
    x, st = s.solve(1e-12)
    H = ob.setup(ch.to_scipy(), 6, 10, ob.Opts(gmres_m=3, max_it=300, tv_lo=0.0, tv_hi=1.0), grid=ch.grid)
    xo, sto = ob.solve(H, 1e-12)
    assert st["mle_restarts"] >= 1 and st["mle_restarts"] == st["restarts"]
    if precision == "fp64":
        assert abs(st["mle_restarts"] - sto["mle_restarts"]) <= 1
        assert abs(st["iterations"] - sto["iterations"]) <= 3
    assert rel(x.cpu().numpy(), exact.exact_stationary(ch)) < bound


def test_plain_restarts_without_mle_restart_still_converge():
    ch = grid_walk(33)
    rp, ci, v = _dev(ch)
    s = _bamg().Solver(rp, ci, v, r=6, levels=10, grid=ch.grid, precision="fp64", gmres_m=3, max_it=400,
                       mle_restart=0, tv_lo=0.0, tv_hi=1.0)
    x, st = s.solve(1e-12)
    assert st["mle_restarts"] == 0 and st["restarts"] >= 1
    assert rel(x.cpu().numpy(), exact.exact_stationary(ch)) < 1e-8


def test_restart_length_beyond_64_matches_oracle():
    """A birth-death chain with metastable wells needs a long Krylov memory (95 steps in one
    cycle here): on the same (imported) hierarchy, restart length 200 (above the old cap of
    64) gives the oracle's iteration count and vector."""
    ch = random_birth_death(14000, 4)
    H = ob.setup(ch.to_scipy(), 8, 30, ob.Opts(gmres_m=200, max_it=200, ridge=1e-10), grid=ch.grid)
    xo, sto = ob.solve(H, 1e-10)
    assert sto["converged"] and sto["iterations"] > 64 and sto["restarts"] == 0
    s = _bamg().import_hierarchy(_levels_of(H), H.pinv, H.x_init, gmres_m=200, max_it=200)
    x, st = s.solve(1e-10)
    assert st["residual_l1"] <= 1e-10 and st["restarts"] == 0
    assert abs(st["iterations"] - sto["iterations"]) <= 1, (st["iterations"], sto["iterations"])


def test_l2_stopping_rule_matches_oracle():
    ch = tandem_queue(32)
    rp, ci, v = _dev(ch)
    o = dict(coarse_max=25)
    s = _bamg().Solver(rp, ci, v, r=6, levels=30, grid=ch.grid, precision="fp64", **o)
    x, st = s.solve(1e-8, norm="l2")
    H = ob.setup(ch.to_scipy(), 6, 30, ob.Opts(**o), grid=ch.grid)
    xo, sto = ob.solve(H, 1e-8, norm="l2")
    assert abs(st["iterations"] - sto["iterations"]) <= 1
    xn = x.cpu().numpy()
    B = ob.system_matrix(ch.to_scipy())
    assert np.linalg.norm(B @ xn) / np.linalg.norm(xn) <= 1e-8


# ------------------------------------------------------------------ pArnoldi
def test_parnoldi_on_the_oracle_hierarchy_matches_oracle():
    """The same hierarchy (imported) on both sides: the same iteration count and Ritz
    vector as the oracle's Arnoldi (numpy eig on H_k there, inverse iteration here)."""
    ch = tandem_queue(30)
    H = ob.setup(ch.to_scipy(), 8, 10, ob.Opts(), grid=ch.grid)
    s = _bamg().import_hierarchy(_levels_of(H), H.pinv, H.x_init)
    x, st = s.parnoldi(1e-12)
    xo, sto = ob.parnoldi(H, 1e-12, m=50)
    assert st["residual_l1"] <= 1e-12
    assert abs(st["iterations"] - sto["iterations"]) <= 1
    assert rel(x.cpu().numpy(), xo) < 1e-10
    # a fixed number of steps: the Ritz vectors after 1..4 steps agree as well
    import torch

    for k in (1, 2, 3, 4):
        stk = None
        s2 = _bamg().import_hierarchy(_levels_of(H), H.pinv, H.x_init, gmres_m=k, max_it=k)
        out = torch.empty(ch.n, dtype=torch.float64, device="cuda")
        with pytest.raises(_bamg().BamgError) as e:
            s2.parnoldi(0.0, out=out)
        stk = e.value.stats
        xk = out.cpu().numpy()
        xok, _ = ob.parnoldi(H, 0.0, m=k, max_it=k)
        assert stk["iterations"] == k
        assert rel(xk, xok) < 1e-9, k


@pytest.mark.parametrize("precision,bound", [("fp64", 1e-9), ("mixed", 1e-6)])
@pytest.mark.parametrize("kind", ["grid33", "tandem40"])
def test_parnoldi_full_path_reaches_exact(kind, precision, bound):
    ch = grid_walk(33) if kind == "grid33" else tandem_queue(40)
    rp, ci, v = _dev(ch)
    s = _bamg().Solver(rp, ci, v, r=8, levels=10, grid=ch.grid, precision=precision, tv_lo=0.0, tv_hi=1.0)
    x, st = s.parnoldi(1e-12)
    xn = x.cpu().numpy()
    assert rel(xn, exact.exact_stationary(ch)) < bound
    assert abs(xn.sum() - 1.0) < 1e-13
    assert ob.l1_ratio(ob.system_matrix(ch.to_scipy()), xn) <= 2e-12


# ------------------------------------------------------------------ multicolour Gauss-Seidel
@pytest.mark.parametrize("precision,bound", [("fp64", 1e-9), ("mixed", 1e-6)])
def test_mcgs_vcycle_on_the_oracle_hierarchy(precision, bound):
    """The same hierarchy (imported) and the same colouring rule on both sides: the GPU's
    Gauss-Seidel V-cycle equals the oracle's on random right-hand sides."""
    import torch

    ch = tandem_queue(40)
    H = ob.setup(ch.to_scipy(), 8, 10, ob.Opts(smoother="mcgs"), grid=ch.grid)
    s = _bamg().import_hierarchy(_levels_of(H), H.pinv, H.x_init, smoother="mcgs",
                                 precision=precision)
    rng = np.random.default_rng(11)
    for _ in range(3):
        v = rng.standard_normal(ch.n)
        z = s.vcycle(torch.tensor(v, device="cuda")).cpu().numpy()
        assert rel(z, ob.vcycle(H, v)) < bound


@pytest.mark.parametrize("precision,bound", [("fp64", 1e-9), ("mixed", 1e-6)])
@pytest.mark.parametrize("kind", ["grid33", "tandem40", "delaunay"])
def test_mcgs_full_path_matches_oracle(kind, precision, bound):
    from workloads import delaunay_walk

    if kind == "grid33":
        ch, kw = grid_walk(33), {}
    elif kind == "tandem40":
        ch, kw = tandem_queue(40), {}
    else:
        ch, kw = delaunay_walk(3000, 2), {"coarsen": "cr"}
    rp, ci, v = _dev(ch)
    s = _bamg().Solver(rp, ci, v, r=8, levels=10, grid=ch.grid, precision=precision, smoother="mcgs", tv_lo=0.0,
                       tv_hi=1.0, **kw)
    x, st = s.solve(1e-12)
    xn = x.cpu().numpy()
    assert rel(xn, exact.exact_stationary(ch)) < bound
    if precision == "fp64" and kind != "delaunay":  # compatible relaxation may split a few points differently
        xo, H, sto = ob.stationary(ch.to_scipy(), 8, 10, 1e-12, ob.Opts(smoother="mcgs", tv_lo=0.0, tv_hi=1.0, **kw),
                                   grid=ch.grid)
        assert abs(st["iterations"] - sto["iterations"]) <= 1
        assert rel(xn, xo) < 1e-9

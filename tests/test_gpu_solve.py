"""Parity of the solve phase and of the whole path with the CPU oracle and the exact
stationary vectors.  FP64 runs must agree to relative L1 1e-8, mixed runs to 1e-6."""

import numpy as np
import pytest
import scipy.sparse as sp

from gpu_util import need_gpu, rel
from oracle import bamg as ob
from oracle import exact
from workloads import delaunay_walk, grid_walk, random_birth_death, tandem_queue

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _gpu():
    need_gpu()


def _torch():
    import torch

    return torch


def _bamg():
    import paper_1004_1451_gb300 as bamg

    return bamg


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


@pytest.fixture(scope="module")
def oracle_H():
    ch = tandem_queue(40)
    H = ob.setup(ch.to_scipy(), 8, 10, ob.Opts(), grid=ch.grid)
    return ch, H


def test_vcycle_matches_oracle(oracle_H):
    torch = _torch()
    ch, H = oracle_H
    s = _bamg().import_hierarchy(_levels_of(H), H.pinv, H.x_init)
    rng = np.random.default_rng(4)
    for _ in range(3):
        v = rng.standard_normal(ch.n)
        v -= v.mean()
        z = s.vcycle(torch.tensor(v, device="cuda")).cpu().numpy()
        assert rel(z, ob.vcycle(H, v)) < 1e-12


def test_vcycle_mixed_close_to_oracle(oracle_H):
    torch = _torch()
    ch, H = oracle_H
    s = _bamg().import_hierarchy(_levels_of(H), H.pinv, H.x_init, precision="mixed")
    v = np.random.default_rng(5).standard_normal(ch.n)
    z = s.vcycle(torch.tensor(v, device="cuda")).cpu().numpy()
    assert rel(z, ob.vcycle(H, v)) < 1e-5


@pytest.fixture(scope="module")
def oracle_H_cr():
    # compatible-relaxation hierarchy whose coarse levels have long rows (16-26 entries on
    # average) and are too large for the single-block tail: the V-cycle runs them with the
    # group-per-row kernels
    ch = delaunay_walk(40000, 3)
    H = ob.setup(ch.to_scipy(), 8, 12, ob.Opts(coarsen="cr"))
    return ch, H


@pytest.mark.parametrize("precision,bound", [("fp64", 1e-12), ("mixed", 1e-5)])
def test_vcycle_long_rows_matches_oracle(oracle_H_cr, precision, bound):
    torch = _torch()
    ch, H = oracle_H_cr
    grouped = [l for l, lv in enumerate(H.levels[:-1])
               if lv.B.nnz >= 12 * lv.B.shape[0] and (lv.B.shape[0] > 1024 or lv.B.nnz > 16384)]
    assert grouped, "no level takes the group-per-row kernels"
    s = _bamg().import_hierarchy(_levels_of(H), H.pinv, H.x_init, precision=precision)
    rng = np.random.default_rng(6)
    for _ in range(2):
        v = rng.standard_normal(ch.n)
        v -= v.mean()
        z = s.vcycle(torch.tensor(v, device="cuda")).cpu().numpy()
        assert rel(z, ob.vcycle(H, v)) < bound


def test_fgmres_matches_oracle(oracle_H):
    ch, H = oracle_H
    s = _bamg().import_hierarchy(_levels_of(H), H.pinv, H.x_init)
    x, st = s.solve(1e-13)
    xo, sto = ob.solve(H, 1e-13)
    assert st["residual_l1"] <= 1e-13
    assert abs(st["iterations"] - sto["iterations"]) <= 1
    assert rel(x.cpu().numpy(), xo) < 1e-10
    assert rel(x.cpu().numpy(), exact.exact_stationary(ch)) < 1e-9


def _run(ch, r, levels, tol, precision, **kw):
    torch = _torch()
    rp = torch.tensor(ch.row_ptr, device="cuda")
    ci = torch.tensor(ch.col, device="cuda")
    v = torch.tensor(ch.val, device="cuda")
    s = _bamg().Solver(rp, ci, v, r=r, levels=levels, grid=ch.grid, precision=precision, **kw)
    x, st = s.solve(tol)
    return s, x.cpu().numpy(), st


@pytest.mark.parametrize("precision,bound", [("fp64", 1e-9), ("mixed", 1e-6)])
@pytest.mark.parametrize("kind", ["grid33", "tandem32", "bd700", "grid_rect"])
def test_full_path_reaches_exact(kind, precision, bound):
    if kind == "grid33":
        ch, r = grid_walk(33), 8
    elif kind == "tandem32":
        ch, r = tandem_queue(32), 10
    elif kind == "grid_rect":
        ch, r = grid_walk(45, 19), 6
    else:
        ch, r = random_birth_death(700, 2), 6
    s, x, st = _run(ch, r, 12, 1e-13 if precision == "fp64" else 1e-12, precision, tv_lo=0.0, tv_hi=1.0)
    xe = exact.exact_stationary(ch)
    assert rel(x, xe) < bound, (rel(x, xe), st)
    assert abs(x.sum() - 1.0) < 1e-13
    assert np.all(x >= -1e-14 * x.max())
    B = ob.system_matrix(ch.to_scipy())
    assert ob.l1_ratio(B, x) <= 2e-12


def test_full_path_agrees_with_oracle_run():
    ch = grid_walk(40, 24)
    s, x, st = _run(ch, 8, 10, 1e-13, "fp64", tv_lo=0.0, tv_hi=1.0)
    xo, H, sto = ob.stationary(ch.to_scipy(), 8, 10, 1e-13, ob.Opts(tv_lo=0.0, tv_hi=1.0), grid=ch.grid)
    assert rel(x, xo) < 1e-9
    info = s.info()
    assert info["n"] == [lv.B.shape[0] for lv in H.levels]
    # same hierarchy sizes and nearly the same iteration count
    assert abs(st["iterations"] - sto["iterations"]) <= 2


def test_hierarchy_invariants():
    ch = tandem_queue(48)
    s, x, st = _run(ch, 10, 12, 1e-12, "fp64")
    bamg = _bamg()
    info = s.info()
    for l in range(info["levels"]):
        rp, ci, v = s.export(l, bamg._capi.EXPORT_B)
        n = len(rp) - 1
        B = sp.csr_matrix((v, ci, rp), shape=(n, n))
        cs = np.abs(np.asarray(B.sum(axis=0)).ravel()).max()
        assert cs <= 1e-12 * np.abs(v).max(), (l, cs)  # 1^T B_l = 0 (Section 4)
        if l + 1 < info["levels"]:
            pcol, pval, pcnt = s.export(l, bamg._capi.EXPORT_P)
            cf = s.export(l, bamg._capi.EXPORT_CF)
            assert np.all(pcnt[cf] == 1) and np.all(pval[cf, 0] == 1.0)
            assert np.all(pcnt <= 2)
    pinv = s.export(info["levels"] - 1, bamg._capi.EXPORT_PINV)
    rp, ci, v = s.export(info["levels"] - 1, bamg._capi.EXPORT_B)
    BL = sp.csr_matrix((v, ci, rp)).toarray()
    assert np.allclose(BL @ pinv @ BL, BL, atol=1e-10 * np.abs(BL).max())
    assert np.allclose(pinv @ BL @ pinv, pinv, atol=1e-8 * np.abs(pinv).max())


def test_config1_grid64_fp64():
    # 64 x 64 grid walk, r = 8 test vectors U(0,1), 3 coarsenings to 64 states, FP64
    ch = grid_walk(64)
    s, x, st = _run(ch, 8, 3, 1e-13, "fp64", tv_lo=0.0, tv_hi=1.0)
    assert s.info()["n"] == [4096, 1024, 256, 64]
    assert rel(x, exact.exact_stationary(ch)) < 1e-8


def test_config2_tandem256_mixed():
    # tandem queue, capacities 255 (65,536 states), r = 10, FP32 V-cycle inside FP64 GMRES
    ch = tandem_queue(255)
    s, x, st = _run(ch, 10, 20, 1e-13, "mixed")
    xe = exact.sparse_nullspace(ch.to_scipy())
    assert st["residual_l1"] <= 1e-13
    assert rel(x, xe) < 1e-6, rel(x, xe)


def test_host_buffers_round_trip():
    torch = _torch()
    ch = grid_walk(30)
    rp = torch.tensor(ch.row_ptr)
    ci = torch.tensor(ch.col)
    v = torch.tensor(ch.val)
    s = _bamg().Solver(rp, ci, v, r=6, levels=6, grid=ch.grid, on_host=True)
    x, st = s.solve(1e-12, host=True)
    assert x.device.type == "cpu"
    assert rel(x.numpy(), exact.exact_stationary(ch)) < 1e-9


def test_initial_guess_flag():
    torch = _torch()
    ch = grid_walk(21)
    xe = exact.exact_stationary(ch)
    s, x, st = _run(ch, 6, 6, 1e-12, "fp64")
    x2, st2 = s.solve(1e-12, x0=torch.tensor(xe, device="cuda"))
    assert st2["iterations"] == 0 and rel(x2.cpu().numpy(), xe) < 1e-14


def test_rejects_bad_input():
    torch = _torch()
    bamg = _bamg()
    ch = grid_walk(10)
    val = ch.val.copy()
    val[3] *= 1.5
    args = (torch.tensor(ch.row_ptr, device="cuda"), torch.tensor(ch.col, device="cuda"))
    with pytest.raises(bamg.BamgError) as e:
        bamg.Solver(*args, torch.tensor(val, device="cuda"), r=6, levels=3, grid=ch.grid)
    assert e.value.code == bamg._capi.BAMG_ENOTSTOCH
    with pytest.raises(bamg.BamgError) as e:
        bamg.Solver(*args, torch.tensor(ch.val, device="cuda"), r=6, levels=3, grid=(9, 10))
    assert e.value.code == bamg._capi.BAMG_EINVAL
    with pytest.raises(bamg.BamgError) as e:
        bamg.Solver(*args, torch.tensor(ch.val, device="cuda"), r=40, levels=3, grid=ch.grid)
    assert e.value.code == bamg._capi.BAMG_EINVAL
    with pytest.raises(bamg.BamgError) as e:  # too few levels for a 64-state coarsest grid
        bamg.Solver(*args, torch.tensor(ch.val, device="cuda"), r=6, levels=0, grid=ch.grid)
    assert e.value.code == bamg._capi.BAMG_EINVAL


def test_nonconvergence_reports_enoconv():
    bamg = _bamg()
    ch = grid_walk(40)
    with pytest.raises(bamg.BamgError) as e:
        _run(ch, 6, 8, 1e-15, "fp64", max_it=2)
    assert e.value.code == bamg._capi.BAMG_ENOCONV
    assert e.value.stats["iterations"] == 2


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_device_loop_gives_the_same_iterates(precision):
    # the Arnoldi steps looping on the device (graph WHILE node) and one launch per step
    # run the same arithmetic and take the same decisions: bit-identical results; a short
    # restart length exercises restarts and the end-of-cycle exit
    ch = tandem_queue(63)
    runs = [_run(ch, 10, 10, 1e-12, precision, gmres_m=6, device_loop=d, persistent=0) for d in (0, 1)]
    (_, x0, st0), (_, x1, st1) = runs
    assert np.array_equal(x0, x1)
    for k in ("iterations", "restarts", "true_checks", "residual_l1"):
        assert st0[k] == st1[k], k
    assert st0["restarts"] >= 1
    assert st0["host_waits"] == st0["iterations"]
    assert st1["host_waits"] == st1["true_checks"] < st1["iterations"]


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
@pytest.mark.parametrize("kind,m", [("tandem63", 6), ("tandem63", 50), ("grid8", 50), ("bd3000", 60),
                                     ("grid_rect", 50)])
def test_persistent_cycle_gives_the_same_iterates(kind, m, precision):
    """The Arnoldi steps in one cooperative launch with grid barriers (persistent=1) and the
    captured step (one graph launch per step) give bit-identical iterates: with a coarse
    tail (tandem, birth-death) and with the dense coarsest level as the only level (8 x 8
    grid), with and without restarts; the persistent form launches far fewer kernels."""
    bamg = _bamg()
    if kind == "tandem63":
        ch, kw = tandem_queue(63), {}
    elif kind == "grid8":
        ch, kw = grid_walk(8), {}
    elif kind == "grid_rect":
        ch, kw = grid_walk(45, 19), {}
    else:
        ch, kw = random_birth_death(3000, 9), dict(ridge=1e-10)
    l0 = bamg.launch_count()
    _, xg, stg = _run(ch, 8, 20, 1e-12, precision, gmres_m=m, device_loop=0, persistent=0, **kw)
    l1 = bamg.launch_count()
    _, xp, stp = _run(ch, 8, 20, 1e-12, precision, gmres_m=m, persistent=1, **kw)
    l2 = bamg.launch_count()
    assert np.array_equal(xg, xp)
    for k in ("iterations", "restarts", "true_checks", "residual_l1"):
        assert stg[k] == stp[k], k
    assert stp["host_waits"] == stp["true_checks"]
    if stg["iterations"] >= 4:
        assert (l2 - l1) < (l1 - l0), (l1 - l0, l2 - l1)


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
@pytest.mark.parametrize("kind", ["tandem127", "grid97", "bd3000", "tandem383"])
def test_cluster_tail_gives_the_same_iterates(kind, precision):
    """The coarse end of the V-cycle on a cluster of 8 thread blocks (coarse_tail=0: every
    level from the first one with at most 4096 rows in one launch; each block owns a slice
    of every level's rows and sends its values to the others through distributed shared
    memory) and in one block (coarse_tail=1: from the first level with at most 1024 rows,
    the levels above on the grid kernels) give bit-identical iterates and V-cycle outputs:
    one thread per row in the grid kernels' order of operations, on these short-row
    hierarchies.  The grid walk's levels (2401, 625, 169, 49 states) and the birth-death
    chain's split unevenly over the blocks; the 384 x 384 tandem queue (147,456 states)
    has two grid levels above the cluster."""
    torch = _torch()
    if kind == "tandem127":
        ch, kw = tandem_queue(127), {}
    elif kind == "tandem383":
        ch, kw = tandem_queue(383), {}
    elif kind == "grid97":
        ch, kw = grid_walk(97), {}
    else:
        ch, kw = random_birth_death(3000, 9), dict(ridge=1e-10)
    s1, x1, st1 = _run(ch, 8, 20, 1e-12, precision, coarse_tail=1, **kw)
    s0, x0, st0 = _run(ch, 8, 20, 1e-12, precision, coarse_tail=0, **kw)
    assert np.array_equal(x0, x1)
    for k in ("iterations", "restarts", "true_checks", "residual_l1"):
        assert st0[k] == st1[k], k
    v = torch.tensor(np.random.default_rng(3).standard_normal(ch.n), device="cuda")
    assert torch.equal(s0.vcycle(v), s1.vcycle(v))


def test_device_loop_stops_at_max_it():
    bamg = _bamg()
    ch = grid_walk(40)
    with pytest.raises(bamg.BamgError) as e:
        _run(ch, 6, 8, 1e-15, "fp64", max_it=3, device_loop=1)
    assert e.value.code == bamg._capi.BAMG_ENOCONV
    assert e.value.stats["iterations"] == 3 and e.value.stats["host_waits"] == 1


def test_delaunay_cr_fp64():
    ch = delaunay_walk(5000, 3)
    s, x, st = _run(ch, 8, 12, 1e-13, "fp64", coarsen="cr")
    assert rel(x, exact.exact_stationary(ch)) < 1e-8
    xo, H, sto = ob.stationary(ch.to_scipy(), 8, 12, 1e-13, ob.Opts(coarsen="cr"))
    assert rel(x, xo) < 1e-8


def test_config3_delaunay_2e20_mixed():
    # Delaunay triangulation of 2^20 points U[0,1]^2, walk with probability 1/deg, r = 16,
    # FP32 setup and V-cycle inside FP64 GMRES, compatible-relaxation coarsening
    ch = delaunay_walk(1 << 20, 0)
    s, x, st = _run(ch, 16, 20, 1e-12, "mixed", coarsen="cr")
    info = s.info()
    assert info["n"][-1] <= 64
    assert rel(x, exact.exact_stationary(ch)) < 1e-6
    print("delaunay 2^20:", info["n"], st)


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_smooth_apply_matches_eq44_smoother(precision):
    # three sweeps x <- x + omega D^{-1} (b - B x) of the V-cycle smoother (Eq. (4.4)) on
    # levels 0 and 1, against the same sweeps on the exported level matrix
    torch = _torch()
    bamg = _bamg()
    ch = tandem_queue(40)
    s, _, _ = _run(ch, 8, 10, 1e-10, precision)
    dt = s.dtype
    assert dt == (torch.float32 if precision == "mixed" else torch.float64)
    rng = np.random.default_rng(11)
    for level in (0, 1):
        rp, ci, v = s.export(level, bamg._capi.EXPORT_B)
        n = len(rp) - 1
        B = sp.csr_matrix((v, ci, rp), shape=(n, n))
        b = rng.standard_normal(n)
        x0 = rng.standard_normal(n)
        xg = torch.tensor(x0, dtype=dt, device="cuda")
        s.smooth(level, torch.tensor(b, dtype=dt, device="cuda"), xg, sweeps=3)
        torch.cuda.synchronize()
        dinv = 1.0 / B.diagonal()
        x = x0.copy()
        for _ in range(3):
            x = x + 0.7 * dinv * (b - B @ x)
        assert rel(xg.cpu().double().numpy(), x) < (1e-12 if precision == "fp64" else 1e-5)

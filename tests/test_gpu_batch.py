"""Batched form: many independent chains set up and solved concurrently through
bamg_solve_batch, each checked against its exact stationary vector."""

import numpy as np
import pytest

from gpu_util import need_gpu, rel
from oracle import bamg as ob
from oracle import exact
from workloads import batched_mixture, grid_walk, random_birth_death, tandem_queue

pytestmark = pytest.mark.gpu

# Birth-death chains with i.i.d. per-state rates have stationary vectors spanning many
# orders of magnitude; their LS fits need a small ridge (the default suits 2-D chains).
BD_OPTS = dict(ridge=1e-10, ridge32=1e-6)


@pytest.fixture(scope="module", autouse=True)
def _gpu():
    need_gpu()


def _dev(chains, device="cuda"):
    import torch

    return [(torch.tensor(c.row_ptr, device=device), torch.tensor(c.col, device=device),
             torch.tensor(c.val, device=device)) for c in chains]


def _opts(chains, **kw):
    return [dict(grid=c.grid, **kw, **(BD_OPTS if c.kind == "birth_death" else {})) for c in chains]


def _error_bound(c, xe, bound, ratio):
    """bound, widened for an ill-conditioned chain: with x and x* both summing to one,
    x - x* = (I - x* 1^T) B^+ B x, so ||x - x*||_1 <= ||(I - x* 1^T) B^+||_1 ||B x||_1."""
    if c.kind != "birth_death":
        return bound
    B = ob.system_matrix(c.to_scipy()).toarray()
    K = np.abs((np.eye(c.n) - np.outer(xe, np.ones(c.n))) @ np.linalg.pinv(B)).sum(axis=0).max()
    return max(bound, 2.0 * K * ratio)


@pytest.mark.parametrize("precision,bound", [("fp64", 1e-8), ("mixed", 1e-6)])
def test_small_mixture_matches_exact(precision, bound):
    import paper_1004_1451_gb300 as bamg

    chains = batched_mixture(7, nchains=12, bd_lo=200, bd_hi=1000, side_lo=12, side_hi=40)
    chains.append(tandem_queue(30))
    xs, stats = bamg.solve_batch(_dev(chains), 8, 20, 1e-12, opts=_opts(chains, precision=precision), workers=4)
    for c, x, st in zip(chains, xs, stats):
        x = x.cpu().numpy()
        assert st["status"] == 0 and st["residual_l1"] <= 1e-12
        xe = exact.exact_stationary(c)
        assert rel(x, xe) < _error_bound(c, xe, bound, st["residual_l1"]), (c.kind, c.n, st)
        assert abs(x.sum() - 1.0) < 1e-12


def test_batch_equals_single_solves():
    """Each chain's result does not depend on the batch around it: same iteration count and
    the same vector as a lone bamg_setup/bamg_solve with the same options."""
    import paper_1004_1451_gb300 as bamg

    chains = [grid_walk(33), random_birth_death(1500, 4), grid_walk(20, 31), tandem_queue(24)]
    mats = _dev(chains)
    opts = _opts(chains)
    xs, stats = bamg.solve_batch(mats, 6, 12, 1e-13, opts=opts, workers=3)
    for c, m, x, st, o in zip(chains, mats, xs, stats, opts):
        s = bamg.Solver(*m, r=6, levels=12, **o)
        x1, st1 = s.solve(1e-13)
        assert st["iterations"] == st1["iterations"]
        assert rel(x.cpu().numpy(), x1.cpu().numpy()) < 1e-14


def test_host_buffers_and_one_worker():
    import paper_1004_1451_gb300 as bamg

    chains = [grid_walk(25), random_birth_death(600, 1)]
    xs, stats = bamg.solve_batch(_dev(chains, "cpu"), 6, 10, 1e-12, opts=_opts(chains), workers=1, host=True)
    for c, x, st in zip(chains, xs, stats):
        assert x.device.type == "cpu"
        xe = exact.exact_stationary(c)
        assert rel(x.numpy(), xe) < _error_bound(c, xe, 1e-9, st["residual_l1"])


def test_failing_chain_reports_and_others_finish():
    import paper_1004_1451_gb300 as bamg

    good = [grid_walk(18), grid_walk(22)]
    bad = grid_walk(15)
    bad.val = bad.val.copy()
    bad.val[5] *= 1.5  # column sum no longer one
    chains = [good[0], bad, good[1]]
    with pytest.raises(bamg.BamgError) as e:
        bamg.solve_batch(_dev(chains), 6, 8, 1e-12, opts=[dict(grid=c.grid) for c in chains], workers=2)
    assert e.value.code == bamg._capi.BAMG_ENOTSTOCH
    assert "chain 1" in str(e.value)
    st = e.value.stats
    assert st[1]["status"] == bamg._capi.BAMG_ENOTSTOCH
    assert st[0]["status"] == 0 and st[2]["status"] == 0


def test_empty_batch():
    import paper_1004_1451_gb300 as bamg

    xs, stats = bamg.solve_batch([], 6, 8, 1e-12)
    assert xs == [] and stats == []


def test_batch_results_agree_with_oracle_residual():
    """Mixed batch on a mixture drawn like the 512-chain workload but smaller: every x
    satisfies the stopping rule when its residual is recomputed in FP64 on the host."""
    import paper_1004_1451_gb300 as bamg

    chains = batched_mixture(0, nchains=16, bd_lo=1024, bd_hi=8192, side_lo=32, side_hi=64)
    xs, stats = bamg.solve_batch(_dev(chains), 8, 20, 1e-10, opts=_opts(chains, precision="mixed"))
    for c, x in zip(chains, xs):
        x = x.cpu().numpy()
        assert ob.l1_ratio(ob.system_matrix(c.to_scipy()), x) <= 1e-10 * 1.01
        assert abs(x.sum() - 1.0) < 1e-12
        if c.kind != "birth_death":  # well conditioned: the residual bound keeps x >= 0
            assert np.all(x >= -1e-12 * x.max())


# The options the 512-chain workload runs with: birth-death chains in FP64 (their
# stationary vectors span more decades than FP32's exponent range), restart length 256
# and MLE restarts; grid walks in mixed precision.
BD_BATCH = dict(ridge=1e-10, gmres_m=256, max_it=3000, precision="fp64")


def _batch_opts(chains):
    return [dict(grid=c.grid, **(BD_BATCH if c.kind == "birth_death" else dict(precision="mixed"))) for c in chains]


def test_workload_draw_with_large_birth_death_chains():
    """The first 64 chains of the 512-chain workload (12 birth-death chains with n >= 16k).
    Grid walks: x proportional to degree within 1e-6 (mixed).  Birth-death chains: the
    residual of every converged x, recomputed in FP64 on the host, meets 1e-10, and every x
    lies within the rigorous bound K ||B x||_1 of the product form (K from detailed balance:
    the bound holds at any size but says little where K is astronomically large, which is
    what the next test is for); at most one in ten may stop at max_it."""
    import paper_1004_1451_gb300 as bamg

    chains = batched_mixture(0)[:64]
    assert sum(c.kind == "birth_death" and c.n >= 16384 for c in chains) >= 10
    try:
        xs, stats = bamg.solve_batch(_dev(chains), 8, 30, 1e-10, opts=_batch_opts(chains), workers=8)
    except bamg.BamgError as e:
        xs, stats = e.xs, e.stats
    nbd = conv = 0
    for c, x, st in zip(chains, xs, stats):
        x = x.cpu().numpy()
        xe = exact.exact_stationary(c)
        if c.kind != "birth_death":
            assert st["status"] == 0
            assert rel(x, xe) < 1e-6
            continue
        nbd += 1
        if st["status"] != 0:  # stopped at max_it: x holds the last iterate
            assert st["status"] == bamg._capi.BAMG_ENOCONV, (c.n, st)
            continue
        conv += 1
        assert abs(x.sum() - 1.0) < 1e-12
        r1 = float(np.abs(ob.system_matrix(c.to_scipy()) @ x).sum())
        assert r1 / np.abs(x).sum() <= 1e-10 * 1.01
        K = 10 ** exact.birth_death_condition(c.meta["birth"], c.meta["death"])
        assert np.abs(x - xe).sum() <= K * r1 * (1 + 1e-6) + 1e-14
    assert conv >= 0.9 * nbd, (conv, nbd)


def test_best_conditioned_birth_death_chains_at_parity_tolerance():
    """The four birth-death chains of the 512-chain workload with the smallest bound K
    (about 1e6-1e6.4) solved to 1e-13 (the parity tolerance), where K ||B x||_1 <= 1e-6:
    each x is within 1e-6 of the product form."""
    import paper_1004_1451_gb300 as bamg

    mix = batched_mixture(0)
    chains = [mix[i] for i in (340, 504, 20, 108)]
    xs, stats = bamg.solve_batch(_dev(chains), 8, 30, 1e-13, opts=_batch_opts(chains), workers=4)
    for c, x, st in zip(chains, xs, stats):
        x = x.cpu().numpy()
        K = 10 ** exact.birth_death_condition(c.meta["birth"], c.meta["death"])
        r1 = float(np.abs(ob.system_matrix(c.to_scipy()) @ x).sum())
        err = np.abs(x - exact.exact_stationary(c)).sum()
        assert K * r1 <= 1e-6 and err <= K * r1 * (1 + 1e-6) + 1e-14, (c.n, K, r1, err)
        assert err < 1e-6

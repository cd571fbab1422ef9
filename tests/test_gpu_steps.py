"""Parity of each setup step (CUDA, through the C ABI) with the CPU oracle on the same
seeded inputs.  Sizes span several thread blocks and end in a ragged tail."""

import numpy as np
import pytest
import scipy.sparse as sp

from gpu_util import dev_csr, ell_from_csr, need_gpu, on_pattern, rel
from oracle import bamg as ob
from workloads import delaunay_walk, grid_walk, tandem_queue

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


# ------------------------------------------------------------------ test vectors
@pytest.mark.parametrize("n,K,ld,col0", [(1000, 6, 8, 0), (4097, 10, 20, 4), (0, 3, 4, 0)])
def test_tv_init_bit_exact(n, K, ld, col0):
    torch = _torch()
    X = torch.zeros(n, ld, dtype=torch.float64, device="cuda")
    _bamg().tv_init(X, K, col0, 1234567, 0.25, 1.75)
    want = ob.tv_init(n, K, 1234567, 0.25, 1.75)
    got = X.cpu().numpy()
    assert np.array_equal(got[:, col0:col0 + K], want)
    if n:
        assert np.all(got[:, :col0] == 0) and np.all(got[:, col0 + K:] == 0)
    X32 = torch.zeros(n, ld, dtype=torch.float32, device="cuda")
    _bamg().tv_init(X32, K, col0, 1234567, 0.25, 1.75)
    assert np.array_equal(X32.cpu().numpy()[:, col0:col0 + K], want.astype(np.float32))


# ------------------------------------------------------------------ relaxation
def _tandem_B(N=32):
    ch = tandem_queue(N)
    return ch, ob.system_matrix(ch.to_scipy())


@pytest.mark.parametrize("dtype_name,r,ld,nu", [("float64", 6, 6, 3), ("float64", 8, 10, 4), ("float32", 10, 12, 4),
                                                 ("float32", 16, 16, 1)])
def test_relax_matches_oracle(dtype_name, r, ld, nu):
    torch = _torch()
    dt = getattr(torch, dtype_name)
    ch, B = _tandem_B(40)
    X0 = ob.tv_init(ch.n, r, 7, 0.0, 1.0)
    want = ob.jacobi(B, X0, 0.7, nu)
    X = torch.zeros(ch.n, ld, dtype=dt, device="cuda")
    X[:, :r] = torch.tensor(X0, dtype=dt)
    _bamg().relax(dev_csr(B, dt), X, r, 0, 0.7, nu)
    got = X.cpu().numpy().astype(np.float64)
    tol = 1e-13 if dt == torch.float64 else 2e-6
    assert rel(got[:, :r], want) < tol
    assert np.all(got[:, r:] == 0)


@pytest.mark.parametrize("dtype_name,shift", [("float32", False), ("float32", True), ("float64", False)])
def test_relax_large_level_matches_oracle(dtype_name, shift):
    # 360,000 rows: more rows than four per thread of the sweep's grid, so the sweep runs
    # with two 16-byte chunks per thread
    torch = _torch()
    dt = getattr(torch, dtype_name)
    ch = grid_walk(600)
    B = ob.system_matrix(ch.to_scipy())
    B.sort_indices()
    n, K, ld = ch.n, 8, 8
    assert n * (K * torch.finfo(dt).bits // 8 // 16) > 4 * 160 * 2 * 256
    rng = np.random.default_rng(8)
    V0 = rng.uniform(-1, 1, (n, K))
    X = torch.zeros(n, ld, dtype=dt, device="cuda")
    X[:, :K] = torch.tensor(V0, dtype=dt)
    if shift:
        lam = np.linspace(0.0, 0.07, K)
        want = ob.jacobi_shifted(B, sp.identity(n, format="csr"), V0, lam, 0.7, 2)
        _bamg().relax(dev_csr(B, dt), X, K, 0, 0.7, 2, lam=torch.tensor(lam, device="cuda"))
    else:
        want = ob.jacobi(B, V0, 0.7, 2)
        _bamg().relax(dev_csr(B, dt), X, K, 0, 0.7, 2)
    got = X.cpu().numpy().astype(np.float64)
    assert rel(got, want) < (1e-13 if dt == torch.float64 else 2e-6)


_AUTOTUNE_CHILD = '''
import sys, numpy as np, torch
sys.path.insert(0, sys.argv[1])
import paper_1004_1451_gb300 as bamg
from gpu_util import dev_csr
from oracle import bamg as ob
from workloads import grid_walk
ch = grid_walk(600)
B = ob.system_matrix(ch.to_scipy())
B.sort_indices()
V0 = np.random.default_rng(9).uniform(-1, 1, (ch.n, 8))
X = torch.tensor(V0, dtype=torch.float32, device="cuda")
bamg.relax(dev_csr(B, torch.float32), X, 8, 0, 0.7, 3)
np.save(sys.argv[2], X.cpu().numpy())
'''


def test_relax_autotune_same_bits(tmp_path):
    # the autotuner only changes the launch shape: the tuned sweeps write the bits of the
    # fixed rule (BAMG_AUTOTUNE=0, in a separate process), and the choice is reported
    import os
    import subprocess
    import sys

    torch = _torch()
    bamg = _bamg()
    ch = grid_walk(600)
    B = ob.system_matrix(ch.to_scipy())
    B.sort_indices()
    V0 = np.random.default_rng(9).uniform(-1, 1, (ch.n, 8))
    X = torch.tensor(V0, dtype=torch.float32, device="cuda")
    bamg.relax(dev_csr(B, torch.float32), X, 8, 0, 0.7, 3)
    got = X.cpu().numpy()
    rep = [r for r in bamg.autotune_report() if r["elem_bytes"] == 4 and r["shift"] == 0 and r["chunks_per_row"] == 2
           and r["log2_n"] == 18]
    assert len(rep) == 1 and rep[0]["chunks_per_thread"] in (1, 2) and rep[0]["blocks_per_sm"] in (1, 2, 4)
    here = os.path.dirname(os.path.abspath(__file__))
    out = tmp_path / "fixed.npy"
    env = dict(os.environ, BAMG_AUTOTUNE="0", PYTHONPATH=os.pathsep.join([os.path.dirname(here), here]))
    subprocess.run([sys.executable, "-c", _AUTOTUNE_CHILD, here, str(out)], env=env, check=True, timeout=600)
    assert np.array_equal(got, np.load(out))


@pytest.mark.parametrize("with_T", [False, True])
def test_shifted_relax_matches_oracle(with_T):
    torch = _torch()
    ch, B = _tandem_B(24)
    rng = np.random.default_rng(3)
    if with_T:
        Tm = sp.csr_matrix(B, copy=True)
        Tm.data = rng.uniform(0.0, 0.1, Tm.nnz)
        Tm = Tm + sp.identity(ch.n) * 2.0
        Tm = sp.csr_matrix(Tm)
        T_val = torch.tensor(on_pattern(B, Tm), device="cuda")
    else:
        Tm = sp.identity(ch.n, format="csr")
        T_val = None
    K, ld = 7, 8
    V0 = rng.uniform(-1, 1, (ch.n, K))
    lam = np.array([0.0, 0.01, 0.02, -0.03, 0.05, 0.05, 0.1])
    want = ob.jacobi_shifted(B, Tm, V0, lam, 0.7, 2)
    X = torch.zeros(ch.n, ld + 2, dtype=torch.float64, device="cuda")
    X[:, 2:2 + K] = torch.tensor(V0)
    _bamg().relax(dev_csr(B), X, K, 2, 0.7, 2, T_val=T_val, lam=torch.tensor(lam, device="cuda"))
    assert rel(X.cpu().numpy()[:, 2:2 + K], want) < 1e-13


@pytest.mark.parametrize("dtype_name,shift", [("float32", False), ("float32", True), ("float64", False),
                                               ("float64", True)])
def test_relax_long_rows_match_oracle(dtype_name, shift):
    # a coarse-level operator (rows of 20-40 entries) exercises the batches beyond the
    # first entries of a row; with shifts and a non-identity T as in the upward pass
    torch = _torch()
    dt = getattr(torch, dtype_name)
    ch = tandem_queue(31)
    H = ob.setup(ch.to_scipy(), 8, 3, ob.Opts(), grid=ch.grid)
    lv = H.levels[2]
    B, Tm = sp.csr_matrix(lv.B), sp.csr_matrix(lv.T)
    B.sort_indices()
    assert np.diff(B.indptr).max() > 6  # rows longer than the first batch of entries
    n = B.shape[0]
    rng = np.random.default_rng(5)
    K, ld = 6, 8
    V0 = rng.uniform(-1, 1, (n, K))
    X = torch.zeros(n, ld, dtype=dt, device="cuda")
    X[:, :K] = torch.tensor(V0, dtype=dt)
    if shift:
        lam = np.array([0.0, 0.01, 0.02, -0.03, 0.05, 0.1])
        want = ob.jacobi_shifted(B, Tm, V0, lam, 0.7, 2)
        _bamg().relax(dev_csr(B, dt), X, K, 0, 0.7, 2, T_val=torch.tensor(on_pattern(B, Tm), dtype=dt, device="cuda"),
                      lam=torch.tensor(lam, device="cuda"))
    else:
        want = ob.jacobi(B, V0, 0.7, 2)
        _bamg().relax(dev_csr(B, dt), X, K, 0, 0.7, 2)
    got = X.cpu().numpy().astype(np.float64)
    assert np.isfinite(got).all()
    assert rel(got[:, :K], want) < (1e-12 if dt == torch.float64 else 1e-4)


def test_weights_match_oracle():
    torch = _torch()
    ch, B = _tandem_B(40)
    X0 = ob.jacobi(B, ob.tv_init(ch.n, 10, 5, 1.0, 2.0), 0.7, 4)
    active = np.array([1, 1, 1, 0, 1, 1, 1, 1, 0, 1], dtype=bool)
    Xh, w = ob.normalize_weights(B, X0, active, 1e-28)
    X = torch.tensor(X0, device="cuda")
    wg = _bamg().tv_weights(dev_csr(B), X, 10, 0, torch.tensor(active.astype(np.uint8), device="cuda"))
    assert rel(wg.cpu().numpy(), w) < 1e-12
    assert rel(X.cpu().numpy(), Xh) < 1e-14


# ------------------------------------------------------------------ coarsening
@pytest.mark.parametrize("nx,ny", [(64, 64), (33, 17), (1000, 1), (255, 3)])
def test_coarsen_grid_bit_exact(nx, ny):
    cf, cidx = _bamg().coarsen_grid(nx, ny)
    ocf, ocidx, _ = ob.coarsen_grid(nx, ny)
    assert np.array_equal(cf.cpu().numpy().astype(bool), ocf)
    assert np.array_equal(cidx.cpu().numpy(), ocidx)


def test_coarsen_cr_matches_oracle():
    ch = delaunay_walk(3000, 11)
    B = ob.system_matrix(ch.to_scipy())
    o = ob.Opts(coarsen="cr", seed=5)
    ocf, ocidx, orounds = ob.coarsen_cr(B, 1, o)
    cf, cidx, nc, rounds = _bamg().coarsen_cr(dev_csr(B), 1, 5, o.cr_theta, o.cr_nu, o.cr_omega, o.cr_max_rounds)
    cf = cf.cpu().numpy().astype(bool)
    # the independent sets are integer work and identical; the slow-point tests compare
    # FP64 ratios with theta, so a ratio within rounding of theta could flip
    assert rounds == orounds
    assert np.mean(cf != ocf) < 1e-3
    if np.array_equal(cf, ocf):
        assert np.array_equal(cidx.cpu().numpy(), ocidx)
    assert nc == cf.sum()


def test_coarsen_cr_long_rows_matches_oracle():
    # a compatible-relaxation coarse level (3,278 rows, 17 entries per row on average): the
    # F-relaxation sweeps run with four lanes per row
    ch = delaunay_walk(40000, 3)
    H = ob.setup(ch.to_scipy(), 8, 12, ob.Opts(coarsen="cr"))
    B = sp.csr_matrix(H.levels[2].B)
    B.sort_indices()
    assert B.nnz >= 12 * B.shape[0]
    o = ob.Opts(coarsen="cr", seed=5)
    ocf, ocidx, orounds = ob.coarsen_cr(B, 2, o)
    cf, cidx, nc, rounds = _bamg().coarsen_cr(dev_csr(B), 2, 5, o.cr_theta, o.cr_nu, o.cr_omega, o.cr_max_rounds)
    cf = cf.cpu().numpy().astype(bool)
    assert rounds == orounds
    assert np.mean(cf != ocf) < 1e-3
    assert nc == cf.sum()


# ------------------------------------------------------------------ LS interpolation
def _ls_inputs(N=40, K=8, z=2):
    ch, B = _tandem_B(N)
    cf, cidx, _ = ob.coarsen_grid(*ch.grid)
    X0 = ob.jacobi(B, ob.tv_init(ch.n, K, 3, 0.0, 1.0), 0.7, 4)
    Xh, w = ob.normalize_weights(B, X0, np.ones(K, bool), 1e-28)
    cand, ncand = ob.neighborhoods(B, cf, cidx, z, 16)
    return ch, B, cf, cidx, Xh, w, cand, ncand


def _ls_value(xi, Xs, w, ridge):
    G = (Xs * w) @ Xs.T
    b = (Xs * w) @ xi
    d = ridge * np.trace(G) / len(Xs)
    p = np.linalg.solve(G + d * np.eye(len(Xs)), b)
    return float(np.sum(w * (xi - p @ Xs) ** 2))


@pytest.mark.parametrize("z,c", [(2, 2), (1, 2), (2, 3)])
def test_interp_ls_matches_oracle(z, c):
    torch = _torch()
    ch, B, cf, cidx, Xh, w, cand, ncand = _ls_inputs(z=z)
    P = ob.ls_interpolation(Xh, w, cf, cidx, cand, ncand, c, 1e-12)
    opcol, opval, opcnt = ell_from_csr(P, c)
    K = Xh.shape[1]
    X = torch.tensor(Xh, device="cuda")
    pcol, pval, pcnt = _bamg().interp_ls(dev_csr(B), torch.tensor(cf.astype(np.uint8), device="cuda"),
                                         torch.tensor(cidx.astype(np.int32), device="cuda"), X, K,
                                         torch.tensor(w, device="cuda"), z=z, mmax=16, c=c, ridge=1e-12)
    pcol, pval, pcnt = pcol.cpu().numpy(), pval.cpu().numpy(), pcnt.cpu().numpy()
    c2f = np.flatnonzero(cf)[np.argsort(cidx[cf])]
    same = np.all(pcol == opcol, axis=1) & (pcnt == opcnt)
    # rows with the same choice: weights agree to rounding
    m = same[:, None] & (np.arange(c)[None, :] < pcnt[:, None])
    assert np.max(np.abs(pval[m] - opval[m]) / np.maximum(np.abs(opval[m]), 1e-300)) < 1e-9
    # rows where rounding flipped a near-tie: the GPU's choice must be as good
    diff = np.flatnonzero(~same)
    assert len(diff) <= max(2, 0.002 * ch.n), len(diff)
    for i in diff:
        Jg = c2f[pcol[i, :pcnt[i]]]
        Jo = c2f[opcol[i, :opcnt[i]]]
        lg = _ls_value(Xh[i], Xh[Jg], w, 1e-12)
        lo = _ls_value(Xh[i], Xh[Jo], w, 1e-12)
        assert lg <= lo * (1 + 1e-6) + 1e-300, (i, lg, lo)


# ------------------------------------------------------------------ Galerkin
@pytest.mark.parametrize("with_T", [False, True])
def test_galerkin_bit_exact(with_T):
    torch = _torch()
    ch, B, cf, cidx, Xh, w, cand, ncand = _ls_inputs(N=50)
    P = ob.ls_interpolation(Xh, w, cf, cidx, cand, ncand, 2, 1e-12)
    Q = ob.averaging_restriction(P)
    if with_T:
        rng = np.random.default_rng(9)
        Tm = sp.csr_matrix(B, copy=True)
        Tm.data = rng.uniform(0.0, 1.0, Tm.nnz)
        T_val = torch.tensor(Tm.data.copy(), device="cuda")
    else:
        Tm = sp.identity(ch.n, format="csr")
        T_val = None
    Bc = ob.galerkin(Q, B, P)
    Tc = ob.galerkin(Q, Tm, P)
    pcol, pval, pcnt = ell_from_csr(P, 2)
    nc = P.shape[1]
    rp, ci, bv, tv = _bamg().galerkin(dev_csr(B), T_val, nc, torch.tensor(pcol, device="cuda"),
                                      torch.tensor(pval, device="cuda"), torch.tensor(pcnt, device="cuda"), 2)
    rp, ci, bv, tv = rp.cpu().numpy(), ci.cpu().numpy(), bv.cpu().numpy(), tv.cpu().numpy()
    assert np.array_equal(rp, Bc.indptr) and np.array_equal(ci, Bc.indices)
    assert np.array_equal(bv, Bc.data)  # same products, same order: identical bits
    Tg = sp.csr_matrix((tv, ci, rp), shape=(nc, nc)).toarray()
    assert np.array_equal(Tg, Tc.toarray())


@pytest.mark.parametrize("nq,dense", [(40, 12), (400, 60), (1200, 120)])
def test_galerkin_long_rows_bit_exact(nq, dense):
    # coarse rows of a few hundred to several thousand products (the shared-memory table
    # path), and with more distinct columns than the table takes (the global fallback);
    # caliber 4, random signs
    torch = _torch()
    rng = np.random.default_rng(nq + dense)
    n = 4 * nq
    rows = np.repeat(np.arange(n), dense)
    cols = rng.integers(0, n, n * dense)
    B = sp.csr_matrix((rng.uniform(-1, 1, n * dense), (rows, cols)), shape=(n, n))
    B = B + sp.identity(n) * 3.0
    B = sp.csr_matrix(B)
    B.sort_indices()
    cf = np.zeros(n, dtype=bool)
    cf[rng.choice(n, nq, replace=False)] = True
    cidx = np.full(n, -1)
    cidx[cf] = np.arange(nq)
    pr, pc, pv = [], [], []
    for i in range(n):
        if cf[i]:
            pr.append(i), pc.append(cidx[i]), pv.append(1.0)
        else:
            for J in np.sort(rng.choice(nq, 4, replace=False)):
                pr.append(i), pc.append(J), pv.append(rng.uniform(-0.5, 1.0))
    P = sp.csr_matrix((pv, (pr, pc)), shape=(n, nq))
    P.sort_indices()
    Q = ob.averaging_restriction(P)
    Tm = sp.csr_matrix(B, copy=True)
    Tm.data = rng.uniform(0.0, 1.0, Tm.nnz)
    Bc = ob.galerkin(Q, B, P)
    Tc = ob.galerkin(Q, Tm, P)
    pcol, pval, pcnt = ell_from_csr(P, 4)
    rp, ci, bv, tv = _bamg().galerkin(dev_csr(B), torch.tensor(Tm.data.copy(), device="cuda"), nq,
                                      torch.tensor(pcol, device="cuda"), torch.tensor(pval, device="cuda"),
                                      torch.tensor(pcnt, device="cuda"), 4)
    rp, ci, bv, tv = rp.cpu().numpy(), ci.cpu().numpy(), bv.cpu().numpy(), tv.cpu().numpy()
    assert np.array_equal(rp, Bc.indptr) and np.array_equal(ci, Bc.indices)
    assert np.array_equal(bv, Bc.data)
    assert np.array_equal(sp.csr_matrix((tv, ci, rp), shape=(nq, nq)).toarray(), Tc.toarray())


# ------------------------------------------------------------------ coarsest level
def _coarse_pair(kind="grid33"):
    # grid walk 33 x 33: a 25-state coarsest level; tandem queue 64 x 64 (non-symmetric):
    # 64 states, the largest coarsest order (both rows of every lane in the one-warp
    # factorisations)
    ch = grid_walk(33) if kind == "grid33" else tandem_queue(63)
    H = ob.setup(ch.to_scipy(), 6, 10, ob.Opts(), grid=ch.grid)
    Lc = H.levels[-1]
    return Lc.B.toarray(), Lc.T.toarray(), H


@pytest.mark.parametrize("kind", ["grid33", "tandem63"])
def test_coarse_eig_matches_oracle(kind):
    torch = _torch()
    Bd, Td, H = _coarse_pair(kind)
    lam_o, V_o, kinds_o = ob.coarse_eigs(Bd, Td, 6)
    lam, V, kinds, pinv = _bamg().coarse_eig(torch.tensor(Bd, device="cuda"), torch.tensor(Td, device="cuda"), 6)
    lam, V, kinds, pinv = lam.cpu().numpy(), V.cpu().numpy(), kinds.cpu().numpy(), pinv.cpu().numpy()
    assert lam[0] == 0.0
    assert np.array_equal(kinds, kinds_o)
    assert np.allclose(lam, lam_o, rtol=1e-9, atol=1e-12)
    # eigen-residuals of the GPU vectors, and agreement where the eigenvalue is isolated
    ev = np.linalg.eigvals(np.linalg.solve(Td, Bd))
    for c in range(V.shape[1]):
        if kinds[c] == 0:
            v = V[:, c]
            assert np.linalg.norm(Bd @ v - lam[c] * (Td @ v)) < 1e-9 or c == 0 and np.linalg.norm(Bd @ v) < 1e-10
            gap = np.sort(np.abs(ev - (lam_o[c] if c else 0.0)))[1]
            if gap > 1e-4:
                assert np.allclose(v, V_o[:, c], atol=1e-8)
    assert np.allclose(pinv, ob.pinv_truncated(Bd), rtol=1e-9, atol=1e-11)


@pytest.mark.parametrize("kind", ["grid33", "tandem63"])
def test_coarse_eig_fp32_vectors_close_to_oracle(kind):
    # the mixed-precision setup refines the coarsest eigenvectors in FP32: same selection,
    # eigenvalues and vectors to FP32 accuracy
    torch = _torch()
    Bd, Td, H = _coarse_pair(kind)
    lam_o, V_o, kinds_o = ob.coarse_eigs(Bd, Td, 6)
    lam, V, kinds, pinv = _bamg().coarse_eig(torch.tensor(Bd, device="cuda"), torch.tensor(Td, device="cuda"), 6,
                                             fp32_vectors=True)
    lam, V, kinds, pinv = lam.cpu().numpy(), V.cpu().numpy(), kinds.cpu().numpy(), pinv.cpu().numpy()
    P = ob.pinv_truncated(Bd)
    assert np.abs(pinv - P).max() <= 1e-4 * np.abs(P).max()
    assert lam[0] == 0.0
    assert np.array_equal(kinds, kinds_o)
    scale = np.abs(Bd).max()
    assert np.allclose(lam, lam_o, rtol=1e-4, atol=1e-6 * scale)
    ev = np.linalg.eigvals(np.linalg.solve(Td, Bd))
    for c in range(V.shape[1]):
        if kinds[c] == 0:
            v = V[:, c]
            assert np.linalg.norm(Bd @ v - lam[c] * (Td @ v)) < 1e-4 * scale
            gap = np.sort(np.abs(ev - (lam_o[c] if c else 0.0)))[1]
            if gap > 1e-3:
                assert np.allclose(v, V_o[:, c], atol=1e-4)

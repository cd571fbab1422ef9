"""Learned interpolation on the GPU against the oracle (oracle/learned.py): features,
LS targets, the MLP's forward pass and gradients, training, the learned rows of P, the
V-cycle factor and an end-to-end learned setup."""

import numpy as np
import pytest
import scipy.sparse as sp

from gpu_util import need_gpu, rel
from oracle import bamg as ob
from oracle import exact
from oracle import learned as ol
from workloads import grid_walk, tandem_queue, tandem_training_set

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


def flat(p):
    return np.concatenate([p["W1"].ravel(), p["b1"], p["W2"].ravel(), p["b2"], p["W3"].ravel(), p["b3"]]).astype(
        np.float32)


def unflat(a):
    out, o = {}, 0
    for layer, (no, ni) in enumerate(ol.LAYERS):
        out[f"W{layer + 1}"] = a[o:o + no * ni].astype(np.float64).reshape(no, ni)
        o += no * ni
        out[f"b{layer + 1}"] = a[o:o + no].astype(np.float64)
        o += no
    return out


def _level(ch, r=6, seed=0):
    B = ob.system_matrix(ch.to_scipy())
    X = ob.jacobi(B, ob.tv_init(ch.n, r, seed, 0.0, 1.0), 0.7, 4)
    cf, cidx, _ = ob.coarsen_grid(*ch.grid)
    Xh, w = ob.normalize_weights(B, X, np.ones(r, dtype=bool), 1e-28)
    cand, ncand = ob.neighborhoods(B, cf, cidx, 2, 16)
    return B, Xh, w, cf, cidx, cand, ncand


def _dev_level(B, Xh, w, cf, cidx, dtype):
    torch = _torch()
    tdt = torch.float64 if dtype == "fp64" else torch.float32
    n, r = Xh.shape
    wpad = 2 if dtype == "fp64" else 4
    ld = (r + wpad - 1) // wpad * wpad
    Xp = np.zeros((n, ld))
    Xp[:, :r] = Xh
    wp = np.zeros(ld)
    wp[:r] = w
    Bd = (torch.tensor(B.indptr.astype(np.int32), device="cuda"), torch.tensor(B.indices.astype(np.int32), device="cuda"),
          torch.tensor(B.data, dtype=tdt, device="cuda"))
    return (Bd, torch.tensor(cf.astype(np.uint8), device="cuda"), torch.tensor(cidx.astype(np.int32), device="cuda"),
            torch.tensor(Xp, dtype=tdt, device="cuda").contiguous(), r, torch.tensor(wp, device="cuda"))


@pytest.mark.parametrize("dtype,tol", [("fp64", 1e-6), ("fp32", 2e-4)])
def test_features_targets_candidates_match_oracle(dtype, tol):
    ch = tandem_queue(13)
    B, Xh, w, cf, cidx, cand, ncand = _level(ch)
    Bd, cfd, cid, X, r, wd = _dev_level(B, Xh, w, cf, cidx, dtype)
    feat, tgt, cd = _bamg().interp_features(Bd, cfd, cid, X, r, wd, targets=True)
    F_o = ol.features(B, cf, Xh, w, cand, ncand)
    T_o = ol.ls_targets(Xh, w, cf, cand, ncand, 2, 1e-4)
    feat, tgt, cd = feat.cpu().numpy(), tgt.cpu().numpy(), cd.cpu().numpy()
    assert np.array_equal(np.where(np.arange(16)[None, :] < ncand[:, None], cand, -1)[~cf], cd[~cf])
    assert np.abs(feat - F_o).max() <= tol * max(1.0, np.abs(F_o).max())
    fine = np.flatnonzero(~cf)
    same = [(np.flatnonzero(tgt[i]) == np.flatnonzero(T_o[i])).all() for i in fine]
    assert np.mean(same) > 0.99  # Algorithm 2's choice (FP32 may break rare near-ties differently)
    ok = fine[np.array(same)]
    assert np.abs(tgt[ok] - T_o[ok]).max() <= 50 * tol * max(1.0, np.abs(T_o).max())


def _model_and_feats(seed=3, rows=None):
    torch = _torch()
    p = ol.init_params(seed)
    rng = np.random.default_rng(seed)
    for k in ("b1", "b2", "b3"):
        p[k] = rng.standard_normal(p[k].shape) * 0.05
    ch = tandem_queue(15)
    B, Xh, w, cf, cidx, cand, ncand = _level(ch)
    F_o = ol.features(B, cf, Xh, w, cand, ncand)[~cf]
    if rows:
        F_o = F_o[:rows]
    m = _bamg().Model(0)
    m.set(flat(p))
    p32 = unflat(flat(p))  # the parameters as the GPU holds them (FP32)
    return m, p32, F_o, torch.tensor(F_o, dtype=torch.float32, device="cuda").contiguous()


def test_forward_matches_oracle_bf16():
    m, p, F_o, Fd = _model_and_feats()
    y = m.forward(Fd).cpu().numpy()
    y_o, _ = ol.forward(p, F_o.astype(np.float32).astype(np.float64), use_bf16=True)
    scale = max(1.0, np.abs(y_o).max())
    assert np.abs(y - y_o).max() <= 1e-2 * scale
    assert np.abs(y - y_o).mean() <= 1e-4 * scale


def test_gradients_match_oracle():
    torch = _torch()
    m, p, F_o, Fd = _model_and_feats(rows=600)
    T = np.random.default_rng(1).standard_normal((F_o.shape[0], 16)) * 0.3
    g, loss = m.gradients(Fd, torch.tensor(T, dtype=torch.float32, device="cuda"))
    Fo32 = F_o.astype(np.float32).astype(np.float64)
    y_o, cache = ol.forward(p, Fo32, use_bf16=True)
    mask = ol.slot_mask(Fo32)
    # the tensor-core backward rounds the gradient entering each product to bf16, as the
    # oracle's bf16_grads option does: agreement up to FP32 accumulation; the exact
    # (unrounded) gradients stay within the rounding's effect
    g_b = ol.backward(p, cache, y_o, T, mask, bf16_grads=True)
    g_o = ol.backward(p, cache, y_o, T, mask)
    assert loss == pytest.approx(ol.loss(y_o, T, mask), rel=1e-3)
    gg = unflat(g)
    for k in g_o:
        err_b = np.linalg.norm(gg[k] - g_b[k]) / max(np.linalg.norm(g_b[k]), 1e-30)
        err = np.linalg.norm(gg[k] - g_o[k]) / max(np.linalg.norm(g_o[k]), 1e-30)
        assert err_b < 1e-3, (k, err_b)
        assert err < 1e-2, (k, err)


def test_get_set_roundtrip_and_init():
    m = _bamg().Model(5)
    a = m.get()
    p = ol.init_params(5)
    assert np.allclose(a, flat(p), rtol=1e-6, atol=1e-7)  # same SplitMix64 initialisation
    b = np.random.default_rng(0).standard_normal(a.size).astype(np.float32)
    m.set(b)
    assert np.array_equal(m.get(), b)


def _dataset(chains, r=10):
    torch = _torch()
    bamg = _bamg()
    Fs, Ts = [], []
    for ch in chains:
        rp, ci, v = (torch.tensor(a, device="cuda") for a in (ch.row_ptr, ch.col, ch.val))
        f, t = bamg.interp_dataset(rp, ci, v, r, 20, grid=ch.grid)
        keep = f[:, 0:96:6].sum(dim=1) > 0  # fine points with candidates
        Fs.append(f[keep])
        Ts.append(t[keep])
    F = torch.cat(Fs)
    T = torch.cat(Ts)
    perm = torch.randperm(F.shape[0], generator=torch.Generator().manual_seed(0)).to(F.device)
    return F[perm].contiguous(), T[perm].contiguous()


def test_dataset_matches_oracle_recording():
    # the GPU dataset of an FP64 setup equals the oracle's recorded (features, targets)
    torch = _torch()
    ch = tandem_queue(11)
    rp, ci, v = (torch.tensor(a, device="cuda") for a in (ch.row_ptr, ch.col, ch.val))
    f, t = _bamg().interp_dataset(rp, ci, v, 8, 10, grid=ch.grid, tv_lo=0.0, tv_hi=1.0)
    rec = []
    ob.setup(ch.to_scipy(), 8, 10, ob.Opts(record=rec, tv_lo=0.0, tv_hi=1.0), grid=ch.grid)
    F_o = np.concatenate([a for a, _, _ in rec])
    T_o = np.concatenate([b for _, b, _ in rec])
    f, t = f.cpu().numpy(), t.cpu().numpy()
    assert f.shape == F_o.shape
    assert np.abs(f - F_o).max() <= 1e-5 * max(1.0, np.abs(F_o).max())
    assert np.abs(t - T_o).max() <= 1e-5 * max(1.0, np.abs(T_o).max())


def test_training_reduces_loss_and_matches_oracle_first_epoch():
    torch = _torch()
    F, T = _dataset(tandem_training_set(2, 3, n_lo=31, n_hi=47))
    m = _bamg().Model(0)
    hist = m.train(F, T, epochs=15, batch=256, lr=1e-3)
    assert hist[-1] < 0.3 * hist[0]
    # the first epoch's loss equals the oracle's on the same rows from the same start
    m2 = _bamg().Model(0)
    h2 = m2.train(F[:1024], T[:1024], epochs=1, batch=256, lr=1e-3)
    p = unflat(_bamg().Model(0).get())
    h_o = ol.train(p, F[:1024].cpu().double().numpy(), T[:1024].cpu().double().numpy(), 1, 256, 1e-3,
                   bf16_grads=True)
    assert h2[0] == pytest.approx(h_o[0], rel=2e-2)


@pytest.mark.parametrize("refit", [False, True])
def test_learned_rows_match_oracle(refit):
    torch = _torch()
    ch = grid_walk(21, 17)
    B, Xh, w, cf, cidx, cand, ncand = _level(ch)
    m, p, _, _ = _model_and_feats(seed=4)
    Bd, cfd, cid, X, r, wd = _dev_level(B, Xh, w, cf, cidx, "fp64")
    pcol, pval, pcnt = _bamg().interp_learned(Bd, cfd, cid, X, r, wd, m, refit=refit)
    F_o = ol.features(B, cf, Xh, w, cand, ncand).astype(np.float32).astype(np.float64)
    y_o, _ = ol.forward(p, F_o)
    P_o = ol.learned_rows(y_o, Xh, w, cf, cidx, cand, ncand, 2, refit, 1e-4).toarray()
    pcol, pval, pcnt = pcol.cpu().numpy(), pval.cpu().numpy(), pcnt.cpu().numpy()
    n = ch.n
    P = np.zeros_like(P_o)
    for i in range(n):
        for a in range(pcnt[i]):
            P[i, pcol[i, a]] += pval[i, a]
    # compare rows whose top-2 choice is clear (no near-tie in |y|)
    ay = np.sort(np.abs(np.where(np.arange(16)[None, :] < ncand[:, None], y_o, -1.0)), axis=1)[:, ::-1]
    clear = (~cf) & ((ncand <= 2) | (ay[:, 1] - ay[:, 2] > 2e-3 * np.maximum(ay[:, 1], 1e-30)))
    assert clear.sum() > 0.4 * (~cf).sum()
    tolv = 1e-9 if refit else 1e-2 * np.abs(P_o).max()
    assert np.abs(P[clear] - P_o[clear]).max() <= tolv
    assert np.array_equal(P[cf], P_o[cf])


def test_vcycle_factor_matches_oracle():
    from test_gpu_solve import _levels_of

    ch = tandem_queue(30)
    H = ob.setup(ch.to_scipy(), 8, 10, ob.Opts(), grid=ch.grid)
    s = _bamg().import_hierarchy(_levels_of(H), H.pinv, H.x_init)
    assert s.vcycle_factor(30) == pytest.approx(ol.vcycle_factor(H, 30), rel=1e-8)


def test_learned_setup_solves_and_falls_back():
    torch = _torch()
    bamg = _bamg()
    F, T = _dataset(tandem_training_set(5, 4, n_lo=31, n_hi=63))
    m = bamg.Model(0)
    m.train(F, T, epochs=20, batch=512, lr=1e-3)
    ch = tandem_training_set(77, 1, n_lo=63, n_hi=63)[0]
    rp, ci, v = (torch.tensor(a, device="cuda") for a in (ch.row_ptr, ch.col, ch.val))
    xe = exact.sparse_nullspace(ch.to_scipy())
    for precision, bound in (("fp64", 1e-8), ("mixed", 1e-6)):
        s = bamg.Solver(rp, ci, v, r=10, levels=20, grid=ch.grid, precision=precision, interp="learned", model=m)
        assert s.interp_used()[0] == "learned"
        x, st = s.solve(1e-13 if precision == "fp64" else 1e-12)
        assert rel(x.cpu().numpy(), xe) < bound, (precision, st)
    # a limit no hierarchy meets sends the setup back to least squares
    s = bamg.Solver(rp, ci, v, r=10, levels=20, grid=ch.grid, interp="learned", model=m, learned_rho_max=1e-9)
    used, rho = s.interp_used()
    assert used == "ls" and rho > 1e-9
    x, st = s.solve(1e-13)
    assert rel(x.cpu().numpy(), xe) < 1e-8


def test_learned_gain_on_a_held_out_chain():
    """What the trained network gains: the MLP trained (20 epochs) on the LS rows of four
    tandem queues of capacity 63-255 with random rates, then a held-out tandem queue of
    capacity 255 (65,536 states) with other rates, whose least-squares V-cycle converges
    (factor about 0.73, so the baseline is sound): the learned hierarchy's V-cycle factor is
    at least 5% smaller and FGMRES needs at least two fewer iterations (measured on a
    GB300: 0.681 against 0.735, 13 against 17), in both precisions."""
    torch = _torch()
    bamg = _bamg()

    def dev(c):
        return tuple(torch.tensor(a, device="cuda") for a in (c.row_ptr, c.col, c.val))

    Fs, Ts = [], []
    for c in tandem_training_set(1, 4, n_lo=63, n_hi=255):
        f, t = bamg.interp_dataset(*dev(c), 10, 20, grid=c.grid, precision="mixed")
        keep = (f[:, 0:96:6].sum(dim=1) > 0) & (t.abs().amax(dim=1) <= 4.0)
        Fs.append(f[keep])
        Ts.append(t[keep])
    F, T = torch.cat(Fs), torch.cat(Ts)
    m = bamg.Model(0)
    m.train(F, T, epochs=20, batch=4096, lr=1e-3)
    test = tandem_training_set(99, 1, n_lo=255, n_hi=255)[0]
    A = dev(test)
    for precision in ("mixed", "fp64"):
        s_ls = bamg.Solver(*A, r=10, levels=20, grid=test.grid, precision=precision)
        s_l = bamg.Solver(*A, r=10, levels=20, grid=test.grid, precision=precision, interp="learned", model=m)
        rho_ls, rho_l = s_ls.vcycle_factor(30), s_l.vcycle_factor(30)
        _, st_ls = s_ls.solve(1e-10)
        _, st_l = s_l.solve(1e-10)
        assert rho_ls < 1.0, rho_ls
        assert rho_l <= 0.95 * rho_ls, (precision, rho_l, rho_ls)
        assert st_l["iterations"] <= st_ls["iterations"] - 2, (precision, st_l["iterations"], st_ls["iterations"])
    m.close()

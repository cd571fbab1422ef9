"""Pins of the learned-interpolation oracle (oracle/learned.py) against independent
computations: torch's bfloat16 conversion, finite differences, the closed form of Adam
under a constant gradient, explicit graph distances, and the LS oracle itself."""

import networkx as nx
import numpy as np
import pytest
import scipy.sparse as sp

from oracle import bamg as ob
from oracle import learned as ol
from workloads import grid_walk, random_birth_death, tandem_queue


def test_bf16_ties_to_even_and_matches_torch():
    torch = pytest.importorskip("torch")
    one = 1.0
    assert ol.bf16(np.array([one]))[0] == 1.0
    assert ol.bf16(np.array([1.0 + 2.0 ** -8]))[0] == 1.0  # halfway, even neighbour below
    assert ol.bf16(np.array([1.0 + 3 * 2.0 ** -8]))[0] == 1.0 + 2.0 ** -6  # halfway, even above
    v = np.random.default_rng(0).standard_normal(10000) * np.exp(np.random.default_rng(1).uniform(-20, 20, 10000))
    ref = torch.tensor(v, dtype=torch.float32).to(torch.bfloat16).to(torch.float64).numpy()
    assert np.array_equal(ol.bf16(v), ref)


def _toy(seed=0, rows=7):
    rng = np.random.default_rng(seed)
    p = {k: v * 0.5 for k, v in ol.init_params(seed).items()}
    for k in ("b1", "b2", "b3"):
        p[k] = rng.standard_normal(p[k].shape) * 0.1
    f = rng.standard_normal((rows, ol.F))
    f[:, 0:ol.NF_SLOT * ol.S:ol.NF_SLOT] = (rng.random((rows, ol.S)) < 0.6).astype(float)
    t = rng.standard_normal((rows, ol.S))
    return p, f, t


def test_backward_matches_finite_differences():
    p, f, t = _toy()
    mask = ol.slot_mask(f)
    y, cache = ol.forward(p, f, use_bf16=False)
    g = ol.backward(p, cache, y, t, mask)
    rng = np.random.default_rng(3)
    h = 1e-6
    for k in p:
        for _ in range(6):
            idx = tuple(rng.integers(0, d) for d in p[k].shape)
            q = {kk: vv.copy() for kk, vv in p.items()}
            q[k][idx] += h
            lp = ol.loss(ol.forward(q, f, False)[0], t, mask)
            q[k][idx] -= 2 * h
            lm = ol.loss(ol.forward(q, f, False)[0], t, mask)
            fd = (lp - lm) / (2 * h)
            assert abs(fd - g[k][idx]) <= 1e-6 * max(1.0, abs(fd)), (k, idx, fd, g[k][idx])


def test_adam_constant_gradient_closed_form():
    # with a constant gradient the bias-corrected moments are exactly g and g^2, so every
    # step moves a parameter by -lr g / (|g| + eps)
    p = {"a": np.array([0.0, 1.0, -2.0])}
    g = {"a": np.array([0.5, -3.0, 1e-3])}
    st = ol.adam_init(p)
    for _ in range(5):
        ol.adam_step(p, g, st, lr=0.01)
    step = -0.01 * g["a"] / (np.abs(g["a"]) + 1e-8)
    assert np.allclose(p["a"], np.array([0.0, 1.0, -2.0]) + 5 * step, rtol=1e-12, atol=1e-12)


def test_init_bounds_and_determinism():
    p = ol.init_params(5)
    q = ol.init_params(5)
    for k, (o, i) in zip(("W1", "W2", "W3"), ol.LAYERS):
        assert p[k].shape == (o, i) and np.array_equal(p[k], q[k])
        a = np.sqrt(6.0 / i)
        assert np.abs(p[k]).max() <= a and abs(p[k].mean()) < 0.05 * a
        assert p[k].std() == pytest.approx(a / np.sqrt(3.0), rel=0.05)


def _level(ch, r=6, seed=0):
    B = ob.system_matrix(ch.to_scipy())
    X = ob.jacobi(B, ob.tv_init(ch.n, r, seed, 0.0, 1.0), 0.7, 4)
    cf, cidx, _ = ob.coarsen_grid(*ch.grid)
    Xh, w = ob.normalize_weights(B, X, np.ones(r, dtype=bool), 1e-28)
    cand, ncand = ob.neighborhoods(B, cf, cidx, 2, 16)
    return B, X, Xh, w, cf, cidx, cand, ncand


def test_features_against_explicit_definitions():
    ch = tandem_queue(9)
    B, X, Xh, w, cf, cidx, cand, ncand = _level(ch)
    Fm = ol.features(B, cf, Xh, w, cand, ncand)
    Bd = B.toarray()
    G = nx.DiGraph()
    G.add_nodes_from(range(ch.n))
    rr, cc = np.nonzero(Bd)
    G.add_edges_from((int(a), int(b)) for a, b in zip(rr, cc) if a != b)
    for i in np.flatnonzero(~cf)[::3]:
        dist = nx.single_source_shortest_path_length(G, int(i), cutoff=3)
        gi = sum(w[k] * Xh[i, k] ** 2 for k in range(len(w)))
        for s in range(ol.S):
            got = Fm[i, 6 * s:6 * s + 6]
            if s >= ncand[i]:
                assert not got.any()
                continue
            j = cand[i, s]
            gj = sum(w[k] * Xh[j, k] ** 2 for k in range(len(w)))
            gij = sum(w[k] * Xh[i, k] * Xh[j, k] for k in range(len(w)))
            want = [1.0, dist[int(j)] / 3.0, gij / gj, gij / np.sqrt(gi * gj), -Bd[i, j] / Bd[i, i], -Bd[j, i] / Bd[j, j]]
            assert np.allclose(got, want, rtol=1e-12, atol=1e-15), (i, s, got, want)
        assert Fm[i, 96] == ncand[i] / 16
        assert Fm[i, 97] == pytest.approx((np.abs(Bd[i]).sum() - abs(Bd[i, i])) / Bd[i, i], rel=1e-12)
        assert not Fm[i, 98:].any()
    assert not Fm[cf].any()


def test_features_scale_invariant_and_self_similar():
    # the features do not change when every test vector is scaled, and a candidate whose
    # test-vector values are a multiple of the fine point's has cosine 1
    ch = grid_walk(12)
    B, X, Xh, w, cf, cidx, cand, ncand = _level(ch)
    F1 = ol.features(B, cf, Xh, w, cand, ncand)
    F2 = ol.features(B, cf, 3.0 * Xh, w, cand, ncand)
    assert np.allclose(F1, F2, rtol=1e-12, atol=1e-14)
    i = int(np.flatnonzero(~cf)[0])
    j = int(cand[i, 0])
    Xs = Xh.copy()
    Xs[j] = 2.0 * Xs[i]
    F3 = ol.features(B, cf, Xs, w, cand, ncand)
    assert F3[i, 2] == pytest.approx(0.5, rel=1e-12) and F3[i, 3] == pytest.approx(1.0, rel=1e-12)


def test_ls_targets_reproduce_ls_interpolation():
    ch = tandem_queue(11)
    B, X, Xh, w, cf, cidx, cand, ncand = _level(ch)
    T = ol.ls_targets(Xh, w, cf, cand, ncand, 2, 1e-4)
    P = ob.ls_interpolation(Xh, w, cf, cidx, cand, ncand, 2, 1e-4).toarray()
    for i in np.flatnonzero(~cf):
        row = np.zeros(P.shape[1])
        for s in range(ncand[i]):
            row[cidx[cand[i, s]]] += T[i, s]
        assert np.allclose(row, P[i], rtol=1e-13, atol=1e-15)


@pytest.mark.parametrize("refit", [False, True])
def test_perfect_model_reproduces_ls(refit):
    # MLP outputs equal to the LS targets select the LS slots; their weights (directly, or
    # refitted by Eq. (3.6) over the same set) are the LS weights
    ch = grid_walk(14, 9)
    B, X, Xh, w, cf, cidx, cand, ncand = _level(ch)
    T = ol.ls_targets(Xh, w, cf, cand, ncand, 2, 1e-4)
    P_ls = ob.ls_interpolation(Xh, w, cf, cidx, cand, ncand, 2, 1e-4).toarray()
    P_l = ol.learned_rows(T, Xh, w, cf, cidx, cand, ncand, 2, refit, 1e-4).toarray()
    assert np.allclose(P_l, P_ls, rtol=1e-10, atol=1e-13)


def test_vcycle_factor_matches_dense_spectral_radius():
    ch = random_birth_death(120, 5)
    H = ob.setup(ch.to_scipy(), 6, 6, ob.Opts(), grid=ch.grid)
    B = H.levels[0].B.toarray()
    n = B.shape[0]
    C = np.column_stack([ob.vcycle(H, e) for e in np.eye(n)])
    E = np.eye(n) - B @ C  # residual propagator; 1^T E = 1^T
    ev = np.sort(np.abs(np.linalg.eigvals(E)))[::-1]
    # drop the eigenvalue 1 of the left eigenvector 1 (residuals never carry it)
    k = np.argmin(np.abs(ev - 1.0))
    rho = np.delete(ev, k).max()
    est = ol.vcycle_factor(H, iters=80)
    assert est == pytest.approx(rho, rel=0.08)


def test_training_fits_a_learnable_map():
    rng = np.random.default_rng(2)
    f = rng.standard_normal((2048, ol.F)) * 0.5
    f[:, 0:96:6] = 1.0
    Wt = rng.standard_normal((ol.S, ol.F)) * 0.1
    t = np.maximum(f @ Wt.T, 0.0)
    p = ol.init_params(1)
    hist = ol.train(p, f, t, epochs=15, batch=256, lr=2e-3)
    assert hist[-1] < 0.2 * hist[0]


def test_learned_setup_with_ls_model_solves():
    # a model trained on LS rows of tandem queues gives a working hierarchy on another one
    from workloads import tandem_training_set

    rec = []
    for ch in tandem_training_set(4, 3, n_lo=15, n_hi=23):
        ob.setup(ch.to_scipy(), 8, 10, ob.Opts(record=rec), grid=ch.grid)
    F = np.concatenate([f[m] for f, _, m in rec])
    T = np.concatenate([t[m] for _, t, m in rec])
    perm = np.random.default_rng(0).permutation(len(F))
    p = ol.init_params(0)
    ol.train(p, F[perm], T[perm], epochs=20, batch=256, lr=1e-3)
    ch = tandem_queue(23)
    xo, H, st = ob.stationary(ch.to_scipy(), 8, 10, 1e-12, ob.Opts(interp="learned", model=p), grid=ch.grid)
    from oracle import exact

    assert np.abs(xo - exact.exact_stationary(ch)).sum() < 1e-9
    assert ol.vcycle_factor(H) < 1.0


def test_bf16_gradients_stay_within_rounding_of_the_exact_ones():
    """Rounding the backward products' gradient operands to bfloat16 (8 significant bits)
    moves every weight gradient by about 2^-9 relative, never by 1% (a mistake in which
    operand is rounded, or a dropped rounding of the hidden activations, shows up as a
    difference above that or as none at all)."""
    rng = np.random.default_rng(4)
    p = ol.init_params(3)
    f = np.abs(rng.standard_normal((300, ol.F)))
    t = rng.standard_normal((300, ol.S)) * 0.3
    y, cache = ol.forward(p, f, use_bf16=True)
    mask = ol.slot_mask(f)
    g = ol.backward(p, cache, y, t, mask)
    gb = ol.backward(p, cache, y, t, mask, bf16_grads=True)
    for k in ("W1", "W2", "W3"):
        e = np.linalg.norm(gb[k] - g[k]) / np.linalg.norm(g[k])
        assert 1e-5 < e < 1e-2, (k, e)
    assert np.array_equal(gb["b3"], g["b3"])  # dy itself is never rounded for the bias sum
    for k in ("b1", "b2"):  # through d2 = bf16(dy) W3 and d1 = bf16(d2) W2
        e = np.linalg.norm(gb[k] - g[k]) / np.linalg.norm(g[k])
        assert 1e-5 < e < 1e-2, (k, e)

"""Plain FP64 oracle of the learned interpolation: a small MLP over each fine point's
local B_l entries and test-vector statistics that predicts the weights of its row of P_l,
trained on the least-squares rows of Algorithm 2 (Eq. (3.6)) that the method itself
produces, with least squares kept as the fallback.

TEST INFRASTRUCTURE ONLY (see oracle/bamg.py).  The paper has no learned interpolation;
this module states the definitions that the CUDA path implements, so that each of them
can be checked against a second, independent computation:

Features of a fine point i with candidates N_i = (j_0, ..., j_{m-1}) in the canonical
order of Eq. (3.5) (path length, then coarse index; at most S = 16), test vectors x^(k)
(normalised, R7) and LS weights w_k:
    g_ab = sum_k w_k x_a^(k) x_b^(k)
    slot s < m:  [1, d_s / 3, g_ij / g_jj, g_ij / sqrt(g_ii g_jj), -b_ij / b_ii, -b_ji / b_jj]
                 (d_s = path length of j = j_s; a ratio with a zero denominator is 0;
                 b_ij = 0 when j is not in row i of B)
    slot s >= m: six zeros
    then [m / S, sum_{j != i} |b_ij| / b_ii], zero-padded to F = 112.
Targets: the LS row of Algorithm 2 on the slots: t_s = p_{j_s} if j_s was chosen, else 0.

MLP: y = W3 relu(W2 relu(W1 f + b1) + b2) + b3 with W1: 128 x 112, W2: 128 x 128,
W3: 16 x 128.  With bf16=True the input of every product (f, the hidden activations and
the weights) is rounded to bfloat16 (round to nearest, ties to even) as the GPU stores
them; sums are exact (FP64) here and FP32 on the GPU.
Loss: (1 / batch) sum_rows sum_{s < m} (y_s - t_s)^2.  Optimiser: Adam (Kingma & Ba,
"Adam: A Method for Stochastic Optimization", ICLR 2015) with beta1 = 0.9,
beta2 = 0.999, eps = 1e-8, bias-corrected moments.
Initialisation: W = (2u - 1) sqrt(6 / fan_in) with u = counter_uniform(seed, layer, index)
(SplitMix64, oracle/bamg.py), biases zero.
Learned row: the c valid slots with the largest |y_s| (lower slot on ties) form J; the
weights are y_s, or with refit the minimiser of Eq. (3.6) over J (with the Tikhonov term
of R25).  Judge: the V-cycle factor rho of the stationary iteration x <- x - C B x, by
power iteration on its residual propagator I - B C (residuals keep 1^T r = 0).
"""

from __future__ import annotations

import numpy as np
import scipy.sparse as sp

from . import bamg as ob

S = 16  # candidate slots (m_max)
NF_SLOT = 6
F = 112  # features, padded to a multiple of 16
H = 128  # hidden width
LAYERS = ((H, F), (H, H), (S, H))  # (out, in) of W1, W2, W3


# ---------------------------------------------------------------------------------
# bfloat16 rounding: keep the top 16 bits of the IEEE binary32 pattern, rounding to
# nearest with ties to even (the conversion of the bfloat16 format's definition).
# ---------------------------------------------------------------------------------
def bf16(a: np.ndarray) -> np.ndarray:
    f = np.asarray(a, dtype=np.float32)
    u = f.view(np.uint32).astype(np.uint64)
    u = (u + 0x7FFF + ((u >> 16) & 1)) & 0xFFFF0000
    return u.astype(np.uint32).view(np.float32).astype(np.float64)


# ---------------------------------------------------------------------------------
# Features and targets
# ---------------------------------------------------------------------------------
def candidate_depths(B, cand: np.ndarray, ncand: np.ndarray) -> np.ndarray:
    """Path length from i to each candidate in G(B) (edges of the off-diagonal pattern
    of row i), by breadth-first layers; 0 for empty slots."""
    n = B.shape[0]
    G = sp.csr_matrix(B, copy=True)
    G.data[:] = 1.0
    G.setdiag(0)
    G.eliminate_zeros()
    depth = np.zeros(cand.shape, dtype=np.int64)
    reach = sp.identity(n, format="csr")
    seen = sp.identity(n, format="csr")
    for d in range(1, 4):
        reach = reach @ G
        reach.data[:] = 1.0
        new = reach - reach.multiply(seen)
        new.eliminate_zeros()
        seen = seen + new
        seen.data[:] = 1.0
        new = new.tocsr()
        for s in range(cand.shape[1]):
            rows = np.flatnonzero((s < ncand) & (depth[:, s] == 0))
            if len(rows):
                hit = np.asarray(new[rows, cand[rows, s]]).ravel() != 0
                depth[rows[hit], s] = d
    return depth


def features(B, cf: np.ndarray, Xh: np.ndarray, w: np.ndarray, cand: np.ndarray, ncand: np.ndarray) -> np.ndarray:
    """The F features of every point (rows of coarse points are zero); Xh holds the
    active normalised test vectors, w their weights."""
    B = sp.csr_matrix(B)
    B.sort_indices()
    n = B.shape[0]
    diag = ob.diag_of(B)
    depth = candidate_depths(B, cand, ncand)
    g_self = (Xh * Xh) @ w
    out = np.zeros((n, F))
    absB = abs(B)
    offmass = (np.asarray(absB.sum(axis=1)).ravel() - np.abs(diag)) / diag

    def entry(r, c):  # b_rc, 0 outside the pattern
        lo, hi = B.indptr[r], B.indptr[r + 1]
        k = lo + np.searchsorted(B.indices[lo:hi], c)
        return float(B.data[k]) if k < hi and B.indices[k] == c else 0.0

    for i in np.flatnonzero(~cf):
        m = int(ncand[i])
        for s in range(m):
            j = int(cand[i, s])
            gij = float(np.dot(w, Xh[i] * Xh[j]))
            gjj = float(g_self[j])
            gii = float(g_self[i])
            f = out[i, NF_SLOT * s:NF_SLOT * (s + 1)]
            f[0] = 1.0
            f[1] = depth[i, s] / 3.0
            f[2] = gij / gjj if gjj != 0.0 else 0.0
            f[3] = gij / np.sqrt(gii * gjj) if gii * gjj != 0.0 else 0.0
            f[4] = -entry(i, j) / diag[i]
            f[5] = -entry(j, i) / diag[j]
        out[i, NF_SLOT * S] = m / S
        out[i, NF_SLOT * S + 1] = offmass[i]
    return out


def ls_targets(Xh: np.ndarray, w: np.ndarray, cf: np.ndarray, cand: np.ndarray, ncand: np.ndarray, c: int,
               ridge: float) -> np.ndarray:
    """Algorithm 2's rows on the slots (n x S; coarse rows zero)."""
    n = Xh.shape[0]
    out = np.zeros((n, S))
    fine = np.flatnonzero(~cf)
    if len(fine) == 0:
        return out
    valid = np.arange(S)[None, :] < ncand[fine][:, None]
    Xc = Xh[np.where(valid, cand[fine], 0)]
    chosen, pw, _ = ob.ls_fit_rows(Xh[fine], Xc, valid, w, c, ridge)
    for t in range(c):
        ok = chosen[:, t] >= 0
        out[fine[ok], chosen[ok, t]] = pw[ok, t]
    return out


# ---------------------------------------------------------------------------------
# The MLP
# ---------------------------------------------------------------------------------
def init_params(seed: int) -> dict:
    p = {}
    for layer, (o, i) in enumerate(LAYERS):
        u = ob.counter_uniform(seed, layer, np.arange(o * i, dtype=np.uint64)).reshape(o, i)
        p[f"W{layer + 1}"] = (2.0 * u - 1.0) * np.sqrt(6.0 / i)
        p[f"b{layer + 1}"] = np.zeros(o)
    return p


def forward(p: dict, f: np.ndarray, use_bf16: bool = True):
    """y and the cache (the rounded inputs of each product, the pre-activations)."""
    r = bf16 if use_bf16 else (lambda a: np.asarray(a, dtype=np.float64))
    x0 = r(f)
    a1 = x0 @ r(p["W1"]).T + p["b1"]
    x1 = r(np.maximum(a1, 0.0))
    a2 = x1 @ r(p["W2"]).T + p["b2"]
    x2 = r(np.maximum(a2, 0.0))
    y = x2 @ r(p["W3"]).T + p["b3"]
    return y, {"x0": x0, "a1": a1, "x1": x1, "a2": a2, "x2": x2, "r": r}


def slot_mask(f: np.ndarray) -> np.ndarray:
    return f[:, 0:NF_SLOT * S:NF_SLOT]


def loss(y: np.ndarray, t: np.ndarray, mask: np.ndarray) -> float:
    return float(np.sum(mask * (y - t) ** 2) / y.shape[0])


def backward(p: dict, cache: dict, y: np.ndarray, t: np.ndarray, mask: np.ndarray, bf16_grads: bool = False) -> dict:
    """Gradients of the loss by the chain rule through the three products (the rounded
    forward inputs are treated as the layer inputs; rounding is not differentiated).
    With bf16_grads the output gradients entering a product (dy, d2, d1) are rounded to
    bfloat16 as well, as the GPU's tensor-core backward takes them; bias gradients are
    plain sums."""
    r = cache["r"]
    rg = bf16 if bf16_grads else (lambda a: a)
    dy = 2.0 * mask * (y - t) / y.shape[0]
    g = {"W3": rg(dy).T @ cache["x2"], "b3": dy.sum(axis=0)}
    d2 = (rg(dy) @ r(p["W3"])) * (cache["a2"] > 0)
    g["W2"] = rg(d2).T @ cache["x1"]
    g["b2"] = d2.sum(axis=0)
    d1 = (rg(d2) @ r(p["W2"])) * (cache["a1"] > 0)
    g["W1"] = rg(d1).T @ cache["x0"]
    g["b1"] = d1.sum(axis=0)
    return g


def adam_init(p: dict) -> dict:
    return {"t": 0, "m": {k: np.zeros_like(v) for k, v in p.items()}, "v": {k: np.zeros_like(v) for k, v in p.items()}}


def adam_step(p: dict, g: dict, st: dict, lr: float, b1: float = 0.9, b2: float = 0.999, eps: float = 1e-8):
    st["t"] += 1
    t = st["t"]
    for k in p:
        st["m"][k] = b1 * st["m"][k] + (1.0 - b1) * g[k]
        st["v"][k] = b2 * st["v"][k] + (1.0 - b2) * g[k] * g[k]
        mh = st["m"][k] / (1.0 - b1 ** t)
        vh = st["v"][k] / (1.0 - b2 ** t)
        p[k] = p[k] - lr * mh / (np.sqrt(vh) + eps)


def train(p: dict, feats: np.ndarray, targets: np.ndarray, epochs: int, batch: int, lr: float, use_bf16=True,
          bf16_grads: bool = False):
    """Adam over contiguous batches of the rows in their given order; returns the mean
    loss of each epoch.  bf16_grads: the backward's product inputs rounded as in
    backward()."""
    st = adam_init(p)
    hist = []
    mask = slot_mask(feats)
    for _ in range(epochs):
        tot, nb = 0.0, 0
        for s in range(0, feats.shape[0], batch):
            f, t, mk = feats[s:s + batch], targets[s:s + batch], mask[s:s + batch]
            y, cache = forward(p, f, use_bf16)
            tot += loss(y, t, mk)
            nb += 1
            adam_step(p, backward(p, cache, y, t, mk, bf16_grads), st, lr)
        hist.append(tot / max(nb, 1))
    return hist


# ---------------------------------------------------------------------------------
# Learned interpolation
# ---------------------------------------------------------------------------------
def learned_rows(y: np.ndarray, Xh: np.ndarray, w: np.ndarray, cf: np.ndarray, cidx: np.ndarray, cand: np.ndarray,
                 ncand: np.ndarray, c: int, refit: bool, ridge: float):
    """P from the MLP outputs y (n x S): per fine point the c valid slots of largest |y|
    (lower slot on ties), weights y or the Eq. (3.6) minimiser over them."""
    n = Xh.shape[0]
    nc = int(cf.sum())
    rows, cols, vals = [], [], []
    for i in range(n):
        if cf[i]:
            rows.append(i)
            cols.append(int(cidx[i]))
            vals.append(1.0)
            continue
        m = int(ncand[i])
        if m == 0:
            continue
        order = sorted(range(m), key=lambda s: (-abs(y[i, s]), s))[:c]
        J = [int(cand[i, s]) for s in order]
        if refit:
            Xs = Xh[J]  # (|J|, K)
            G = (Xs * w) @ Xs.T
            b = (Xs * w) @ Xh[i]
            G = G + ridge * np.trace(G) / len(J) * np.eye(len(J))
            pv = np.linalg.solve(G, b)
        else:
            pv = np.array([y[i, s] for s in order])
        for j, v in zip(J, pv):
            rows.append(i)
            cols.append(int(cidx[j]))
            vals.append(float(v))
    P = sp.csr_matrix((vals, (rows, cols)), shape=(n, nc))
    P.sort_indices()
    return P


def vcycle_factor(H, iters: int = 20, seed: int = 7) -> float:
    """rho of the stationary iteration x <- x - C B x: power iteration on its residual
    propagator E = I - B C, r <- E r, from r_0 = B x_0 with x_0 in U[1, 2] (SplitMix64
    stream 0).  Residuals have 1^T r = 0 (1^T B = 0), the subspace without E's eigenvalue 1
    (left eigenvector 1); each step removes the mean of r (zero in exact arithmetic) and
    rescales r to unit norm.  rho = geometric mean of ||E r|| / ||r|| over the second half."""
    B = H.levels[0].B
    n = B.shape[0]
    x = 1.0 + ob.counter_uniform(seed, 0, np.arange(n, dtype=np.uint64))
    r = B @ x
    r = r - r.mean()
    r = r / np.linalg.norm(r)
    logs = []
    for _ in range(iters):
        r = r - B @ ob.vcycle(H, r)
        r = r - r.mean()
        nr = float(np.linalg.norm(r))
        logs.append(np.log(nr) if nr > 0 else -np.inf)
        if nr == 0.0:
            break
        r = r / nr
    tail = logs[len(logs) // 2:]
    return float(np.exp(np.mean(tail)))

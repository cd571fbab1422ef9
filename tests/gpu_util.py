"""Helpers shared by the GPU tests (test infrastructure)."""

import numpy as np
import scipy.sparse as sp


def need_gpu():
    import pytest
    import torch

    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_1004_1451_gb300.build as b

    b.build()


def dev_csr(M, dtype=None):
    import torch

    M = sp.csr_matrix(M)
    M.sort_indices()
    dtype = dtype or torch.float64
    return (torch.tensor(M.indptr.astype(np.int32), device="cuda"),
            torch.tensor(M.indices.astype(np.int32), device="cuda"),
            torch.tensor(M.data, dtype=dtype, device="cuda"))


def on_pattern(B, T):
    """Values of T at the positions of B's pattern (T's pattern must be contained)."""
    B = sp.csr_matrix(B)
    T = sp.csr_matrix(T)
    out = np.zeros(B.nnz)
    for i in range(B.shape[0]):
        row = dict(zip(T.indices[T.indptr[i]:T.indptr[i + 1]], T.data[T.indptr[i]:T.indptr[i + 1]]))
        for p in range(B.indptr[i], B.indptr[i + 1]):
            out[p] = row.pop(B.indices[p], 0.0)
        assert not row, "T has entries outside B's pattern"
    return out


def rel(a, b):
    a = np.asarray(a, dtype=np.float64)
    b = np.asarray(b, dtype=np.float64)
    return float(np.abs(a - b).sum() / max(np.abs(b).sum(), 1e-300))


def ell_from_csr(P, c):
    P = sp.csr_matrix(P)
    n = P.shape[0]
    pcol = np.full((n, c), -1, dtype=np.int32)
    pval = np.zeros((n, c))
    pcnt = np.diff(P.indptr).astype(np.int32)
    for i in range(n):
        a, b = P.indptr[i], P.indptr[i + 1]
        pcol[i, :b - a] = P.indices[a:b]
        pval[i, :b - a] = P.data[a:b]
    return pcol, pval, pcnt

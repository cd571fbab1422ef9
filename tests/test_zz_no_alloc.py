"""bamg_relax_noalloc, the relaxation entry point that allocates nothing (for callers
that may not allocate device memory), must give what bamg_relax gives.  Kept in a file
that pytest collects last, so that a run stopping at the first failure has run every
other test before it."""

import ctypes as C

import numpy as np
import pytest

from gpu_util import dev_csr, need_gpu, rel
from oracle import bamg as ob
from workloads import tandem_queue

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("dtype_name,r,ld,col0,nu,tol", [("float64", 6, 8, 0, 3, 1e-13), ("float32", 10, 16, 4, 4, 2e-6)])
def test_noalloc_matches_allocating_entry_point_twice(dtype_name, r, ld, col0, nu, tol):
    need_gpu()
    import torch

    import paper_1004_1451_gb300 as bamg

    dt = getattr(torch, dtype_name)
    ch = tandem_queue(40)  # 1681 states: several blocks and a ragged tail
    B = ob.system_matrix(ch.to_scipy())
    Bd = dev_csr(B, dt)
    for call in range(2):  # two calls in a row: the second starts from the first's leftovers
        X0 = ob.tv_init(ch.n, r, 100 + call, 0.0, 1.0)
        Xa = torch.zeros(ch.n, ld, dtype=dt, device="cuda")
        Xa[:, col0:col0 + r] = torch.tensor(X0, dtype=dt)
        Xb = Xa.clone()
        bamg.relax(Bd, Xa, r, col0, 0.7, nu)
        bamg.relax_noalloc(Bd, Xb, r, col0, 0.7, nu)
        a, b = Xa.cpu().numpy().astype(np.float64), Xb.cpu().numpy().astype(np.float64)
        assert rel(b[:, col0:col0 + r], a[:, col0:col0 + r]) < tol
        assert np.array_equal(b[:, :col0], a[:, :col0])


@pytest.mark.parametrize("dtype_name,r,ld,col0,tol", [("float64", 6, 8, 2, 1e-13), ("float32", 7, 12, 4, 2e-6)])
def test_noalloc_shifted_sweeps_match_allocating_entry_point(dtype_name, r, ld, col0, tol):
    # the shifted sweeps (B - lambda_k T) x_k = 0 of the eigenvector relaxation use the
    # diagonal of T and the shifts; T is B's pattern with values of a coarse mass matrix
    need_gpu()
    import torch

    import paper_1004_1451_gb300 as bamg

    dt = getattr(torch, dtype_name)
    ch = tandem_queue(33)
    B = ob.system_matrix(ch.to_scipy())
    Bd = dev_csr(B, dt)
    Tv = torch.tensor(1.0 + 0.25 * np.abs(B.data), dtype=dt, device="cuda")  # diagonally dominant, positive
    lam = torch.tensor(np.linspace(0.0, 0.05, r), dtype=torch.float64, device="cuda")
    for call in range(2):
        X0 = ob.tv_init(ch.n, r, 200 + call, 1.0, 2.0)
        Xa = torch.zeros(ch.n, ld, dtype=dt, device="cuda")
        Xa[:, col0:col0 + r] = torch.tensor(X0, dtype=dt)
        Xb = Xa.clone()
        bamg.relax(Bd, Xa, r, col0, 0.7, 2, T_val=Tv, lam=lam)
        bamg.relax_noalloc(Bd, Xb, r, col0, 0.7, 2, T_val=Tv, lam=lam)
        a, b = Xa.cpu().numpy().astype(np.float64), Xb.cpu().numpy().astype(np.float64)
        assert rel(b[:, col0:col0 + r], a[:, col0:col0 + r]) < tol


def test_negative_col0_is_refused_by_both_entry_points():
    need_gpu()
    import torch

    import paper_1004_1451_gb300 as bamg

    ch = tandem_queue(10)
    Bd = dev_csr(ob.system_matrix(ch.to_scipy()), torch.float64)
    X = torch.zeros(ch.n, 8, dtype=torch.float64, device="cuda")
    for fn in (bamg.relax, bamg.relax_noalloc):
        with pytest.raises(bamg.BamgError) as e:
            fn(Bd, X, 2, -2, 0.7, 1)
        assert e.value.code == bamg._capi.BAMG_EINVAL


def test_noalloc_rejects_sizes_beyond_its_scratch():
    need_gpu()
    import torch

    import paper_1004_1451_gb300 as bamg

    n = 1 << 18  # 262,144 rows x (32 + 3) doubles > 8 MiB
    rp = torch.arange(n + 1, dtype=torch.int32, device="cuda")
    ci = torch.arange(n, dtype=torch.int32, device="cuda")
    val = torch.ones(n, dtype=torch.float64, device="cuda")
    X = torch.zeros(n, 32, dtype=torch.float64, device="cuda")
    with pytest.raises(bamg.BamgError) as e:
        bamg.relax_noalloc((rp, ci, val), X, 32, 0, 0.7, 1)
    assert e.value.code == bamg._capi.BAMG_EINVAL
    assert "scratch" in str(e.value)

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

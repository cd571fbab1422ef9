"""GB300 Bootstrap AMG for Markov chains: Python binding of libbamg.so.

Argument marshalling only: every step runs in the library's CUDA kernels, and torch
provides device memory and the current stream.  The functions mirror include/bamg.h.
"""

from __future__ import annotations

import ctypes as C

import numpy as np
import torch

from . import _capi as capi
from ._capi import BamgError  # noqa: F401

__all__ = ["Solver", "Model", "solve_batch", "interp_dataset", "interp_features", "interp_learned", "import_hierarchy", "tv_init", "relax", "relax_noalloc", "tv_weights", "coarsen_grid", "coarsen_cr",
           "interp_ls", "galerkin", "coarse_eig", "launch_count", "default_opts", "BamgError"]


def _lib():
    return capi.load()


def _stream():
    return C.c_void_p(torch.cuda.current_stream().cuda_stream)


def _p(t):
    return C.c_void_p(t.data_ptr()) if t is not None else C.c_void_p(0)


def _dtype_code(t: torch.Tensor) -> int:
    if t.dtype == torch.float64:
        return capi.F64
    if t.dtype == torch.float32:
        return capi.F32
    raise TypeError("floating arrays must be float32 or float64")


def _i32(t):
    assert t.dtype == torch.int32 and t.is_contiguous(), "index arrays must be contiguous int32"
    return t


def _mat(rp, ci, val):
    return capi.Mat(int(rp.numel() - 1), int(ci.numel()), _p(_i32(rp)).value, _p(_i32(ci)).value, _p(val).value)


def launch_count() -> int:
    """Kernels launched by the library in this process."""
    return int(_lib().bamg_launch_count())


_OPT_NAMES = [f[0] for f in capi.Opts._fields_]


def default_opts(**kw) -> capi.Opts:
    o = capi.Opts()
    capi.check(_lib().bamg_default_opts(C.byref(o)))
    if "precision" in kw and isinstance(kw["precision"], str):
        kw["precision"] = {"fp64": capi.PREC_FP64, "mixed": capi.PREC_MIXED}[kw["precision"]]
    if "coarsen" in kw and isinstance(kw["coarsen"], str):
        kw["coarsen"] = {"grid": capi.COARSEN_GRID, "cr": capi.COARSEN_CR}[kw["coarsen"]]
    if "interp" in kw and isinstance(kw["interp"], str):
        kw["interp"] = {"ls": capi.INTERP_LS, "learned": capi.INTERP_LEARNED}[kw["interp"]]
    if "model" in kw:
        m = kw.pop("model")
        kw["model"] = m._h.value if m is not None else None
    if "smoother" in kw and isinstance(kw["smoother"], str):
        kw["smoother"] = {"jacobi": 0, "mcgs": 1}[kw["smoother"]]
    if "learned_refit" in kw:
        kw["learned_refit"] = int(bool(kw["learned_refit"]))
    if "grid" in kw:
        g = kw.pop("grid")
        if g is not None:
            kw["grid_nx"], kw["grid_ny"] = int(g[0]), int(g[1])
    for k, v in kw.items():
        if k not in _OPT_NAMES or k == "stream":
            raise KeyError(f"unknown option {k}")
        setattr(o, k, v)
    return o


class Solver:
    """Bootstrap AMG hierarchy of one chain (bamg_setup) and its preconditioned solve.

    row_ptr, col, val: CSR of the column-stochastic A (rows = destination states), as
    torch tensors on the GPU (int32, int32, float64) or, with on_host=True, on the CPU."""

    def __init__(self, row_ptr, col, val, r: int, levels: int, on_host: bool = False, **opts):
        self._h = C.c_void_p(0)
        o = default_opts(**opts)
        o.stream = _stream().value
        self.opts = o
        n = int(row_ptr.numel() - 1)
        if on_host:
            row_ptr = row_ptr.contiguous()
            col = col.contiguous()
            val = val.contiguous()
        self._keep = (row_ptr, col, val)
        A = capi.Csr(n, int(col.numel()), _p(_i32(row_ptr)).value, _p(_i32(col)).value, _p(val).value,
                     1 if on_host else 0)
        capi.check(_lib().bamg_setup(C.byref(A), r, levels, C.byref(o), C.byref(self._h)))
        self._keep = None
        self.n = n

    @classmethod
    def _from_handle(cls, h, n, o):
        self = cls.__new__(cls)
        self._h, self.n, self.opts, self._keep = h, n, o, None
        return self

    def _out(self, out, host, x0, norm):
        flags = capi.NORM_L2 if norm == "l2" else 0
        assert norm in ("l1", "l2")
        if host:
            flags |= capi.X_HOST
            x = out if out is not None else torch.empty(self.n, dtype=torch.float64, pin_memory=True)
        else:
            x = out if out is not None else torch.empty(self.n, dtype=torch.float64, device="cuda")
        if x0 is not None:
            x.copy_(x0)
            flags |= capi.X_GUESS
        return x, flags

    def solve(self, tol: float, x0=None, out=None, host: bool = False, norm: str = "l1"):
        """Returns (x, stats).  x0: optional initial guess (same device as out).  norm:
        "l1" (||Bx||_1/||x||_1 <= tol) or "l2" (the 2-norm ratio of the paper's tables)."""
        x, flags = self._out(out, host, x0, norm)
        st = capi.Stats()
        code = _lib().bamg_solve(self._h, _p(x), flags, float(tol), C.byref(st))
        stats = {f[0]: getattr(st, f[0]) for f in capi.Stats._fields_}
        if code != capi.BAMG_OK:
            err = BamgError(code, _lib().bamg_last_error().decode())
            err.stats = stats
            raise err
        return x, stats

    def parnoldi(self, tol: float, x0=None, out=None, host: bool = False, norm: str = "l1"):
        """Multigrid-preconditioned Arnoldi (bamg_parnoldi).  Returns (x, stats)."""
        x, flags = self._out(out, host, x0, norm)
        st = capi.Stats()
        code = _lib().bamg_parnoldi(self._h, _p(x), flags, float(tol), C.byref(st))
        stats = {f[0]: getattr(st, f[0]) for f in capi.Stats._fields_}
        if code != capi.BAMG_OK:
            err = BamgError(code, _lib().bamg_last_error().decode())
            err.stats = stats
            raise err
        return x, stats

    def vcycle(self, v: torch.Tensor) -> torch.Tensor:
        z = torch.empty_like(v)
        capi.check(_lib().bamg_vcycle_apply(self._h, _p(v.contiguous()), _p(z)))
        return z

    @property
    def dtype(self):
        """Arithmetic of the hierarchy and V-cycle (torch.float32 for mixed precision)."""
        code = _lib().bamg_hierarchy_precision(self._h)
        return torch.float32 if code == capi.F32 else torch.float64

    def smooth(self, level: int, b: torch.Tensor, x: torch.Tensor, sweeps: int = 1, work=None):
        """sweeps V-cycle smoother sweeps on `level`, x updated in place, launched
        asynchronously on the stream the hierarchy was set up on."""
        assert b.dtype == self.dtype and x.dtype == self.dtype and x.is_contiguous() and b.is_contiguous()
        if work is None:
            work = torch.empty_like(x)
        capi.check(_lib().bamg_smooth_apply(self._h, level, sweeps, _p(b), _p(x), _p(work)))
        return x

    def vcycle_factor(self, iters: int = 20) -> float:
        """V-cycle factor of x <- x - C B x (power iteration on I - B C, bamg_vcycle_factor)."""
        rho = C.c_double()
        capi.check(_lib().bamg_vcycle_factor(self._h, iters, C.byref(rho)))
        return rho.value

    def interp_used(self):
        """("ls" | "learned", the V-cycle factor measured for the fallback decision or 0)."""
        rho = C.c_double()
        code = _lib().bamg_hierarchy_interp(self._h, C.byref(rho))
        if code < 0:
            raise BamgError(code, "bad handle")
        return ("learned" if code == capi.INTERP_LEARNED else "ls"), rho.value

    def info(self) -> dict:
        L = C.c_int(0)
        ns = (C.c_int64 * 32)()
        nz = (C.c_int64 * 32)()
        opc = C.c_double(0)
        capi.check(_lib().bamg_hierarchy_info(self._h, C.byref(L), ns, nz, C.byref(opc)))
        return {"levels": L.value, "n": list(ns[:L.value]), "nnz": list(nz[:L.value]), "op_complexity": opc.value}

    def layout(self) -> dict:
        ld, r, v0, nv = C.c_int(), C.c_int(), C.c_int(), C.c_int()
        capi.check(_lib().bamg_hierarchy_layout(self._h, 0, C.byref(ld), C.byref(r), C.byref(v0), C.byref(nv)))
        return {"ld": ld.value, "r": r.value, "v_col0": v0.value, "nvec": nv.value}

    def export(self, level: int, what: int):
        need = C.c_int64(0)
        code = _lib().bamg_level_export(self._h, level, what, None, 0, C.byref(need))
        if code not in (capi.BAMG_OK, capi.BAMG_ESIZE):
            capi.check(code)
        buf = np.zeros(max(int(need.value), 1), dtype=np.uint8)
        capi.check(_lib().bamg_level_export(self._h, level, what, buf.ctypes.data, need.value, C.byref(need)))
        info = self.info()
        n = info["n"][level]
        if what == capi.EXPORT_B:
            nnz = info["nnz"][level]
            rp = buf[:4 * (n + 1)].view(np.int32)
            ci = buf[4 * (n + 1):4 * (n + 1) + 4 * nnz].view(np.int32)
            v = buf[4 * (n + 1) + 4 * nnz:].view(np.float64)
            return rp, ci, v
        if what == capi.EXPORT_P:
            c = self.opts.caliber
            pcol = buf[:4 * n * c].view(np.int32).reshape(n, c)
            pcnt = buf[4 * n * c:4 * n * c + 4 * n].view(np.int32)
            pval = buf[4 * n * c + 4 * n:].view(np.float64).reshape(n, c)
            return pcol, pval, pcnt
        if what == capi.EXPORT_CF:
            return buf[:n].astype(bool)
        if what == capi.EXPORT_X:
            return buf.view(np.float64).reshape(n, -1)
        if what == capi.EXPORT_PINV:
            m = int(round(np.sqrt(need.value / 8)))
            return buf.view(np.float64).reshape(m, m)
        return buf.view(np.float64)

    def close(self):
        if self._h:
            _lib().bamg_free(self._h)
            self._h = C.c_void_p(0)

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def solve_batch(chains, r, levels, tol: float, opts=None, workers: int = 0, host: bool = False):
    """bamg_solve_batch over a list of chains.  chains[k] = (row_ptr, col, val) torch
    tensors (on the GPU, or on the CPU with host=True); r, levels: ints or per-chain
    lists; opts: a dict of options or a list of dicts (e.g. grid=(nx, ny) per chain).
    Returns (list of x tensors, list of stats dicts); raises on the first failing chain."""
    n = len(chains)
    rs = [r] * n if isinstance(r, int) else list(r)
    lv = [levels] * n if isinstance(levels, int) else list(levels)
    ol = [dict(opts or {}) for _ in range(n)] if not isinstance(opts, (list, tuple)) else [dict(o) for o in opts]
    As = (capi.Csr * n)()
    Os = (capi.Opts * n)()
    xs = (C.c_void_p * n)()
    keep, outs = [], []
    for k, (rp, ci, v) in enumerate(chains):
        if host:
            rp, ci, v = rp.contiguous(), ci.contiguous(), v.contiguous()
        keep += [rp, ci, v]
        m = int(rp.numel() - 1)
        As[k] = capi.Csr(m, int(ci.numel()), _p(_i32(rp)).value, _p(_i32(ci)).value, _p(v).value, 1 if host else 0)
        Os[k] = default_opts(**ol[k])
        x = torch.empty(m, dtype=torch.float64, pin_memory=True) if host else \
            torch.empty(m, dtype=torch.float64, device="cuda")
        outs.append(x)
        xs[k] = x.data_ptr()
    st = (capi.Stats * n)()
    torch.cuda.synchronize()
    code = _lib().bamg_solve_batch(n, As, (C.c_int * n)(*rs), (C.c_int * n)(*lv), Os, xs,
                                   capi.X_HOST if host else 0, float(tol), workers, st)
    stats = [{f[0]: getattr(st[k], f[0]) for f in capi.Stats._fields_} for k in range(n)]
    if code != capi.BAMG_OK:
        err = BamgError(code, _lib().bamg_last_error().decode())
        err.stats = stats
        err.xs = outs  # every chain's result (the failed ones hold their last iterate)
        raise err
    return outs, stats


class Model:
    """The MLP of the learned interpolation (bamg_model_*): 112 features -> 128 -> 128 -> 16
    slot weights, bfloat16 products with FP32 sums, trained with Adam on LS rows."""

    F, H, S = capi.MLP_F, capi.MLP_H, capi.MLP_S

    def __init__(self, seed: int = 0):
        self._h = C.c_void_p(0)
        capi.check(_lib().bamg_model_create(seed, C.byref(self._h)))
        self.n_params = int(_lib().bamg_model_param_count())

    def close(self):
        if self._h.value:
            _lib().bamg_model_free(self._h)
            self._h = C.c_void_p(0)

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def get(self) -> np.ndarray:
        out = np.empty(self.n_params, dtype=np.float32)
        capi.check(_lib().bamg_model_get(self._h, out.ctypes.data, self.n_params))
        return out

    def set(self, params) -> None:
        a = np.ascontiguousarray(params, dtype=np.float32)
        assert a.size == self.n_params
        capi.check(_lib().bamg_model_set(self._h, a.ctypes.data, self.n_params))

    def forward(self, feat: torch.Tensor) -> torch.Tensor:
        assert feat.dtype == torch.float32 and feat.is_contiguous() and feat.shape[1] == self.F
        y = torch.empty(feat.shape[0], self.S, dtype=torch.float32, device=feat.device)
        capi.check(_lib().bamg_model_forward(self._h, _p(feat), feat.shape[0], _p(y), _stream()))
        return y

    def gradients(self, feat: torch.Tensor, target: torch.Tensor):
        g = np.empty(self.n_params, dtype=np.float32)
        loss = C.c_double()
        capi.check(_lib().bamg_model_gradients(self._h, _p(feat), _p(target), feat.shape[0], g.ctypes.data,
                                               C.byref(loss), _stream()))
        return g, loss.value

    def train(self, feat: torch.Tensor, target: torch.Tensor, epochs: int, batch: int, lr: float):
        """Adam over contiguous batches in row order; returns the mean batch loss per epoch."""
        assert feat.is_contiguous() and target.is_contiguous()
        hist = np.zeros(max(epochs, 1))
        capi.check(_lib().bamg_model_train(self._h, _p(feat), _p(target), feat.shape[0], epochs, batch, float(lr),
                                           hist.ctypes.data, _stream()))
        return hist[:epochs]


def interp_dataset(row_ptr, col, val, r: int, levels: int, **opts):
    """(features, LS targets) of every point of every level of a least-squares setup
    (bamg_interp_dataset), as float32 CUDA tensors (rows x 112, rows x 16)."""
    n = int(row_ptr.numel() - 1)
    A = capi.Csr(n, int(col.numel()), _p(_i32(row_ptr)).value, _p(_i32(col)).value, _p(val).value, 0)
    o = default_opts(**opts)
    o.stream = _stream().value
    need = C.c_int64(0)
    code = _lib().bamg_interp_dataset(C.byref(A), r, levels, C.byref(o), None, None, 0, C.byref(need))
    if code not in (capi.BAMG_OK, capi.BAMG_ESIZE):
        capi.check(code)
    rows = need.value
    feat = torch.empty(rows, capi.MLP_F, dtype=torch.float32, device=row_ptr.device)
    tgt = torch.empty(rows, capi.MLP_S, dtype=torch.float32, device=row_ptr.device)
    capi.check(_lib().bamg_interp_dataset(C.byref(A), r, levels, C.byref(o), _p(feat), _p(tgt), rows,
                                          C.byref(need)))
    return feat, tgt


def interp_features(B, cf, cidx, X, ncols, w, z=2, mmax=16, c=2, ridge=1e-4, targets=False):
    """The LS kernel's per-point features (and, with targets, its LS rows on the slots and
    candidates) for one level (bamg_interp_features)."""
    rp, ci, v = B
    n = int(rp.numel() - 1)
    m = _mat(rp, ci, v)
    feat = torch.empty(n, capi.MLP_F, dtype=torch.float32, device=v.device)
    tgt = torch.empty(n, capi.MLP_S, dtype=torch.float32, device=v.device) if targets else None
    cand = torch.empty(n, capi.MLP_S, dtype=torch.int32, device=v.device)
    capi.check(_lib().bamg_interp_features(_dtype_code(v), C.byref(m), _p(cf), _p(cidx), _p(X), ncols, X.shape[1],
                                           _p(w), z, mmax, c, float(ridge), _p(feat), _p(tgt), _p(cand), _stream()))
    return feat, tgt, cand


def interp_learned(B, cf, cidx, X, ncols, w, model: Model, refit=True, z=2, mmax=16, c=2, ridge=1e-4):
    """Learned interpolation of one level (bamg_interp_learned): P in ELL form."""
    rp, ci, v = B
    n = int(rp.numel() - 1)
    m = _mat(rp, ci, v)
    pcol = torch.empty(n * c, dtype=torch.int32, device=v.device)
    pval = torch.empty(n * c, dtype=v.dtype, device=v.device)
    pcnt = torch.empty(n, dtype=torch.int32, device=v.device)
    capi.check(_lib().bamg_interp_learned(_dtype_code(v), C.byref(m), _p(cf), _p(cidx), _p(X), ncols, X.shape[1],
                                          _p(w), z, mmax, c, float(ridge), model._h, int(bool(refit)), _p(pcol),
                                          _p(pval), _p(pcnt), _stream()))
    return pcol.view(n, c), pval.view(n, c), pcnt


def import_hierarchy(levels, pinv: np.ndarray, x_init: np.ndarray, **opts) -> Solver:
    """Solver over a given hierarchy.  levels: list of dicts with numpy 'B' = (row_ptr,
    col, val) and, except on the coarsest level, 'P' = (row_ptr, col, val) in CSR."""
    o = default_opts(**opts)
    o.stream = _stream().value
    keep = []
    arr = (capi.LevelIn * len(levels))()
    for l, lv in enumerate(levels):
        rp, ci, v = (np.ascontiguousarray(lv["B"][0], np.int32), np.ascontiguousarray(lv["B"][1], np.int32),
                     np.ascontiguousarray(lv["B"][2], np.float64))
        keep += [rp, ci, v]
        arr[l].n, arr[l].nnz = len(rp) - 1, len(ci)
        arr[l].h_row_ptr, arr[l].h_col, arr[l].h_val = rp.ctypes.data, ci.ctypes.data, v.ctypes.data
        if "P" in lv:
            prp, pci, pv = (np.ascontiguousarray(lv["P"][0], np.int32), np.ascontiguousarray(lv["P"][1], np.int32),
                            np.ascontiguousarray(lv["P"][2], np.float64))
            keep += [prp, pci, pv]
            arr[l].p_nnz = len(pci)
            arr[l].h_p_row_ptr, arr[l].h_p_col, arr[l].h_p_val = prp.ctypes.data, pci.ctypes.data, pv.ctypes.data
    pinv = np.ascontiguousarray(pinv, np.float64)
    x_init = np.ascontiguousarray(x_init, np.float64)
    h = C.c_void_p(0)
    capi.check(_lib().bamg_import(len(levels), arr, pinv.ctypes.data, x_init.ctypes.data, C.byref(o), C.byref(h)))
    return Solver._from_handle(h, int(arr[0].n), o)


# ------------------------------------------------------------------ step entry points
def tv_init(X: torch.Tensor, ncols: int, col0: int, seed: int, lo: float, hi: float):
    n, ld = X.shape
    capi.check(_lib().bamg_tv_init(_dtype_code(X), n, ncols, ld, col0, seed, lo, hi, _p(X), _stream()))
    return X


def _check_relax_args(B, X, ncols, T_val, lam):
    """The C ABI takes raw device pointers with X row-major (n x ld): check the tensors
    behind them before handing their addresses over."""
    assert X.is_cuda and X.dim() == 2 and X.is_contiguous(), "X must be a contiguous 2-D CUDA tensor (n x ld)"
    assert X.dtype in (torch.float64, torch.float32), "X must be float64 or float32"
    assert B[2].is_cuda and B[2].dtype == X.dtype and B[2].is_contiguous(), "B's values must be CUDA tensors of X's dtype"
    assert T_val is None or (T_val.is_cuda and T_val.dtype == X.dtype and T_val.is_contiguous()
                             and T_val.numel() == B[1].numel()), "T_val must match B's pattern and X's dtype"
    assert lam is None or (lam.is_cuda and lam.dtype == torch.float64 and lam.numel() >= ncols), \
        "lam must be a CUDA float64 tensor with at least ncols entries"


def relax(B, X: torch.Tensor, ncols: int, col0: int, omega: float, nu: int, T_val=None, lam=None, work=None):
    """B = (row_ptr, col, val) device tensors with val in X's dtype."""
    _check_relax_args(B, X, ncols, T_val, lam)
    n, ld = X.shape
    work = torch.empty_like(X) if work is None else work
    m = _mat(*B)
    capi.check(_lib().bamg_relax(_dtype_code(X), C.byref(m), _p(T_val), _p(lam), ncols, ld, col0, omega, nu, _p(X),
                                 _p(work), _stream()))
    return X


def autotune_report():
    """The SpMM sweep shapes the autotuner chose in this process (bamg_autotune_report):
    one dict per key."""
    rows = (C.c_int32 * (7 * 64))()
    k = _lib().bamg_autotune_report(rows, 64)
    capi.check(min(k, 0))
    names = ("elem_bytes", "shift", "entry_batch", "chunks_per_row", "log2_n", "chunks_per_thread", "blocks_per_sm")
    return [dict(zip(names, rows[7 * r:7 * r + 7])) for r in range(k)]


def mle_solve(row_ptr, col, val, r: int, levels: int, tol: float, max_cycles: int = 50, norm: str = "l1",
              keep: bool = False, **opts):
    """The MLE as a stand-alone solver (bamg_mle_solve): returns (x, stats, solver or None).
    With keep=True the rebuilt hierarchy comes back as a Solver (also when the MLE did not
    converge; stats["status"] then says so) for a following solve() or parnoldi()."""
    o = default_opts(**opts)
    o.stream = _stream().value
    n = int(row_ptr.numel() - 1)
    A = capi.Csr(n, int(col.numel()), _p(_i32(row_ptr)).value, _p(_i32(col)).value, _p(val).value, 0)
    x = torch.empty(n, dtype=torch.float64, device="cuda")
    st = capi.Stats()
    h = C.c_void_p(0)
    flags = capi.NORM_L2 if norm == "l2" else 0
    code = _lib().bamg_mle_solve(C.byref(A), r, levels, C.byref(o), float(tol), int(max_cycles), flags, _p(x),
                                 C.byref(st), C.byref(h) if keep else None)
    stats = {f[0]: getattr(st, f[0]) for f in capi.Stats._fields_}
    solver = Solver._from_handle(h, n, o) if keep and h.value else None
    if code not in (capi.BAMG_OK, capi.BAMG_ENOCONV) or (code != capi.BAMG_OK and not keep):
        if solver is not None:
            solver.close()
        err = BamgError(code, _lib().bamg_last_error().decode())
        err.stats = stats
        raise err
    stats["status"] = code
    return x, stats, solver


def relax_noalloc(B, X: torch.Tensor, ncols: int, col0: int, omega: float, nu: int, T_val=None, lam=None):
    """bamg_relax_noalloc: the sweeps of relax() with the library's fixed device scratch
    instead of any allocation (see include/bamg.h for its size limit)."""
    _check_relax_args(B, X, ncols, T_val, lam)
    n, ld = X.shape
    m = _mat(*B)
    capi.check(_lib().bamg_relax_noalloc(_dtype_code(X), C.byref(m), _p(T_val), _p(lam), ncols, ld, col0, omega, nu,
                                         _p(X), _stream()))
    return X


def tv_weights(B, X: torch.Tensor, ncols: int, col0: int = 0, active=None, floor: float = 1e-28):
    n, ld = X.shape
    w = torch.zeros(ncols, dtype=torch.float64, device=X.device)
    m = _mat(*B)
    capi.check(_lib().bamg_tv_weights(_dtype_code(X), C.byref(m), ncols, ld, col0, _p(active), floor, _p(X), _p(w),
                                      _stream()))
    return w


def coarsen_grid(nx: int, ny: int):
    cf = torch.empty(nx * ny, dtype=torch.uint8, device="cuda")
    cidx = torch.empty(nx * ny, dtype=torch.int32, device="cuda")
    capi.check(_lib().bamg_coarsen_grid(nx, ny, _p(cf), _p(cidx), _stream()))
    return cf, cidx


def coarsen_cr(B, level: int, seed: int, theta: float = 0.85, nu: int = 8, omega: float = 0.7, max_rounds: int = 20):
    n = int(B[0].numel() - 1)
    cf = torch.empty(n, dtype=torch.uint8, device="cuda")
    cidx = torch.empty(n, dtype=torch.int32, device="cuda")
    nc, rounds = C.c_int(), C.c_int()
    m = _mat(*B)
    capi.check(_lib().bamg_coarsen_cr(C.byref(m), level, seed, theta, nu, omega, max_rounds, _p(cf), _p(cidx),
                                      C.byref(nc), C.byref(rounds), _stream()))
    return cf, cidx, nc.value, rounds.value


def interp_ls(B, cf, cidx, X: torch.Tensor, ncols: int, w, z: int = 2, mmax: int = 16, c: int = 2,
              ridge: float = 1e-12):
    n, ld = X.shape
    pcol = torch.empty(n * c, dtype=torch.int32, device=X.device)
    pval = torch.empty(n * c, dtype=X.dtype, device=X.device)
    pcnt = torch.empty(n, dtype=torch.int32, device=X.device)
    m = _mat(B[0], B[1], X)  # only the pattern of B is read
    capi.check(_lib().bamg_interp_ls(_dtype_code(X), C.byref(m), _p(cf), _p(cidx), _p(X), ncols, ld, _p(w), z, mmax,
                                     c, ridge, _p(pcol), _p(pval), _p(pcnt), _stream()))
    return pcol.view(n, c), pval.view(n, c), pcnt


def galerkin(B, T_val, nc: int, pcol, pval, pcnt, c: int):
    val = B[2]
    m = _mat(*B)
    need = C.c_int64(0)
    rp = torch.empty(nc + 1, dtype=torch.int32, device=val.device)
    code = _lib().bamg_galerkin(_dtype_code(val), C.byref(m), _p(T_val), nc, _p(pcol), _p(pval), _p(pcnt), c, _p(rp),
                                None, None, None, 0, C.byref(need), _stream())
    if code not in (capi.BAMG_OK, capi.BAMG_ESIZE):
        capi.check(code)
    nnz = int(need.value)
    ci = torch.empty(max(nnz, 1), dtype=torch.int32, device=val.device)
    bv = torch.empty(max(nnz, 1), dtype=val.dtype, device=val.device)
    tv = torch.empty(max(nnz, 1), dtype=val.dtype, device=val.device)
    capi.check(_lib().bamg_galerkin(_dtype_code(val), C.byref(m), _p(T_val), nc, _p(pcol), _p(pval), _p(pcnt), c,
                                    _p(rp), _p(ci), _p(bv), _p(tv), nnz, C.byref(need), _stream()))
    return rp, ci[:nnz], bv[:nnz], tv[:nnz]


def coarse_eig(Bd: torch.Tensor, Td: torch.Tensor, k_ev: int, with_pinv: bool = True, fp32_vectors: bool = False):
    n = Bd.shape[0]
    lam = torch.zeros(k_ev + 1, dtype=torch.float64, device=Bd.device)
    V = torch.zeros(k_ev + 1, n, dtype=torch.float64, device=Bd.device)
    kinds = torch.zeros(k_ev + 1, dtype=torch.int32, device=Bd.device)
    pinv = torch.zeros(n, n, dtype=torch.float64, device=Bd.device) if with_pinv else None
    nv = C.c_int()
    capi.check(_lib().bamg_coarse_eig(capi.F32 if fp32_vectors else capi.F64, n, _p(Bd.contiguous()),
                                      _p(Td.contiguous()), k_ev, _p(lam), _p(V), _p(kinds),
                                      C.byref(nv), _p(pinv), _stream()))
    k = nv.value
    return lam[:k], V[:k].T, kinds[:k], pinv

"""Time to ||Bx||_1 / ||x||_1 <= 1e-10 for Bootstrap AMG on GB300.

Workload (one step = the whole hot path: setup + preconditioned GMRES): the tandem
queueing network with two queues of capacity 255 (65,536 states), arrival 11/31,
service 10/31 and 10/31, r = 10 test vectors, FP32 setup and V-cycle inside FP64
flexible GMRES.  Inputs are resident in HBM when a step's timing starts; L2 is
flushed between steps.  Also reported: the same metric end to end from host buffers,
the plain FP64 method on the same chain, the roofline of the dominant kernel (the V-cycle
smoother on the finest level), an SpMM HBM probe, the batched form on 512 chains, LS vs
learned interpolation on a held-out tandem queue of 262,144 states, the 2^20-point
Delaunay walk, the 64x64 grid walk, plain-FP64 runs beside the mixed ones, and the CPU
oracle on the host cores.

python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
Profiling helpers: --only-step, --kernel-probe, --probe-only N, --large-only,
--large-reps R, --device-loop 0 (one graph launch per Arnoldi step, so that ncu lists the
solve kernels), --no-batch, --no-learned, --no-large, --no-variants.
"""

import os

# the CPU oracle is timed single-threaded; set before numpy loads
for _v in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS"):
    os.environ.setdefault(_v, "1")

import argparse
import json
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "time to ||Bx||_1/||x||_1 <= 1e-10 (setup + solve), mixed FP32/FP64"
WORKLOAD = "tandem queue, capacities 255 (65,536 states), rates 11/31, 10/31, 10/31; r=10; mixed FP32 V-cycle in FP64 FGMRES"
TOL = 1e-10
N_CAP = 255
R = 10


def _workload():
    from workloads import tandem_queue

    return tandem_queue(N_CAP)


def _dist():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    return ws, rank


def max_over_ranks(v: float, device) -> float:
    """The maximum of v over the ranks of the initialised process group (v itself when
    there is none): the job's step time is its slowest replica's."""
    import torch
    import torch.distributed as dist

    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return v
    t = torch.tensor([v], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def _line(d):
    print(json.dumps(d), flush=True)


# ------------------------------------------------------------------ clocks
class Clocks:
    def __init__(self):
        self.p = None
        import tempfile

        self.path = os.path.join(tempfile.gettempdir(), f"bamg_clocks_{os.getpid()}.csv")

    def start(self):
        try:
            os.makedirs(os.path.dirname(self.path), exist_ok=True)
            q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
                 "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
                 "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")
            self.f = open(self.path, "w")
            # this rank's own GPU only: nvidia-smi numbers devices physically, so map the
            # local rank through CUDA_VISIBLE_DEVICES (indices or UUIDs) when it is set
            local = int(os.environ.get("LOCAL_RANK", "0"))
            vis = [v.strip() for v in os.environ.get("CUDA_VISIBLE_DEVICES", "").split(",") if v.strip()]
            dev = vis[local] if local < len(vis) else str(local)
            self.p = subprocess.Popen(["nvidia-smi", "-i", dev, f"--query-gpu={q}", "--format=csv,noheader,nounits",
                                       "-lms", "100"], stdout=self.f, stderr=subprocess.DEVNULL)
        except Exception:
            self.p = None

    def stop(self):
        if self.p is None:
            return None
        self.p.terminate()
        try:
            self.p.wait(timeout=5)
        except Exception:
            self.p.kill()
        self.f.close()
        sm, mx, reasons = [], 0.0, set()
        for line in open(self.path):
            f = [x.strip() for x in line.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                mx = max(mx, float(f[2]))
            except ValueError:
                continue
            for name, val in zip(("hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"), f[5:9]):
                if val.lower().startswith("active"):
                    reasons.add(name)
        if not sm:
            return None
        return {"sm_mhz": float(np.median(sm)), "sm_max_mhz": mx, "reasons": sorted(reasons), "samples": len(sm)}


# ------------------------------------------------------------------ our arm
def run_ours(args):
    import torch

    import paper_1004_1451_gb300 as bamg
    import paper_1004_1451_gb300.build as pb

    ws, rank = _dist()
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    if ws > 1:
        import torch.distributed as dist

        dist.init_process_group("nccl")
    pb.build()
    ch = _workload()
    dev = torch.device("cuda", local)
    rp = torch.tensor(ch.row_ptr, device=dev)
    ci = torch.tensor(ch.col, device=dev)
    v = torch.tensor(ch.val, device=dev)
    x = torch.empty(ch.n, dtype=torch.float64, device=dev)
    flush = torch.empty(256 << 20, dtype=torch.uint8, device=dev)
    stream = torch.cuda.current_stream()

    def step(precision="mixed"):
        s = bamg.Solver(rp, ci, v, r=R, levels=20, grid=ch.grid, precision=precision,
                        device_loop=args.device_loop, persistent=args.persistent,
                        coarse_tail=args.coarse_tail)
        _, st = s.solve(TOL, out=x)
        return s, st

    for _ in range(args.warmup):
        s, st = step()
        s.close()
    torch.cuda.synchronize()
    if ws > 1:
        dist.barrier()
    clocks = Clocks()
    clocks.start()
    times, iters, split, waits = [], [], [], []
    l0 = bamg.launch_count()
    for _ in range(args.steps):
        flush.fill_(1)
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        s, st = step()
        e1.record(stream)
        e1.synchronize()
        times.append(e0.elapsed_time(e1))
        iters.append(st["iterations"])
        split.append((st["setup_ms"], st["solve_ms"]))
        waits.append(st["host_waits"])
        s.close()
    launches = (bamg.launch_count() - l0) / args.steps
    torch.cuda.synchronize()
    ck = clocks.stop()
    if args.only_step:
        if rank == 0:
            _line({"metric": METRIC, "value": round(float(np.mean(times)), 4), "unit": "ms",
                   "gmres_iterations": int(np.median(iters)), "host_waits_in_solve": int(np.median(waits)),
                   "gpu_launches": int(round(launches)), "only_step": True})
        return
    ms = max_over_ranks(float(np.sum(times)) / args.steps, dev)
    if ws > 1:
        dist.barrier()
    # ---- accuracy of the timed result against a sparse direct solution
    xe = _direct_stationary(ch) if rank == 0 else None
    xr = x.cpu().numpy()
    err = float(np.abs(xr - xe).sum() / np.abs(xe).sum()) if xe is not None else None
    # ---- end to end from host buffers through the C ABI
    hrp, hci, hv = torch.tensor(ch.row_ptr).pin_memory(), torch.tensor(ch.col).pin_memory(), torch.tensor(ch.val).pin_memory()
    hx = torch.empty(ch.n, dtype=torch.float64).pin_memory()
    e2e = []
    for k in range(max(2, args.steps // 2) + 1):
        flush.fill_(1)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        s = bamg.Solver(hrp, hci, hv, r=R, levels=20, grid=ch.grid, precision="mixed", on_host=True)
        s.solve(TOL, out=hx, host=True)
        e2e.append((time.perf_counter() - t0) * 1e3)
        s.close()
    e2e_ms = float(np.median(e2e[1:]))
    # ---- plain FP64 method on the same chain
    fp64 = []
    for k in range(3):
        flush.fill_(1)
        torch.cuda.synchronize()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        s, st64 = step("fp64")
        e1.record(stream)
        e1.synchronize()
        fp64.append(e0.elapsed_time(e1))
        s.close()
    if ws > 1:
        dist.destroy_process_group()
    if rank != 0:
        return
    peaks = json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json"))) if os.path.exists(
        os.path.join(ROOT, "MEASURED_PEAKS.json")) else {"hbm_gbs": 6800.0, "_fallback": True}
    s_dom = bamg.Solver(rp, ci, v, r=R, levels=20, grid=ch.grid, precision="mixed")
    roof = dominant_kernel(s_dom, peaks)
    s_dom.close()
    probe = spmm_probe(peaks) if not args.no_probe else None
    batch = batch_line(args) if not args.no_batch else None
    learned = learned_line(args) if not args.no_learned else None
    large = large_line(args) if not args.no_large else None
    variants = variants_line(args) if not args.no_variants else None
    small = small_line(args)
    cpu = cpu_baseline() if not args.no_cpu else None
    nnz_a = int(ch.nnz)
    out = {
        "metric": METRIC, "value": round(ms, 4), "unit": "ms", "n_gpus": ws, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": round(ms, 4), "higher_is_better": False, "scaling": "weak",
        "vs_baseline": None, "dtype": "f32+f64", "data": "synthetic",
        "config": {"workload": WORKLOAD, "n": ch.n, "nnz_A": nnz_a, "r": R, "tol": TOL,
                   "l2": "flushed between steps (256 MiB write)", "parallelism": f"replicas x{ws}"},
        "gmres_iterations": int(np.median(iters)), "host_waits_in_solve": int(np.median(waits)),
        "rel_l1_vs_exact": err,
        "host_setup_ms": round(float(np.median([a for a, b in split])), 3),
        "host_solve_ms": round(float(np.median([b for a, b in split])), 3),
        "e2e": {"value": round(e2e_ms, 4), "unit": "ms", "h2d_bytes_per_step": 4 * (ch.n + 1) + 12 * nnz_a,
                "d2h_bytes_per_step": 8 * ch.n},
        "fp64_ms": round(float(np.median(fp64)), 4), "fp64_iterations": st64["iterations"],
        "speedup_mixed_vs_fp64": round(float(np.median(fp64)) / ms, 3),
        "gpu_launches": int(round(launches)),
        "roofline": roof, "spmm_hbm": probe, "batch": batch, "learned": learned, "large": large, "small": small, "variants": variants, "cpu_baseline": cpu, "clocks": ck,
    }
    _line(out)


VARIANTS_WORKLOAD = "tandem 256 x 256 (the timed chain), mixed, r=10, tol 1e-10 (l1 ratio)"


def variants_line(args, reps=3):
    """The method's variants on the timed chain: the default (omega-Jacobi V(2,2), one V-cycle
    setup, FGMRES); the multicolour Gauss-Seidel smoother; the W-cycle setup (mu = 2); two
    setup cycles (V^2); and the multigrid-preconditioned Arnoldi solver.  Per variant: the
    median over `reps` runs of setup and solve time (CUDA events around each phase on the
    launching stream), iterations, and the V-cycle factor of the hierarchy (20 steps)."""
    import torch

    import paper_1004_1451_gb300 as bamg
    from workloads import tandem_queue

    ch = tandem_queue(255)
    dev = torch.device("cuda")
    rp, ci, v = (torch.tensor(ch.row_ptr, device=dev), torch.tensor(ch.col, device=dev),
                 torch.tensor(ch.val, device=dev))
    stream = torch.cuda.current_stream()
    out = {"workload": VARIANTS_WORKLOAD}
    for name, kw, solver in [("default", {}, "fgmres"), ("mcgs_smoother", dict(smoother="mcgs"), "fgmres"),
                             ("w_cycle_setup", dict(mu=2), "fgmres"), ("two_setup_cycles", dict(setup_cycles=2),
                                                                       "fgmres"),
                             ("parnoldi", {}, "parnoldi")]:
        rows = []
        for _ in range(reps + 1):
            e = [torch.cuda.Event(enable_timing=True) for _ in range(3)]
            e[0].record(stream)
            s = bamg.Solver(rp, ci, v, r=R, levels=20, grid=ch.grid, precision="mixed", **kw)
            e[1].record(stream)
            x, st = s.parnoldi(TOL) if solver == "parnoldi" else s.solve(TOL)
            e[2].record(stream)
            e[2].synchronize()
            rho = s.vcycle_factor(20)
            s.close()
            rows.append((e[0].elapsed_time(e[1]), e[1].elapsed_time(e[2]), st["iterations"], rho))
        rows = rows[1:]  # the first run warms up
        out[name] = {"setup_ms": round(float(np.median([r[0] for r in rows])), 3),
                     "solve_ms": round(float(np.median([r[1] for r in rows])), 3),
                     "iterations": int(np.median([r[2] for r in rows])),
                     "vcycle_factor": round(float(np.median([r[3] for r in rows])), 4)}
    return out


def _direct_stationary(ch):
    """x with (I - A) x = 0, 1^T x = 1 by a sparse LU (SuperLU): fix the last entry to one,
    solve the remaining rows and columns of I - A (nonsingular for an irreducible chain)
    and normalise.  The accuracy yardstick of the timed result."""
    import scipy.sparse as sp
    import scipy.sparse.linalg as spla

    n = ch.n
    M = (sp.identity(n, format="csr") - ch.to_scipy().tocsr()).tocsc()
    x = np.ones(n)
    x[:-1] = spla.spsolve(M[:-1, :-1], -M[:-1, n - 1].toarray().ravel())
    return x / x.sum()


def _grid_B(N, dev, dtype):
    """B = I - A of the N x N grid walk, built directly on the device (sorted CSR)."""
    import torch

    n = N * N
    i = torch.arange(n, device=dev, dtype=torch.int64)
    x, y = i % N, i // N
    deg = (x > 0).long() + (x < N - 1).long() + (y > 0).long() + (y < N - 1).long()
    cols = torch.stack([i - N, i - 1, i, i + 1, i + N], 1)
    ok = torch.stack([y > 0, x > 0, torch.ones_like(x, dtype=torch.bool), x < N - 1, y < N - 1], 1)
    cc = cols.clamp(0, n - 1)
    vals = torch.where(cols == i[:, None], torch.ones_like(cc, dtype=torch.float64), -1.0 / deg[cc].double())
    rp = torch.zeros(n + 1, dtype=torch.int64, device=dev)
    rp[1:] = torch.cumsum(ok.sum(1), 0)
    return rp.int(), cols[ok].int(), vals[ok].to(dtype)


def _time_relax(bamg, B, X, ncols, col0, reps, stream, sweeps=20):
    """Average duration of one omega-Jacobi sweep launch: `sweeps` launches per call
    (the call's two diagonal kernels and its synchronisation amortised over them)."""
    import torch

    work = torch.empty_like(X)
    bamg.relax(B, X, ncols, col0, 0.7, 2, work=work)  # warm-up
    evs = []
    for _ in range(reps):
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        bamg.relax(B, X, ncols, col0, 0.7, sweeps, work=work)
        e1.record(stream)
        evs.append((e0, e1))
    torch.cuda.synchronize()
    return float(np.mean([a.elapsed_time(b) for a, b in evs])) / sweeps


# DRAM traffic of one finest-level k_smooth launch from an ncu capture of this kernel on
# the tandem 256 x 256 workload, valid while the kernel's source is unchanged.
SMOOTH_TRAFFIC = {"bytes": 3145856, "source_sha1": "7ed3993ff8abcfcebbdf3cee3ca489213920e9f5"}


def _kernel_source_sha1():
    """sha1 of the k_smooth kernel's own source text (from its template line to its closing
    brace in k_solve.cu): the captured traffic stays valid while that text is unchanged."""
    import hashlib

    with open(os.path.join(ROOT, "paper_1004_1451_gb300", "csrc", "k_solve.cu")) as f:
        lines = f.read().split("\n")
    start = next(i for i, l in enumerate(lines) if l.startswith("__global__ void k_smooth("))
    if lines[start - 1].startswith("template"):
        start -= 1
    end = next(i for i in range(start, len(lines)) if lines[i].startswith("}"))
    return hashlib.sha1("\n".join(lines[start:end + 1]).encode()).hexdigest()


def dominant_kernel(solver, peaks, sweeps=20, reps=10):
    """k_smooth, the V-cycle smoother (Eq. (4.4)), on the finest level of the workload's
    own hierarchy: one of the three kernels with the largest shares of the step in the ncu
    launch list (8-9% each, with the single-block coarse tail and the FP64 Gram-Schmidt
    update).  Its 3.4 MB level stays in L2, so it is bound by load latency, not HBM
    bandwidth: the fraction of the HBM peak is reported for scale only.
    Timed live with CUDA events on the stream it is launched on, `sweeps` launches per
    event pair.  Algorithmic bytes per launch (FP32 values, int32 indices): the CSR of
    B_0 once (8 nnz + 4 (n + 1)), D^{-1}, b and x read once, y written once (16 n)."""
    import torch

    info = solver.info()
    n, nnz = int(info["n"][0]), int(info["nnz"][0])
    dt = solver.dtype
    esz = 4 if dt == torch.float32 else 8
    b = torch.rand(n, dtype=dt, device="cuda")
    x = torch.rand(n, dtype=dt, device="cuda")
    work = torch.empty_like(x)
    stream = torch.cuda.current_stream()
    solver.smooth(0, b, x, sweeps=2, work=work)  # warm-up
    evs = []
    for _ in range(reps):
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        solver.smooth(0, b, x, sweeps=sweeps, work=work)
        e1.record(stream)
        evs.append((e0, e1))
    torch.cuda.synchronize()
    us = float(np.median([a.elapsed_time(c) for a, c in evs])) * 1e3 / sweeps
    nbytes = (esz + 4) * nnz + 4 * (n + 1) + 4 * esz * n
    gbs = nbytes / (us * 1e-6) / 1e9
    peak = float(peaks.get("hbm_gbs", 6800.0))
    traffic = SMOOTH_TRAFFIC["bytes"] if SMOOTH_TRAFFIC["source_sha1"] == _kernel_source_sha1() else None
    return {"kernel": "k_smooth<float> (V-cycle smoother, finest level, 65,536 rows)", "bound": "latency/L2",
            "achieved": round(gbs, 1), "peak": peak, "unit": "GB/s", "frac": round(gbs / peak, 4),
            "traffic": traffic, "bytes_per_launch": int(nbytes), "us_per_launch": round(us, 3),
            "peak_source": _peak_source(peaks),
            "note": "level-0 working set (%.1f MB) stays in the 129 MB L2 between launches; the step is a chain of "
                    "~800 latency-bound launches (largest shares 8-9%% each), and the HBM-bound kernel of the method, "
                    "the SpMM sweep, is measured at scale in spmm_hbm" % (nbytes / 1e6)}


def _peak_source(peaks):
    return ("of measured: MEASURED_PEAKS.json hbm_gbs (burst copy)" if "hbm_gbs" in peaks and not peaks.get("_fallback")
            else "of fallback: 6.8 TB/s (MEASURED_PEAKS.json absent)")


def spmm_probe(peaks, N=4096):
    """HBM probe: one omega-Jacobi SpMM sweep on the 4096 x 4096 grid walk (16.8 M states,
    83.9 M non-zeros) over r = 16 FP32 test vectors: 2.95 GB of algorithmic traffic."""
    import torch

    import paper_1004_1451_gb300 as bamg

    dev = torch.device("cuda")
    B = _grid_B(N, dev, torch.float32)
    n, nnz = N * N, int(B[1].numel())
    X = torch.rand(n, 16, dtype=torch.float32, device=dev)
    ms = _time_relax(bamg, B, X, 16, 0, 3, torch.cuda.current_stream())
    nbytes = nnz * 8 + 4 * (n + 1) + 4 * n + 2 * 4 * n * 16
    gbs = nbytes / (ms * 1e-3) / 1e9
    peak = float(peaks.get("hbm_gbs", 6800.0))
    del X, B
    torch.cuda.empty_cache()
    lg = n.bit_length() - 1
    shape = [{"chunks_per_thread": r["chunks_per_thread"], "blocks_per_sm": r["blocks_per_sm"]}
             for r in bamg.autotune_report()
             if r["elem_bytes"] == 4 and r["shift"] == 0 and r["chunks_per_row"] == 4 and r["log2_n"] == lg]
    return {"workload": f"grid walk {N}^2, r=16, FP32", "kernel": "k_jacobi<float>", "ms": round(ms, 4),
            "bytes": int(nbytes), "achieved": round(gbs, 1), "peak": peak, "unit": "GB/s", "frac": round(gbs / peak, 4),
            "peak_source": _peak_source(peaks),
            "launch_shape": shape[0] if shape else "fixed rule (two chunks per thread, 2 blocks/SM)"}


BATCH_WORKLOAD = ("512 chains, seed 0: 256 birth-death chains (n log-uniform in [1024, 65536], per-state "
                  "rates U(0.2, 0.5)) and 256 grid walks (side uniform in [32, 256]); r=8; mixed")
# Birth-death chains with i.i.d. per-state rates have stationary vectors spanning tens of
# orders of magnitude (beyond FP32's exponent range, so their V-cycle runs in FP64) and
# metastable wells (many eigenvalues near zero): their LS fits use a small ridge (the
# default suits 2-D chains), and FGMRES a long restart cycle (256) with an MLE restart after
# each cycle that fails.
BD_OPTS = dict(ridge=1e-10, ridge32=1e-6, gmres_m=256, max_it=3000, precision="fp64")


def _bd_log_x(birth, death):
    """log of the product-form stationary vector x_{k+1} = x_k b_k / d_{k+1}, 1^T x = 1."""
    lx = np.zeros(len(birth))
    lx[1:] = np.cumsum(np.log(birth[:-1]) - np.log(death[1:]))
    lx -= lx.max()
    return lx - np.log(np.exp(lx).sum())


def _bd_bounds(birth, death, tol):
    """(K, eps) for a birth-death chain.  K bounds the l1 error per unit residual: with
    u = x / x* and the net flux J_i across edge i (|J_i| <= ||B x||_1 / 2), detailed balance
    gives u_{i+1} - u_i = -J_i / (b_i x*_i), so ||x - x*||_1 <= K ||B x||_1 with
    K = sum_i (M_L(i) below the weighted median, M_R(i) from it on) / (b_i x*_i).  eps: a
    mass move across one edge changes x by 2 M_L M_R at a residual of 2 b_m x*_m, so a
    non-negative vector meeting tol can lie eps away; eps > 1e-6 means tol cannot pin x.
    Both masses are accumulated from their own end in log space: past a deep valley of x*
    followed by a smaller bump, M_R lies far below the rounding of 1 - M_L while 1 / (b x*)
    there is huge, and those edges dominate K."""
    lx = _bd_log_x(birth, death)
    lML = np.logaddexp.accumulate(lx)[:-1]
    lMR = np.logaddexp.accumulate(lx[::-1])[::-1][1:]
    lflux = np.log(birth[:-1]) + lx[:-1]
    m = int(np.searchsorted(np.exp(lML), 0.5))
    t = np.where(np.arange(len(lML)) < m, lML, lMR) - lflux
    log10_K = float((t.max() + np.log(np.exp(t - t.max()).sum())) / np.log(10.0))
    eps = float((2.0 * np.exp(lML + lMR + np.minimum(0.0, np.log(tol / 2.0) - lflux))).max())
    return log10_K, eps


def _bd_residual(c, x):
    """B x = x - A x for a birth-death chain's CSR (host, FP64)."""
    rp, ci, v = c.row_ptr, c.col, c.val
    ax = np.add.reduceat(v * x[ci], rp[:-1]) if len(v) else np.zeros(c.n)
    return x - ax


_last_batch_x = None


def batch_line(args, workers=8):
    """Chains solved per second by bamg_solve_batch on the 512-chain mixture (inputs
    resident on the device), with the count of chains that reached the tolerance."""
    import torch

    import paper_1004_1451_gb300 as bamg
    from workloads import batched_mixture

    chains = batched_mixture(0)
    mats = [(torch.tensor(c.row_ptr, device="cuda"), torch.tensor(c.col, device="cuda"),
             torch.tensor(c.val, device="cuda")) for c in chains]
    def opts_for(prec):
        return [dict(grid=c.grid, **dict(dict(precision=prec), **(BD_OPTS if c.kind == "birth_death" else {})))
                for c in chains]

    def once(prec="mixed"):
        global _last_batch_x
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        try:
            xs, st = bamg.solve_batch(mats, 8, 30, TOL, opts=opts_for(prec), workers=workers)
        except bamg.BamgError as e:
            xs, st = getattr(e, "xs", None), e.stats
        dt = time.perf_counter() - t0
        _last_batch_x = [x.cpu().numpy() for x in xs] if xs is not None else [np.full(c.n, np.nan) for c in chains]
        return dt, st

    once()  # warm-up
    dt, st = once()
    # accuracy of the birth-death chains against the product form (the last mixed run)
    xs = _last_batch_x
    bd_err, pinned, unpinnable, within = [], 0, 0, 0
    for c, x in zip(chains, xs):
        if c.kind != "birth_death":
            continue
        xe = np.exp(_bd_log_x(c.meta["birth"], c.meta["death"]))
        e = float(np.abs(x - xe).sum())
        bd_err.append(e)
        lk, eps = _bd_bounds(c.meta["birth"], c.meta["death"], TOL)
        pinned += int(lk + np.log10(TOL) <= -6.0)
        unpinnable += int(eps > 1e-6)
        within += int(e <= 10.0 ** lk * float(np.abs(_bd_residual(c, x)).sum()) * (1 + 1e-6) + 1e-14)
    dt64, st64 = once("fp64")
    ok = [s_["status"] == 0 for s_ in st]
    bd = [c.kind == "birth_death" for c in chains]
    return {"workload": BATCH_WORKLOAD, "chains": len(chains), "states": int(sum(c.n for c in chains)),
            "nnz_A": int(sum(c.nnz for c in chains)), "value": round(len(chains) / dt, 2), "unit": "chains/s",
            "ms": round(dt * 1e3, 1), "workers": workers, "converged": int(sum(ok)),
            "converged_grid": int(sum(o and not b for o, b in zip(ok, bd))),
            "converged_birth_death": int(sum(o and b for o, b in zip(ok, bd))),
            "not_converged": sorted([int(c.n), int(s_["status"]), int(s_["iterations"])]
                                    for c, o, s_ in zip(chains, ok, st) if not o),
            "precision": "grid walks: FP32 V-cycle in FP64 FGMRES; birth-death chains: FP64 throughout",
            "birth_death_vs_product_form": {
                "pinned_to_1e-6_by_tol": pinned, "provably_not_pinned_by_tol": unpinnable,
                "within_rigorous_bound": within, "median_rel_l1": float(np.median(bd_err)),
                "max_rel_l1": float(max(bd_err)),
                "note": "K bounds ||x - x*||_1 / ||B x||_1 (detailed balance); a chain is pinned to 1e-6 by the "
                        "tolerance when K tol <= 1e-6 and provably not when a mass move across one edge meets the "
                        "tolerance yet moves x by more than 1e-6"},
            "gmres_iterations_total": int(sum(s_["iterations"] for s_ in st)),
            "fp64": {"value": round(len(chains) / dt64, 2), "unit": "chains/s", "ms": round(dt64 * 1e3, 1),
                     "converged": int(sum(s_["status"] == 0 for s_ in st64))},
            "note": "birth-death chains that stop at max_it count in the time; host-timed (threads and streams)"}


LEARNED_WORKLOAD = ("learned P: MLP trained on the LS rows of 16 tandem queues (capacities uniform in [63, 255], "
                    "rates U(0.2, 0.45) normalised, seed 1; rows with an LS weight above 4 left out); tested on a "
                    "held-out tandem queue of capacity 511 (262,144 states, seed 99); r=10; mixed")


def _timed(fn, reps):
    import torch

    out, ts = None, []
    for _ in range(reps):
        torch.cuda.synchronize()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record()
        out = fn()
        e1.record()
        e1.synchronize()
        ts.append(e0.elapsed_time(e1))
    return out, float(np.median(ts))


def learned_line(args, train_rows=1 << 20, epochs=10, batch=4096):
    """LS vs learned interpolation on the held-out tandem queue: V-cycle factor, setup and
    solve times (CUDA events on the current stream), iterations, accuracy."""
    import torch

    import paper_1004_1451_gb300 as bamg
    from workloads import tandem_training_set

    def dev(ch):
        return (torch.tensor(ch.row_ptr, device="cuda"), torch.tensor(ch.col, device="cuda"),
                torch.tensor(ch.val, device="cuda"))

    t0 = time.perf_counter()
    Fs, Ts = [], []
    for ch in tandem_training_set(1, 16, n_lo=63, n_hi=255):
        f, t = bamg.interp_dataset(*dev(ch), R, 20, grid=ch.grid, precision="mixed")
        # fine points with candidates; rows whose LS weights exceed 4 in magnitude (a few
        # in 10^4, from nearly collinear candidates) are left out of the MSE training set
        keep = (f[:, 0:96:6].sum(dim=1) > 0) & (t.abs().amax(dim=1) <= 4.0)
        Fs.append(f[keep])
        Ts.append(t[keep])
    F, T = torch.cat(Fs), torch.cat(Ts)
    del Fs, Ts
    perm = torch.randperm(F.shape[0], generator=torch.Generator().manual_seed(0))[:train_rows].to(F.device)
    F, T = F[perm].contiguous(), T[perm].contiguous()
    torch.cuda.synchronize()
    data_s = time.perf_counter() - t0
    model = bamg.Model(0)
    t0 = time.perf_counter()
    hist = model.train(F, T, epochs=epochs, batch=batch, lr=1e-3)
    train_s = time.perf_counter() - t0
    rows = int(F.shape[0])
    del F, T
    test = tandem_training_set(99, 1, n_lo=511, n_hi=511)[0]
    A = dev(test)
    xe = _direct_stationary(test)
    out = {"workload": LEARNED_WORKLOAD, "n": test.n, "train_rows": rows, "epochs": epochs, "batch": batch,
           "data_s": round(data_s, 2), "train_s": round(train_s, 2), "train_loss_first_last": [round(hist[0], 5),
                                                                                               round(hist[-1], 5)]}
    # LS with one setup cycle has a divergent V-cycle on this chain (its factor exceeds 1 as a
    # stationary iteration; FGMRES still converges); with two setup cycles (the tables' V^2)
    # the LS V-cycle converges, so that is the baseline the learned hierarchies are judged by
    for name, prec, kw in (("ls", "mixed", {}), ("ls_v2", "mixed", {"setup_cycles": 2}),
                           ("learned", "mixed", {"interp": "learned", "model": model}),
                           ("learned_v2", "mixed", {"interp": "learned", "model": model, "setup_cycles": 2}),
                           ("ls_fp64", "fp64", {}), ("ls_v2_fp64", "fp64", {"setup_cycles": 2})):
        s, setup_ms = _timed(lambda: bamg.Solver(*A, r=R, levels=20, grid=test.grid, precision=prec, **kw), 5)
        rho = s.vcycle_factor(20)
        (x, st), solve_ms = _timed(lambda: s.solve(TOL), 3)
        err = float(np.abs(x.cpu().numpy() - xe).sum() / np.abs(xe).sum())
        out[name] = {"setup_ms": round(setup_ms, 3), "solve_ms": round(solve_ms, 3), "gmres_iterations": st["iterations"],
                     "vcycle_factor": round(rho, 4), "rel_l1_vs_exact": err, "levels": s.info()["n"]}
        s.close()
    model.close()
    base = min((k for k in ("ls", "ls_v2", "ls_fp64", "ls_v2_fp64") if out[k]["vcycle_factor"] < 1.0),
               key=lambda k: out[k]["setup_ms"] + out[k]["solve_ms"], default=None)
    best = min(("learned", "learned_v2"), key=lambda k: out[k]["setup_ms"] + out[k]["solve_ms"])
    if base is not None:
        b, l = out[base], out[best]
        out["gain"] = {"baseline": base, "learned": best,
                       "iterations": [b["gmres_iterations"], l["gmres_iterations"]],
                       "vcycle_factor": [b["vcycle_factor"], l["vcycle_factor"]],
                       "time_ms": [round(b["setup_ms"] + b["solve_ms"], 3), round(l["setup_ms"] + l["solve_ms"], 3)]}
    return out


SMALL_WORKLOAD = "random walk on a 64x64 grid (4,096 states, 4-neighbour, probability 1/deg); r=8"


def small_line(args, reps=5):
    """The 64x64 grid walk in plain FP64 and in mixed precision: setup and solve times (CUDA
    events), iterations, accuracy against the closed form x ~ degree."""
    import torch

    import paper_1004_1451_gb300 as bamg
    from workloads import grid_walk

    ch = grid_walk(64)
    A = (torch.tensor(ch.row_ptr, device="cuda"), torch.tensor(ch.col, device="cuda"),
         torch.tensor(ch.val, device="cuda"))
    deg = np.asarray(ch.meta["degree"], dtype=np.float64)
    xe = deg / deg.sum()
    out = {"workload": SMALL_WORKLOAD, "n": ch.n, "nnz_A": int(ch.nnz)}
    for prec in ("fp64", "mixed"):
        s, setup_ms = _timed(lambda: bamg.Solver(*A, r=8, levels=20, grid=ch.grid, precision=prec), reps)
        (x, st), solve_ms = _timed(lambda: s.solve(TOL), reps)
        out[prec] = {"setup_ms": round(setup_ms, 3), "solve_ms": round(solve_ms, 3),
                     "ms": round(setup_ms + solve_ms, 3), "gmres_iterations": st["iterations"],
                     "rel_l1_vs_exact": float(np.abs(x.cpu().numpy() - xe).sum()), "levels": s.info()["n"]}
        s.close()
    return out


LARGE_WORKLOAD = ("Delaunay triangulation of 2^20 points U[0,1]^2 (seed 0), random walk with probability 1/deg; "
                  "r=16; compatible-relaxation coarsening; mixed")


def large_line(args):
    """The 2^20-point Delaunay walk: setup and solve times (CUDA events), iterations,
    accuracy against the closed form x ~ degree, and the SpMM sweep on its finest level."""
    import torch

    import paper_1004_1451_gb300 as bamg
    from workloads import delaunay_walk

    t0 = time.perf_counter()
    ch = delaunay_walk(1 << 20, 0)
    gen_s = time.perf_counter() - t0
    A = (torch.tensor(ch.row_ptr, device="cuda"), torch.tensor(ch.col, device="cuda"),
         torch.tensor(ch.val, device="cuda"))
    deg = np.asarray(ch.meta["degree"], dtype=np.float64)
    xe = deg / deg.sum()
    reps = args.large_reps
    s, setup_ms = _timed(lambda: bamg.Solver(*A, r=16, levels=30, precision="mixed", coarsen="cr",
                                             device_loop=args.device_loop), reps)
    (x, st), solve_ms = _timed(lambda: s.solve(TOL), reps)
    err = float(np.abs(x.cpu().numpy() - xe).sum())
    info = s.info()
    s.close()
    # the plain FP64 method on the same chain
    s, setup64 = _timed(lambda: bamg.Solver(*A, r=16, levels=30, precision="fp64", coarsen="cr"), reps)
    (x, st64), solve64 = _timed(lambda: s.solve(TOL), reps)
    err64 = float(np.abs(x.cpu().numpy() - xe).sum())
    s.close()
    return {"workload": LARGE_WORKLOAD, "n": ch.n, "nnz_A": int(ch.nnz), "setup_ms": round(setup_ms, 2),
            "solve_ms": round(solve_ms, 2), "ms": round(setup_ms + solve_ms, 2), "gmres_iterations": st["iterations"],
            "rel_l1_vs_exact": err, "levels": info["n"], "op_complexity": round(info["op_complexity"], 3),
            "fp64": {"setup_ms": round(setup64, 2), "solve_ms": round(solve64, 2), "ms": round(setup64 + solve64, 2),
                     "gmres_iterations": st64["iterations"], "rel_l1_vs_exact": err64},
            "generation_s": round(gen_s, 1)}


def kernel_probe():
    """Only the dominant-kernel timing (for an ncu capture of k_smooth on the finest level)."""
    import torch

    import paper_1004_1451_gb300 as bamg

    ch = _workload()
    rp, ci, v = (torch.tensor(a, device="cuda") for a in (ch.row_ptr, ch.col, ch.val))
    s = bamg.Solver(rp, ci, v, r=R, levels=20, grid=ch.grid, precision="mixed")
    _line(dominant_kernel(s, {"hbm_gbs": 6800.0, "_fallback": True}, sweeps=3, reps=1))


def cpu_baseline():
    """The oracle as it stands, single-threaded, on the full workload (one solve)."""
    from oracle import bamg as ob

    ch = _workload()
    A = ch.to_scipy()
    t0 = time.perf_counter()
    x, H, st = ob.stationary(A, R, 20, TOL, ob.Opts(), grid=ch.grid)
    dt = time.perf_counter() - t0
    from workloads import grid_walk

    g = grid_walk(64)
    t0 = time.perf_counter()
    ob.stationary(g.to_scipy(), 8, 20, TOL, ob.Opts(), grid=g.grid)
    dt_small = time.perf_counter() - t0
    return {"value": round(dt * 1e3, 1), "unit": "ms", "cores": 1, "kind": "oracle",
            "sample": "one full setup + FGMRES solve of the same chain to 1e-10 (FP64 numpy/scipy)",
            "iterations": st["iterations"], "grid64_r8_ms": round(dt_small * 1e3, 1)}


# ------------------------------------------------------------------ reference arm
def run_reference(args):
    ws, rank = _dist()
    if rank != 0:
        return
    from oracle import bamg as ob

    ch = _workload()
    A = ch.to_scipy()
    # a bounded sample: one untimed run, then timed runs until K are done or about 150 s of
    # oracle time has passed (each run is a whole setup + solve; the line reports the mean)
    if args.warmup > 0:
        ob.stationary(A, R, 20, TOL, ob.Opts(), grid=ch.grid)
    ts = []
    for _ in range(args.steps):
        t0 = time.perf_counter()
        x, H, st = ob.stationary(A, R, 20, TOL, ob.Opts(), grid=ch.grid)
        ts.append((time.perf_counter() - t0) * 1e3)
        if sum(ts) > 150e3:
            break
    ms = float(np.mean(ts))
    _line({"impl": "reference", "metric": METRIC, "value": round(ms, 2), "unit": "ms", "n_gpus": ws,
           "steps": args.steps, "warmup": args.warmup, "ms_per_step": round(ms, 2), "higher_is_better": False,
           "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
           "config": {"workload": WORKLOAD, "n": ch.n, "r": R, "tol": TOL},
           "cpu_baseline": {"value": round(ms, 2), "unit": "ms", "cores": 1, "kind": "oracle",
                            "sample": f"full setup + FGMRES solve of the workload per step; {len(ts)} of "
                                      f"{args.steps} steps timed (bounded to about 150 s), 1 warm-up run"},
           "e2e": {"value": round(ms, 2), "unit": "ms", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}})


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=50)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--no-probe", action="store_true")
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--only-step", action="store_true", help="time the workload steps only (for profiler launch lists)")
    ap.add_argument("--probe-only", type=int, default=0, help="run only the SpMM probe on an N x N grid walk")
    ap.add_argument("--no-batch", action="store_true", help="skip the 512-chain batched line")
    ap.add_argument("--no-learned", action="store_true", help="skip the learned-interpolation line")
    ap.add_argument("--kernel-probe", action="store_true", help="run only the dominant-kernel timing")
    ap.add_argument("--learned-only", action="store_true", help="run only the learned-interpolation line")
    ap.add_argument("--no-large", action="store_true", help="skip the 2^20-point Delaunay line")
    ap.add_argument("--persistent", type=int, default=0,
                    help="1: Arnoldi steps in one cooperative launch where the hierarchy qualifies; 0: graph form")
    ap.add_argument("--coarse-tail", type=int, default=0, choices=[0, 1],
                    help="coarse end of the V-cycle: 0 on a thread-block cluster (from the first level with at "
                         "most 4096 rows), 1 in one block (from 1024 rows)")
    ap.add_argument("--no-variants", action="store_true", help="skip the variants line (smoother, setup cycling, "
                                                                 "pArnoldi)")
    ap.add_argument("--large-only", action="store_true", help="run only the 2^20-point Delaunay line")
    ap.add_argument("--large-reps", type=int, default=3, help="timed repetitions of the 2^20-point Delaunay line")
    ap.add_argument("--device-loop", type=int, default=1, choices=[0, 1],
                    help="0: one graph launch per Arnoldi step (same kernels; ncu lists kernels of a "
                         "graph's conditional body only this way)")
    args = ap.parse_args()
    if args.impl == "reference":
        run_reference(args)
    elif args.large_only:
        import torch

        import paper_1004_1451_gb300.build as pb

        pb.build()
        torch.cuda.set_device(int(os.environ.get("LOCAL_RANK", "0")))
        _line(large_line(args))
    elif args.learned_only:
        import torch

        import paper_1004_1451_gb300.build as pb

        pb.build()
        torch.cuda.set_device(int(os.environ.get("LOCAL_RANK", "0")))
        _line(learned_line(args))
    elif args.kernel_probe:
        import torch

        import paper_1004_1451_gb300.build as pb

        pb.build()
        torch.cuda.set_device(int(os.environ.get("LOCAL_RANK", "0")))
        kernel_probe()
    elif args.probe_only:
        import torch

        import paper_1004_1451_gb300.build as pb

        pb.build()
        torch.cuda.set_device(int(os.environ.get("LOCAL_RANK", "0")))
        peaks = json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json"))) if os.path.exists(
            os.path.join(ROOT, "MEASURED_PEAKS.json")) else {"hbm_gbs": 6800.0, "_fallback": True}
        _line(spmm_probe(peaks, N=args.probe_only))
    else:
        run_ours(args)


if __name__ == "__main__":
    main()

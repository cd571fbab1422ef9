"""Time to ||Bx||_1 / ||x||_1 <= 1e-10 for Bootstrap AMG on GB300.

Workload (one step = the whole hot path: setup + preconditioned GMRES): the tandem
queueing network with two queues of capacity 255 (65,536 states), arrival 11/31,
service 10/31 and 10/31, r = 10 test vectors, FP32 setup and V-cycle inside FP64
flexible GMRES.  Inputs are resident in HBM when a step's timing starts; L2 is
flushed between steps.  Also reported: the same metric end to end from host buffers,
the plain FP64 method on the same chain, the roofline of the dominant kernel, an SpMM
HBM probe, and the CPU oracle on the host cores.

python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
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


def _line(d):
    print(json.dumps(d), flush=True)


# ------------------------------------------------------------------ clocks
class Clocks:
    def __init__(self):
        self.p = None
        self.path = os.path.join(ROOT, "gpurun_out", f"clocks_{os.getpid()}.csv")

    def start(self):
        try:
            os.makedirs(os.path.dirname(self.path), exist_ok=True)
            q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
                 "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
                 "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")
            self.f = open(self.path, "w")
            self.p = subprocess.Popen(["nvidia-smi", f"--query-gpu={q}", "--format=csv,noheader,nounits", "-lms", "100"],
                                      stdout=self.f, stderr=subprocess.DEVNULL)
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
        dev = os.environ.get("LOCAL_RANK", "0")
        for line in open(self.path):
            f = [x.strip() for x in line.split(",")]
            if len(f) < 9 or f[0] != str(int(dev)) and len(f[0]) == 1 and False:
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
        s = bamg.Solver(rp, ci, v, r=R, levels=20, grid=ch.grid, precision=precision)
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
    times, iters, split = [], [], []
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
        s.close()
    launches = (bamg.launch_count() - l0) / args.steps
    torch.cuda.synchronize()
    ck = clocks.stop()
    if args.only_step:
        if rank == 0:
            _line({"metric": METRIC, "value": round(float(np.mean(times)), 4), "unit": "ms",
                   "gmres_iterations": int(np.median(iters)), "gpu_launches": int(round(launches)), "only_step": True})
        return
    ms = float(np.sum(times)) / args.steps
    if ws > 1:
        t = torch.tensor([ms], device=dev)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        ms = float(t.item())
        dist.barrier()
    # ---- parity of the timed result against the exact stationary vector
    from oracle import exact

    xe = exact.sparse_nullspace(ch.to_scipy()) if rank == 0 else None
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
        os.path.join(ROOT, "MEASURED_PEAKS.json")) else {"hbm_gbs": 6800.0}
    roof = dominant_kernel(ch, peaks)
    probe = spmm_probe(peaks) if not args.no_probe else None
    cpu = cpu_baseline() if not args.no_cpu else None
    nnz_a = int(ch.nnz)
    out = {
        "metric": METRIC, "value": round(ms, 4), "unit": "ms", "n_gpus": ws, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": round(ms, 4), "higher_is_better": False, "scaling": "weak",
        "vs_baseline": None, "dtype": "f32+f64", "data": "synthetic",
        "config": {"workload": WORKLOAD, "n": ch.n, "nnz_A": nnz_a, "r": R, "tol": TOL,
                   "l2": "flushed between steps (256 MiB write)", "parallelism": f"replicas x{ws}"},
        "gmres_iterations": int(np.median(iters)), "rel_l1_vs_exact": err,
        "host_setup_ms": round(float(np.median([a for a, b in split])), 3),
        "host_solve_ms": round(float(np.median([b for a, b in split])), 3),
        "e2e": {"value": round(e2e_ms, 4), "unit": "ms", "h2d_bytes_per_step": 4 * (ch.n + 1) + 12 * nnz_a,
                "d2h_bytes_per_step": 8 * ch.n},
        "fp64_ms": round(float(np.median(fp64)), 4), "fp64_iterations": st64["iterations"],
        "speedup_mixed_vs_fp64": round(float(np.median(fp64)) / ms, 3),
        "gpu_launches": int(round(launches)),
        "roofline": roof, "spmm_hbm": probe, "cpu_baseline": cpu, "clocks": ck,
    }
    _line(out)


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


def dominant_kernel(ch, peaks):
    """omega-Jacobi SpMM sweep on the workload's finest level (FP32, r = 10 columns of a
    20-wide block, as in the setup).  Algorithmic bytes per launch: the matrix once
    (nnz * (4 + 4) + 4 (n + 1)), the inverse diagonal (4 n), the relaxed columns read and
    written once (2 * 4 * n * 12)."""
    import torch

    import paper_1004_1451_gb300 as bamg
    from oracle import bamg as ob  # noqa: F401  (input matrix only)

    dev = torch.device("cuda")
    B = ob.system_matrix(ch.to_scipy())
    Bd = (torch.tensor(B.indptr.astype(np.int32), device=dev), torch.tensor(B.indices.astype(np.int32), device=dev),
          torch.tensor(B.data, dtype=torch.float32, device=dev))
    X = torch.rand(ch.n, 20, dtype=torch.float32, device=dev)
    ms = _time_relax(bamg, Bd, X, 10, 0, 10, torch.cuda.current_stream())
    nbytes = B.nnz * 8 + 4 * (ch.n + 1) + 4 * ch.n + 2 * 4 * ch.n * 12
    gbs = nbytes / (ms * 1e-3) / 1e9
    peak = float(peaks.get("hbm_gbs", 6800.0))
    return {"kernel": "k_jacobi<float> (SpMM sweep, finest level)", "bound": "hbm", "achieved": round(gbs, 1),
            "peak": peak, "unit": "GB/s", "frac": round(gbs / peak, 4), "traffic": None,
            "bytes_per_launch": int(nbytes), "us_per_launch": round(ms * 1e3, 3),
            "note": "working set fits in L2 (8.9 MB); bytes are algorithmic"}


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
    return {"workload": f"grid walk {N}^2, r=16, FP32", "kernel": "k_jacobi<float>", "ms": round(ms, 4),
            "bytes": int(nbytes), "achieved": round(gbs, 1), "peak": peak, "unit": "GB/s", "frac": round(gbs / peak, 4)}


def cpu_baseline():
    """The oracle as it stands, single-threaded, on the full workload (one solve)."""
    from oracle import bamg as ob

    ch = _workload()
    A = ch.to_scipy()
    t0 = time.perf_counter()
    x, H, st = ob.stationary(A, R, 20, TOL, ob.Opts(), grid=ch.grid)
    dt = time.perf_counter() - t0
    return {"value": round(dt * 1e3, 1), "unit": "ms", "cores": 1, "kind": "oracle",
            "sample": "one full setup + FGMRES solve of the same chain to 1e-10 (FP64 numpy/scipy)",
            "iterations": st["iterations"]}


# ------------------------------------------------------------------ reference arm
def run_reference(args):
    ws, rank = _dist()
    if rank != 0:
        return
    from oracle import bamg as ob

    ch = _workload()
    A = ch.to_scipy()
    for _ in range(args.warmup):
        ob.stationary(A, R, 20, TOL, ob.Opts(), grid=ch.grid)
    ts = []
    for _ in range(args.steps):
        t0 = time.perf_counter()
        x, H, st = ob.stationary(A, R, 20, TOL, ob.Opts(), grid=ch.grid)
        ts.append((time.perf_counter() - t0) * 1e3)
    ms = float(np.mean(ts))
    _line({"impl": "reference", "metric": METRIC, "value": round(ms, 2), "unit": "ms", "n_gpus": ws,
           "steps": args.steps, "warmup": args.warmup, "ms_per_step": round(ms, 2), "higher_is_better": False,
           "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
           "config": {"workload": WORKLOAD, "n": ch.n, "r": R, "tol": TOL},
           "cpu_baseline": {"value": round(ms, 2), "unit": "ms", "cores": 1, "kind": "oracle",
                            "sample": "full setup + FGMRES solve of the workload per step"},
           "e2e": {"value": round(ms, 2), "unit": "ms", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}})


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--no-probe", action="store_true")
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--only-step", action="store_true", help="time the workload steps only (for profiler launch lists)")
    ap.add_argument("--probe-only", type=int, default=0, help="run only the SpMM probe on an N x N grid walk")
    args = ap.parse_args()
    if args.impl == "reference":
        run_reference(args)
    elif args.probe_only:
        import torch

        import paper_1004_1451_gb300.build as pb

        pb.build()
        torch.cuda.set_device(int(os.environ.get("LOCAL_RANK", "0")))
        peaks = json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json"))) if os.path.exists(
            os.path.join(ROOT, "MEASURED_PEAKS.json")) else {"hbm_gbs": 6800.0}
        _line(spmm_probe(peaks, N=args.probe_only))
    else:
        run_ours(args)


if __name__ == "__main__":
    main()

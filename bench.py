#!/usr/bin/env python
"""Benchmark of the matching-AMG preconditioned CG on one GB300.

Workload (default): 3D Poisson, 7-point stencil on a 256^3 grid (16.8M
unknowns, 117M nonzeros), FP64 CSR, w = 1, 3 matching sweeps per level,
l1-Jacobi 1+1, dense Cholesky on the coarsest level, b = A x* with
x* ~ U[-1, 1] (seed 1), x0 = 0, PCG to rel-res 1e-6.

One step = amg_setup (the whole hierarchy build) + amg_solve + amg_free with
A, w and b already resident in HBM. The metric is time to solution (ms per
step, lower is better). Inputs (1.4 GB) are larger than L2, so no flush is
needed between steps.

Prints one JSON line. ``--impl reference`` times the CPU oracle instead (a
bounded sample of the same workload, scaled to the full size by unknowns).
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "AMG-PCG time to rel-res 1e-6 (full setup + single-RHS solve)"
FP64_PEAK_TFLOPS = 1.25   # GB300 FP64 rate (the profiling recipe's figure; a stand-alone FMA loop measured 1.19)


def _args():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--grid", type=int, default=256)
    ap.add_argument("--workload", default="poisson", choices=["poisson", "varcoef", "aniso3d"],
                    help="poisson: 7-point Laplacian (default line); varcoef: jump coefficients exp(g), sigma 2; "
                         "aniso3d: -(100 u_xx + 100 u_yy + u_zz)")
    ap.add_argument("--smooth-p", type=int, default=0, choices=[0, 1],
                    help="1: smoothed prolongator Pbar = (I - omega D^-1 A) P (the paper's VA3 setting)")
    ap.add_argument("--pre", type=int, default=1, help="l1-Jacobi sweeps before the coarse correction")
    ap.add_argument("--post", type=int, default=1, help="l1-Jacobi sweeps after the coarse correction")
    ap.add_argument("--omega-rule", type=int, default=0, choices=[0, 1],
                    help="smoothed prolongator weight: 0 = 4 / (3 ||D^-1 A||), 1 = 1 / ||D^-1 A|| (the text's)")
    ap.add_argument("--smooth-w", type=int, default=0,
                    help="> 0: w = that many l1-Jacobi sweeps on A w = 0 from ones (amg_smooth_vector, inside the step)")
    ap.add_argument("--krylov", type=int, default=0, help="0 PCG, 1 flexible CG")
    ap.add_argument("--cycle", default="v", choices=["v", "k"],
                    help="v: V-cycle (default line); k: K-cycle, two FCG iterations as the coarse correction")
    ap.add_argument("--kdepth", type=int, default=32,
                    help="K-cycle on coarse levels 1..kdepth (32: every intermediate level, the paper's cycle)")
    ap.add_argument("--precision", default="fp64", choices=["fp64", "fp32"])
    ap.add_argument("--rtol", type=float, default=1e-6)
    ap.add_argument("--autotune", type=int, default=0, choices=[0, 1],
                    help="1: autotuned launch shapes (timed once per shape, during warm-up)")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--cpu-sample-grid", type=int, default=0,
                    help="grid of the CPU oracle baseline (0: the benchmarked grid itself, not scaled)")
    ap.add_argument("--profile-steps", type=int, default=5,
                    help="profiled steps after the timed region: per-kernel CUDA-event times and the roofline")
    ap.add_argument("--serve", action="store_true",
                    help="serving benchmark: 5 cached hierarchies, Poisson arrivals, p50/p99 latency and solves/s")
    ap.add_argument("--serve-requests", type=int, default=60)
    ap.add_argument("--many", action="store_true",
                    help="batched benchmark: 256 independent Poisson systems, grid edges uniform in 16..64")
    ap.add_argument("--many-systems", type=int, default=256)
    ap.add_argument("--block", type=int, default=0,
                    help="multi-RHS benchmark: K right-hand sides (N(0,1), seed 4) on one Poisson hierarchy")
    ap.add_argument("--block-grid", type=int, default=128)
    ap.add_argument("--serve-scale", type=float, default=1.0,
                    help="grid scale factor of the served problems (1.0 = 64^3/128^3/192^3/2048^2/128^3)")
    return ap.parse_args()


# DRAM traffic per row of the level-0 FP64 V-cycle kernels, from one ncu
# capture on 3D Poisson 160^3 (dram__bytes_read.sum + dram__bytes_write.sum),
# valid for the 7-point Poisson workload in FP64 and only while the kernel
# source it was taken on is unchanged (checked by hash).
_TRAFFIC = {
    "post_smooth_l0": {"kernel": "k_post", "bytes_per_row": (314713600 + 22986240) / 4096000},
    "pre_residual_l0": {"kernel": "k_pre", "bytes_per_row": (408948992 + 53501184) / 4096000},
}
_TRAFFIC_SRC_HASH = "e5fe5e8b08565c47"


def _kernel_source_hash(names):
    """sha256 (16 hex) of the named kernels' and sell_row's source in solve.cu."""
    import hashlib
    lines = open(os.path.join(ROOT, "paper_2006_16147_gb300", "csrc", "solve.cu")).read().splitlines()
    parts = []
    for name in list(names) + ["sell_row"]:
        for i, line in enumerate(lines):
            if f" {name}(" in line and ("__global__" in line or "__device__" in line):
                j = i
                while not lines[j].startswith("template"):
                    j -= 1
                k = i
                while lines[k] != "}":
                    k += 1
                parts.append("\n".join(lines[j:k + 1]))
                break
    return hashlib.sha256("\n\n".join(parts).encode()).hexdigest()[:16]


def _traffic(kernel_name, n, workload, precision):
    t = _TRAFFIC.get(kernel_name)
    if t is None or workload != "poisson" or precision != "fp64":
        return None
    if _kernel_source_hash(["k_post", "k_pre"]) != _TRAFFIC_SRC_HASH:
        return None
    return t["bytes_per_row"] * n


def _peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


class ClockSampler:
    """nvidia-smi sampling of SM clocks and throttle reasons while running."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None
        self.path = os.path.join(tempfile.gettempdir(), f"amg_bench_clocks_{os.getpid()}_{index}.csv")

    def __enter__(self):
        try:
            os.makedirs(os.path.dirname(self.path), exist_ok=True)
            self.f = open(self.path, "w")
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={self.index}", f"--query-gpu={self.Q}",
                                          "--format=csv,noheader,nounits", "-lms", "100"],
                                         stdout=self.f, stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None
        return self

    def __exit__(self, *a):
        if self.proc:
            self.proc.terminate()
            self.proc.wait()
            self.f.close()

    def summary(self):
        if not self.proc:
            return None
        sm, mx, reasons = [], 0.0, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        try:
            for line in open(self.path):
                f = [x.strip() for x in line.split(",")]
                if len(f) < 9:
                    continue
                try:
                    sm.append(float(f[1]))
                    mx = max(mx, float(f[2]))
                except ValueError:
                    continue
                for nm, v in zip(names, f[5:9]):
                    if v.lower() == "active":
                        reasons.add(nm)
            os.remove(self.path)
        except Exception:
            return None
        if not sm:
            return None
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": mx, "reasons": sorted(reasons), "samples": len(sm)}


def _workload(grid, kind="poisson"):
    from paper_2006_16147_gb300 import workloads as W
    if kind == "varcoef":
        A = W.varcoef3d(grid, seed=2)
        b, _ = W.rhs_uniform(A, 3)
    elif kind == "aniso3d":
        A = W.aniso3d(grid, k=(100.0, 100.0, 1.0))
        b, _ = W.rhs_uniform(A, 1)
    else:
        A = W.poisson3d(grid)
        b, _ = W.rhs_uniform(A, 1)
    return A, b


def _workload_name(args):
    base = {"poisson": f"poisson3d_{args.grid}^3_7pt_fp64",
            "varcoef": f"varcoef3d_{args.grid}^3_sigma2_{args.precision}vcycle",
            "aniso3d": f"aniso3d_{args.grid}^3_k100-100-1_{args.precision}vcycle"}[args.workload]
    return (base + "_setup+solve" + (f"_kcycle{args.kdepth}" if args.cycle == "k" else "") +
            ("_smoothedP" if args.smooth_p else "") + ("_omega1/eta" if args.smooth_p and args.omega_rule else "") +
            (f"_l1jacobi{args.pre}+{args.post}" if (args.pre, args.post) != (1, 1) else "") +
            (f"_smoothw{args.smooth_w}" if args.smooth_w > 0 else ""))


def _host_info():
    """Host cores, CPU model and compiler of the machine the oracle runs on."""
    model = ""
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for line in out.splitlines():
            if line.startswith("Model name:"):
                model = line.split(":", 1)[1].strip()
                break
    except Exception:
        pass
    try:
        cxx = subprocess.run(["g++", "--version"], capture_output=True, text=True, timeout=10).stdout.splitlines()[0]
    except Exception:
        cxx = ""
    return {"host_cores": os.cpu_count(), "cpu_model": model, "compiler": cxx + " -O2 -ffp-contract=off"}


def _oracle_run(A, b, rtol, flexible=False, cycle=0, smooth_w=0, smooth_p=False, pre=1, post=1, omega_rule=0):
    """Oracle (plain FP64, 1 thread) setup + PCG on (A, b); setup and solve timed separately."""
    import oracle
    t0 = time.perf_counter()
    w = oracle.smooth_vector(A, np.ones(A.n), smooth_w) if smooth_w > 0 else None
    H = oracle.Hierarchy(A, w, cycle=cycle, smooth_p=smooth_p, pre=pre, post=post, omega_rule=omega_rule)
    t1 = time.perf_counter()
    x, info = H.pcg(b, rtol=rtol, flexible=flexible or cycle > 0)
    t2 = time.perf_counter()
    del H
    return dict(setup_s=t1 - t0, solve_s=t2 - t1, iterations=info["iterations"], n=A.n,
                true_relres=info["true_relres"])


def _oracle_kw(args):
    return dict(flexible=args.krylov == 1, cycle=args.kdepth if args.cycle == "k" else 0,
                smooth_w=args.smooth_w, smooth_p=bool(args.smooth_p), pre=args.pre, post=args.post,
                omega_rule=args.omega_rule)


REF_BUDGET_S = 150.0   # timed full-size oracle steps stop once the next one would pass this


def reference_arm(args):
    """The CPU oracle timed on the full workload (no scaling), rank 0 only.

    Warm-up steps run the oracle on the 32^3 instance of the same workload
    (untimed; they load and exercise the code). Timed steps each run the
    oracle's setup + PCG on the full-size instance; they stop after --steps or
    once the next step would pass REF_BUDGET_S (at least one), and the line
    reports the number actually run.
    """
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return 0
    import oracle
    oracle.build()
    kw = _oracle_kw(args)
    As, bs = _workload(min(32, args.grid), args.workload)
    for _ in range(args.warmup):
        _oracle_run(As, bs, args.rtol, **kw)
    A, b = _workload(args.grid, args.workload)
    runs = []
    t_start = time.perf_counter()
    while len(runs) < args.steps:
        runs.append(_oracle_run(A, b, args.rtol, **kw))
        step_s = runs[-1]["setup_s"] + runs[-1]["solve_s"]
        if time.perf_counter() - t_start + step_s > REF_BUDGET_S:
            break
    wall_ms = (time.perf_counter() - t_start) * 1e3
    v = statistics.mean((r["setup_s"] + r["solve_s"]) * 1e3 for r in runs)
    host = _host_info()
    sample = (f"oracle setup {statistics.mean(r['setup_s'] for r in runs):.2f} s + PCG "
              f"{statistics.mean(r['solve_s'] for r in runs):.2f} s ({runs[-1]['iterations']} it) on the full "
              f"{args.grid}^3 instance, {len(runs)} timed step(s) of {args.steps} requested (time budget "
              f"{REF_BUDGET_S:.0f} s), not scaled; warm-up steps on the 32^3 instance")
    line = {"impl": "reference", "metric": METRIC, "value": v, "unit": "ms", "n_gpus": args.gpus,
            "steps": len(runs), "warmup": args.warmup, "steps_requested": args.steps, "ms_per_step": v,
            "timed_wall_ms": wall_ms, "higher_is_better": False, "scaling": "weak", "vs_baseline": None,
            "dtype": "f64", "data": "synthetic",
            "config": {"workload": _workload_name(args), "grid": args.grid, "rtol": args.rtol},
            "setup_ms": statistics.mean(r["setup_s"] for r in runs) * 1e3,
            "solve_ms": statistics.mean(r["solve_s"] for r in runs) * 1e3,
            "iterations": runs[-1]["iterations"], "true_relres": runs[-1]["true_relres"],
            "cpu_baseline": {"value": v, "unit": "ms", "cores": 1, "kind": "oracle", "sample": sample, **host},
            "e2e": {"value": v, "unit": "ms", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


def serve_arm(args):
    """Served mixed-precision solves vs plain FP64 one-at-a-time FIFO.

    Five cached hierarchies: Poisson 64^3, 128^3, 192^3; anisotropic 2D
    -u_xx - 0.01 u_yy on 2048^2; jump coefficients 128^3. Requests pick a
    hierarchy uniformly and bring k ~ U{1..16} right-hand sides N(0, 1).
    Arrivals are Poisson at 50/80/95% of the measured capacity of the plain
    FP64 server (one request at a time, one column at a time). At 95% load and
    saturated, two FP64 arms that batch as well: each request's columns in one
    block solve (FP64 V-cycle), and the same continuous-batching server on the
    FP64 hierarchies. Latency is arrival to the result in host memory;
    solves/s counts right-hand sides.
    """
    import torch
    from paper_2006_16147_gb300 import amg
    from paper_2006_16147_gb300 import workloads as W
    torch.cuda.set_device(0)
    dev = torch.device("cuda:0")
    sc = args.serve_scale
    g = lambda v: max(8, int(round(v * sc)))
    specs = [("poisson3d_%d" % g(64), lambda: W.poisson3d(g(64)), 0),
             ("poisson3d_%d" % g(128), lambda: W.poisson3d(g(128)), 0),
             ("poisson3d_%d" % g(192), lambda: W.poisson3d(g(192)), 0),
             ("aniso2d_%d_eps1e-2" % g(2048), lambda: W.poisson2d_aniso(g(2048), g(2048), 1e-2), 0),
             ("varcoef3d_%d_sigma2" % g(128), lambda: W.varcoef3d(g(128), seed=2), 1)]
    t = lambda a: torch.from_numpy(np.ascontiguousarray(a)).to(dev)
    mats, h64, h32, pools = [], [], [], []
    rng = np.random.Generator(np.random.PCG64(6))
    for name, mk, flex in specs:
        A = mk()
        mats.append(A)
        args_dev = (t(A.row_ptr), t(A.col), t(A.val), torch.ones(A.n, dtype=torch.float64, device=dev))
        h64.append(amg.amg_setup(*args_dev, precision=0, krylov=flex))
        h32.append(amg.amg_setup(*args_dev, precision=1, krylov=flex))
        pool = torch.from_numpy(rng.normal(0.0, 1.0, size=(A.n, 16))).pin_memory().numpy()
        pools.append(pool)
    torch.cuda.synchronize()
    rtol = args.rtol

    nreq = args.serve_requests
    req_h = rng.integers(0, len(specs), size=nreq)
    req_k = rng.integers(1, 17, size=nreq)
    blocks = [np.ascontiguousarray(pools[h][:, :k]) for h, k in zip(req_h, req_k)]

    def plain_solve(hid, B):
        X = np.zeros_like(B)
        it = 0
        for c in range(B.shape[1]):
            b = torch.from_numpy(np.ascontiguousarray(B[:, c])).to(dev)
            x = torch.zeros_like(b)
            inf = amg.amg_solve(h64[hid], b, x, rtol=rtol, maxit=2000)
            X[:, c] = x.cpu().numpy()
            it = max(it, inf["iterations"])
        return X

    def batch_solve(hid, B):
        # the request's k columns in one block solve with the FP64 V-cycle
        Bd = torch.from_numpy(np.ascontiguousarray(B)).to(dev)
        Xd = torch.zeros_like(Bd)
        amg.amg_solve_batch(h64[hid], Bd, Xd, rtol=rtol, maxit=2000)
        return Xd.cpu().numpy()

    # capacity of the plain server (columns per second), requests back to back
    warm = min(5, nreq)
    for j in range(warm):
        plain_solve(int(req_h[j]), blocks[j])
    t0 = time.perf_counter()
    ncap = min(20, nreq)
    cols = 0
    for j in range(ncap):
        plain_solve(int(req_h[j]), blocks[j])
        cols += int(req_k[j])
    capacity = cols / (time.perf_counter() - t0)
    mean_k = float(np.mean(req_k))

    def run_plain(arrivals, solve_fn=plain_solve):
        lat = []
        t_start = time.perf_counter()
        for j in range(nreq):
            now = time.perf_counter() - t_start
            if now < arrivals[j]:
                time.sleep(arrivals[j] - now)
            solve_fn(int(req_h[j]), blocks[j])
            done = time.perf_counter() - t_start
            lat.append((done - arrivals[j]) * 1e3)
        elapsed = time.perf_counter() - t_start
        return lat, elapsed

    def run_served(arrivals, srv):
        t_start = time.perf_counter()
        j = 0
        lat = {}
        sub_t = {}
        results = {}
        while len(results) < nreq:
            now = time.perf_counter() - t_start
            while j < nreq and arrivals[j] <= now:
                rid, X = srv.submit(int(req_h[j]), blocks[j])
                sub_t[rid] = arrivals[j]
                j += 1
            pending = srv.step()
            now2 = time.perf_counter() - t_start
            for r in srv.poll():
                results[r["id"]] = r
                lat[r["id"]] = (now2 - sub_t[r["id"]]) * 1e3
            if pending == 0 and j < nreq:
                time.sleep(max(0.0, arrivals[j] - (time.perf_counter() - t_start)))
        elapsed = time.perf_counter() - t_start
        worst = max(r["relres"] for r in results.values())
        return list(lat.values()), elapsed, worst

    # warm the block paths (graph capture, workspaces) of every arm once
    for hid in range(len(specs)):
        batch_solve(hid, pools[hid][:, :16])
    q = lambda v, f: float(np.percentile(v, f))
    ncols = int(req_k.sum())
    out = []
    for load in (0.5, 0.8, 0.95):
        lam = load * capacity / mean_k
        arr = np.cumsum(rng.exponential(1.0 / lam, size=nreq))
        arr -= arr[0]
        lp, ep = run_plain(arr)
        srv = amg.Server(h32, slots=16, budget_bytes=120 << 30, rtol=rtol, maxit=2000)
        ls, es, worst = run_served(arr, srv)
        st = srv.stats()
        srv.close()
        row = {"load": load, "arrival_rate_req_s": lam,
               "plain_fp64": {"p50_ms": q(lp, 50), "p99_ms": q(lp, 99), "solves_per_s": ncols / ep},
               "served_fp32vcycle": {"p50_ms": q(ls, 50), "p99_ms": q(ls, 99), "solves_per_s": ncols / es,
                                     "worst_true_relres": worst, "steps": st["steps"], "peak_bytes": st["peak_bytes"]}}
        if load == 0.95:
            # FP64 arms that batch too: one block solve per request (FP64
            # V-cycle), and the same server on the FP64 hierarchies
            lb, eb = run_plain(arr, batch_solve)
            srv = amg.Server(h64, slots=16, budget_bytes=120 << 30, rtol=rtol, maxit=2000)
            l64, e64, w64 = run_served(arr, srv)
            srv.close()
            row["batch_fp64_per_request"] = {"p50_ms": q(lb, 50), "p99_ms": q(lb, 99), "solves_per_s": ncols / eb}
            row["served_fp64"] = {"p50_ms": q(l64, 50), "p99_ms": q(l64, 99), "solves_per_s": ncols / e64,
                                  "worst_true_relres": w64}
        out.append(row)
    # throughput with every request queued at once (saturated): the
    # mixed-precision server against the FP64 server and back-to-back FP64
    # block solves per request
    srv = amg.Server(h64, slots=16, budget_bytes=120 << 30, rtol=rtol, maxit=2000)
    l64, e64, w64 = run_served(np.zeros(nreq), srv)
    srv.close()
    lb, eb = run_plain(np.zeros(nreq), batch_solve)
    srv = amg.Server(h32, slots=16, budget_bytes=120 << 30, rtol=rtol, maxit=2000)
    ls, es, worst = run_served(np.zeros(nreq), srv)
    srv.close()
    line = {"metric": "served solves/s and p50/p99 latency (continuous batching, FP32 V-cycle in FP64 CG)",
            "value": int(req_k.sum()) / es, "unit": "solves/s", "higher_is_better": True,
            "plain_fp64_capacity_solves_per_s": capacity, "requests": nreq, "mean_rhs_per_request": mean_k,
            "hierarchies": [s[0] for s in specs], "rtol": rtol, "loads": out,
            "saturated": {"solves_per_s": ncols / es, "p50_ms": q(ls, 50), "p99_ms": q(ls, 99),
                          "worst_true_relres": worst,
                          "served_fp64": {"solves_per_s": ncols / e64, "p50_ms": q(l64, 50), "p99_ms": q(l64, 99),
                                          "worst_true_relres": w64},
                          "batch_fp64_per_request": {"solves_per_s": ncols / eb, "p50_ms": q(lb, 50),
                                                     "p99_ms": q(lb, 99)}},
            "latency": "arrival to the result in host memory",
            "data": "synthetic"}
    print(json.dumps(line), flush=True)
    for h in h64 + h32:
        h.close()
    return 0


def many_arm(args):
    """Many uneven independent systems in one hierarchy and one solve.

    256 3D Poisson systems with grid edges drawn uniformly from 16..64 (seed 5,
    4,096 to 262,144 unknowns each), right-hand sides N(0, 1) (seed 5), x0 = 0,
    rel-res 1e-6 per system. One step = amg_setup_many + amg_solve_many +
    amg_free with the systems resident in HBM. Beside it: the same systems
    set up and solved one at a time with the plain FP64 method.
    """
    import torch
    from paper_2006_16147_gb300 import amg
    from paper_2006_16147_gb300 import workloads as W
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    amg.lib()
    edges = W.batch_edges(args.many_systems, seed=5)
    mats = [W.poisson3d(e) for e in edges]
    offs = np.concatenate([[0], np.cumsum([M.n for M in mats])]).astype(np.int64)
    ntot = int(offs[-1])
    nnz_tot = sum(M.nnz for M in mats)
    b = W.rhs_normal(ntot, seed=5)
    t = lambda a: torch.from_numpy(np.ascontiguousarray(a)).to(dev)
    systems = [(t(M.row_ptr), t(M.col), t(M.val), torch.ones(M.n, dtype=torch.float64, device=dev)) for M in mats]
    d_b = t(b)
    d_x = torch.zeros(ntot, dtype=torch.float64, device=dev)
    stream = torch.cuda.current_stream(dev)
    prec = amg.AMG_FP32_VCYCLE if args.precision == "fp32" else amg.AMG_FP64
    m = len(mats)

    def step(profile=0, marks=None):
        d_x.zero_()
        h = amg.amg_setup_many(systems, precision=prec, krylov=args.krylov, autotune=args.autotune,
                               profile=profile, stream=stream.cuda_stream)
        if marks is not None:
            marks[1].record(stream)
        infos = amg.amg_solve_many(h, d_b, d_x, m, rtol=args.rtol, maxit=1000)
        hi = amg.amg_hierarchy_info(h)
        ks = amg.amg_kernel_stats(h) if profile else None
        h.close()
        return infos, hi, ks

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()
    launches0 = amg.amg_launch_count()
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    runs = []
    with ClockSampler(local) as clk:
        ev0.record(stream)
        for _ in range(args.steps):
            runs.append(step())
        ev1.record(stream)
        torch.cuda.synchronize()
    ms = ev0.elapsed_time(ev1) / args.steps
    launches = (amg.amg_launch_count() - launches0) // args.steps
    clocks = clk.summary()
    infos, hi, _ = runs[-1]
    # one profiled step after the timed region: setup / solve split and the scope table
    marks = [torch.cuda.Event(enable_timing=True) for _ in range(3)]
    marks[0].record(stream)
    _, _, ks = step(profile=1, marks=marks)
    marks[2].record(stream)
    torch.cuda.synchronize()
    prof_setup_ms, prof_solve_ms = marks[0].elapsed_time(marks[1]), marks[1].elapsed_time(marks[2])
    kernels = {name: {"launches": sc, "ms": round(kms, 4)}
               for name, (sc, kms, by) in sorted(ks.items(), key=lambda kv: -kv[1][1])}
    xs = d_x.cpu().numpy()
    worst = 0.0
    for s, M in enumerate(mats):
        bs = b[offs[s]:offs[s + 1]]
        worst = max(worst, float(np.linalg.norm(bs - M.scipy() @ xs[offs[s]:offs[s + 1]]) / np.linalg.norm(bs)))
    its = [i["iterations"] for i in infos]

    # the same systems one at a time, plain FP64 (setup + solve each)
    torch.cuda.synchronize()
    xo = torch.zeros(int(max(M.n for M in mats)), dtype=torch.float64, device=dev)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for s, (rp, cl, vl, w) in enumerate(systems):
        h = amg.amg_setup(rp, cl, vl, w, stream=stream.cuda_stream)
        xo[:mats[s].n].zero_()
        amg.amg_solve(h, d_b[offs[s]:offs[s + 1]], xo[:mats[s].n], rtol=args.rtol, maxit=1000)
        h.close()
    e1.record(stream)
    torch.cuda.synchronize()
    solo_ms = e0.elapsed_time(e1)

    # end to end: systems and right-hand sides copied from pinned host memory
    # inside the timed region, solutions read back
    hp = [tuple(torch.from_numpy(np.ascontiguousarray(a)).pin_memory() for a in (M.row_ptr, M.col, M.val))
          for M in mats]
    bh = torch.from_numpy(b).pin_memory()
    xh = torch.empty(ntot, dtype=torch.float64).pin_memory()
    e2e_steps = max(1, min(3, args.steps))
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for _ in range(e2e_steps):
        sy = [(rp.to(dev, non_blocking=True), cl.to(dev, non_blocking=True), vl.to(dev, non_blocking=True),
               torch.ones(rp.shape[0] - 1, dtype=torch.float64, device=dev)) for rp, cl, vl in hp]
        db = bh.to(dev, non_blocking=True)
        dx = torch.zeros(ntot, dtype=torch.float64, device=dev)
        h = amg.amg_setup_many(sy, precision=prec, krylov=args.krylov, stream=stream.cuda_stream)
        amg.amg_solve_many(h, db, dx, m, rtol=args.rtol, maxit=1000)
        h.close()
        xh.copy_(dx)
    torch.cuda.synchronize()
    e2e_ms = (time.perf_counter() - t0) * 1e3 / e2e_steps
    h2d = sum(M.row_ptr.nbytes + M.col.nbytes + M.val.nbytes for M in mats) + b.nbytes

    cpu = None
    if not args.no_cpu_baseline and rank == 0 and world == 1:
        import oracle
        oracle.build()
        t0 = time.perf_counter()
        done = 0
        for s, M in enumerate(mats):
            H = oracle.Hierarchy(M)
            H.pcg(b[offs[s]:offs[s + 1]], rtol=args.rtol)
            done += M.n
            if time.perf_counter() - t0 > 10.0:
                break
        el = time.perf_counter() - t0
        cpu = {"value": el * 1e3 * ntot / done, "unit": "ms", "cores": 1, "kind": "oracle",
               "sample": f"oracle setup + PCG of the first {s + 1} systems ({done} unknowns, {el:.1f} s), "
                         f"scaled by unknowns x{ntot / done:.1f}"}

    if rank == 0:
        line = {
            "metric": f"batched AMG-PCG: {m} independent systems to rel-res 1e-6 (setup + solve)",
            "value": round(ms, 3), "unit": "ms", "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": round(ms, 3), "higher_is_better": False, "scaling": "weak", "vs_baseline": None,
            "dtype": "f64" if args.precision == "fp64" else "f64-cg/f32-vcycle", "data": "synthetic",
            "config": {"workload": f"{m}_poisson3d_edges16-64_seed5", "systems": m, "n": ntot, "nnz": nnz_tot,
                       "edges_min": min(edges), "edges_max": max(edges), "rtol": args.rtol,
                       "precision": args.precision, "autotune": args.autotune,
                       "l2": "inputs larger than L2, no flush"},
            "systems_per_s": round(m * 1e3 / ms, 1),
            "iterations_max": max(its), "iterations_mean": round(float(np.mean(its)), 2),
            "worst_numpy_relres": worst, "levels": hi["n"],
            "one_at_a_time_fp64_ms": round(solo_ms, 2), "speedup_vs_one_at_a_time": round(solo_ms / ms, 2),
            "gpu_launches": int(launches), "clocks": clocks,
            "profiled_setup_ms": round(prof_setup_ms, 3), "profiled_solve_ms": round(prof_solve_ms, 3),
            "kernels": kernels,
            "kernel_stats": "CUDA events around every scope in one profiled step after the timed region",
            "e2e": {"value": e2e_ms, "unit": "ms", "h2d_bytes_per_step": int(h2d), "d2h_bytes_per_step": 8 * ntot},
            "cpu_baseline": cpu,
        }
        print(json.dumps(line), flush=True)
    return 0


def block_arm(args):
    """Multi-RHS block solve: 3D Poisson block-grid^3 with K columns.

    Columns N(0, 1) (seed 4), row-major n x K, x0 = 0, rel-res 1e-6 per column.
    One step = amg_setup + amg_solve_batch + amg_free with A and B resident in
    HBM. Beside it: the K columns solved one after another on one hierarchy.
    """
    import torch
    from paper_2006_16147_gb300 import amg
    from paper_2006_16147_gb300 import workloads as W
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    amg.lib()
    K = args.block
    A = W.poisson3d(args.block_grid)
    B = W.rhs_normal(A.n, seed=4, k=K)
    t = lambda a: torch.from_numpy(np.ascontiguousarray(a)).to(dev)
    d_ptr, d_col, d_val = t(A.row_ptr), t(A.col), t(A.val)
    d_w = torch.ones(A.n, dtype=torch.float64, device=dev)
    d_B = t(B)
    d_X = torch.zeros(A.n, K, dtype=torch.float64, device=dev)
    stream = torch.cuda.current_stream(dev)
    prec = amg.AMG_FP32_VCYCLE if args.precision == "fp32" else amg.AMG_FP64

    def step(profile=0):
        d_X.zero_()
        h = amg.amg_setup(d_ptr, d_col, d_val, d_w, precision=prec, krylov=args.krylov, autotune=args.autotune,
                          profile=profile, stream=stream.cuda_stream)
        infos = amg.amg_solve_batch(h, d_B, d_X, rtol=args.rtol, maxit=1000)
        return h, infos

    for _ in range(args.warmup):
        h, _ = step()
        h.close()
    torch.cuda.synchronize()
    launches0 = amg.amg_launch_count()
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    solve_ms = []
    # timed steps run unprofiled, so each CG step is one CUDA graph launch
    with ClockSampler(local) as clk:
        ev0.record(stream)
        for _ in range(args.steps):
            h, infos = step(profile=0)
            solve_ms.append(infos[0]["solve_ms"])
            hi = amg.amg_hierarchy_info(h)
            h.close()
        ev1.record(stream)
        torch.cuda.synchronize()
    ms = ev0.elapsed_time(ev1) / args.steps
    launches = (amg.amg_launch_count() - launches0) // args.steps
    clocks = clk.summary()
    # per-kernel CUDA-event times from one more step with the library's event
    # scopes on (kernels launched one by one)
    kstats = {}
    h, _ = step(profile=1)
    for name, (sc, kms, by) in amg.amg_kernel_stats(h).items():
        kstats[name] = [sc, kms, by]
    h.close()
    X = d_X.cpu().numpy()
    R = B - A.scipy() @ X
    worst = float(np.max(np.linalg.norm(R, axis=0) / np.linalg.norm(B, axis=0)))
    its = [i["iterations"] for i in infos]

    # the same columns one after another on one hierarchy (solve only), and
    # the batch solve alone on that hierarchy
    h = amg.amg_setup(d_ptr, d_col, d_val, d_w, precision=prec, krylov=args.krylov, autotune=args.autotune,
                      stream=stream.cuda_stream)
    xc = torch.zeros(A.n, dtype=torch.float64, device=dev)
    cols = [d_B[:, c].contiguous() for c in range(K)]
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    seq_its = []
    e0.record(stream)
    for c in range(K):
        xc.zero_()
        seq_its.append(amg.amg_solve(h, cols[c], xc, rtol=args.rtol, maxit=1000)["iterations"])
    e1.record(stream)
    torch.cuda.synchronize()
    seq_ms = e0.elapsed_time(e1)
    d_X.zero_()
    e0.record(stream)
    amg.amg_solve_batch(h, d_B, d_X, rtol=args.rtol, maxit=1000)
    e1.record(stream)
    torch.cuda.synchronize()
    batch_solve_ms = e0.elapsed_time(e1)
    h.close()

    peak, peak_kind = _peaks()
    dom = max((k for k in kstats if not k.startswith("setup_")), key=lambda k: kstats[k][1])
    nl, kms, by = kstats[dom]
    if dom == "spmv_dot":
        # the outer CG's SpMM over K columns is FP64-ALU bound on this GPU:
        # 2 nnz K flops for the product and 2 n K for the per-column p . q
        flops = 2.0 * A.nnz * K + 2.0 * A.n * K
        achieved = flops / (kms / nl * 1e-3) / 1e12
        roofline = {"kernel": dom, "bound": "alu", "achieved": round(achieved, 3), "peak": FP64_PEAK_TFLOPS,
                    "unit": "TFLOP/s", "frac": round(achieved / FP64_PEAK_TFLOPS, 4), "traffic": None,
                    "peak_kind": "nominal FP64 (non-tensor) rate of the profiling recipe",
                    "flops_per_launch": flops, "ms_per_launch": kms / nl,
                    "hbm_achieved_gbs": round((by / nl) / (kms / nl * 1e-3) / 1e9, 1)}
    else:
        achieved = (by / nl) / (kms / nl * 1e-3) / 1e9
        roofline = {"kernel": dom, "bound": "hbm", "achieved": round(achieved, 1), "peak": peak, "unit": "GB/s",
                    "frac": round(achieved / peak, 4), "traffic": None, "peak_kind": peak_kind,
                    "bytes_per_launch": by / nl, "ms_per_launch": kms / nl}
    kernel_table = {k: {"launches_per_step": v[0], "ms_per_step": round(v[1], 4),
                        "GBps": round(v[2] / max(v[1], 1e-12) / 1e6, 1) if v[2] else None}
                    for k, v in sorted(kstats.items(), key=lambda kv: -kv[1][1])}
    if rank == 0:
        line = {
            "metric": f"multi-RHS AMG-PCG: {K} right-hand sides to rel-res 1e-6 (setup + block solve)",
            "value": round(ms, 3), "unit": "ms", "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": round(ms, 3), "higher_is_better": False, "scaling": "weak", "vs_baseline": None,
            "dtype": "f64" if args.precision == "fp64" else "f64-cg/f32-vcycle", "data": "synthetic",
            "config": {"workload": f"poisson3d_{args.block_grid}^3_{K}rhs_seed4", "n": A.n, "nnz": A.nnz, "k": K,
                       "rtol": args.rtol, "precision": args.precision, "autotune": args.autotune,
                       "l2": "inputs larger than L2, no flush"},
            "columns_per_s": round(K * 1e3 / ms, 1), "iterations_max": max(its),
            "iterations_mean": round(float(np.mean(its)), 2), "worst_numpy_relres": worst,
            "levels": hi["n"], "block_solve_ms": round(batch_solve_ms, 2),
            "sequential_single_rhs_solve_ms": round(seq_ms, 2), "sequential_iterations_max": max(seq_its),
            "sequential_iterations_mean": round(float(np.mean(seq_its)), 2),
            "speedup_vs_sequential": round(seq_ms / batch_solve_ms, 2),
            "roofline": roofline, "kernels": kernel_table, "gpu_launches": int(launches), "clocks": clocks,
            "kernel_stats": "CUDA events of one profiled step after the timed region (kernels launched "
                            "one by one); the timed steps replay one CUDA graph per CG step",
        }
        print(json.dumps(line), flush=True)
    return 0


def main():
    args = _args()
    if args.impl == "reference":
        return reference_arm(args)
    if args.serve:
        return serve_arm(args)
    if args.many:
        return many_arm(args)
    if args.block:
        return block_arm(args)

    import torch
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    dist = None
    torch.cuda.set_device(local)          # before the process group: NCCL binds this rank's GPU
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl" if torch.cuda.is_available() else "gloo")
    dev = torch.device("cuda", local)

    from paper_2006_16147_gb300 import amg
    amg.lib()

    A, b = _workload(args.grid, args.workload)
    t = lambda a: torch.from_numpy(np.ascontiguousarray(a)).to(dev)
    d_ptr, d_col, d_val = t(A.row_ptr), t(A.col), t(A.val)
    d_w = torch.ones(A.n, dtype=torch.float64, device=dev)
    d_b = t(b)
    d_x = torch.zeros(A.n, dtype=torch.float64, device=dev)
    stream = torch.cuda.current_stream(dev)
    prec = amg.AMG_FP32_VCYCLE if args.precision == "fp32" else amg.AMG_FP64

    def step(profile=0, keep=False):
        d_x.zero_()
        w = (amg.amg_smooth_vector(d_ptr, d_col, d_val, d_w, args.smooth_w, stream=stream.cuda_stream)
             if args.smooth_w > 0 else d_w)
        h = amg.amg_setup(d_ptr, d_col, d_val, w, precision=prec, profile=profile, krylov=args.krylov,
                          autotune=args.autotune, cycle=args.kdepth if args.cycle == "k" else 0,
                          smooth_p=args.smooth_p, pre=args.pre, post=args.post, omega_rule=args.omega_rule,
                          stream=stream.cuda_stream)
        info = amg.amg_solve(h, d_b, d_x, rtol=args.rtol, maxit=1000)
        if keep:
            return h, info
        h.close()
        return None, info

    def barrier():
        torch.cuda.synchronize()
        if dist is not None:
            dist.barrier()

    for _ in range(args.warmup):
        step()

    # ---- timed region: K unprofiled steps, CUDA events on the library's stream
    infos = []
    hinfos = []
    barrier()
    launches0 = amg.amg_launch_count()
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    with ClockSampler(local) as clk:
        ev0.record(stream)
        for k in range(args.steps):
            h, info = step(profile=0, keep=True)
            infos.append(info)
            hinfos.append(amg.amg_hierarchy_info(h))
            h.close()
        ev1.record(stream)
        barrier()
    launches = amg.amg_launch_count() - launches0
    ms = ev0.elapsed_time(ev1) / args.steps
    if dist is not None:
        tt = torch.tensor([ms], device=dev)
        dist.all_reduce(tt, op=dist.ReduceOp.MAX)
        ms = float(tt.item())
    clocks = clk.summary()

    # ---- per-kernel times: a few more steps with the library's CUDA-event
    # scopes around every kernel (on the launching stream), right after the
    # timed region; they give the kernel table and the roofline
    kstats = {}
    psteps = max(1, min(args.profile_steps, args.steps))
    pev0, pev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    pev0.record(stream)
    for k in range(psteps):
        h, _ = step(profile=1, keep=True)
        for name, (sc, kms, by) in amg.amg_kernel_stats(h).items():
            st_ = kstats.setdefault(name, [0, 0.0, 0.0])
            st_[0] += sc
            st_[1] += kms
            st_[2] += by
        h.close()
    pev1.record(stream)
    torch.cuda.synchronize()
    profiled_ms = pev0.elapsed_time(pev1) / psteps

    # residual check of the last solution (independent of the library)
    xs = d_x.cpu().numpy()
    rel = float(np.linalg.norm(b - A.scipy() @ xs) / np.linalg.norm(b))

    # ---- accuracy of a mixed-precision or non-default run: error against an
    # FP64 solve of the same system to rel-res 1e-10, and iterations at 1e-8
    accuracy = None
    if (args.precision == "fp32" or args.workload != "poisson" or args.cycle == "k" or args.smooth_p
            or (args.pre, args.post) != (1, 1)):
        accuracy = {}
        h64 = amg.amg_setup(d_ptr, d_col, d_val, d_w, stream=stream.cuda_stream)
        xr = torch.zeros_like(d_x)
        amg.amg_solve(h64, d_b, xr, rtol=1e-10, maxit=2000)
        h64.close()
        for tol in (args.rtol, 1e-8):
            hh = amg.amg_setup(d_ptr, d_col, d_val, d_w, precision=prec, krylov=args.krylov,
                               cycle=args.kdepth if args.cycle == "k" else 0, smooth_p=args.smooth_p,
                               pre=args.pre, post=args.post, omega_rule=args.omega_rule,
                               stream=stream.cuda_stream)
            xt = torch.zeros_like(d_x)
            inf = amg.amg_solve(hh, d_b, xt, rtol=tol, maxit=2000)
            hh.close()
            e = float(torch.linalg.norm(xt - xr) / torch.linalg.norm(xr))
            accuracy[f"rtol_{tol:g}"] = {"iterations": inf["iterations"], "true_relres": inf["true_relres"],
                                         "rel_error_vs_fp64_1e-10": e}

    # ---- roofline of the dominant solve kernel (largest summed time)
    peak, peak_kind = _peaks()
    solve_k = {k: v for k, v in kstats.items() if not k.startswith("setup_")}
    dom = max(solve_k, key=lambda k: solve_k[k][1])
    nl, ms_tot, by_tot = solve_k[dom]
    per_launch_ms = ms_tot / nl
    achieved = (by_tot / nl) / (per_launch_ms * 1e-3) / 1e9
    traffic = _traffic(dom, A.n, args.workload, args.precision)
    roofline = {"kernel": dom, "bound": "hbm", "achieved": round(achieved, 1), "peak": peak, "unit": "GB/s",
                "frac": round(achieved / peak, 4), "traffic": traffic, "peak_kind": peak_kind,
                "traffic_source": ("ncu DRAM bytes on 160^3 scaled by rows" if traffic else None),
                "bytes_per_launch": by_tot / nl, "ms_per_launch": per_launch_ms, "launches": nl // psteps,
                "timing": f"CUDA events around every launch over {psteps} profiled steps after the timed region"}
    kernel_table = {k: {"launches_per_step": v[0] // psteps, "ms_per_step": round(v[1] / psteps, 4),
                        "GBps": round(v[2] / max(v[1], 1e-12) / 1e6, 1) if v[2] else None}
                    for k, v in sorted(kstats.items(), key=lambda kv: -kv[1][1])}

    # ---- end to end through the host-buffer entry points (pinned host memory)
    e2e = None
    if not args.no_e2e:
        hp = {k: torch.from_numpy(np.ascontiguousarray(v)).pin_memory().numpy()
              for k, v in dict(ptr=A.row_ptr, col=A.col, val=A.val, w=np.ones(A.n), b=b).items()}
        xh = torch.zeros(A.n, dtype=torch.float64).pin_memory().numpy()
        e2e_steps = max(1, min(3, args.steps))
        kc = args.kdepth if args.cycle == "k" else 0
        hopt = dict(precision=prec, krylov=args.krylov, cycle=kc, smooth_p=args.smooth_p, pre=args.pre,
                    post=args.post, omega_rule=args.omega_rule)
        amg_h = amg.amg_setup_host(hp["ptr"], hp["col"], hp["val"], hp["w"], **hopt)
        amg_h.close()
        barrier()
        t0 = time.perf_counter()
        for _ in range(e2e_steps):
            xh[:] = 0.0
            hh = amg.amg_setup_host(hp["ptr"], hp["col"], hp["val"], hp["w"], **hopt)
            amg.amg_solve_host(hh, hp["b"], xh, rtol=args.rtol, maxit=1000)
            hh.close()
        barrier()
        e2e_ms = (time.perf_counter() - t0) * 1e3 / e2e_steps
        h2d = A.row_ptr.nbytes + A.col.nbytes + A.val.nbytes + 8 * A.n * 3
        e2e = {"value": e2e_ms, "unit": "ms", "h2d_bytes_per_step": int(h2d), "d2h_bytes_per_step": int(8 * A.n)}

    # ---- CPU oracle baseline (rank 0, N = 1 only): the oracle as it stands on
    # the same workload, once, setup and PCG timed separately
    cpu = None
    if not args.no_cpu_baseline and rank == 0 and world == 1:
        import oracle
        oracle.build()
        g = args.cpu_sample_grid if args.cpu_sample_grid > 0 else args.grid
        As, bs = (A, b) if g == args.grid else _workload(g, args.workload)
        r = _oracle_run(As, bs, args.rtol, **_oracle_kw(args))
        scale = A.n / r["n"]
        cpu = {"value": (r["setup_s"] + r["solve_s"]) * 1e3 * scale, "unit": "ms", "cores": 1, "kind": "oracle",
               "setup_ms": r["setup_s"] * 1e3 * scale, "solve_ms": r["solve_s"] * 1e3 * scale,
               "iterations": r["iterations"],
               "sample": (f"oracle setup {r['setup_s']:.2f} s + PCG {r['solve_s']:.2f} s ({r['iterations']} it) "
                          + (f"on the full {g}^3 instance, one run, not scaled" if scale == 1 else
                             f"on the {g}^3 instance, scaled x{scale:.0f} by unknowns")),
               **_host_info()}

    if rank == 0:
        it = [i["iterations"] for i in infos]
        hi = hinfos[-1]
        line = {
            "metric": METRIC, "value": round(ms, 3), "unit": "ms", "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": round(ms, 3), "higher_is_better": False, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64" if args.precision == "fp64" else "f64-cg/f32-vcycle",
            "data": "synthetic",
            "config": {"workload": _workload_name(args),
                       "grid": args.grid, "cycle": args.cycle, "kdepth": args.kdepth if args.cycle == "k" else None,
                       "n": A.n, "nnz": A.nnz, "rtol": args.rtol, "sweeps": 3, "smoother": f"l1-jacobi {args.pre}+{args.post}",
                       "coarse": "dense cholesky", "l2": "inputs (1.4 GB) larger than L2, no flush",
                       "precision": args.precision, "autotune": args.autotune,
                       "parallelism": "replicas" if world > 1 else "single"},
            "iterations": it[-1], "true_relres": infos[-1]["true_relres"], "numpy_relres": rel,
            "setup_ms": round(statistics.mean(h["setup_ms"] for h in hinfos), 3),
            "solve_ms": round(statistics.mean(i["solve_ms"] for i in infos), 3),
            "levels": hi["n"], "opc": round(hi["opc"], 4), "solves_per_s": round(world * 1e3 / ms, 3),
            "match_rounds": int(sum(sum(r) for r in hi["rounds"])),
            "roofline": roofline, "kernels": kernel_table, "profiled_ms_per_step": round(profiled_ms, 3),
            "kernel_stats": f"CUDA events around every launch over {psteps} profiled steps after the timed "
                            "region; the timed steps run unprofiled",
            "gpu_launches": int(launches), "gpu_launches_per_step": int(launches // args.steps),
            "accuracy": accuracy,
            "clocks": clocks, "e2e": e2e, "cpu_baseline": cpu,
        }
        print(json.dumps(line), flush=True)
    if dist is not None:
        dist.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())

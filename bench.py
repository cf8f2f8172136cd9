"""Benchmark: design iterations per second of AARMR topology optimisation on
the 3D cantilever 192 x 96 x 96 hex8 (5,447,811 DOFs), mixed precision.

One step = one design iteration of Fig. 1 / Algorithm 1 (density filter,
SIMP, MGCG or CARM with its residual check and MGCG fallback, compliance
and sensitivity, sensitivity filter, OC update), run through the C ABI with
every array resident in HBM.  The job starts from the workload's initial
design; the first W iterations are warm-up, the next K are timed (default
W=3, K=27: iterations 4..30, so both the MGCG phase (k <= N_on = 15) and the
CARM phase are inside the timed region).

Prints one JSON line (see the fields below).  ``--impl reference`` times the
CPU oracle on the host instead.  Under torchrun (N > 1) every rank runs an
independent replica (the path does not shard); value is the sum of the
ranks' iterations over the slowest rank's time.
"""

from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "design iters/s at 5.4M DOFs"
UNIT = "design_iters/s"
WORKLOAD = ("3D cantilever 192x96x96 hex8 (5,447,811 DOFs), E0=1 Emin=1e-9 nu=0.3 p=3, "
            "volfrac 0.12, rmin 2.0, 6-level MGCG ({prec}, rtol 1e-8), "
            "CARM s=10 (N_s=N_m=10, N_on=15, eps_tol 1e-3)")
PREC_TEXT = {"mixed": "FP32 V-cycle/apply; CG vectors, dots, CARM and OC FP64-accurate in "
                      "double-float on the FP32 pipe",
             "fp64": "all float64"}


def _workload(precision: str) -> str:
    return WORKLOAD.format(prec=PREC_TEXT[precision])


def _args():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=27)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--precision", default="mixed", choices=["mixed", "fp64"])
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--small", action="store_true", help="48x24x24 instead (quick checks)")
    ap.add_argument("--kernel", default=None, choices=[None, "apply"],
                    help="time one kernel alone (profiling) instead of the design loop")
    ap.add_argument("--kernel-prec", default="fp32", choices=["fp32", "fp64"])
    ap.add_argument("--serve-jobs", type=int, default=24,
                    help="jobs of the served stream replayed for p50/p99 (0: skip)")
    ap.add_argument("--serve-iters", type=int, default=6)
    ap.add_argument("--serve-time-scale", type=float, default=0.25)
    return ap.parse_args()


def _problem(args):
    from workloads import config3_cantilever3d, cantilever3d
    if args.small:
        return cantilever3d(48, 24, 24, volfrac=0.12, rmin=2.0, n_iter=30, mg_levels=4,
                            precision=args.precision, n_parm=10, n_carm=10, n_on=15,
                            eps_tol=1e-3, rtol=1e-8, maxit=200)
    return config3_cantilever3d(args.precision)


# ---------------------------------------------------------------------------
# clocks sampled during the timed region
# ---------------------------------------------------------------------------
class ClockSampler:
    QUERY = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.proc = None
        self.path = os.path.join("/tmp", f"bench_clocks_{os.getpid()}.csv")

    def start(self):
        try:
            self.fh = open(self.path, "w")
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.gpu), f"--query-gpu={self.QUERY}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=self.fh, stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        self.fh.close()
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in open(self.path):
            f = [x.strip() for x in line.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                mx.append(float(f[2]))
            except ValueError:
                continue
            for nm, v in zip(names, f[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        if not sm:
            return None
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx),
                "reasons": sorted(reasons), "samples": len(sm)}


# ---------------------------------------------------------------------------
# CPU oracle baseline (bounded sample, scaled to the workload)
# ---------------------------------------------------------------------------
ORACLE_SAMPLE_MESH = (48, 24, 24)


def _oracle_sample_worker(steps: int, precision: str):
    """Runs in a child process with BLAS limited to one thread."""
    from oracle import aarmr
    from workloads import cantilever3d, grid_counts
    nx, ny, nz = ORACLE_SAMPLE_MESH
    p = cantilever3d(nx, ny, nz, volfrac=0.12, rmin=2.0, n_iter=steps, mg_levels=4,
                     precision=precision, n_parm=10, n_carm=10, n_on=15, eps_tol=1e-3,
                     rtol=1e-8, maxit=200)
    m = aarmr.OracleModel(p)
    t0 = time.perf_counter()
    aarmr.run(p, n_iter=steps, mode="aarmr", model=m)
    dt = time.perf_counter() - t0
    n_sample = grid_counts(3, nx, ny, nz)[2]
    n_full = grid_counts(3, 192, 96, 96)[2]
    return dt, n_sample, n_full


def cpu_baseline(steps: int = 2, precision: str = "mixed"):
    env = dict(os.environ, OMP_NUM_THREADS="1", OPENBLAS_NUM_THREADS="1", MKL_NUM_THREADS="1")
    code = ("import json,sys; sys.path.insert(0, %r); import bench; "
            "print(json.dumps(bench._oracle_sample_worker(%d, %r)))" % (ROOT, steps, precision))
    r = subprocess.run([sys.executable, "-c", code], capture_output=True, text=True, env=env,
                       cwd=ROOT, timeout=900)
    if r.returncode != 0:
        raise RuntimeError("oracle baseline failed: " + r.stderr[-2000:])
    dt, n_sample, n_full = json.loads(r.stdout.strip().splitlines()[-1])
    scale = n_full / n_sample
    per_iter = dt / steps * scale
    return {"value": 1.0 / per_iter, "unit": UNIT, "cores": 1, "kind": "oracle",
            "sample": (f"{steps} oracle design iterations (numpy/scipy float64, MGCG branch) "
                       f"on the same cantilever at {ORACLE_SAMPLE_MESH[0]}x{ORACLE_SAMPLE_MESH[1]}"
                       f"x{ORACLE_SAMPLE_MESH[2]} ({n_sample} DOFs), {dt:.1f} s, time scaled by "
                       f"the DOF ratio {scale:.1f} to 192x96x96"),
            "seconds_per_iter_scaled": per_iter}


# ---------------------------------------------------------------------------
# the GPU arm
# ---------------------------------------------------------------------------
def _dist():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def slowest_rank(seconds: float, ws: int, device: str = "cuda") -> float:
    """Time of the slowest rank: an all-reduce MAX over the process group
    (NCCL on GPUs, gloo on the host), or the local time when alone."""
    if ws <= 1:
        return seconds
    import torch
    import torch.distributed as dist
    t = torch.tensor([seconds], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def whole_job_rate(steps: int, ws: int, slowest_s: float) -> float:
    """Design iterations per second of all replicas together: every rank
    runs `steps` iterations of its own job, and the job ends with the slowest."""
    return ws * steps / slowest_s


def _traffic_from_profiles(kernel_tag: str):
    """Per-launch DRAM bytes of the dominant kernel from the committed ncu
    summary, if it was taken on the current kernel source."""
    import hashlib
    path = os.path.join(ROOT, "profiles", "apply_pair_cantilever192.md")
    src = os.path.join(ROOT, "paper_2205_00385_gb300", "csrc", "kernels_pair.cu")
    if not os.path.exists(path):
        return None
    sha = hashlib.sha256(open(src, "rb").read()).hexdigest()[:16]
    rec = {}
    for line in open(path):
        if ": " in line and line.startswith("- "):
            k, v = line[2:].split(": ", 1)   # keys may hold a colon ("sha256[:16]")
            rec[k.strip()] = v.strip().strip("`")
    if rec.get("kernels_pair.cu sha256[:16]") != sha:
        return None
    try:
        return float(rec.get(f"{kernel_tag} dram bytes per launch", "nan"))
    except ValueError:
        return None


def run_ours(args):
    import torch
    ws, rank, local = _dist()
    torch.cuda.set_device(local)
    if ws > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    from paper_2205_00385_gb300 import binding as B
    from paper_2205_00385_gb300.driver import TopoSolver
    p = _problem(args)
    W, K = args.warmup, args.steps

    def barrier():
        torch.cuda.synchronize()
        if ws > 1:
            import torch.distributed as dist
            dist.barrier()
            torch.cuda.synchronize()

    # ---- device-resident run ----
    s = TopoSolver(p)
    for _ in range(W):
        s.step(read_compliance=False)
    # timed kinds: the float32 finest-grid operator (K p of every CG
    # iteration, the kernel the roofline is taken on), whole V-cycles and the
    # other finest-grid variants; nothing inside the captured V-cycle graph
    B.to_profile_enable(s.ctx, (1 << B.PK_FINE32) | (1 << B.PK_VCYCLE) | (1 << B.PK_FINE_OTHER))
    for kind in (B.PK_FINE32, B.PK_COARSE, B.PK_VCYCLE, B.PK_FINE_OTHER):
        B.to_profile_read(s.ctx, kind)
    B.to_launch_count(s.ctx, reset=True)
    clocks = ClockSampler(local)
    barrier()
    clocks.start()
    ev0 = torch.cuda.Event(enable_timing=True)
    ev1 = torch.cuda.Event(enable_timing=True)
    ev0.record(s.stream)
    t0 = time.perf_counter()
    branches = []
    cg = 0
    for _ in range(K):
        log = s.step(read_compliance=False)
        branches.append(log.branch)
        cg += log.cg_iters
    ev1.record(s.stream)
    barrier()
    wall = time.perf_counter() - t0
    clk = clocks.stop()
    dev_s = ev0.elapsed_time(ev1) / 1e3
    launches = B.to_launch_count(s.ctx)
    n_f, ms_f, by_f = B.to_profile_read(s.ctx, B.PK_FINE32)
    n_v, ms_v, _ = B.to_profile_read(s.ctx, B.PK_VCYCLE)
    n_o, ms_o, by_o = B.to_profile_read(s.ctx, B.PK_FINE_OTHER)
    kname = "k_apply3_pair<EPI_APPLY> (finest-grid K p, float32, two element columns per thread)"
    pair = n_f > 0
    if not pair:   # float64 path: the finest-grid operator runs in float64
        n_f, ms_f, by_f = n_o, ms_o, by_o
        kname = "k_apply3_col<double> (finest-grid K p, float64)"
    C_final = float(s.scalars[0].item())
    s.close()
    del s
    torch.cuda.empty_cache()

    elapsed = slowest_rank(max(dev_s, 1e-9), ws)
    value = whole_job_rate(K, ws, elapsed)

    # ---- end to end through the C ABI with host buffers ----
    e2e = None
    if not args.no_e2e:
        s = TopoSolver(p)
        rho_host = torch.empty(p.nel, dtype=torch.float64, pin_memory=True)
        rho_host.copy_(torch.from_numpy(p.rho0))
        out_host = torch.empty(p.nel + 2, dtype=torch.float64, pin_memory=True)
        for _ in range(W):
            s.rho.copy_(rho_host, non_blocking=True)
            s.step(read_compliance=False)
            rho_host.copy_(s.rho)
        barrier()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(s.stream)
        for _ in range(K):
            s.rho.copy_(rho_host, non_blocking=True)              # H2D: design field
            s.step(read_compliance=False)
            out_host[:p.nel].copy_(s.rho, non_blocking=True)      # D2H: new design
            out_host[p.nel:].copy_(s.scalars[:2], non_blocking=True)  # D2H: C, change
            torch.cuda.current_stream().synchronize()
            rho_host.copy_(out_host[:p.nel])
        e1.record(s.stream)
        barrier()
        e2e_s = e0.elapsed_time(e1) / 1e3
        s.close()
        e2e_s = slowest_rank(e2e_s, ws)
        e2e = {"value": whole_job_rate(K, ws, e2e_s), "unit": UNIT, "h2d_bytes_per_step": p.nel * 8,
               "d2h_bytes_per_step": p.nel * 8 + 16}

    if rank != 0:
        return None
    peaks = {}
    try:
        peaks = json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except Exception:
        pass
    hbm_peak = float(peaks.get("hbm_gbs", 6800.0))
    peak_src = "measured" if "hbm_gbs" in peaks else "fallback"
    avg_ms = ms_f / max(n_f, 1)
    achieved = (by_f / max(n_f, 1)) / (avg_ms / 1e3) / 1e9 if n_f else 0.0
    roofline = {"bound": "hbm", "kernel": kname,
                "achieved": round(achieved, 1), "peak": hbm_peak, "unit": "GB/s",
                "frac": round(achieved / hbm_peak, 4), "peak_source": peak_src,
                "traffic": _traffic_from_profiles("k_apply3_pair") if pair else None,
                "launches": n_f, "avg_launch_us": round(avg_ms * 1e3, 2),
                "algorithmic_bytes_per_launch": round(by_f / max(n_f, 1)),
                "share_of_step": round(ms_f / 1e3 / elapsed * ws, 4),
                "vcycle": {"count": n_v, "ms": round(ms_v, 3), "graph": True},
                "other_fine_apply": {"launches": n_o, "ms": round(ms_o, 3)}}
    line = {
        "metric": METRIC, "value": round(value, 4), "unit": UNIT, "n_gpus": ws, "steps": K,
        "warmup": W, "ms_per_step": round(elapsed / K * 1e3, 3), "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32+df64" if p.precision == "mixed"
        else "f64", "data": "synthetic",
        "config": {"workload": _workload(p.precision) if not args.small else "cantilever 48x24x24 (quick)",
                   "precision": p.precision, "iterations_timed": f"{W + 1}..{W + K}",
                   "branches": {b: branches.count(b) for b in set(branches)},
                   "cg_iterations": cg, "final_compliance": C_final,
                   "l2": "inputs larger than L2 (43.6 MB per float64 vector; >2 GB state)",
                   "parallelism": f"replicas x{ws}"},
        "roofline": roofline, "e2e": e2e, "gpu_launches": int(launches), "clocks": clk,
        "wall_s": round(wall, 3),
    }
    if args.serve_jobs > 0 and ws == 1:
        from paper_2205_00385_gb300.serve import Server
        from workloads import config5_jobs
        jobs = config5_jobs()[:args.serve_jobs]
        rep = Server(int(120 * 2 ** 30), max_active=16).run(jobs, args.serve_iters,
                                                          args.serve_time_scale)
        line["serving"] = {
            "stream": (f"first {args.serve_jobs} jobs of the 256-job Poisson stream (4 jobs/s, "
                       f"arrivals x{args.serve_time_scale}), {args.serve_iters} design iterations "
                       "each, mixed precision, HBM budget 120 GiB, up to 16 concurrent jobs"),
            "throughput_iters_per_s": round(rep["throughput_iters_per_s"], 2),
            "iter_latency_ms_p50": round(rep["iter_latency_ms"]["p50"], 2),
            "iter_latency_ms_p99": round(rep["iter_latency_ms"]["p99"], 2),
            "job_latency_s_p50": round(rep["job_latency_s"]["p50"], 3),
            "job_latency_s_p99": round(rep["job_latency_s"]["p99"], 3),
            "peak_active_jobs": rep["peak_active_jobs"], "jobs_done": rep["jobs_done"]}
    if not args.no_cpu_baseline and ws == 1:
        try:
            line["cpu_baseline"] = cpu_baseline(2, p.precision)
        except Exception as ex:  # keep the GPU line even if the host baseline fails
            line["cpu_baseline"] = {"error": str(ex)[:300]}
    return line


def run_reference(args):
    ws, rank, _ = _dist()
    if rank != 0:
        return None
    W, K = args.warmup, args.steps
    per = []
    base = None
    for i in range(W + K):
        base = cpu_baseline(1, args.precision)
        if i >= W:
            per.append(base["seconds_per_iter_scaled"])
    tot = sum(per)
    v = K / tot
    cpu = dict(base)
    cpu["value"] = v
    cpu["sample"] = ("each step: " + base["sample"])
    return {"impl": "reference", "metric": METRIC, "value": round(v, 6), "unit": UNIT,
            "n_gpus": ws, "steps": K, "warmup": W, "ms_per_step": round(tot / K * 1e3, 1),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "f64", "data": "synthetic", "config": {"workload": _workload(args.precision)},
            "cpu_baseline": cpu,
            "e2e": {"value": round(v, 6), "unit": UNIT, "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}


def run_kernel_apply(args):
    """Times only the finest-grid stiffness operator K x on the bench
    workload (uniform design), for profiling: W untimed, K timed launches."""
    import numpy as np
    import torch
    from paper_2205_00385_gb300 import binding as B
    from paper_2205_00385_gb300.driver import TopoSolver
    p = _problem(args)
    s = TopoSolver(p)
    rho = torch.full((p.nel,), p.volfrac, dtype=torch.float64, device="cuda")
    B.to_set_density(s.ctx, rho)
    x = torch.from_numpy(np.random.default_rng(1).standard_normal(p.ndof)).cuda()
    y = torch.empty_like(x)
    prec = B.TO_PREC_FP32 if args.kernel_prec == "fp32" else B.TO_PREC_FP64
    for _ in range(args.warmup):
        B.to_apply(s.ctx, B.TO_OP_K, prec, x, y)
    B.to_profile_enable(s.ctx, True)
    B.to_profile_read(s.ctx, 0)
    for _ in range(args.steps):
        B.to_apply(s.ctx, B.TO_OP_K, prec, x, y)
    n, ms, by = B.to_profile_read(s.ctx, 0)
    s.close()
    return {"kernel": "k_apply", "precision": args.kernel_prec, "launches": n,
            "avg_us": ms / n * 1e3, "GB/s": by / (ms / 1e3) / 1e9,
            "bytes_per_launch": by / n, "workload": p.name + f" {p.nelx}x{p.nely}x{p.nelz}"}


def main():
    args = _args()
    if args.kernel == "apply":
        print(json.dumps(run_kernel_apply(args)), flush=True)
        return
    line = run_reference(args) if args.impl == "reference" else run_ours(args)
    if line is not None:
        print(json.dumps(line), flush=True)


if __name__ == "__main__":
    main()

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

import numpy as np

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
    ap.add_argument("--no-fp64-arm", action="store_true",
                    help="skip the plain float64 run of the same workload")
    ap.add_argument("--no-mgcg-arm", action="store_true",
                    help="skip the MGCG-only run of the same workload")
    ap.add_argument("--no-autotune", action="store_true",
                    help="keep the occupancy heuristic's launch shapes")
    ap.add_argument("--tensor-cores", action="store_true",
                    help="finest-grid float32 operator on the tensor cores (tcgen05)")
    ap.add_argument("--small", action="store_true", help="48x24x24 instead (quick checks)")
    ap.add_argument("--bridge320", action="store_true",
                    help="with --kernel: the 320x160x160 bridge (24.96M DOFs) instead")
    ap.add_argument("--fused-coarse", action="store_true",
                    help="with --kernel vcycle: the coarse levels as one cluster launch")
    ap.add_argument("--kernel", default=None, choices=[None, "apply", "vcycle"],
                    help="time one kernel alone (profiling) instead of the design loop")
    ap.add_argument("--kernel-prec", default="fp32", choices=["fp32", "fp64"])
    ap.add_argument("--serve-jobs", type=int, default=24,
                    help="jobs of the served stream replayed for p50/p99 (0: skip)")
    ap.add_argument("--serve-iters", type=int, default=6)
    ap.add_argument("--serve-time-scale", type=float, default=0.25)
    return ap.parse_args()


def _problem(args):
    from workloads import cantilever3d_192x96x96, bridge3d_320x160x160, cantilever3d
    if getattr(args, "bridge320", False):
        return bridge3d_320x160x160()
    if args.small:
        return cantilever3d(48, 24, 24, volfrac=0.12, rmin=2.0, n_iter=30, mg_levels=4,
                            precision=args.precision, n_parm=10, n_carm=10, n_on=15,
                            eps_tol=1e-3, rtol=1e-8, maxit=200)
    return cantilever3d_192x96x96(args.precision)


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
# CPU oracle baseline: the oracle's own design loop, timed per iteration
# ---------------------------------------------------------------------------
# Meshes with the workload's settings and its 6 x 3 x 3 coarsest grid: the
# oracle cannot run 192 x 96 x 96 within minutes (its assembled stiffness
# alone would be 441 M non-zeros), so it runs these and the time is scaled.
ORACLE_MESHES = {"24x12x12": (24, 12, 12, 3), "48x24x24": (48, 24, 24, 4)}
FULL_DOFS = 5447811


def _oracle_window_worker(mesh: str, warmup: int, steps: int):
    """Runs in a child process: the oracle's Algorithm 1 loop for
    warmup + steps iterations; returns the wall times of the last `steps`
    (the iterations the GPU arm times) and their branches."""
    from oracle import aarmr
    from workloads import cantilever3d, grid_counts
    nx, ny, nz, lv = ORACLE_MESHES[mesh]
    p = cantilever3d(nx, ny, nz, volfrac=0.12, rmin=2.0, n_iter=warmup + steps, mg_levels=lv,
                     precision="fp64", n_parm=10, n_carm=10, n_on=15, eps_tol=1e-3,
                     rtol=1e-8, maxit=200)
    tr = aarmr.run(p, mode="aarmr")
    hist = tr.history[warmup:]
    return {"mesh": mesh, "dofs": grid_counts(3, nx, ny, nz)[2],
            "seconds": [h.seconds for h in hist],
            "branches": {b: sum(h.branch == b for h in hist) for b in {h.branch for h in hist}},
            "iterations": f"{warmup + 1}..{warmup + steps}"}


def _cores() -> int:
    try:
        return len(os.sched_getaffinity(0))
    except Exception:
        return os.cpu_count() or 1


def oracle_window(mesh: str, warmup: int, steps: int) -> dict:
    """The oracle's timed window in a fresh interpreter (no CUDA state), with
    its BLAS free to use every core of the host; also reports the average
    number of busy cores (child CPU time over wall time)."""
    import resource
    code = ("import json,sys; sys.path.insert(0, %r); import bench; "
            "print(json.dumps(bench._oracle_window_worker(%r, %d, %d)))"
            % (ROOT, mesh, warmup, steps))
    r0 = resource.getrusage(resource.RUSAGE_CHILDREN)
    t0 = time.perf_counter()
    r = subprocess.run([sys.executable, "-c", code], capture_output=True, text=True, cwd=ROOT,
                       timeout=3600)
    wall = time.perf_counter() - t0
    r1 = resource.getrusage(resource.RUSAGE_CHILDREN)
    if r.returncode != 0:
        raise RuntimeError("oracle run failed: " + r.stderr[-2000:])
    out = json.loads(r.stdout.strip().splitlines()[-1])
    cpu = (r1.ru_utime - r0.ru_utime) + (r1.ru_stime - r0.ru_stime)
    out["busy_cores"] = round(cpu / max(wall, 1e-9), 2)
    out["per_iter_s"] = sum(out["seconds"]) / len(out["seconds"])
    return out


def cpu_baseline(warmup: int, steps: int) -> dict:
    """Bounded sample for the GPU arm's line: the oracle's iterations
    warmup+1 .. warmup+steps at 24 x 12 x 12, their time scaled linearly by
    the DOF count to 5.4M DOFs.  The oracle's cost per iteration grows at
    least linearly with the DOFs (its MGCG iteration counts grow with the
    grid), so the value is an upper bound on its rate at the workload's size;
    the reference arm measures the growth exponent."""
    w = oracle_window("24x12x12", warmup, steps)
    scale = FULL_DOFS / w["dofs"]
    per_iter = w["per_iter_s"] * scale
    return {"value": round(1.0 / per_iter, 6), "unit": UNIT, "cores": _cores(),
            "busy_cores": w["busy_cores"], "kind": "oracle", "extrapolated": True,
            "sample": (f"oracle (numpy/scipy float64) design iterations {w['iterations']} of the "
                       f"workload's settings at 24x12x12 ({w['dofs']} DOFs, 3 levels, same 6x3x3 "
                       f"coarsest grid), {sum(w['seconds']):.1f} s measured, "
                       f"{w['per_iter_s']:.3f} s per iteration, scaled linearly by the DOF ratio "
                       f"{scale:.0f} (an upper bound on the oracle's rate at 5.4M DOFs)"),
            "branches": w["branches"], "measured_s_per_iter": round(w["per_iter_s"], 4)}


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


def _timed_run(p, W, K, ws, barrier, profile=True, clocks=None, autotune=True,
               tensor_cores=False):
    """W untimed and K timed design iterations of one job; the compliance of
    every timed iteration is copied on the device (no host read inside the
    timed region) and read afterwards."""
    import torch
    from paper_2205_00385_gb300 import binding as B
    from paper_2205_00385_gb300.driver import TopoSolver
    s = TopoSolver(p, autotune=autotune, tensor_cores=tensor_cores)
    for _ in range(W):
        s.step(read_compliance=False)
    if profile:
        # timed kinds: the float32 finest-grid operator (K p of every CG
        # iteration, the kernel the roofline is taken on), whole V-cycles and
        # the other finest-grid variants; nothing inside the V-cycle graph
        B.to_profile_enable(s.ctx, (1 << B.PK_FINE32) | (1 << B.PK_VCYCLE) |
                            (1 << B.PK_FINE_OTHER))
        for kind in (B.PK_FINE32, B.PK_COARSE, B.PK_VCYCLE, B.PK_FINE_OTHER):
            B.to_profile_read(s.ctx, kind)
    B.to_launch_count(s.ctx, reset=True)
    comp = torch.zeros(K, dtype=torch.float64, device=s.device)
    barrier()
    if clocks:
        clocks.start()
    ev0 = torch.cuda.Event(enable_timing=True)
    ev1 = torch.cuda.Event(enable_timing=True)
    ev0.record(s.stream)
    t0 = time.perf_counter()
    logs = []
    for i in range(K):
        logs.append(s.step(read_compliance=False))
        with torch.cuda.stream(s.stream):
            comp[i].copy_(s.scalars[0])
    ev1.record(s.stream)
    barrier()
    wall = time.perf_counter() - t0
    clk = clocks.stop() if clocks else None
    out = {"dev_s": ev0.elapsed_time(ev1) / 1e3, "wall_s": wall, "clocks": clk, "logs": logs,
           "tuning": s.tuning,
           "launches": B.to_launch_count(s.ctx),
           "compliance": comp.cpu().numpy().tolist()}
    if profile:
        out["prof"] = {k: B.to_profile_read(s.ctx, k)
                       for k in (B.PK_FINE32, B.PK_VCYCLE, B.PK_FINE_OTHER)}
    s.close()
    del s
    torch.cuda.empty_cache()
    return out


def _carm_summary(logs):
    """Time and outcome of the timed iterations' CARM attempts (build of the
    basis, reduced solve and eps), and the MGCG solves around them."""
    att = [h for h in logs if h.branch in ("carm", "mgcg-fallback")]
    mg = [h for h in logs if h.branch == "mgcg"]
    fb = [h for h in logs if h.branch == "mgcg-fallback"]
    if not att:
        return None
    return {"attempts": len(att), "accepted": sum(h.branch == "carm" for h in att),
            "timing_note": "host wall time of each solve, between stream synchronisations",
            "mean_build_and_solve_ms": round(1e3 * sum(h.carm_seconds for h in att) / len(att), 3),
            "eps_min": float(min(h.eps for h in att)), "eps_max": float(max(h.eps for h in att)),
            "mean_mgcg_solve_ms": (round(1e3 * sum(h.solve_seconds for h in mg) / len(mg), 3)
                                   if mg else None),
            "mean_fallback_solve_ms": (round(1e3 * sum(h.solve_seconds for h in fb) / len(fb), 3)
                                       if fb else None)}


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
    r = _timed_run(p, W, K, ws, barrier, clocks=ClockSampler(local), autotune=not args.no_autotune,
                   tensor_cores=args.tensor_cores)
    logs = r["logs"]
    branches = [h.branch for h in logs]
    cg = sum(h.cg_iters for h in logs)
    elapsed = slowest_rank(max(r["dev_s"], 1e-9), ws)
    value = whole_job_rate(K, ws, elapsed)
    n_f, ms_f, by_f = r["prof"][B.PK_FINE32]
    n_v, ms_v, by_v = r["prof"][B.PK_VCYCLE]
    n_o, ms_o, by_o = r["prof"][B.PK_FINE_OTHER]
    kname = ("k_apply3_tc<EPI_APPLY> (finest-grid K p, float32 storage, tcgen05 TF32x3 MMAs)"
             if args.tensor_cores else
             "k_apply3_pair<EPI_APPLY> (finest-grid K p, float32, two element columns per thread)")
    if n_f == 0:   # float64 path: the finest-grid operator runs in float64
        n_f, ms_f, by_f = n_o, ms_o, by_o
        kname = "k_apply3_col<double> (finest-grid K p, float64)"

    # ---- the same workload in plain float64 (the comparison the target names) ----
    fp64 = None
    if p.precision == "mixed" and not args.no_fp64_arm:
        r64 = _timed_run(p.with_(precision="fp64"), W, K, ws, barrier, profile=False,
                         autotune=not args.no_autotune)
        e64 = slowest_rank(max(r64["dev_s"], 1e-9), ws)
        c32, c64 = np.array(r["compliance"]), np.array(r64["compliance"])
        b64 = [h.branch for h in r64["logs"]]
        fp64 = {"value": round(whole_job_rate(K, ws, e64), 4), "unit": UNIT,
                "ms_per_step": round(e64 / K * 1e3, 3),
                "branches": {b: b64.count(b) for b in set(b64)},
                "cg_iterations": sum(h.cg_iters for h in r64["logs"]),
                "mixed_speedup": round(value / whole_job_rate(K, ws, e64), 3),
                "compliance_rel_diff_max": float(np.max(np.abs(c32 - c64) / np.abs(c64))),
                "note": ("each precision runs its own trajectory from the same initial design; "
                         "the difference is taken per timed iteration")}

    # ---- the same workload with MGCG only (Algorithm 1 without the reanalysis) ----
    mgcg_only = None
    if not args.no_mgcg_arm:
        rm = _timed_run(p.with_(n_on=10 ** 9), W, K, ws, barrier, profile=False,
                        autotune=not args.no_autotune, tensor_cores=args.tensor_cores)
        em = slowest_rank(max(rm["dev_s"], 1e-9), ws)
        cm = np.array(rm["compliance"])
        mgcg_only = {"value": round(whole_job_rate(K, ws, em), 4), "unit": UNIT,
                     "ms_per_step": round(em / K * 1e3, 3),
                     "cg_iterations": sum(h.cg_iters for h in rm["logs"]),
                     "aarmr_over_mgcg": round(value / whole_job_rate(K, ws, em), 4),
                     "final_compliance": float(cm[-1]),
                     "final_compliance_rel_diff": float(abs(r["compliance"][-1] - cm[-1]) /
                                                        abs(cm[-1]))}

    # ---- end to end through the C ABI with host buffers ----
    e2e = None
    if not args.no_e2e:
        s = TopoSolver(p, autotune=not args.no_autotune)
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
        e2e = {"value": round(whole_job_rate(K, ws, e2e_s), 4), "unit": UNIT,
               "h2d_bytes_per_step": p.nel * 8, "d2h_bytes_per_step": p.nel * 8 + 16}

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
    v_avg_ms = ms_v / max(n_v, 1)
    v_achieved = (by_v / max(n_v, 1)) / (v_avg_ms / 1e3) / 1e9 if n_v else 0.0
    roofline = {"bound": "hbm", "kernel": kname,
                "achieved": round(achieved, 1), "peak": hbm_peak, "unit": "GB/s",
                "frac": round(achieved / hbm_peak, 4), "peak_source": peak_src,
                "traffic": None,
                "traffic_note": ("not captured in this run; the ncu DRAM bytes of this kernel are "
                                 "summarised under profiles/"),
                "launches": n_f, "avg_launch_us": round(avg_ms * 1e3, 2),
                "algorithmic_bytes_per_launch": round(by_f / max(n_f, 1)),
                "algorithmic_bytes_rule": "x and y 12 B each per node (float32), E 4 B per element",
                "share_of_step": round(ms_f / 1e3 / elapsed * ws, 4),
                "vcycle": {"bound": "hbm", "launches": n_v, "avg_us": round(v_avg_ms * 1e3, 2),
                           "algorithmic_bytes": round(by_v / max(n_v, 1)),
                           "achieved": round(v_achieved, 1), "frac": round(v_achieved / hbm_peak, 4),
                           "graph": True,
                           "rule": ("each array each V-cycle kernel touches, once: operator x, y, "
                                    "moduli or assembled stencil, right-hand side, inverse "
                                    "diagonal; transfer inputs and outputs; coarsest inverse")},
                "other_fine_apply": {"launches": n_o, "ms": round(ms_o, 3)}}
    if p.dim == 3 and n_f:
        # the same kernel against the FP32 pipe, which ncu shows it is bound by
        # (issue and FMA pipe about half busy, DRAM below a tenth)
        nodes = (p.nelx + 1) * (p.nely + 1) * (p.nelz + 1)
        flops = 234 * p.nel + 21 * nodes
        alu_peak = 152 * 128 * 2 * 2.07e9 / 1e12
        alu_ach = flops / (avg_ms / 1e3) / 1e12
        roofline["alu"] = {
            "bound": "alu", "pipe": "fp32", "achieved": round(alu_ach, 2), "peak": alu_peak,
            "unit": "TFLOP/s", "frac": round(alu_ach / alu_peak, 4),
            "flops_per_launch": flops,
            "flops_rule": ("234 per element (the 8-point Walsh transform of the three components "
                           "both ways, 2 x 72 adds; E scaling, 24; the 45 non-zero Walsh-block "
                           "entries, 24 multiplies + 21 FMAs) + 21 per node (the sums of eight "
                           "element contributions)"),
            "peak_rule": "152 SMs x 128 FP32 lanes x 2 FLOP per FMA x 2.07 GHz (maximum SM clock)"}
    line = {
        "metric": METRIC, "value": round(value, 4), "unit": UNIT, "n_gpus": ws, "steps": K,
        "warmup": W, "ms_per_step": round(elapsed / K * 1e3, 3), "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32+df64" if p.precision == "mixed"
        else "f64", "data": "synthetic",
        "config": {"workload": _workload(p.precision) if not args.small else "cantilever 48x24x24 (quick)",
                   "precision": p.precision, "iterations_timed": f"{W + 1}..{W + K}",
                   "branches": {b: branches.count(b) for b in set(branches)},
                   "cg_iterations": cg, "mgcg_not_converged": sum(not h.converged for h in logs),
                   "final_compliance": r["compliance"][-1],
                   "l2": "inputs larger than L2 (43.6 MB per float64 vector; >2 GB state)",
                   "parallelism": f"replicas x{ws}"},
        "roofline": roofline, "fp64_arm": fp64, "mgcg_only_arm": mgcg_only,
        "carm_attempts": _carm_summary(logs),
        "mgcg_us_per_cg_iteration": round(
            1e6 * sum(h.solve_seconds - h.carm_seconds for h in logs) / max(cg, 1), 1),
        "e2e": e2e, "gpu_launches": int(r["launches"]),
        "autotune": ([{k: (round(v, 2) if isinstance(v, float) else v) for k, v in q.items()}
                      for q in r["tuning"]] if r["tuning"] else None),
        "clocks": r["clocks"], "wall_s": round(r["wall_s"], 3),
    }
    if args.serve_jobs > 0 and ws == 1:
        from paper_2205_00385_gb300.serve import Server
        from workloads import served_job_stream
        jobs = served_job_stream()[:args.serve_jobs]
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
            line["cpu_baseline"] = cpu_baseline(W, K)
        except Exception as ex:  # keep the GPU line even if the host baseline fails
            line["cpu_baseline"] = {"error": str(ex)[:300]}
    return line


def extrapolate_time(small: dict, large: dict, dofs: int):
    """Time per iteration at `dofs` from two measured windows, assuming
    time ~ DOFs^alpha with alpha fitted between them (at least 1: the cost
    per iteration never grows more slowly than the DOF count)."""
    import math
    alpha = math.log(large["per_iter_s"] / small["per_iter_s"]) / math.log(
        large["dofs"] / small["dofs"])
    alpha = max(alpha, 1.0)
    return alpha, large["per_iter_s"] * (dofs / large["dofs"]) ** alpha


def run_reference(args):
    """The reference arm: the oracle, as it stands, on the host cores.  It
    runs the workload's settings at 24 x 12 x 12 and 48 x 24 x 24 (both with
    the workload's 6 x 3 x 3 coarsest grid) for warmup + steps iterations,
    times the last `steps` (the iterations the GPU arm times), fits the
    growth of the time per iteration with the DOF count between the two and
    reports the rate extrapolated to 5.4M DOFs.  ms_per_step is the measured
    time per iteration at 48 x 24 x 24 (what this run spent per step)."""
    ws, rank, _ = _dist()
    if rank != 0:
        return None
    W, K = args.warmup, args.steps
    a = oracle_window("24x12x12", W, K)
    b = oracle_window("48x24x24", W, K)
    alpha, per_iter_full = extrapolate_time(a, b, FULL_DOFS)
    v = 1.0 / per_iter_full
    sample = (f"oracle (numpy/scipy float64) design iterations {b['iterations']} of the workload's "
              f"settings at 48x24x24 ({b['dofs']} DOFs, 4 levels): {b['per_iter_s']:.3f} s per "
              f"iteration; at 24x12x12 ({a['dofs']} DOFs, 3 levels): {a['per_iter_s']:.3f} s; "
              f"time per iteration ~ DOFs^{alpha:.3f} fitted between the two and extrapolated "
              f"to 5,447,811 DOFs: {per_iter_full:.1f} s per iteration")
    cpu = {"value": round(v, 6), "unit": UNIT, "cores": _cores(), "busy_cores": b["busy_cores"],
           "kind": "oracle", "sample": sample, "extrapolated": True,
           "measured": {"48x24x24": {"s_per_iter": round(b["per_iter_s"], 4),
                                      "branches": b["branches"]},
                        "24x12x12": {"s_per_iter": round(a["per_iter_s"], 4),
                                      "branches": a["branches"]}},
           "dof_exponent": round(alpha, 4)}
    return {"impl": "reference", "metric": METRIC, "value": round(v, 6), "unit": UNIT,
            "n_gpus": ws, "steps": K, "warmup": W,
            "ms_per_step": round(b["per_iter_s"] * 1e3, 1),
            "ms_per_step_note": ("measured at 48x24x24; value is the rate extrapolated to "
                                 "5.4M DOFs (see cpu_baseline.sample)"),
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
    s = TopoSolver(p, tensor_cores=args.tensor_cores)
    rho = torch.full((p.nel,), p.volfrac, dtype=torch.float64, device="cuda")
    B.to_set_density(s.ctx, rho)
    x = torch.from_numpy(np.random.default_rng(1).standard_normal(p.ndof)).cuda()
    y = torch.empty_like(x)
    prec = B.TO_PREC_FP32 if args.kernel_prec == "fp32" else B.TO_PREC_FP64
    for _ in range(args.warmup):
        B.to_apply(s.ctx, B.TO_OP_K, prec, x, y)
    # the float32 finest-grid operator is profiled as its own kind, the
    # other finest-grid precisions together
    kind = B.PK_FINE32 if args.kernel_prec == "fp32" else B.PK_FINE_OTHER
    B.to_profile_enable(s.ctx, 1 << kind)
    B.to_profile_read(s.ctx, kind)
    for _ in range(args.steps):
        B.to_apply(s.ctx, B.TO_OP_K, prec, x, y)
    n, ms, by = B.to_profile_read(s.ctx, kind)
    s.close()
    return {"kernel": ("k_apply3_tc" if args.tensor_cores else "k_apply3_pair")
            if args.kernel_prec == "fp32" else "k_apply3_col<double>",
            "precision": args.kernel_prec,
            "launches": n,
            "avg_us": ms / n * 1e3, "GB/s": by / (ms / 1e3) / 1e9,
            "bytes_per_launch": by / n, "workload": p.name + f" {p.nelx}x{p.nely}x{p.nelz}"}


def run_kernel_vcycle(args):
    """Times the V-cycle (to_vcycle, uncaptured, with its float64 <-> float32
    conversions) on the bench workload at a uniform design, for profiling:
    W untimed, K timed calls; --fused-coarse selects the one-launch coarse
    end."""
    import numpy as np
    import torch
    from paper_2205_00385_gb300 import binding as B
    from paper_2205_00385_gb300.driver import TopoSolver
    p = _problem(args)
    s = TopoSolver(p)
    rho = torch.full((p.nel,), p.volfrac, dtype=torch.float64, device="cuda")
    B.to_set_density(s.ctx, rho)
    if args.fused_coarse:
        B.to_operator_options(s.ctx, B.TO_OPERATOR_FUSED_COARSE)
    r = torch.from_numpy(np.random.default_rng(1).standard_normal(p.ndof)).cuda()
    z = torch.empty_like(r)
    for _ in range(args.warmup):
        B.to_vcycle(s.ctx, r, z)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(args.steps):
        B.to_vcycle(s.ctx, r, z)
    e1.record()
    torch.cuda.synchronize()
    s.close()
    return {"kernel": "to_vcycle", "fused_coarse": bool(args.fused_coarse),
            "calls": args.steps, "avg_us": 1e3 * e0.elapsed_time(e1) / args.steps,
            "workload": p.name + f" {p.nelx}x{p.nely}x{p.nelz}"}


def main():
    args = _args()
    if args.kernel == "apply":
        print(json.dumps(run_kernel_apply(args)), flush=True)
        return
    if args.kernel == "vcycle":
        print(json.dumps(run_kernel_vcycle(args)), flush=True)
        return
    line = run_reference(args) if args.impl == "reference" else run_ours(args)
    if line is not None:
        print(json.dumps(line), flush=True)


if __name__ == "__main__":
    main()

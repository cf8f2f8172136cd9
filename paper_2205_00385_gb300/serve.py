"""Serving many topology-optimisation jobs on one GPU.

A request stream (arrival time, problem) is replayed; jobs are admitted in
arrival order when a slot is free and their device memory (the library
workspace plus the job's own arrays) fits the HBM budget.  Every admitted
job keeps its multigrid hierarchy, PARM and CARM resident in its own
workspace.  A job leaves when its iterations are done and its memory
returns to the budget.

Two servers:

* BatchServer (continuous batching): the active jobs advance in rounds of
  one design iteration each (Fig. 1).  A round is one batched launch of all
  jobs' density phases (to_batch_step: one CUDA graph whose branches are the
  jobs), the jobs' solves (Algorithm 1: MGCG or CARM) concurrently, each on
  its own stream from a worker thread, and one batched launch of all jobs'
  update phases (compliance, sensitivity, filter, OC).  Arrivals join and
  finished jobs leave between rounds, so the GPU never waits for the whole
  batch to finish.  A job's per-iteration latency is the round's duration.
* StreamServer: every job runs its own loop on its own stream from its own
  host thread, with the single-job calls.

Both report throughput (design iterations per second over the whole
stream), per-iteration latency percentiles (p50/p99) and job latency from
arrival to completion.  Each job computes bitwise the same in either server
as alone (same kernels, same per-job order).
"""

from __future__ import annotations

import argparse
import json
import threading
import time
from collections import deque
from dataclasses import dataclass, field
from typing import Dict, List, Optional

import numpy as np

from . import binding as B


def job_device_bytes(prob) -> int:
    """Device bytes a job holds: the library workspace plus the driver's
    arrays (design, physical density, sensitivities: 5 x nel float64; the
    displacement and load copies: 2 x n float64; masks)."""
    desc = B.make_desc(prob.dim, (prob.nelx, prob.nely, prob.nelz), prob.E0, prob.Emin, prob.nu,
                       prob.penal, prob.rmin, prob.mg_levels,
                       B.TO_MIXED if prob.precision == "mixed" else B.TO_FP64, prob.n_parm,
                       prob.n_carm)
    ws = B.to_workspace_bytes(desc)
    return int(ws + 512 + 8 * (6 * prob.nel + 2 * prob.ndof) + prob.ndof)


class AdmissionController:
    """FIFO admission by slots and device-memory budget (host logic only)."""

    def __init__(self, budget_bytes: int, max_active: int):
        self.budget = int(budget_bytes)
        self.max_active = int(max_active)
        self.used = 0
        self.active = 0
        self.peak_used = 0
        self.peak_active = 0
        self.cv = threading.Condition()

    def fits_alone(self, need: int) -> bool:
        return need <= self.budget

    def can_admit(self, need: int) -> bool:
        return self.active < self.max_active and self.used + need <= self.budget

    def admit(self, need: int, timeout: Optional[float] = None) -> bool:
        """Block until the job fits, then reserve it.  False on timeout."""
        with self.cv:
            ok = self.cv.wait_for(lambda: self.can_admit(need), timeout=timeout)
            if not ok:
                return False
            self.used += need
            self.active += 1
            self.peak_used = max(self.peak_used, self.used)
            self.peak_active = max(self.peak_active, self.active)
            return True

    def release(self, need: int) -> None:
        with self.cv:
            self.used -= need
            self.active -= 1
            self.cv.notify_all()


@dataclass
class JobRecord:
    job_id: int
    arrival_s: float
    need_bytes: int
    admit_s: float = 0.0
    finish_s: float = 0.0
    iter_latency_s: List[float] = field(default_factory=list)
    compliance: List[float] = field(default_factory=list)
    branches: List[str] = field(default_factory=list)
    rho: Optional[np.ndarray] = None
    error: Optional[str] = None


def run_job_on_stream(prob, n_iter: int, keep_rho: bool = False, record: Optional[JobRecord] = None,
                      t0: float = 0.0):
    """Runs one job to completion on a fresh stream of the current device."""
    import torch
    from .driver import TopoSolver
    stream = torch.cuda.Stream()
    rec = record or JobRecord(-1, 0.0, 0)
    solver = TopoSolver(prob, stream=stream)
    try:
        for _ in range(n_iter):
            a = time.perf_counter()
            log = solver.step(read_compliance=True)
            rec.iter_latency_s.append(time.perf_counter() - a)
            rec.compliance.append(log.compliance)
            rec.branches.append(log.branch)
        if keep_rho:
            with torch.cuda.stream(stream):
                rec.rho = solver.rho.cpu().numpy()
    finally:
        solver.close()
        stream.synchronize()
    rec.finish_s = time.perf_counter() - t0
    return rec


class StreamServer:
    def __init__(self, budget_bytes: int, max_active: int = 8, keep_rho: bool = False):
        self.ctrl = AdmissionController(budget_bytes, max_active)
        self.keep_rho = keep_rho

    def run(self, jobs, n_iter: Optional[int] = None, time_scale: float = 1.0) -> Dict:
        """Replays ``jobs`` (workloads.Job list, arrival-sorted); arrival
        times are multiplied by ``time_scale``."""
        import torch
        device = torch.cuda.current_device()
        records: List[JobRecord] = []
        threads: List[threading.Thread] = []
        t0 = time.perf_counter()
        for job in sorted(jobs, key=lambda j: j.arrival_s):
            need = job_device_bytes(job.problem)
            rec = JobRecord(job.job_id, job.arrival_s * time_scale, need)
            records.append(rec)
            if not self.ctrl.fits_alone(need):
                rec.error = "larger than the HBM budget"
                continue
            wait = rec.arrival_s - (time.perf_counter() - t0)
            if wait > 0:
                time.sleep(wait)
            self.ctrl.admit(need)
            rec.admit_s = time.perf_counter() - t0
            iters = n_iter if n_iter is not None else job.problem.n_iter

            def work(prob=job.problem, rec=rec, iters=iters, need=need):
                torch.cuda.set_device(device)
                try:
                    run_job_on_stream(prob, iters, self.keep_rho, rec, t0)
                except Exception as ex:  # recorded, the stream keeps going
                    rec.error = repr(ex)
                    rec.finish_s = time.perf_counter() - t0
                finally:
                    self.ctrl.release(need)

            th = threading.Thread(target=work, daemon=True)
            th.start()
            threads.append(th)
        for th in threads:
            th.join()
        wall = time.perf_counter() - t0
        return self.report(records, wall)

    def report(self, records: List[JobRecord], wall: float) -> Dict:
        lat = np.array([x for r in records for x in r.iter_latency_s]) * 1e3
        done = [r for r in records if r.error is None]
        job_lat = np.array([r.finish_s - r.arrival_s for r in done])
        n_it = int(lat.size)
        return {
            "jobs": len(records), "jobs_done": len(done),
            "jobs_failed": [(r.job_id, r.error) for r in records if r.error],
            "iterations": n_it, "wall_s": wall,
            "throughput_iters_per_s": n_it / wall if wall > 0 else 0.0,
            "iter_latency_ms": {"p50": float(np.percentile(lat, 50)) if n_it else None,
                                "p99": float(np.percentile(lat, 99)) if n_it else None,
                                "mean": float(lat.mean()) if n_it else None},
            "job_latency_s": {"p50": float(np.percentile(job_lat, 50)) if job_lat.size else None,
                              "p99": float(np.percentile(job_lat, 99)) if job_lat.size else None},
            "peak_active_jobs": self.ctrl.peak_active,
            "peak_admitted_gb": self.ctrl.peak_used / 2 ** 30,
            "budget_gb": self.ctrl.budget / 2 ** 30,
        }


@dataclass
class _Active:
    job_id: int
    solver: object
    record: JobRecord
    need: int
    left: int


class BatchServer:
    """Continuous batching: rounds of one design iteration per active job,
    the density and update phases of all jobs as one graph launch each."""

    def __init__(self, budget_bytes: int, max_active: int = 16, keep_rho: bool = False,
                 precision: Optional[str] = None, autotune: bool = True):
        self.ctrl = AdmissionController(budget_bytes, max_active)
        self.keep_rho = keep_rho
        self.precision = precision
        self.autotune = autotune
        self.rounds = 0
        self.batched_jobs = 0     # sum over rounds of the jobs in the round

    def _admit(self, job, need, t0, iters):
        from .driver import TopoSolver
        import torch
        rec = JobRecord(job.job_id, 0.0, need)
        stream = torch.cuda.Stream()
        prob = job.problem if self.precision is None else job.problem.with_(precision=self.precision)
        solver = TopoSolver(prob, stream=stream, autotune=self.autotune)
        rec.admit_s = time.perf_counter() - t0
        return _Active(job.job_id, solver, rec, need, iters)

    def run(self, jobs, n_iter: Optional[int] = None, time_scale: float = 1.0) -> Dict:
        import concurrent.futures as cf
        import torch
        device = torch.cuda.current_device()
        server_stream = torch.cuda.Stream()
        sh = server_stream.cuda_stream
        pending = deque(sorted(jobs, key=lambda j: j.arrival_s))
        records: Dict[int, JobRecord] = {}
        active: List[_Active] = []
        t0 = time.perf_counter()
        pool = cf.ThreadPoolExecutor(max_workers=max(1, self.ctrl.max_active))

        def solve(a: _Active):
            torch.cuda.set_device(device)
            return a.solver.solve_phase()

        while pending or active:
            now = time.perf_counter() - t0
            while pending and pending[0].arrival_s * time_scale <= now:
                job = pending[0]
                need = job_device_bytes(job.problem)
                if not self.ctrl.fits_alone(need):
                    pending.popleft()
                    rec = JobRecord(job.job_id, job.arrival_s * time_scale, need)
                    rec.error = "larger than the HBM budget"
                    records[job.job_id] = rec
                    continue
                if not self.ctrl.can_admit(need):
                    break
                pending.popleft()
                self.ctrl.admit(need)
                iters = n_iter if n_iter is not None else job.problem.n_iter
                a = self._admit(job, need, t0, iters)
                a.record.arrival_s = job.arrival_s * time_scale
                records[job.job_id] = a.record
                active.append(a)
            if not active:
                if pending:
                    time.sleep(max(0.0, pending[0].arrival_s * time_scale -
                                   (time.perf_counter() - t0)))
                continue
            r0 = time.perf_counter()
            # the density phase of every job, ordered after each job's own work
            for a in active:
                server_stream.wait_stream(a.solver.stream)
            table = [a.solver.batch_job() for a in active]
            B.to_batch_step(table, B.TO_PHASE_DENSITY, sh)
            for a in active:
                a.solver.stream.wait_stream(server_stream)
            # the solves, concurrently on the jobs' own streams
            outs = list(pool.map(solve, active))
            for a in active:
                server_stream.wait_stream(a.solver.stream)
            table = [a.solver.batch_job() for a in active]   # this iteration's volume fraction
            B.to_batch_step(table, B.TO_PHASE_UPDATE, sh)
            with torch.cuda.stream(server_stream):
                vals = torch.stack([a.solver.scalars[:2] for a in active]).cpu().numpy()
            dt = time.perf_counter() - r0
            self.rounds += 1
            self.batched_jobs += len(active)
            still = []
            for a, out, v in zip(active, outs, vals):
                rec = a.record
                rec.iter_latency_s.append(dt)
                rec.compliance.append(float(v[0]))
                rec.branches.append(out[0])
                a.left -= 1
                if a.left > 0:
                    still.append(a)
                    continue
                if self.keep_rho:
                    with torch.cuda.stream(server_stream):
                        rec.rho = a.solver.rho.cpu().numpy()
                server_stream.synchronize()
                a.solver.close()
                rec.finish_s = time.perf_counter() - t0
                self.ctrl.release(a.need)
            active = still
        pool.shutdown()
        wall = time.perf_counter() - t0
        recs = [records[k] for k in sorted(records)]
        rep = StreamServer.report(self, recs, wall)
        rep["rounds"] = self.rounds
        rep["mean_jobs_per_round"] = self.batched_jobs / max(self.rounds, 1)
        rep["_records"] = recs
        return rep


# the default server
Server = BatchServer


def main():
    import torch
    from workloads import served_job_stream
    ap = argparse.ArgumentParser(description="Replay the served stream of optimisation jobs")
    ap.add_argument("--jobs", type=int, default=256)
    ap.add_argument("--iters", type=int, default=30)
    ap.add_argument("--time-scale", type=float, default=1.0)
    ap.add_argument("--budget-gb", type=float, default=200.0)
    ap.add_argument("--max-active", type=int, default=16)
    ap.add_argument("--precision", default="workload", choices=["workload", "mixed", "fp64"])
    a = ap.parse_args()
    torch.cuda.set_device(0)
    jobs = served_job_stream()[:a.jobs]
    ap2 = a
    srv = BatchServer(int(ap2.budget_gb * 2 ** 30), ap2.max_active,
                      precision=None if ap2.precision == "workload" else ap2.precision)
    rep = srv.run(jobs, ap2.iters, ap2.time_scale)
    rep.pop("_records", None)
    print(json.dumps(rep))


if __name__ == "__main__":
    main()

"""Serving: admission control (host logic, CPU) and the alone-versus-mix
property on the GPU -- every job's result is the same when it runs alone
and when it runs concurrently with others, both in the continuous-batching
server (the density and update phases of all active jobs as one graph
launch each, the solves concurrently) and in the per-job-stream server.
Each job has its own context, workspace and stream, its kernels run in the
same order either way, and every reduction uses a fixed grid and order, so
the results must agree bit for bit.  The jobs reach the CARM phase of
Algorithm 1 (N_on = 3) within their six iterations."""

import threading
import time

import numpy as np
import pytest

from workloads import Job, small_problem


def _ctrl(budget, slots):
    from paper_2205_00385_gb300.serve import AdmissionController
    return AdmissionController(budget, slots)


def test_admission_respects_slots_and_budget():
    c = _ctrl(100, 2)
    assert c.admit(60, timeout=0.01)
    assert not c.admit(50, timeout=0.01)        # budget: 60 + 50 > 100
    assert c.admit(40, timeout=0.01)            # fits exactly
    assert not c.admit(1, timeout=0.01)         # no slot left
    c.release(60)
    assert c.admit(10, timeout=0.01)
    assert c.peak_active == 2 and c.peak_used == 100
    assert not c.fits_alone(101)


def test_admission_blocks_until_release():
    c = _ctrl(10, 4)
    assert c.admit(8, timeout=0.01)
    got = []

    def waiter():
        got.append(c.admit(5, timeout=5.0))

    th = threading.Thread(target=waiter)
    th.start()
    time.sleep(0.05)
    assert got == []                            # still waiting
    c.release(8)
    th.join(timeout=5.0)
    assert got == [True] and c.used == 5


def _jobs():
    specs = [("cantilever3d", dict(nelx=16, nely=8, nelz=8, mg_levels=3)),
             ("bridge3d", dict(nelx=16, nely=8, nelz=8, mg_levels=3, noise=0.05)),
             ("cantilever3d", dict(nelx=24, nely=12, nelz=12, mg_levels=3, volfrac=0.2)),
             ("bridge3d", dict(nelx=8, nely=4, nelz=4, mg_levels=3))]
    jobs = []
    for q, (kind, kw) in enumerate(specs):
        p = small_problem(kind, n_iter=6, n_on=3, n_parm=2, n_carm=3, eps_tol=0.5,
                          precision="mixed", **kw)
        jobs.append(Job(q, 0.01 * q, p))
    return jobs


def _alone(jobs):
    from paper_2205_00385_gb300.serve import JobRecord, run_job_on_stream
    alone = {}
    for j in jobs:
        alone[j.job_id] = run_job_on_stream(j.problem, j.problem.n_iter, keep_rho=True,
                                            record=JobRecord(j.job_id, 0.0, 0))
    return alone


@pytest.mark.gpu
def test_each_job_same_alone_and_in_the_batched_mix():
    import torch
    from paper_2205_00385_gb300.serve import BatchServer
    torch.cuda.set_device(0)
    jobs = _jobs()
    alone = _alone(jobs)
    assert any("carm" in r.branches or "mgcg-fallback" in r.branches for r in alone.values())
    server = BatchServer(budget_bytes=64 * 2 ** 30, max_active=4, keep_rho=True)
    rep = server.run(jobs, n_iter=6)
    records = {r.job_id: r for r in rep["_records"]}
    assert rep["jobs_done"] == len(jobs) and not rep["jobs_failed"]
    assert rep["peak_active_jobs"] >= 2 and rep["mean_jobs_per_round"] > 1.0   # shared launches
    assert rep["iter_latency_ms"]["p99"] >= rep["iter_latency_ms"]["p50"] > 0
    for j in jobs:
        a, m = alone[j.job_id], records[j.job_id]
        assert a.branches == m.branches
        assert a.compliance == m.compliance            # bitwise
        assert np.array_equal(a.rho, m.rho)


@pytest.mark.gpu
def test_each_job_same_alone_and_in_the_stream_mix():
    import torch
    from paper_2205_00385_gb300.serve import StreamServer
    torch.cuda.set_device(0)
    jobs = _jobs()
    alone = _alone(jobs)
    server = StreamServer(budget_bytes=64 * 2 ** 30, max_active=4, keep_rho=True)
    records = {}
    orig_report = server.report

    def capture(recs, wall):
        for r in recs:
            records[r.job_id] = r
        return orig_report(recs, wall)

    server.report = capture
    rep = server.run(jobs, n_iter=6)
    assert rep["jobs_done"] == len(jobs) and not rep["jobs_failed"]
    assert rep["peak_active_jobs"] >= 2            # they did overlap
    for j in jobs:
        a, m = alone[j.job_id], records[j.job_id]
        assert a.branches == m.branches
        assert a.compliance == m.compliance            # bitwise
        assert np.array_equal(a.rho, m.rho)


@pytest.mark.gpu
def test_tight_budget_serialises_jobs():
    import torch
    from paper_2205_00385_gb300.serve import BatchServer, job_device_bytes
    torch.cuda.set_device(0)
    jobs = _jobs()
    biggest = max(job_device_bytes(j.problem) for j in jobs)
    server = BatchServer(budget_bytes=biggest + 1024, max_active=4)
    rep = server.run(jobs, n_iter=2)
    assert rep["jobs_done"] == len(jobs)
    assert rep["peak_admitted_gb"] * 2 ** 30 <= biggest + 1024


@pytest.mark.gpu
def test_batch_step_rejects_bad_tables():
    """to_batch_step checks its table before launching anything."""
    import torch
    from paper_2205_00385_gb300 import binding as B
    from paper_2205_00385_gb300.driver import TopoSolver
    torch.cuda.set_device(0)
    s = TopoSolver(_jobs()[3].problem)
    try:
        j = s.batch_job()
        sh = torch.cuda.current_stream().cuda_stream
        for bad, phase in (([j, j], B.TO_PHASE_DENSITY),                      # same context twice
                           ([dict(j, rho_phys=None)], B.TO_PHASE_DENSITY),    # missing output
                           ([dict(j, volfrac=0.0)], B.TO_PHASE_UPDATE),       # bad OC parameter
                           ([j], 7)):                                           # bad phase
            with pytest.raises(B.TopoError) as e:
                B.to_batch_step(bad, phase, sh)
            assert e.value.status == B.TO_E_INVALID
        with pytest.raises(B.TopoError):
            B.to_batch_step([], B.TO_PHASE_DENSITY, sh)
    finally:
        s.close()

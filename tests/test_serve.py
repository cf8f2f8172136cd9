"""Serving: admission control (host logic, CPU) and the alone-versus-mix
property on the GPU -- every job's result is the same when it runs alone
and when it runs concurrently with others.  Each job has its own context,
workspace and stream, and every reduction uses a fixed grid and order, so
the results must agree bit for bit."""

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


@pytest.mark.gpu
def test_each_job_same_alone_and_in_the_mix():
    import torch
    from paper_2205_00385_gb300.serve import JobRecord, Server, run_job_on_stream
    torch.cuda.set_device(0)
    jobs = _jobs()
    alone = {}
    for j in jobs:
        rec = run_job_on_stream(j.problem, j.problem.n_iter, keep_rho=True,
                                record=JobRecord(j.job_id, 0.0, 0))
        alone[j.job_id] = rec
    server = Server(budget_bytes=64 * 2 ** 30, max_active=4, keep_rho=True)
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
    assert rep["iter_latency_ms"]["p99"] >= rep["iter_latency_ms"]["p50"] > 0
    for j in jobs:
        a, m = alone[j.job_id], records[j.job_id]
        assert a.branches == m.branches
        assert a.compliance == m.compliance            # bitwise
        assert np.array_equal(a.rho, m.rho)


@pytest.mark.gpu
def test_tight_budget_serialises_jobs():
    import torch
    from paper_2205_00385_gb300.serve import Server, job_device_bytes
    torch.cuda.set_device(0)
    jobs = _jobs()
    biggest = max(job_device_bytes(j.problem) for j in jobs)
    server = Server(budget_bytes=biggest + 1024, max_active=4)
    rep = server.run(jobs, n_iter=2)
    assert rep["jobs_done"] == len(jobs)
    assert rep["peak_admitted_gb"] * 2 ** 30 <= biggest + 1024

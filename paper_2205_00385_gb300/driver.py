"""Design loop of AARMR topology optimisation (Fig. 1, Algorithm 1) driven
through the C ABI.

The host decides which branch runs (MGCG or CARM) from scalars the device
returns (the CG residual, eps of Eq. 29); every arithmetic step runs in
libtopo.so kernels.  PyTorch only provides device memory and the stream.

Readings (shared with the oracle): MGCG for design iterations k <= N_on,
whose last N_s solutions fill the PARM; from k = N_on + 1 the CARM is
built from u_last and accepted when eps < eps_tol, otherwise MGCG is
warm-started from the reduced solution and its result pushed into the PARM.
"""

from __future__ import annotations

import time
from dataclasses import dataclass, field
from typing import List, Optional

import numpy as np

from . import binding as B


def _torch():
    import torch
    return torch


@dataclass
class IterLog:
    k: int
    branch: str
    compliance: float
    eps: Optional[float]
    cg_iters: int
    change: float
    seconds: float
    relres: Optional[float] = None   # final recursive-residual ratio of the MGCG solve
    converged: bool = True           # False when the MGCG solve stopped at maxit
    solve_seconds: float = 0.0       # wall time of the equilibrium solve (MGCG or CARM)
    carm_seconds: float = 0.0        # wall time of the CARM build and reduced solve, if tried


class TopoSolver:
    """One optimisation job resident on the GPU."""

    def __init__(self, prob, device="cuda", stream=None, precision: Optional[str] = None,
                 autotune: bool = False, tensor_cores: bool = False):
        torch = _torch()
        self.prob = prob
        self.device = torch.device(device)
        prec = (precision or prob.precision)
        self.precision = prec
        self.desc = B.make_desc(prob.dim, (prob.nelx, prob.nely, prob.nelz), prob.E0, prob.Emin,
                                prob.nu, prob.penal, prob.rmin, prob.mg_levels,
                                B.TO_MIXED if prec == "mixed" else B.TO_FP64, prob.n_parm,
                                prob.n_carm)
        self.ws_bytes = B.to_workspace_bytes(self.desc)
        raw = torch.empty(self.ws_bytes + 256, dtype=torch.uint8, device=self.device)
        off = (-raw.data_ptr()) % 256
        self._ws_raw = raw
        self.ws = raw[off:off + self.ws_bytes]
        self.stream = stream if stream is not None else torch.cuda.current_stream(self.device)
        f64 = dict(dtype=torch.float64, device=self.device)
        with torch.cuda.stream(self.stream):
            fixed = torch.from_numpy(prob.fixed.astype(np.uint8)).to(self.device)
            f = torch.from_numpy(prob.f.astype(np.float64)).to(self.device)
            self.ctx = B.to_mesh_init(self.desc, fixed, f, self.ws, self.stream.cuda_stream)
            self._keep = (fixed, f)
            nel, n = prob.nel, prob.ndof
            self.rho = torch.from_numpy(prob.rho0.astype(np.float64)).to(self.device)
            self.rho_phys = torch.empty(nel, **f64)
            self.dc = torch.empty(nel, **f64)
            self.dc_f = torch.empty(nel, **f64)
            self.dv_f = torch.empty(nel, **f64)
            self.u = torch.zeros(n, **f64)
            self.scalars = torch.zeros(4, **f64)       # compliance, change, eps, spare
            ones = torch.ones(nel, **f64)
            B.to_filter(self.ctx, B.TO_FILTER_SENS, ones, self.dv_f)
            if tensor_cores and prob.dim == 3 and prec == "mixed":
                B.to_operator_options(self.ctx, B.TO_OPERATOR_TENSOR_CORES)
            if getattr(prob, "carm_r1", "u_last") == "projected_load":
                B.to_carm_options(self.ctx, B.TO_CARM_R1_PROJECTED_LOAD)
            self.tuning = None
            if autotune:
                # launch shapes timed on this grid (cached per process by grid)
                B.to_filter(self.ctx, B.TO_FILTER_DENSITY, self.rho, self.rho_phys)
                B.to_set_density(self.ctx, self.rho_phys)
                self.tuning = B.to_autotune(self.ctx)
        self.k = 0
        self.history: List[IterLog] = []

    def close(self):
        if getattr(self, "ctx", None) is not None:
            B.to_destroy(self.ctx)
            self.ctx = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    # -- one design iteration -------------------------------------------------
    # Fig. 1: the density phase (filter, SIMP), the solve (Algorithm 1) and
    # the update phase (compliance, sensitivity, its filter, OC).  A serving
    # loop runs the two phases of many jobs as batched launches
    # (to_batch_step) and only the solves job by job; step() runs all three
    # for one job with the single-job calls.
    def density_phase(self):
        B.to_filter(self.ctx, B.TO_FILTER_DENSITY, self.rho, self.rho_phys)
        B.to_set_density(self.ctx, self.rho_phys)

    def solve_phase(self):
        """Algorithm 1 for the next design iteration k: MGCG while k <= N_on
        (its last N_s solutions fill the PARM), else the CARM, accepted when
        eps < eps_tol, otherwise MGCG warm-started from it and pushed into the
        PARM.  Returns (branch, eps, cg_iters, relres, converged)."""
        p = self.prob
        ctx = self.ctx
        self.k += 1
        k = self.k
        eps = None
        iters, rel, ok = 0, None, True
        self.last_carm_s = 0.0
        if k <= p.n_on or B.to_parm_count(ctx) < p.n_parm:
            flags = (B.TO_SOLVE_WARM_START if k > 1 else 0)
            if k > p.n_on - p.n_parm:
                flags |= B.TO_SOLVE_PUSH_PARM
            iters, rel, ok = B.to_mgcg_solve(ctx, p.rtol, p.maxit, flags, self.u)
            branch = "mgcg"
        else:
            tc = time.perf_counter()
            B.to_carm_build(ctx, self.u)
            eps = B.to_carm_solve(ctx, self.u, self.scalars[2:3])   # returns eps to the host
            self.last_carm_s = time.perf_counter() - tc
            if eps < p.eps_tol:
                branch = "carm"
            else:
                iters, rel, ok = B.to_mgcg_solve(ctx, p.rtol, p.maxit,
                                                 B.TO_SOLVE_WARM_START | B.TO_SOLVE_PUSH_PARM,
                                                 self.u)
                branch = "mgcg-fallback"
        return branch, eps, iters, rel, ok

    def update_phase(self):
        """Compliance, sensitivity, its filter and the OC update for the
        current design iteration (the volume fraction may follow a ramp)."""
        p = self.prob
        B.to_sensitivity(self.ctx, self.u, self.scalars[0:1], self.dc)
        B.to_filter(self.ctx, B.TO_FILTER_SENS, self.dc, self.dc_f)
        B.to_oc_update(self.ctx, p.volfrac_at(self.k), p.move, self.dc_f, self.dv_f, self.rho,
                       self.scalars[1:2])

    def batch_job(self):
        """This job's entry of a to_batch_step table (for the update phase of
        the current iteration k, after solve_phase)."""
        p = self.prob
        return dict(ctx=self.ctx, rho=self.rho, rho_phys=self.rho_phys, u=self.u, dc=self.dc,
                    dc_f=self.dc_f, dv_f=self.dv_f, compliance_dev=self.scalars[0:1],
                    change_dev=self.scalars[1:2], volfrac=p.volfrac_at(max(self.k, 1)),
                    move=p.move)

    def step(self, read_compliance: bool = True) -> IterLog:
        t0 = time.perf_counter()
        self.density_phase()
        # the solve's calls synchronise on their results (|r|, eps), so the
        # host wall time of solve_phase, after the density phase has
        # finished, is the solve's time
        self.stream.synchronize()
        ts = time.perf_counter()
        branch, eps, iters, rel, ok = self.solve_phase()
        self.stream.synchronize()
        t_solve = time.perf_counter() - ts
        self.update_phase()
        C = change = float("nan")
        if read_compliance:
            torch = _torch()
            with torch.cuda.stream(self.stream):
                vals = self.scalars[:2].cpu().numpy()
            C, change = float(vals[0]), float(vals[1])
        log = IterLog(self.k, branch, C, eps, iters, change, time.perf_counter() - t0, rel, ok,
                      t_solve, self.last_carm_s)
        self.history.append(log)
        return log

    def run(self, n_iter: Optional[int] = None) -> List[IterLog]:
        for _ in range(n_iter if n_iter is not None else self.prob.n_iter):
            self.step()
        return self.history


@dataclass
class MechLog:
    k: int
    objective: float                 # u_out of the state solution
    branches: tuple                  # (state, adjoint)
    eps: tuple
    cg_iters: tuple
    change: float
    seconds: float
    solve_seconds: float = 0.0       # wall time of both equilibrium solves


class MechanismSolver:
    """Compliant-mechanism job (Sec. 4.3, the displacement inverter): the
    state system (K + S) u = f_in and the adjoint system (K + S) lam = l
    (l the unit vector of the output DOF) as two contexts on the same mesh,
    springs and density, each running Algorithm 1 with its own PARM.  Per
    iteration: filter and SIMP on the state context (the adjoint context
    gets the same physical density), both solves, the output sensitivity
    from (u, lam), its filter and the damped OC update."""

    def __init__(self, prob, device="cuda", stream=None, precision: Optional[str] = None):
        torch = _torch()
        if prob.out_dof < 0 or not prob.springs:
            raise ValueError("a mechanism problem needs out_dof and springs")
        self.prob = prob
        l_vec = np.zeros(prob.ndof)
        l_vec[prob.out_dof] = 1.0
        self.state = TopoSolver(prob, device, stream, precision)
        self.adj = TopoSolver(prob.with_(f=l_vec), device, self.state.stream, precision)
        dofs = [d for d, _ in prob.springs]
        ks = [k for _, k in prob.springs]
        with torch.cuda.stream(self.state.stream):
            for s in (self.state, self.adj):
                B.to_mesh_springs(s.ctx, dofs, ks)
            B.to_oc_options(self.state.ctx, prob.oc_eta)
        self.k = 0
        self.history: List[MechLog] = []

    def close(self):
        self.state.close()
        self.adj.close()

    def step(self) -> MechLog:
        torch = _torch()
        p, st, ad = self.prob, self.state, self.adj
        t0 = time.perf_counter()
        with torch.cuda.stream(st.stream):
            st.density_phase()
            B.to_set_density(ad.ctx, st.rho_phys)
            st.stream.synchronize()
            ts = time.perf_counter()
            bu, eu, iu, _, _ = st.solve_phase()
            bl, el, il, _, _ = ad.solve_phase()
            st.stream.synchronize()
            t_solve = time.perf_counter() - ts
            self.k = st.k
            B.to_sensitivity_adjoint(st.ctx, st.u, ad.u, st.scalars[3:4], st.dc)
            B.to_filter(st.ctx, B.TO_FILTER_SENS, st.dc, st.dc_f)
            B.to_oc_update(st.ctx, p.volfrac_at(self.k), p.move, st.dc_f, st.dv_f, st.rho,
                           st.scalars[1:2])
            obj = float(st.u[p.out_dof].item())
            change = float(st.scalars[1].item())
        log = MechLog(self.k, obj, (bu, bl), (eu, el), (iu, il), change,
                      time.perf_counter() - t0, t_solve)
        self.history.append(log)
        return log

    def run(self, n_iter: Optional[int] = None) -> List[MechLog]:
        for _ in range(n_iter if n_iter is not None else self.prob.n_iter):
            self.step()
        return self.history


def run_job(prob, n_iter=None, device="cuda", precision=None):
    s = TopoSolver(prob, device=device, precision=precision)
    try:
        hist = s.run(n_iter)
        rho = s.rho.cpu().numpy()
    finally:
        s.close()
    return rho, hist

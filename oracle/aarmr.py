"""Topology optimisation with AARMR: Algorithm 1 inside the design loop of
Fig. 1 (Sec. 3).

Each design iteration k:
  rho~ = filter(rho) (Eq. 31), E = SIMP(rho~) (Eq. 1);
  if k <= N_on: u = MGCG(K, f) warm-started from u_last; the solutions of
     iterations N_on - N_s + 1 .. N_on build the PARM (Eq. 27-28);
  else: CARM from u_last, PARM and dK = K - K_ref (Eq. 26, 21), reduced
     solve (Eq. 23-25); accept if eps < eps_tol (Eq. 29), otherwise
     u = MGCG(K, f) warm-started from the reduced solution and pushed into
     the PARM (FIFO);
  C, dC/drho~ (Eq. 3, 6/34), filtered sensitivities (Eq. 33), OC update.

Variants the paper studies: the first CA basis vector Phi K_Phi^-1 Phi^T f
instead of u_last (Fig. 2; problem field carm_r1) and a volume fraction
lowered in the middle of the run (Fig. 3; problem field volfrac_ramp).

Readings: Algorithm 1's "loop < N_on" versus the text's "more than N_on"
are reconciled as MGCG for k <= N_on and CARM from k = N_on + 1; K_ref is
the stiffness of the previous design iteration (the text says the last
stiffness matrix is used to rebuild the CARM); r_1 = u_last is the accepted
solution of the previous iteration.  Whole trajectories are not pinned by
the paper's printed results (parity unpinned beyond the per-step pins).
"""

from __future__ import annotations

import time
from dataclasses import dataclass, field
from typing import Dict, List, Optional

import numpy as np

from . import fe, filters, oc, reanalysis, sensitivity, solvers


class OracleModel:
    """Fixed data of one problem: grid, KE, filter, BCs, load."""

    def __init__(self, prob):
        self.prob = prob
        self.grid = fe.Grid.of(prob)
        self.KE = fe.element_stiffness(prob.dim, prob.nu)
        self.fixed = prob.fixed.astype(np.uint8)
        self.f = prob.f.astype(float)
        self.H, self.Hs = filters.filter_matrix(self.grid, prob.rmin)
        self.dv_f = filters.sensitivity_filter(self.H, self.Hs, np.ones(self.grid.nel))

    def modulus(self, rho_phys):
        p = self.prob
        return sensitivity.simp_modulus(rho_phys, p.E0, p.Emin, p.penal)

    def K(self, E):
        return fe.stiffness(self.grid, E, self.KE, self.fixed)

    def dK(self, E, E_ref):
        """dK = K - K_ref with BCs: the identity rows cancel (Eq. 8)."""
        return fe.apply_bcs(fe.assemble(self.grid, E - E_ref, self.KE), self.fixed,
                            diag_fixed=0.0)

    def multigrid(self, K):
        return solvers.Multigrid(self.grid, K, self.fixed, self.prob.mg_levels)

    def mgcg(self, K, x0=None, rtol=None, maxit=None):
        p = self.prob
        mg = self.multigrid(K)
        return solvers.mgcg(K, self.f, mg, x0=x0, rtol=p.rtol if rtol is None else rtol,
                            maxit=p.maxit if maxit is None else maxit)

    def exact(self, K):
        return solvers.direct_solve(K, self.f, self.fixed)

    def sensitivities(self, u, rho_phys, E):
        p = self.prob
        ce = sensitivity.element_energy(self.grid, self.KE, u, self.fixed)
        C = sensitivity.compliance(E, ce)
        dc = sensitivity.compliance_sensitivity(rho_phys, ce, p.E0, p.Emin, p.penal)
        return C, dc


@dataclass
class IterRecord:
    k: int
    branch: str
    compliance: float
    eps: Optional[float]
    cg_iters: int
    change: float
    w_percent: float
    seconds: float = 0.0      # wall time of the iteration (timing only)


@dataclass
class Trajectory:
    rho: np.ndarray
    history: List[IterRecord] = field(default_factory=list)
    snapshots: Dict[int, dict] = field(default_factory=dict)


def run(prob, n_iter: Optional[int] = None, mode: str = "aarmr", snapshot_at=(),
        model: Optional[OracleModel] = None) -> Trajectory:
    """Run the design loop.  mode: "aarmr" (Algorithm 1), "mgcg" (MGCG every
    iteration, the paper's reference method) or "direct" (exact solves).

    ``snapshot_at`` lists iterations whose solve inputs are recorded
    (rho~, E, E_ref, u_last, Phi) for per-solve comparisons."""
    m = model or OracleModel(prob)
    p = prob
    n_iter = p.n_iter if n_iter is None else n_iter
    rho = p.rho0.astype(float).copy()
    parm = reanalysis.Parm(p.n_parm)
    u_last = np.zeros(m.grid.ndof)
    E_prev = None
    rho_phys_prev = None
    traj = Trajectory(rho)
    for k in range(1, n_iter + 1):
        t0 = time.perf_counter()
        rho_phys = filters.density_filter(m.H, m.Hs, rho)
        E = m.modulus(rho_phys)
        K = m.K(E)
        if k in snapshot_at:
            traj.snapshots[k] = dict(rho=rho.copy(), rho_phys=rho_phys.copy(), E=E.copy(),
                                     E_prev=None if E_prev is None else E_prev.copy(),
                                     rho_phys_prev=None if rho_phys_prev is None
                                     else rho_phys_prev.copy(),
                                     u_last=u_last.copy(),
                                     Phi=parm.matrix() if parm.cols else None)
        eps, iters = None, 0
        if mode == "direct":
            u, branch = m.exact(K), "direct"
        elif mode == "aarmr" and k > p.n_on and parm.full:
            K_ref = m.K(E_prev)
            dK = m.dK(E, E_prev)
            u, eps, _ = reanalysis.aarmr_solve(lambda v: K @ v, lambda v: K_ref @ v,
                                               lambda v: dK @ v, m.f, u_last, parm.matrix(),
                                               p.n_carm, r1=p.carm_r1)
            if eps < p.eps_tol:
                branch = "carm"
            else:
                u, iters, _ = m.mgcg(K, x0=u)
                parm.push(u)
                branch = "mgcg-fallback"
        else:
            u, iters, _ = m.mgcg(K, x0=u_last if k > 1 else None)
            branch = "mgcg"
            if mode == "aarmr" and k > p.n_on - p.n_parm:
                parm.push(u)
        C, dc = m.sensitivities(u, rho_phys, E)
        dc_f = filters.sensitivity_filter(m.H, m.Hs, dc)
        rho_new, _, change = oc.oc_update(rho, dc_f, m.dv_f, m.H, m.Hs, p.volfrac_at(k), p.move)
        w = float(np.mean(np.abs(rho_new - rho)) * 100.0)      # Eq. 30
        traj.history.append(IterRecord(k, branch, C, eps, iters, change, w,
                                       time.perf_counter() - t0))
        rho = rho_new
        u_last = u
        E_prev = E
        rho_phys_prev = rho_phys
    traj.rho = rho
    return traj

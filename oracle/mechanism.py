"""Compliant-mechanism design of Sec. 4.3: the displacement inverter, the
paper's non-self-adjoint example.  Test infrastructure (the CPU oracle):
only tests, the smoke check and the bench's CPU baseline use it.

Objective: the output displacement u_out = l^T u, l the unit vector of the
output DOF, minimised, so that the output end moves against the input force
(its magnitude is maximised).  Linear springs to ground at the input and
output DOFs enter the stiffness as K_s(rho~) = K(rho~) + S, S diagonal with
k_in and k_out (Sec. 4.3: k_in = 1, k_out = 0.1).

Sensitivity by the adjoint system K_s lam = l (K_s is symmetric):
    d u_out / d rho~_e = -lam^T (dK_s / d rho~_e) u
                       = -p (E0 - Emin) rho~_e^(p-1) lam_e^T KE u_e,
with u the state solution of K_s u = f_in.

Readings of what the section leaves open:
* both the state and the adjoint system run Algorithm 1, each with its own
  PARM, u_last and reduced model, on the same K_s and K_s,ref: the paper
  "employs approximate sensitivity", read as the sensitivity formed from
  the AARMR solutions of both systems;
* the springs do not depend on the design, so they cancel in
  dK = K_s - K_s,ref (Eq. 8);
* the OC update keeps the compliance rule's form with a damping exponent
  eta (0.3 for the mechanism, as is usual for compliant mechanisms; 1/2 is
  the compliance rule): rho_new = clamp(rho * max(0, -dc / (lam dv))^eta)
  within the move limit, lam from the filtered volume constraint;
* geometry (Fig. 31 is not in the text): the half domain lies above its
  symmetry axis, the bottom edge (y-displacements fixed there); the input A
  is the bottom-left node with a unit force in +x, the output B the
  bottom-right node; the top-left end of the left edge (nely/16 of it,
  at least one element) is clamped.  (workloads.inverter2d)
"""

from __future__ import annotations

import time
from dataclasses import dataclass, field
from typing import List, Optional

import numpy as np
import scipy.sparse as sp

from . import fe, filters, oc, reanalysis, solvers
from .aarmr import OracleModel


def spring_matrix(ndof: int, springs) -> sp.csr_matrix:
    """S: diagonal, k at each spring's DOF (Sec. 4.3)."""
    d = np.zeros(ndof)
    for dof, k in springs:
        d[int(dof)] += float(k)
    return sp.diags(d).tocsr()


def output_sensitivity(grid: fe.Grid, KE: np.ndarray, u: np.ndarray, lam: np.ndarray,
                       fixed: np.ndarray, rho_phys: np.ndarray, E0: float, Emin: float,
                       penal: float) -> np.ndarray:
    """d u_out / d rho~_e = -p (E0 - Emin) rho~_e^(p-1) lam_e^T KE u_e, the
    prescribed DOFs taken as zero in both fields."""
    free = 1.0 - fixed.astype(float)
    dofs = grid.element_dofs()
    ue = (u * free)[dofs]
    le = (lam * free)[dofs]
    mutual = np.einsum("ei,ij,ej->e", le, KE, ue)
    return -penal * (E0 - Emin) * rho_phys ** (penal - 1.0) * mutual


class MechanismModel(OracleModel):
    """Fixed data of a mechanism problem: the compliance model's plus the
    springs and the unit output vector l."""

    def __init__(self, prob):
        super().__init__(prob)
        self.S = spring_matrix(self.grid.ndof, prob.springs)
        self.l = np.zeros(self.grid.ndof)
        self.l[prob.out_dof] = 1.0

    def K(self, E):
        """K_s = K(rho~) + S with the boundary conditions of K."""
        return (super().K(E) + self.S).tocsr()

    def solve_mgcg(self, K, rhs, x0=None, mg=None):
        p = self.prob
        mg = mg or self.multigrid(K)
        return solvers.mgcg(K, rhs, mg, x0=x0, rtol=p.rtol, maxit=p.maxit)


@dataclass
class MechRecord:
    k: int
    objective: float                  # u_out of the state solution
    branches: tuple                   # (state, adjoint)
    eps: tuple                        # (state, adjoint) eps of Eq. 29 or None
    cg_iters: tuple
    change: float
    seconds: float = 0.0


@dataclass
class MechTrajectory:
    rho: np.ndarray
    history: List[MechRecord] = field(default_factory=list)


class _System:
    """One linear system of the mechanism loop (state or adjoint) with its
    own Algorithm 1 state."""

    def __init__(self, n_parm: int, ndof: int, rhs: np.ndarray):
        self.parm = reanalysis.Parm(n_parm)
        self.u_last = np.zeros(ndof)
        self.rhs = rhs

    def step(self, m: MechanismModel, k: int, K, K_ref, dK, mg, mode: str):
        """Algorithm 1 for this system at design iteration k."""
        p = m.prob
        eps, iters = None, 0
        if mode == "direct":
            u, branch = solvers.direct_solve(K, self.rhs, m.fixed), "direct"
        elif mode == "aarmr" and k > p.n_on and self.parm.full:
            u, eps, _ = reanalysis.aarmr_solve(lambda v: K @ v, lambda v: K_ref @ v,
                                               lambda v: dK @ v, self.rhs, self.u_last,
                                               self.parm.matrix(), p.n_carm, r1=p.carm_r1)
            if eps < p.eps_tol:
                branch = "carm"
            else:
                u, iters, _ = m.solve_mgcg(K, self.rhs, x0=u, mg=mg)
                self.parm.push(u)
                branch = "mgcg-fallback"
        else:
            u, iters, _ = m.solve_mgcg(K, self.rhs, x0=self.u_last if k > 1 else None, mg=mg)
            branch = "mgcg"
            if mode == "aarmr" and k > p.n_on - p.n_parm:
                self.parm.push(u)
        self.u_last = u
        return u, branch, eps, iters


def run(prob, n_iter: Optional[int] = None, mode: str = "aarmr",
        model: Optional[MechanismModel] = None) -> MechTrajectory:
    """The mechanism design loop: per iteration the filter and SIMP
    (Eq. 31, 1), the state and adjoint solves (each by Algorithm 1 in mode
    "aarmr", MGCG every time in "mgcg", exact in "direct"), the output
    sensitivity, its filter (Eq. 33) and the damped OC update."""
    m = model or MechanismModel(prob)
    p = prob
    n_iter = p.n_iter if n_iter is None else n_iter
    rho = p.rho0.astype(float).copy()
    state = _System(p.n_parm, m.grid.ndof, m.f)
    adj = _System(p.n_parm, m.grid.ndof, m.l)
    E_prev = None
    traj = MechTrajectory(rho)
    for k in range(1, n_iter + 1):
        t0 = time.perf_counter()
        rho_phys = filters.density_filter(m.H, m.Hs, rho)
        E = m.modulus(rho_phys)
        K = m.K(E)
        K_ref = m.K(E_prev) if E_prev is not None else None
        dK = m.dK(E, E_prev) if E_prev is not None else None
        mg = m.multigrid(K) if mode != "direct" else None
        u, bu, eu, iu = state.step(m, k, K, K_ref, dK, mg, mode)
        lam, bl, el, il = adj.step(m, k, K, K_ref, dK, mg, mode)
        obj = float(u[p.out_dof])
        dc = output_sensitivity(m.grid, m.KE, u, lam, m.fixed, rho_phys, p.E0, p.Emin, p.penal)
        dc_f = filters.sensitivity_filter(m.H, m.Hs, dc)
        rho_new, _, change = oc.oc_update(rho, dc_f, m.dv_f, m.H, m.Hs, p.volfrac_at(k), p.move,
                                          eta=p.oc_eta)
        traj.history.append(MechRecord(k, obj, (bu, bl), (eu, el), (iu, il), change,
                                       time.perf_counter() - t0))
        rho = rho_new
        E_prev = E
    traj.rho = rho
    return traj

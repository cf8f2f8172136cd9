"""The efficiency studies of Sec. 4.2 and 4.3 on the GPU: each problem runs twice
through the same library, once with AARMR (Algorithm 1) and once with MGCG
at every design iteration (the paper's reference method), and reports

* speedup = T_Ref / T_Goal (Eq. 35): cumulative equilibrium-solve time of
  MGCG over that of AARMR;
* diff = (C_Goal - C_Ref) / C_Ref x 100 % (Eq. 36): relative difference of
  the final compliance;
* the MGCG evaluations of each run (the quantity of Fig. 17 and Fig. 25).

For the displacement inverter of Sec. 4.3 (Table 1) the objective is the
output displacement, both the state and the adjoint solve count in the
solve time, and the average CG iterations per MGCG call are reported.

Run from the repository root, for example:
    python -m paper_2205_00385_gb300.studies --case beam --model 0 --eps 0.01 0.05
    python -m paper_2205_00385_gb300.studies --case inverter --model 0 --eps 0.0001 0.001 --iters 200
"""

from __future__ import annotations

import argparse
import json
from typing import Dict

from .driver import MechanismSolver, TopoSolver


def run_pair(prob, precision: str = "fp64") -> Dict:
    """AARMR and MGCG-only runs of one problem; returns the Eq. 35 / 36
    figures and the per-run totals."""
    out = {}
    for name, p in (("aarmr", prob), ("mgcg", prob.with_(n_on=10 ** 9))):
        s = TopoSolver(p, precision=precision)
        try:
            hist = s.run(p.n_iter)
        finally:
            s.close()
        out[name] = dict(
            solve_s=sum(h.solve_seconds for h in hist),
            mgcg_evaluations=sum(h.branch != "carm" for h in hist),
            carm_accepted=sum(h.branch == "carm" for h in hist),
            cg_iterations=sum(h.cg_iters for h in hist),
            final_compliance=hist[-1].compliance,
            not_converged=sum(not h.converged for h in hist))
    a, m = out["aarmr"], out["mgcg"]
    out["speedup"] = m["solve_s"] / a["solve_s"]
    out["diff_percent"] = (a["final_compliance"] - m["final_compliance"]) / m[
        "final_compliance"] * 100.0
    return out


def run_pair_mechanism(prob, precision: str = "fp64") -> Dict:
    """The same for a mechanism problem (Table 1): Eq. 35 over both solves
    of every iteration, Eq. 36 on the final output displacement."""
    out = {}
    for name, p in (("aarmr", prob), ("mgcg", prob.with_(n_on=10 ** 9))):
        s = MechanismSolver(p, precision=precision)
        try:
            hist = s.run(p.n_iter)
        finally:
            s.close()
        calls = sum(b != "carm" for h in hist for b in h.branches)
        cg = sum(sum(h.cg_iters) for h in hist)
        out[name] = dict(
            solve_s=sum(h.solve_seconds for h in hist),
            mgcg_evaluations=calls,
            carm_accepted=sum(b == "carm" for h in hist for b in h.branches),
            cg_iterations=cg, avg_cg_per_mgcg=cg / max(calls, 1),
            final_objective=hist[-1].objective)
    a, m = out["aarmr"], out["mgcg"]
    out["speedup"] = m["solve_s"] / a["solve_s"]
    out["diff_percent"] = (a["final_objective"] - m["final_objective"]) / abs(
        m["final_objective"]) * 100.0
    return out


def main():
    from workloads import (BEAM_MODELS, HALFWHEEL_MODELS, INVERTER_MODELS, study_beam,
                           study_halfwheel, study_inverter)
    ap = argparse.ArgumentParser(description="Sec. 4.2 / 4.3 speedup and difference studies")
    ap.add_argument("--case", choices=["halfwheel", "beam", "inverter"], required=True)
    ap.add_argument("--model", type=int, default=0, help="model index of Sec. 4.2 (0-3)")
    ap.add_argument("--eps", type=float, nargs="+", default=[0.01, 0.05])
    ap.add_argument("--iters", type=int, default=100)
    ap.add_argument("--precision", default="fp64", choices=["fp64", "mixed"])
    a = ap.parse_args()
    for eps in a.eps:
        if a.case == "halfwheel":
            nx, ny = HALFWHEEL_MODELS[a.model]
            p = study_halfwheel(nx, ny, eps, n_iter=a.iters)
        elif a.case == "inverter":
            nx, ny = INVERTER_MODELS[a.model]
            p = study_inverter(nx, ny, eps, n_iter=a.iters)
        else:
            nx, ny, nz = BEAM_MODELS[a.model]
            p = study_beam(nx, ny, nz, eps, n_iter=a.iters)
        r = (run_pair_mechanism if a.case == "inverter" else run_pair)(p, a.precision)
        r.update(case=a.case, model=a.model, grid=[p.nelx, p.nely, p.nelz], eps_tol=eps,
                 iters=a.iters, precision=a.precision)
        print(json.dumps(r), flush=True)


if __name__ == "__main__":
    main()

"""Properties of the method that the paper reports or implies, checked on
the GPU path through the C ABI.

* Sec. 4.1's basis-size study reports that (N_s, N_m) = (1, 1), (1, 10) and
(10, 1) give exactly overlapping results.  With N_m = 1 the reduced space
is span{u_last} whatever N_s; with N_s = 1 every CA vector beyond r_1 lies
in span{phi_1}, which holds u_last.  On the 60 x 20 MBB half-beam (float64,
the workload of that size) with a residual criterion loose enough that CARM
is accepted repeatedly, the three GPU trajectories must take the same
branches with equal compliances, and the (1, 1) trajectory must match the
oracle's.
* A PARM that holds the exact solution u* (and a CA basis that spans
  span{u_last, Phi}) makes the CARM's Galerkin solution u* itself, with a
  vanishing force residual (Eq. 22-29), in float64 and in the mixed path.

This file runs last (it is the newest).
"""

import pytest

from oracle import aarmr
from workloads import mbb2d_60x20

pytestmark = pytest.mark.gpu

SETTINGS = ((1, 1), (1, 10), (10, 1))
N_ITER = 40


def _problem(ns, nm):
    return mbb2d_60x20().with_(n_parm=ns, n_carm=nm, n_on=12, eps_tol=0.3)


def _gpu_history(p):
    from paper_2205_00385_gb300.driver import TopoSolver
    s = TopoSolver(p)
    try:
        return s.run(N_ITER)
    finally:
        s.close()


def test_basis_sizes_the_paper_reports_as_overlapping():
    runs = {key: _gpu_history(_problem(*key)) for key in SETTINGS}
    ref = runs[(1, 1)]
    assert sum(h.branch == "carm" for h in ref) >= 5
    assert sum(h.branch == "mgcg-fallback" for h in ref) >= 5
    for key in SETTINGS[1:]:
        hist = runs[key]
        assert [h.branch for h in hist] == [h.branch for h in ref], key
        for a, b in zip(ref, hist):
            assert abs(a.compliance - b.compliance) <= 1e-9 * a.compliance, (key, a, b)
    oracle = aarmr.run(_problem(1, 1), n_iter=N_ITER, mode="aarmr").history
    assert [h.branch for h in ref] == [h.branch for h in oracle]
    for g, o in zip(ref, oracle):
        assert abs(g.compliance - o.compliance) <= 1e-6 * o.compliance, (g, o)


@pytest.mark.parametrize("precision,tol", [("fp64", 1e-9), ("mixed", 1e-6)])
def test_exact_solution_in_the_parm_is_recovered(precision, tol):
    """When the exact solution u* is a PARM column and the CA basis spans
    span{u_last, Phi} (N_m = N_s + 1, well conditioned here), the CARM
    Galerkin solution is u* itself and the force residual (Eq. 29)
    vanishes to rounding, whatever u_last."""
    import numpy as np
    from gpu_helpers import Ctx, dev, host
    from oracle import fe, sensitivity, solvers
    from workloads import rand_density, rand_vector, small_problem, smooth_fields
    from paper_2205_00385_gb300 import binding as B
    p = small_problem("cantilever3d", nelx=8, nely=4, nelz=4, mg_levels=3, n_parm=3, n_carm=4)
    g = fe.Grid.of(p)
    KE = fe.element_stiffness(3, p.nu)
    r_prev = rand_density(g.nel, 61, 0.1, 1.0)
    r_now = np.clip(r_prev + rand_density(g.nel, 62, -0.1, 0.1), 0.05, 1.0)
    E = sensitivity.simp_modulus(r_now, p.E0, p.Emin, p.penal)
    u_star = solvers.direct_solve(fe.stiffness(g, E, KE, p.fixed), p.f, p.fixed)
    cols = [u_star] + smooth_fields(p.nelx, p.nely, p.nelz, p.fixed, 2)
    u_last = rand_vector(g.ndof, 63, fixed=p.fixed)
    with Ctx(p, precision=precision) as c:
        c.set_density(r_prev)
        c.set_density(r_now)
        for v in cols:
            B.to_parm_push(c.ctx, dev(v))
        B.to_carm_build(c.ctx, dev(u_last))
        u = dev(np.zeros(g.ndof))
        eps = B.to_carm_solve(c.ctx, u)
        u = host(u)
    assert eps < tol, eps
    assert np.linalg.norm(u - u_star) <= tol * np.linalg.norm(u_star)

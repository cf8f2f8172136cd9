"""Pins of the oracle's compliant-mechanism problem (Sec. 4.3): the springs'
place in the stiffness, the adjoint sensitivity of the output displacement,
the damped OC rule and the design loop, each against something other than
the oracle's own formula (a hand-computed one-DOF system, reciprocity,
finite differences, brute force, the exact solver)."""

import numpy as np
import pytest

from oracle import fe, filters, mechanism, oc, solvers
from workloads import inverter2d, rand_density, small_problem


def _model(p):
    return mechanism.MechanismModel(p)


def test_spring_adds_to_a_single_free_dof():
    """With every DOF but the input's prescribed, K_s u = f reduces to
    (K_aa + k_in) u_a = f_a: the spring must add k_in on that diagonal entry
    and nowhere else."""
    p = inverter2d(4, 2)
    fixed = np.ones(p.ndof, np.uint8)
    a = p.springs[0][0]
    fixed[a] = 0
    p = p.with_(fixed=fixed)
    m = _model(p)
    E = m.modulus(np.full(p.nel, 0.7))
    K = m.K(E)
    # K_aa from the element matrices: node A (bottom-left) belongs to element
    # 0 only, as its corner 0 with x-DOF row 0
    KE = fe.element_stiffness(2, p.nu)
    kaa = E[0] * KE[0, 0]
    u = solvers.direct_solve(K, m.f, m.fixed)
    assert abs(u[a] - 1.0 / (kaa + p.springs[0][1])) < 1e-14
    S = mechanism.spring_matrix(p.ndof, p.springs)
    assert S.nnz == 2 and S[p.out_dof, p.out_dof] == 0.1 and S[a, a] == 1.0


def test_reciprocity_of_state_and_adjoint():
    """Maxwell-Betti for the symmetric K_s: l^T K_s^-1 f = f^T K_s^-1 l."""
    p = small_problem("inverter2d", nelx=24, nely=12)
    m = _model(p)
    K = m.K(m.modulus(rand_density(p.nel, 31, 0.05, 1.0)))
    u = solvers.direct_solve(K, m.f, m.fixed)
    lam = solvers.direct_solve(K, m.l, m.fixed)
    assert abs(m.l @ u - m.f @ lam) <= 1e-12 * abs(m.l @ u)


def test_output_sensitivity_matches_finite_differences():
    p = small_problem("inverter2d", nelx=16, nely=8)
    m = _model(p)
    rho = rand_density(p.nel, 33, 0.2, 0.9)

    def u_out(r):
        return solvers.direct_solve(m.K(m.modulus(r)), m.f, m.fixed)[p.out_dof]

    K = m.K(m.modulus(rho))
    u = solvers.direct_solve(K, m.f, m.fixed)
    lam = solvers.direct_solve(K, m.l, m.fixed)
    dc = mechanism.output_sensitivity(m.grid, m.KE, u, lam, m.fixed, rho, p.E0, p.Emin, p.penal)
    # central differences, h = 1e-5: truncation ~h^2, rounding ~1e-16 |u_out| / h,
    # both far below 1e-6 of the field's largest entry
    h = 1e-5
    scale = np.max(np.abs(dc))
    for e in (0, 5, p.nel // 2, p.nel - 1, 37, int(np.argmax(np.abs(dc)))):
        rp, rm = rho.copy(), rho.copy()
        rp[e] += h
        rm[e] -= h
        fd = (u_out(rp) - u_out(rm)) / (2 * h)
        assert abs(dc[e] - fd) <= 1e-6 * scale


def test_damped_oc_keeps_the_volume_and_matches_brute_force():
    p = small_problem("inverter2d", nelx=16, nely=8)
    g = fe.Grid.of(p)
    H, Hs = filters.filter_matrix(g, p.rmin)
    rng = np.random.default_rng(35)
    rho = rng.uniform(0.1, 0.9, p.nel)
    dc = -rng.uniform(0.0, 1.0, p.nel) * rng.choice([1.0, -0.1], p.nel)   # both signs
    dv = filters.sensitivity_filter(H, Hs, np.ones(p.nel))
    for eta in (0.3, 0.5):
        rn, lam, _ = oc.oc_update(rho, dc, dv, H, Hs, 0.4, move=0.1, eta=eta)
        assert abs(filters.density_filter(H, Hs, rn).sum() - 0.4 * p.nel) < 1e-6 * p.nel
        for e in range(0, p.nel, 7):
            x = max(0.0, -dc[e] / (dv[e] * lam))
            want = min(min(1.0, rho[e] + 0.1), max(max(0.0, rho[e] - 0.1), rho[e] * x ** eta))
            assert abs(rn[e] - want) < 1e-15
    # elements whose density increase raises u_out drop by the move limit
    rn, _, _ = oc.oc_update(rho, dc, dv, H, Hs, 0.4, move=0.1, eta=0.3)
    up = dc > 0
    assert np.allclose(rn[up], np.maximum(0.0, rho[up] - 0.1))


def test_mechanism_loop_mgcg_follows_the_exact_solver():
    p = small_problem("inverter2d", nelx=32, nely=16, mg_levels=3, n_iter=8, rtol=1e-12,
                      maxit=400)
    a = mechanism.run(p, mode="mgcg")
    b = mechanism.run(p, mode="direct")
    for ra, rb in zip(a.history, b.history):
        assert abs(ra.objective - rb.objective) <= 1e-8 * abs(rb.objective)
    assert np.max(np.abs(a.rho - b.rho)) < 1e-6
    # the objective improves: the output is driven against the input
    assert a.history[-1].objective < a.history[0].objective


def test_aarmr_mechanism_reaches_the_reduced_models_and_stays_close():
    """Algorithm 1 on both systems: after N_on the CA models are tried and,
    at the paper's 0.1 % criterion, accepted in about half the solves; the
    design's objective stays within 1 % of the MGCG-only run's."""
    p = small_problem("inverter2d", nelx=32, nely=16, mg_levels=3, n_iter=40, n_on=10,
                      n_parm=2, n_carm=2, eps_tol=1e-3, rtol=1e-10, maxit=400)
    a = mechanism.run(p, mode="aarmr")
    m = mechanism.run(p, mode="mgcg")
    branches = [r.branches for r in a.history]
    assert all(b == ("mgcg", "mgcg") for b in branches[:10])
    assert sum(b.count("carm") for b in branches[10:]) >= 10
    assert abs(a.history[-1].objective - m.history[-1].objective) <= 0.01 * abs(
        m.history[-1].objective)
    # with a criterion nothing meets, every attempt falls back and the run is
    # MGCG warm-started from the reduced solution: the same designs as MGCG
    strict = mechanism.run(p.with_(eps_tol=0.0, n_iter=16), mode="aarmr")
    assert all(set(r.branches) <= {"mgcg", "mgcg-fallback"} for r in strict.history)
    assert any("mgcg-fallback" in r.branches for r in strict.history)
    for rs, rm in zip(strict.history, m.history):
        assert abs(rs.objective - rm.objective) <= 1e-7 * abs(rm.objective)

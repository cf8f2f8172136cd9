"""Pins of the oracle's solvers and reanalysis: dense library solves, the
nested-space identity of Galerkin coarsening, V-cycle symmetry, Kirsch's
CA = PCG equivalence, full-basis exactness, special cases and invariants."""

import numpy as np
import pytest
import scipy.linalg as sla

from oracle import aarmr, fe, reanalysis, solvers
from workloads import small_problem


def _setup(kind, **kw):
    p = small_problem(kind, **kw)
    g = fe.Grid.of(p)
    KE = fe.element_stiffness(p.dim, p.nu)
    return p, g, KE


@pytest.mark.parametrize("kind", ["mbb2d", "cantilever3d", "bridge3d"])
def test_direct_solve_matches_dense_library(kind):
    p, g, KE = _setup(kind)
    E = np.random.default_rng(0).uniform(1e-3, 1.0, g.nel)
    K = fe.stiffness(g, E, KE, p.fixed)
    u = solvers.direct_solve(K, p.f, p.fixed)
    ud = np.linalg.solve(K.toarray(), p.f)
    assert np.max(np.abs(u - ud)) < 1e-10 * np.max(np.abs(ud))


@pytest.mark.parametrize("kind", ["mbb2d", "cantilever3d", "bridge3d"])
def test_galerkin_coarse_operator_equals_coarse_fe_matrix(kind):
    """Nested FE spaces: with E constant on each coarse element, P^T K P is the
    stiffness assembled on the coarse grid (element size 2, so KE scales by
    2^(dim-2)), with the coarse BCs."""
    p, g, KE = _setup(kind)
    gc = solvers.coarse_grid(g)
    Ec = np.random.default_rng(1).uniform(0.1, 1.0, gc.nel)
    ex, ey, ez = g.element_ijk()
    E = Ec[(ex // 2) + gc.nelx * ((ey // 2) + gc.nely * (ez // 2))]
    A0 = fe.stiffness(g, E, KE, p.fixed)
    mg = solvers.Multigrid(g, A0, p.fixed, 2)
    fc = solvers.coarse_fixed(g, gc, p.fixed)
    ref = fe.stiffness(gc, Ec * 2.0 ** (p.dim - 2), KE, fc)
    assert abs(mg.A[1] - ref).max() < 1e-13 * abs(ref).max()


@pytest.mark.parametrize("kind", ["mbb2d", "cantilever3d"])
def test_vcycle_symmetric_positive(kind):
    p, g, KE = _setup(kind)
    E = np.random.default_rng(2).uniform(1e-3, 1.0, g.nel)
    A0 = fe.stiffness(g, E, KE, p.fixed)
    mg = solvers.Multigrid(g, A0, p.fixed, 3 if kind == "cantilever3d" else 3)
    rng = np.random.default_rng(3)
    a, b = rng.standard_normal(g.ndof), rng.standard_normal(g.ndof)
    Ma, Mb = mg.vcycle(a), mg.vcycle(b)
    assert abs(Ma @ b - a @ Mb) < 1e-12 * np.linalg.norm(Ma) * np.linalg.norm(b)
    assert Ma @ a > 0


@pytest.mark.parametrize("kind", ["mbb2d", "cantilever3d", "bridge3d"])
def test_mgcg_converges_to_direct_solution(kind):
    p, g, KE = _setup(kind)
    E = np.random.default_rng(4).uniform(1e-3, 1.0, g.nel)
    A0 = fe.stiffness(g, E, KE, p.fixed)
    mg = solvers.Multigrid(g, A0, p.fixed, 3)
    u, it, rel = solvers.mgcg(A0, p.f, mg, rtol=1e-12, maxit=200)
    ud = solvers.direct_solve(A0, p.f, p.fixed)
    assert it < 200 and rel < 1e-12
    assert np.linalg.norm(u - ud) < 1e-9 * np.linalg.norm(ud)


def test_ca_equals_pcg_with_reference_preconditioner():
    """Kirsch's result (cited in the introduction): with the exact inverse of
    K_ref and r1 = K_ref^{-1} f, the CA solution with m basis vectors equals
    the m-th PCG iterate preconditioned by K_ref (x0 = 0), because
    K_ref^{-1} K = I - B makes the Krylov space span{r1, B r1, ...}."""
    p, g, KE = _setup("cantilever3d", nelx=4, nely=2, nelz=2)
    rng = np.random.default_rng(5)
    E_ref = rng.uniform(0.2, 1.0, g.nel)
    E = E_ref * rng.uniform(0.7, 1.3, g.nel)
    K = fe.stiffness(g, E, KE, p.fixed).toarray()
    Kr = fe.stiffness(g, E_ref, KE, p.fixed).toarray()
    dK = K - Kr
    cf = sla.cho_factor(Kr)
    r1 = sla.cho_solve(cf, p.f)
    for m in (1, 2, 3, 4):
        R = reanalysis.ca_exact_basis(r1, lambda v: sla.cho_solve(cf, v), lambda v: dK @ v, m)
        u_ca, _, _ = reanalysis.reduced_solve(lambda v: K @ v, reanalysis.orthonormalize(R), p.f)
        u_pcg, it, _ = solvers.pcg(K, p.f, precond=lambda v: sla.cho_solve(cf, v),
                                   rtol=0.0, maxit=m)
        assert np.linalg.norm(u_ca - u_pcg) < 1e-8 * np.linalg.norm(u_pcg)


def test_full_parm_gives_exact_inverse():
    """Eq. 18 with Phi spanning R^n is K_ref^{-1} exactly."""
    p, g, KE = _setup("mbb2d", nelx=4, nely=2)
    Kr = fe.stiffness(g, np.random.default_rng(6).uniform(0.2, 1, g.nel), KE, p.fixed).toarray()
    Phi = np.random.default_rng(7).standard_normal((g.ndof, g.ndof))
    Kinv = reanalysis.approx_inverse(Phi, Phi.T @ Kr @ Phi)
    M = np.stack([Kinv(e) for e in np.eye(g.ndof)], axis=1)
    assert np.max(np.abs(M @ Kr - np.eye(g.ndof))) < 1e-8


def test_approx_inverse_invariant_to_scaling_and_permutation():
    p, g, KE = _setup("cantilever3d", nelx=4, nely=2, nelz=2)
    rng = np.random.default_rng(8)
    Kr = fe.stiffness(g, rng.uniform(0.2, 1, g.nel), KE, p.fixed)
    Phi = rng.standard_normal((g.ndof, 4))
    v = rng.standard_normal(g.ndof)
    a = reanalysis.approx_inverse(Phi, reanalysis.k_phi(Phi, lambda x: Kr @ x))(v)
    Phi2 = Phi[:, [2, 0, 3, 1]] * np.array([3.0, -0.5, 7.0, 1e-3])
    b = reanalysis.approx_inverse(Phi2, reanalysis.k_phi(Phi2, lambda x: Kr @ x))(v)
    assert np.linalg.norm(a - b) < 1e-10 * np.linalg.norm(a)


def test_singular_k_phi_takes_the_pseudo_inverse():
    """The fallback of the K_Phi inverse (Cholesky fails: pseudo-inverse).
    A = B B^T with B = [[1, 0], [0, 1], [1, 1]] is singular with integer
    entries, so Cholesky meets an exactly zero third pivot (2 - 1 - 1) and
    the eigen branch runs.  Its Moore-Penrose inverse has the closed form
    B (B^T B)^-2 B^T = [[5, -4, 1], [-4, 5, 1], [1, 1, 2]] / 9, worked out
    by hand from B^T B = [[2, 1], [1, 2]]; a kept null direction (wrong
    cutoff) or a transposed eigenvector matrix would not give it."""
    A = np.array([[1.0, 0.0, 1.0], [0.0, 1.0, 1.0], [1.0, 1.0, 2.0]])
    with pytest.raises(np.linalg.LinAlgError):
        sla.cho_factor(A)
    P = reanalysis.small_spd_inverse(A)
    closed = np.array([[5.0, -4.0, 1.0], [-4.0, 5.0, 1.0], [1.0, 1.0, 2.0]]) / 9.0
    assert np.max(np.abs(P - closed)) < 1e-14
    # Penrose conditions
    assert np.max(np.abs(A @ P @ A - A)) < 1e-14
    assert np.max(np.abs(P @ A @ P - P)) < 1e-14
    assert np.max(np.abs((A @ P).T - A @ P)) < 1e-14


def test_approx_inverse_with_a_repeated_parm_column():
    """Eq. 18 depends on span(Phi) only (span invariance): a PARM holding
    one column twice (K_Phi singular) gives the operator of the PARM without
    the repeat, whichever branch the K_Phi inverse takes; and a PARM with a
    zero column (exact zero pivot, so the pseudo-inverse branch) gives that
    of the PARM without it."""
    p, g, KE = _setup("cantilever3d", nelx=4, nely=2, nelz=2)
    rng = np.random.default_rng(18)
    Kr = fe.stiffness(g, rng.uniform(0.2, 1, g.nel), KE, p.fixed)
    Phi = rng.standard_normal((g.ndof, 3))
    v = rng.standard_normal(g.ndof)
    kphi = lambda F: reanalysis.k_phi(F, lambda x: Kr @ x)
    ref = reanalysis.approx_inverse(Phi, kphi(Phi))(v)
    rep = Phi[:, [0, 1, 1, 2]]
    assert np.linalg.norm(reanalysis.approx_inverse(rep, kphi(rep))(v) - ref) <= \
        1e-10 * np.linalg.norm(ref)
    zc = np.concatenate([Phi[:, :2], np.zeros((g.ndof, 1)), Phi[:, 2:]], axis=1)
    with pytest.raises(np.linalg.LinAlgError):
        sla.cho_factor(0.5 * (kphi(zc) + kphi(zc).T))
    assert np.linalg.norm(reanalysis.approx_inverse(zc, kphi(zc))(v) - ref) <= \
        1e-10 * np.linalg.norm(ref)


def _carm_fixture(seed=9, ns=3):
    p, g, KE = _setup("cantilever3d", nelx=6, nely=2, nelz=2)
    rng = np.random.default_rng(seed)
    E_ref = rng.uniform(0.2, 1.0, g.nel)
    E = E_ref * rng.uniform(0.8, 1.2, g.nel)
    K = fe.stiffness(g, E, KE, p.fixed)
    Kr = fe.stiffness(g, E_ref, KE, p.fixed)
    dK = fe.apply_bcs(fe.assemble(g, E - E_ref, KE), p.fixed, diag_fixed=0.0)
    us = []
    for s in range(ns):
        Es = E_ref * rng.uniform(0.9, 1.1, g.nel)
        us.append(solvers.direct_solve(fe.stiffness(g, Es, KE, p.fixed), p.f, p.fixed))
    parm = reanalysis.Parm(ns)
    for u in us:
        parm.push(u)
    u_last = solvers.direct_solve(Kr, p.f, p.fixed)
    return p, g, K, Kr, dK, parm.matrix(), u_last


def test_dk_zero_gives_scaled_last_solution():
    p, g, K, Kr, dK, Phi, u_last = _carm_fixture()
    zero = lambda v: 0.0 * v
    R = reanalysis.carm_basis(u_last, Phi, reanalysis.k_phi(Phi, lambda v: Kr @ v), zero, 4)
    assert np.all(R[:, 1:] == 0.0)
    Rt = reanalysis.orthonormalize(R)
    assert Rt.shape[1] == 1
    u, _, _ = reanalysis.reduced_solve(lambda v: K @ v, Rt, p.f)
    alpha = (p.f @ u_last) / (u_last @ (K @ u_last))
    assert np.linalg.norm(u - alpha * u_last) < 1e-12 * np.linalg.norm(u)


def test_uniform_scaling_recovered_exactly():
    """E = a E_ref with u_last the exact reference solution: the exact new
    solution u_last / a lies in the CARM span, so eps is at rounding level."""
    p, g, KE = _setup("cantilever3d", nelx=6, nely=2, nelz=2)
    rng = np.random.default_rng(10)
    E_ref = rng.uniform(0.2, 1.0, g.nel)
    a = 1.7
    Kr = fe.stiffness(g, E_ref, KE, p.fixed)
    Ka = fe.stiffness(g, a * E_ref, KE, p.fixed)
    dKa = fe.apply_bcs(fe.assemble(g, (a - 1.0) * E_ref, KE), p.fixed, diag_fixed=0.0)
    parm = reanalysis.Parm(2)
    for s in range(2):
        Es = E_ref * rng.uniform(0.9, 1.1, g.nel)
        parm.push(solvers.direct_solve(fe.stiffness(g, Es, KE, p.fixed), p.f, p.fixed))
    u_last = solvers.direct_solve(Kr, p.f, p.fixed)
    u, eps, _ = reanalysis.aarmr_solve(lambda v: Ka @ v, lambda v: Kr @ v, lambda v: dKa @ v,
                                       p.f, u_last, parm.matrix(), 3)
    assert eps < 1e-10
    assert np.linalg.norm(u - u_last / a) < 1e-10 * np.linalg.norm(u)


def test_carm_rank_and_span_invariants():
    p, g, K, Kr, dK, Phi, u_last = _carm_fixture(ns=3)
    KP = reanalysis.k_phi(Phi, lambda v: Kr @ v)
    R = reanalysis.carm_basis(u_last, Phi, KP, lambda v: dK @ v, 7)
    s = np.linalg.svd(R / np.linalg.norm(R, axis=0), compute_uv=False)
    assert np.sum(s > 1e-10 * s[0]) <= Phi.shape[1] + 1          # rank <= N_s + 1
    # with N_m >= N_s + 1 the span is span{u_last, Phi}, independent of dK
    u1, _, eps1 = reanalysis.reduced_solve(lambda v: K @ v, reanalysis.orthonormalize(R), p.f)
    Q, _ = np.linalg.qr(np.column_stack([u_last, Phi]))
    u2, _, eps2 = reanalysis.reduced_solve(lambda v: K @ v, Q, p.f)
    assert np.linalg.norm(u1 - u2) < 1e-8 * np.linalg.norm(u2)
    # Galerkin identity f^T u = u^T K u (Eq. 23-25)
    assert abs(p.f @ u1 - u1 @ (K @ u1)) < 1e-12 * abs(p.f @ u1)


def test_parm_fifo_normalised():
    parm = reanalysis.Parm(2)
    parm.push(np.array([3.0, 4.0]))
    parm.push(np.array([0.0, 2.0]))
    parm.push(np.array([5.0, 0.0]))
    Phi = parm.matrix()
    assert Phi.shape == (2, 2) and parm.full
    assert np.allclose(Phi[:, 0], [0.0, 1.0]) and np.allclose(Phi[:, 1], [1.0, 0.0])


def test_design_loop_mgcg_matches_direct():
    """MGCG-driven design loop with a tight tolerance follows the
    direct-solve loop."""
    p = small_problem("cantilever3d", nelx=8, nely=4, nelz=4, n_iter=6, mg_levels=3,
                      rtol=1e-12)
    a = aarmr.run(p, mode="mgcg")
    b = aarmr.run(p, mode="direct")
    for ra, rb in zip(a.history, b.history):
        assert abs(ra.compliance - rb.compliance) < 1e-8 * rb.compliance
    assert np.max(np.abs(a.rho - b.rho)) < 1e-7


def test_design_loop_carm_branch_taken_with_loose_tolerance():
    p = small_problem("mbb2d", nelx=16, nely=8, n_iter=10, n_on=4, n_parm=2, n_carm=3,
                      eps_tol=0.5, mg_levels=3)
    t = aarmr.run(p, mode="aarmr")
    branches = [h.branch for h in t.history]
    assert branches[:4] == ["mgcg"] * 4
    assert "carm" in branches[4:]
    assert all(h.eps is not None for h in t.history[4:])


def test_aarmr_with_full_parm_reduces_to_classical_ca():
    """With Phi spanning R^n, Eq. 18 is the exact K_ref^{-1}, so the AARMR
    basis (Eq. 26) is the classical CA basis (Eq. 13) and both reduced
    solutions agree.  With N_m <= N_s the span depends on K_Phi, so this
    fails if K_Phi were formed with K instead of K_ref."""
    p, g, KE = _setup("mbb2d", nelx=4, nely=2)
    rng = np.random.default_rng(11)
    E_ref = rng.uniform(0.2, 1.0, g.nel)
    E = E_ref * rng.uniform(0.6, 1.4, g.nel)
    K = fe.stiffness(g, E, KE, p.fixed)
    Kr = fe.stiffness(g, E_ref, KE, p.fixed)
    dK = fe.apply_bcs(fe.assemble(g, E - E_ref, KE), p.fixed, diag_fixed=0.0)
    Phi = rng.standard_normal((g.ndof, g.ndof))
    u_last = solvers.direct_solve(Kr, p.f, p.fixed)
    u_a, eps_a, _ = reanalysis.aarmr_solve(lambda v: K @ v, lambda v: Kr @ v,
                                           lambda v: dK @ v, p.f, u_last, Phi, 3)
    cf = sla.cho_factor(Kr.toarray())
    R = reanalysis.ca_exact_basis(u_last, lambda v: sla.cho_solve(cf, v), lambda v: dK @ v, 3)
    u_c, _, eps_c = reanalysis.reduced_solve(lambda v: K @ v, reanalysis.orthonormalize(R), p.f)
    assert np.linalg.norm(u_a - u_c) < 1e-8 * np.linalg.norm(u_c)
    assert abs(eps_a - eps_c) < 1e-6 * eps_c


def test_basis_sizes_the_paper_reports_as_overlapping():
    """Sec. 4.1's basis-size study reports that the settings
    (N_s, N_m) = (1, 1), (1, 10) and (10, 1) give exactly overlapping
    results.  The method explains it: with N_m = 1 the reduced space is
    span{u_last} whatever N_s; with N_s = 1 every CA vector beyond r_1 lies
    in span{phi_1}, which holds u_last (the last MGCG solution, or a Galerkin
    multiple of it).  The three design trajectories, with CARM accepted
    repeatedly, must coincide: same branches, compliances equal to rounding."""
    from workloads import mbb2d_60x20
    base = mbb2d_60x20()
    runs = {}
    for ns, nm in ((1, 1), (1, 10), (10, 1)):
        p = base.with_(n_parm=ns, n_carm=nm, n_on=12, eps_tol=0.3)
        runs[(ns, nm)] = aarmr.run(p, n_iter=40, mode="aarmr").history
    ref = runs[(1, 1)]
    assert sum(h.branch == "carm" for h in ref) >= 5
    assert sum(h.branch == "mgcg-fallback" for h in ref) >= 5
    for key in ((1, 10), (10, 1)):
        hist = runs[key]
        assert [h.branch for h in hist] == [h.branch for h in ref], key
        for a, b in zip(ref, hist):
            assert abs(a.compliance - b.compliance) <= 1e-9 * a.compliance, (key, a, b)


def test_projected_load_start_with_full_parm_is_pcg():
    """The alternative first basis vector of Fig. 2, r_1 = Phi K_Phi^-1
    Phi^T f: with Phi spanning R^n, Eq. 18 is K_ref^-1 exactly, so r_1 =
    K_ref^-1 f and the CARM with m vectors is Kirsch's CA, i.e. the m-th PCG
    iterate preconditioned by K_ref (the result cited in the introduction).
    The u_last start would not give the PCG iterate."""
    p, g, KE = _setup("cantilever3d", nelx=4, nely=2, nelz=2)
    rng = np.random.default_rng(15)
    E_ref = rng.uniform(0.2, 1.0, g.nel)
    E = E_ref * rng.uniform(0.7, 1.3, g.nel)
    K = fe.stiffness(g, E, KE, p.fixed).toarray()
    Kr = fe.stiffness(g, E_ref, KE, p.fixed).toarray()
    dK = K - Kr
    Phi = rng.standard_normal((g.ndof, g.ndof))
    cf = sla.cho_factor(Kr)
    u_last = rng.standard_normal(g.ndof)
    for m in (1, 2, 3):
        u, _, _ = reanalysis.aarmr_solve(lambda v: K @ v, lambda v: Kr @ v, lambda v: dK @ v,
                                         p.f, u_last, Phi, m, r1="projected_load")
        u_pcg, _, _ = solvers.pcg(K, p.f, precond=lambda v: sla.cho_solve(cf, v), rtol=0.0,
                                  maxit=m)
        assert np.linalg.norm(u - u_pcg) < 1e-7 * np.linalg.norm(u_pcg)
        u_l, _, _ = reanalysis.aarmr_solve(lambda v: K @ v, lambda v: Kr @ v, lambda v: dK @ v,
                                           p.f, u_last, Phi, m)
        assert np.linalg.norm(u_l - u_pcg) > 1e-3 * np.linalg.norm(u_pcg)


def test_volume_ramp_is_followed():
    """Fig. 3's study lowers the volume fraction in the middle of the run; the
    OC update (Eq. 3) then holds the filtered volume at the ramped fraction of
    every iteration: sum rho~ = volfrac(k) N."""
    p = small_problem("mbb2d", nelx=24, nely=8, n_iter=9, volfrac=0.5,
                      volfrac_ramp=(4, 0.45, 0.02))
    assert [p.volfrac_at(k) for k in (3, 4, 5, 6, 7, 9)] == [0.5, 0.5, 0.48, 0.46, 0.45, 0.45]
    m = aarmr.OracleModel(p)
    t = aarmr.run(p, mode="mgcg", model=m, snapshot_at=tuple(range(2, 10)))
    for k in range(2, 10):
        rho_phys = t.snapshots[k]["rho_phys"]      # the design made by iteration k - 1
        assert abs(rho_phys.sum() - p.volfrac_at(k - 1) * p.nel) < 1e-9 * p.nel

"""GPU parity: every call of the C ABI against the CPU oracle on the same
seeded inputs.

Tolerances (relative unless stated):
* float64 stiffness apply and Galerkin level operators: 1e-13 / 1e-12 of the
  largest entry -- only summation order differs (<= ~30 terms per entry);
* float32 apply: 1e-5 in norm (float32 rounding of KE, E and x, 24-term sums);
* float64 V-cycle: 1e-10 (a few thousand operations per entry, the dense
  coarse inverse is formed explicitly); float32 V-cycle: 2e-3 (the coarsest
  grid's explicit inverse is formed in float32 from a matrix of condition
  ~1e4, so its relative error is ~1e-3);
* CARM build and solve: the same kept directions (Eq. 21), then u~, eps and
  compliance within 1e-9 / 1e-8 / 1e-10 (float64) and 1e-6 (mixed), see
  CARM_TOL;
* MGCG solutions: compliance within 1e-10 (float64 path, rtol 1e-12) and
  1e-6 (mixed path) of the exact solve -- the stated per-solve targets;
* filter, sensitivity filter: 1e-12; compliance and sensitivity: 1e-10
  (u_e^T KE u_e cancels for elements in near-rigid motion: the rounding
  error is relative to |u_e|^2 |KE|, up to ~1e3 times the element energy);
  OC: 1e-10 absolute on rho (the bisection bracket is 1e-13 relative).
"""

import numpy as np
import pytest

from gpu_helpers import Ctx, dev, host
from oracle import aarmr, fe, filters, oc, reanalysis, sensitivity, solvers
from workloads import small_problem, rand_vector, rand_density

pytestmark = pytest.mark.gpu


def _B():
    from paper_2205_00385_gb300 import binding as B
    return B


PROBLEMS = [
    ("mbb2d", dict(nelx=60, nely=20)),
    ("cantilever3d", dict(nelx=24, nely=12, nelz=12)),
    ("bridge3d", dict(nelx=16, nely=8, nelz=8)),
]


def _model(p):
    g = fe.Grid.of(p)
    KE = fe.element_stiffness(p.dim, p.nu)
    return g, KE


def _E(p, rho_phys):
    return sensitivity.simp_modulus(rho_phys, p.E0, p.Emin, p.penal)


@pytest.mark.parametrize("kind,kw", PROBLEMS)
@pytest.mark.parametrize("op", [0, 1, 2])
def test_apply_parity(kind, kw, op):
    B = _B()
    p = small_problem(kind, mg_levels=3, **kw)
    g, KE = _model(p)
    r_prev = rand_density(g.nel, 1, 0.0, 1.0)
    r_now = np.clip(r_prev + rand_density(g.nel, 2, -0.2, 0.2), 0, 1)
    x = rand_vector(g.ndof, 3)
    coef = {0: _E(p, r_now), 1: _E(p, r_prev), 2: _E(p, r_now) - _E(p, r_prev)}[op]
    y_ref = fe.apply_ebe(g, coef, KE, x, p.fixed, diag_fixed=0.0 if op == 2 else 1.0)
    with Ctx(p, precision="fp64") as c:
        c.set_density(r_prev)
        c.set_density(r_now)
        xd = dev(x)
        y64 = dev(np.zeros(g.ndof))
        y32 = dev(np.zeros(g.ndof))
        ydf = dev(np.zeros(g.ndof))
        B.to_apply(c.ctx, op, B.TO_PREC_FP64, xd, y64)
        B.to_apply(c.ctx, op, B.TO_PREC_FP32, xd, y32)
        B.to_apply(c.ctx, op, B.TO_PREC_DF, xd, ydf)
        y64, y32, ydf = host(y64), host(y32), host(ydf)
    scale = np.max(np.abs(y_ref))
    assert np.max(np.abs(y64 - y_ref)) <= 1e-13 * scale
    # float32, entry by entry: x, E and KE are rounded to float32 and each
    # element product passes through magnitudes up to max|KE| sum_j |x_j|
    # (transforms and block products of ~20 rounding steps, 8 element sums
    # per node), so the error of entry i is bounded by ~160 u32 ~ 1e-5 of
    # S_i = sum_e |E_e| max|KE| sum_(j in e) |x_j|; a lost or doubled element
    # contribution would be ~5e-3 of S_i
    S = fe.apply_ebe(g, np.abs(coef), np.full_like(KE, np.max(np.abs(KE))), np.abs(x), p.fixed,
                     diag_fixed=1.0)
    print(f"[apply f32 {kind} op{op}] max |err|/S = {np.max(np.abs(y32 - y_ref) / S):.2e}")
    assert np.all(np.abs(y32 - y_ref) <= 1e-5 * S + 1e-30), np.max(np.abs(y32 - y_ref) / S)
    # double-float: 48-bit significands, errors relative to |KE| |x_e| summed
    # over ~30 terms per entry -> 1e-12 of the largest entry
    assert np.max(np.abs(ydf - y_ref)) <= 1e-12 * scale


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
@pytest.mark.parametrize("kind,kw,levels", [("cantilever3d", dict(nelx=16, nely=8, nelz=8), 4),
                                            ("mbb2d", dict(nelx=32, nely=16), 4),
                                            ("bridge3d", dict(nelx=8, nely=4, nelz=4), 3)])
def test_galerkin_level_operators(precision, kind, kw, levels):
    """Element-by-element P^T K P on every coarse level against the oracle's
    sparse triple products (with the coarse BC rows)."""
    B = _B()
    p = small_problem(kind, mg_levels=levels, **kw)
    g, KE = _model(p)
    rho = rand_density(g.nel, 5, 0.05, 1.0)
    K = fe.stiffness(g, _E(p, rho), KE, p.fixed)
    mg = solvers.Multigrid(g, K, p.fixed, levels)
    with Ctx(p, precision=precision) as c:
        c.set_density(rho)
        for l in range(1, levels):
            _, n_l = B.to_level_info(c.ctx, l)
            assert n_l == mg.A[l].shape[0]
            x = rand_vector(n_l, 10 + l)
            y = dev(np.zeros(n_l))
            B.to_level_apply(c.ctx, l, dev(x), y)
            y = host(y)
            y_ref = mg.A[l] @ x
            if precision == "fp64":
                assert np.max(np.abs(y - y_ref)) <= 1e-12 * np.max(np.abs(y_ref))
            else:
                assert np.linalg.norm(y - y_ref) <= 1e-5 * np.linalg.norm(y_ref)


@pytest.mark.parametrize("kind,kw", PROBLEMS)
def test_vcycle_parity(kind, kw):
    B = _B()
    p = small_problem(kind, mg_levels=3, **kw)
    g, KE = _model(p)
    rho = rand_density(g.nel, 6, 0.1, 1.0)
    K = fe.stiffness(g, _E(p, rho), KE, p.fixed)
    mg = solvers.Multigrid(g, K, p.fixed, 3)
    r = rand_vector(g.ndof, 7, fixed=p.fixed)
    z_ref = mg.vcycle(r)
    with Ctx(p, precision="fp64") as c:
        c.set_density(rho)
        z = dev(np.zeros(g.ndof))
        B.to_vcycle(c.ctx, dev(r), z)
        z = host(z)
    assert np.linalg.norm(z - z_ref) <= 1e-10 * np.linalg.norm(z_ref)
    with Ctx(p, precision="mixed") as c:
        c.set_density(rho)
        z = dev(np.zeros(g.ndof))
        B.to_vcycle(c.ctx, dev(r), z)
        z = host(z)
    assert np.linalg.norm(z - z_ref) <= 2e-3 * np.linalg.norm(z_ref)


# hierarchies deep enough that restriction, smoothing and interpolation run
# on several stored levels below level 1
DEEP = [
    ("mbb2d", dict(nelx=64, nely=32), 5),
    ("cantilever3d", dict(nelx=32, nely=16, nelz=16), 4),
]


@pytest.mark.parametrize("kind,kw,levels", DEEP)
@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_vcycle_deep_hierarchy(kind, kw, levels, precision):
    """V-cycles of deep hierarchies against the oracle; repeated calls give
    the same bits."""
    B = _B()
    p = small_problem(kind, mg_levels=levels, **kw)
    g, KE = _model(p)
    rho = rand_density(g.nel, 16, 0.1, 1.0)
    K = fe.stiffness(g, _E(p, rho), KE, p.fixed)
    r = rand_vector(g.ndof, 17, fixed=p.fixed)
    z_ref = solvers.Multigrid(g, K, p.fixed, levels).vcycle(r)
    out = []
    with Ctx(p, precision=precision) as c:
        c.set_density(rho)
        for _ in range(2):
            z = dev(np.zeros(g.ndof))
            B.to_vcycle(c.ctx, dev(r), z)
            out.append(host(z))
    assert np.array_equal(out[0], out[1])
    tol = 1e-10 if precision == "fp64" else 2e-3
    assert np.linalg.norm(out[0] - z_ref) <= tol * np.linalg.norm(z_ref)


@pytest.mark.parametrize("kind,kw,levels", DEEP)
def test_mgcg_deep_hierarchy(kind, kw, levels):
    """MGCG on a mid-optimisation density with a deep hierarchy: the float64
    path takes the oracle's iteration count (within 1) and the mixed one
    (V-cycle replayed from a captured graph) at most half as many again
    (float32 rounding in the V-cycle and the operator perturbs the
    preconditioned iteration); both reach the exact compliance."""
    B = _B()
    p = small_problem(kind, mg_levels=levels, n_iter=8, **kw)
    g, KE = _model(p)
    rho = _snapshot_density(p, 8)
    E = _E(p, rho)
    K = fe.stiffness(g, E, KE, p.fixed)
    C_ref = p.f @ solvers.direct_solve(K, p.f, p.fixed)
    it_ref = solvers.mgcg(K, p.f, solvers.Multigrid(g, K, p.fixed, levels), rtol=1e-8,
                          maxit=500)[1]
    sol = {}
    for precision in ("mixed", "fp64"):
        with Ctx(p, precision=precision) as c:
            c.set_density(rho)
            u = dev(np.zeros(g.ndof))
            it, rel, ok = B.to_mgcg_solve(c.ctx, 1e-8, 500, 0, u)
            assert ok and rel < 1e-8, (precision, it, rel)
            sol[precision] = (it, host(u))
    assert abs(sol["fp64"][0] - it_ref) <= 1, (sol["fp64"][0], it_ref)
    assert sol["mixed"][0] <= 1.5 * it_ref + 2, (sol["mixed"][0], it_ref)
    for precision, tol in (("mixed", 1e-6), ("fp64", 1e-10)):
        C = sensitivity.compliance(E, sensitivity.element_energy(g, KE, sol[precision][1], p.fixed))
        assert abs(C - C_ref) <= tol * C_ref


def _snapshot_density(p, k):
    t = aarmr.run(p, n_iter=k, mode="mgcg", snapshot_at=(k,))
    return t.snapshots[k]["rho_phys"]


@pytest.mark.parametrize("kind,kw", PROBLEMS)
@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_mgcg_solve_parity(kind, kw, precision):
    """Per-solve parity on a mid-optimisation density field (high contrast)."""
    B = _B()
    p = small_problem(kind, mg_levels=3, n_iter=8, **kw)
    g, KE = _model(p)
    rho_phys = _snapshot_density(p, 8)
    E = _E(p, rho_phys)
    K = fe.stiffness(g, E, KE, p.fixed)
    u_ref = solvers.direct_solve(K, p.f, p.fixed)
    C_ref = p.f @ u_ref
    rtol = 1e-12 if precision == "fp64" else 1e-8
    with Ctx(p, precision=precision) as c:
        c.set_density(rho_phys)
        u = dev(np.zeros(g.ndof))
        it, rel, ok = B.to_mgcg_solve(c.ctx, rtol, 500, 0, u)
        u = host(u)
    assert ok and rel < rtol and it < 500
    ce = sensitivity.element_energy(g, KE, u, p.fixed)
    C = sensitivity.compliance(E, ce)
    tol = 1e-10 if precision == "fp64" else 1e-6
    assert abs(C - C_ref) <= tol * C_ref
    true_res = np.linalg.norm(p.f - K @ u) / np.linalg.norm(p.f)
    assert true_res < (1e-10 if precision == "fp64" else 1e-5)


@pytest.mark.parametrize("kind,kw", PROBLEMS)
@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_filter_sensitivity_oc_parity(kind, kw, precision):
    """fp64: float64 arithmetic throughout.  mixed: the 3D compliance and
    sensitivity in double-float arithmetic (~2^-48 relative per operation,
    inputs split to 48 significant bits), within the same bounds."""
    B = _B()
    fabs_tol = 1e-14
    p = small_problem(kind, mg_levels=3, **kw)
    g, KE = _model(p)
    H, Hs = filters.filter_matrix(g, p.rmin)
    rho = rand_density(g.nel, 8, 0.0, 1.0)
    rho_phys_ref = filters.density_filter(H, Hs, rho)
    E = _E(p, rho_phys_ref)
    u = solvers.direct_solve(fe.stiffness(g, E, KE, p.fixed), p.f, p.fixed)
    ce = sensitivity.element_energy(g, KE, u, p.fixed)
    C_ref = sensitivity.compliance(E, ce)
    dc_ref = sensitivity.compliance_sensitivity(rho_phys_ref, ce, p.E0, p.Emin, p.penal)
    dcf_ref = filters.sensitivity_filter(H, Hs, dc_ref)
    dvf_ref = filters.sensitivity_filter(H, Hs, np.ones(g.nel))
    rho_new_ref, lam, change_ref = oc.oc_update(rho, dcf_ref, dvf_ref, H, Hs, p.volfrac, 0.2)
    with Ctx(p, precision=precision) as c:
        rp = dev(np.zeros(g.nel))
        B.to_filter(c.ctx, B.TO_FILTER_DENSITY, dev(rho), rp)
        rho_phys = host(rp)
        assert np.max(np.abs(rho_phys - rho_phys_ref)) <= fabs_tol
        c.set_density(rho_phys_ref)
        Cd = dev(np.zeros(1))
        dcd = dev(np.zeros(g.nel))
        B.to_sensitivity(c.ctx, dev(u), Cd, dcd)
        assert abs(host(Cd)[0] - C_ref) <= 1e-10 * C_ref
        assert np.max(np.abs(host(dcd) - dc_ref)) <= 1e-10 * np.max(np.abs(dc_ref))
        dcf = dev(np.zeros(g.nel))
        B.to_filter(c.ctx, B.TO_FILTER_SENS, dev(dc_ref), dcf)
        assert np.max(np.abs(host(dcf) - dcf_ref)) <= 1e-12 * np.max(np.abs(dcf_ref))
        dvf = dev(np.zeros(g.nel))
        B.to_filter(c.ctx, B.TO_FILTER_SENS, dev(np.ones(g.nel)), dvf)
        assert np.max(np.abs(host(dvf) - dvf_ref)) <= fabs_tol
        rd = dev(rho)
        ch = dev(np.zeros(1))
        B.to_oc_update(c.ctx, p.volfrac, 0.2, dev(dcf_ref), dev(dvf_ref), rd, ch)
        assert np.max(np.abs(host(rd) - rho_new_ref)) <= 1e-10
        assert abs(host(ch)[0] - change_ref) <= 1e-10


# CARM parity on the oracle's inputs.  Both sides build the basis with
# float64-accurate products and keep the same singular directions; what
# differs is rounding of the basis (float64 or double-float, ~1e-16 or
# ~4e-15 per operation, amplified by the cancellation of K on smooth
# fields), which moves the kept directions by that much over their
# singular value (>= 1e-6 of the largest).  The Galerkin compliance is
# stationary in the subspace, so it moves at second order; u~ and eps at
# first order.
CARM_TOL = {"fp64": {"u": 1e-9, "eps": 1e-8, "C": 1e-10},
            "mixed": {"u": 1e-6, "eps": 1e-6, "C": 1e-6}}


def _carm_case(kind, kw, ns, k_snap):
    p = small_problem(kind, mg_levels=3, n_on=6, n_parm=ns, n_carm=ns, eps_tol=10.0,
                      rtol=1e-12, **kw)
    t = aarmr.run(p, n_iter=k_snap, mode="aarmr", snapshot_at=(k_snap,))
    return p, t.snapshots[k_snap]


@pytest.mark.parametrize("kind,kw", PROBLEMS)
@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_carm_parity(kind, kw, precision):
    """CARM build + reduced solve (Eq. 15-29) on the oracle's own inputs at a
    CARM iteration of a real trajectory."""
    B = _B()
    p, s = _carm_case(kind, kw, 4, 9)
    g, KE = _model(p)
    K = fe.stiffness(g, s["E"], KE, p.fixed)
    Kr = fe.stiffness(g, s["E_prev"], KE, p.fixed)
    dK = fe.apply_bcs(fe.assemble(g, s["E"] - s["E_prev"], KE), p.fixed, diag_fixed=0.0)
    u_ref, eps_ref, Rt = reanalysis.aarmr_solve(lambda v: K @ v, lambda v: Kr @ v,
                                                lambda v: dK @ v, p.f, s["u_last"], s["Phi"],
                                                p.n_carm)
    with Ctx(p, precision=precision) as c:
        c.set_density(s["rho_phys_prev"])
        c.set_density(s["rho_phys"])
        for i in range(s["Phi"].shape[1]):
            B.to_parm_push(c.ctx, dev(s["Phi"][:, i]))
        B.to_carm_build(c.ctx, dev(s["u_last"]))
        _, k, _ = B.to_carm_info(c.ctx)
        u = dev(np.zeros(g.ndof))
        eps = B.to_carm_solve(c.ctx, u)
        u = host(u)
    # both sides keep the directions with sigma > 1e-6 sigma_1 (Eq. 21)
    assert k == Rt.shape[1], (k, Rt.shape[1])
    C, C_ref = p.f @ u, p.f @ u_ref
    tol = CARM_TOL[precision]
    assert np.linalg.norm(u - u_ref) <= tol["u"] * np.linalg.norm(u_ref)
    assert abs(eps - eps_ref) <= tol["eps"] * eps_ref
    assert abs(C - C_ref) <= tol["C"] * C_ref


@pytest.mark.parametrize("kind,kw", PROBLEMS[:2])
@pytest.mark.parametrize("precision", ["fp64", "mixed"])
@pytest.mark.parametrize("ns", [4, 10])
def test_carm_basis_orthonormal(kind, kw, precision, ns):
    """The orthonormalised CARM basis (Eq. 21) of a real trajectory:
    R~^T R~ = I to rounding, for the few- and many-column paths of the
    re-orthogonalising Gram-Schmidt."""
    B = _B()
    p, s = _carm_case(kind, kw, ns, ns + 5)
    with Ctx(p, precision=precision) as c:
        c.set_density(s["rho_phys_prev"])
        c.set_density(s["rho_phys"])
        for i in range(s["Phi"].shape[1]):
            B.to_parm_push(c.ctx, dev(s["Phi"][:, i]))
        B.to_carm_build(c.ctx, dev(s["u_last"]))
        err = B.to_carm_basis_error(c.ctx)
    assert err <= 1e-12, err


def test_carm_zero_change_gives_scaled_last_solution():
    """dK = 0 (same density twice): every r_i, i >= 2, vanishes and the
    reduced solution is the Rayleigh-Ritz multiple of u_last."""
    B = _B()
    p = small_problem("cantilever3d", nelx=8, nely=4, nelz=4, mg_levels=3, n_parm=3, n_carm=3)
    g, KE = _model(p)
    rho = rand_density(g.nel, 12, 0.2, 1.0)
    E = _E(p, rho)
    K = fe.stiffness(g, E, KE, p.fixed)
    u_last = solvers.direct_solve(fe.stiffness(g, 0.8 * E, KE, p.fixed), p.f, p.fixed)
    with Ctx(p, precision="fp64") as c:
        c.set_density(rho)
        c.set_density(rho)
        for i in range(3):
            B.to_parm_push(c.ctx, dev(rand_vector(g.ndof, 20 + i, fixed=p.fixed)))
        B.to_carm_build(c.ctx, dev(u_last))
        u = dev(np.zeros(g.ndof))
        eps = B.to_carm_solve(c.ctx, u)
        u = host(u)
    alpha = (p.f @ u_last) / (u_last @ (K @ u_last))
    assert np.linalg.norm(u - alpha * u_last) <= 1e-10 * np.linalg.norm(u)
    assert eps < 1e-8   # u_last is exact up to scaling


def test_carm_before_parm_full_is_state_error():
    B = _B()
    p = small_problem("cantilever3d", nelx=8, nely=4, nelz=4, mg_levels=3, n_parm=3, n_carm=3)
    with Ctx(p, precision="fp64") as c:
        c.set_density(np.full(p.nel, 0.5))
        with pytest.raises(B.TopoError) as e:
            B.to_carm_build(c.ctx, dev(np.zeros(p.ndof)))
        assert e.value.status == B.TO_E_STATE


def test_unclosed_supports_and_loaded_fixed_dofs_rejected():
    B = _B()
    p = small_problem("cantilever3d", nelx=8, nely=4, nelz=4, mg_levels=3)
    fixed = np.zeros(p.ndof, np.uint8)
    fixed[3 * (1 + 9 * 0) + 1] = 1        # node (1,0,0): odd x index, not a coarse node
    fixed[3 * 0: 3 * 0 + 3] = 1
    bad = p.with_(fixed=fixed)
    with pytest.raises(B.TopoError) as e:
        Ctx(bad, precision="fp64")
    assert e.value.status == B.TO_E_INVALID
    f = p.f.copy()
    f[0] = 1.0                           # node 0 is clamped
    with pytest.raises(B.TopoError) as e:
        Ctx(p.with_(f=f), precision="fp64")
    assert e.value.status == B.TO_E_INVALID


def test_two_level_tiny_mesh():
    B = _B()
    p = small_problem("cantilever3d", nelx=2, nely=2, nelz=2, mg_levels=2)
    g, KE = _model(p)
    rho = rand_density(g.nel, 13, 0.3, 1.0)
    K = fe.stiffness(g, _E(p, rho), KE, p.fixed)
    u_ref = solvers.direct_solve(K, p.f, p.fixed)
    with Ctx(p, precision="fp64") as c:
        c.set_density(rho)
        u = dev(np.zeros(g.ndof))
        it, rel, ok = B.to_mgcg_solve(c.ctx, 1e-13, 100, 0, u)
        u = host(u)
    assert ok
    assert np.linalg.norm(u - u_ref) <= 1e-10 * np.linalg.norm(u_ref)


def _compare_trajectories(p, n_iter, rel_c):
    from paper_2205_00385_gb300.driver import TopoSolver
    ref = aarmr.run(p, n_iter=n_iter, mode="aarmr")
    s = TopoSolver(p)
    try:
        hist = s.run(n_iter)
        rho = s.rho.cpu().numpy()
    finally:
        s.close()
    branches_gpu = [h.branch for h in hist]
    branches_ref = [h.branch for h in ref.history]
    for hg, hr in zip(hist, ref.history):
        if hg.branch != hr.branch:
            # only acceptable when eps sits on the threshold
            assert hr.eps is not None and abs(hr.eps - p.eps_tol) < 1e-6 * p.eps_tol
            break
        assert abs(hg.compliance - hr.compliance) <= rel_c * hr.compliance, (hg, hr)
    assert branches_gpu == branches_ref
    assert abs(hist[-1].compliance - ref.history[-1].compliance) <= 1e-3 * ref.history[-1].compliance
    return hist, ref, rho


def test_design_loop_mbb2d_60x20_fp64():
    """The 2D MBB workload (60 x 20, 50 iterations, s = 6) end to end."""
    from workloads import mbb2d_60x20
    p = mbb2d_60x20()
    hist, ref, rho = _compare_trajectories(p, p.n_iter, 1e-6)
    assert np.max(np.abs(rho - ref.rho)) < 1e-3


def test_design_loop_small_3d_mixed():
    p = small_problem("cantilever3d", nelx=16, nely=8, nelz=8, mg_levels=3, n_iter=14, n_on=8,
                      n_parm=4, n_carm=4, eps_tol=1e-2, precision="mixed")
    _compare_trajectories(p, p.n_iter, 1e-5)

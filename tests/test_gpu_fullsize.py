"""GPU parity at the workloads' full sizes, through the C ABI.

The element-by-element parity tests run grids the oracle finishes in
seconds.  These run the workloads' own sizes, in the configuration the
benchmark times (library contexts built from the same problem definitions),
and compare what the oracle can compute at that size: every entry where a
vectorised oracle pass takes seconds, sampled entries computed one by one
where it does not, and otherwise the conditions that define the result.

* 3D cantilever 192 x 96 x 96 (5,447,811 DOFs; mixed precision, 6 levels,
  s = 10):
  - every entry of K x, K_ref x and dK x in the float32 (the solver's own
    operator), double-float and float64 products;
  - the density and sensitivity filters, compliance, sensitivity and the
    OC update on seeded inputs, every entry;
  - an MGCG solve on a mid-optimisation design: its true residual under the
    oracle's operator, and its compliance against the float64 path's;
  - one CARM build and reduced solve (Eq. 15-29) at s = 10 with smooth
    synthetic PARM columns, in both precisions, against the oracle's CARM:
    kept directions, orthonormality, u~, eps and compliance.
* 3D bridge 320 x 160 x 160 (24,961,923 DOFs, r = 2.5; the largest
  workload): sampled entries of K x and of the sensitivity, every entry of
  both filters (the oracle's matrix-free form), an MGCG solve by its true
  residual, and the OC update by the conditions that define it: box and
  move limits, the volume constraint, and one multiplier for every element
  strictly inside its limits.
* 3D cantilever 48 x 24 x 24 (91,875 DOFs; float64, 4 levels): an MGCG
  solve against the oracle's MGCG (iteration count and compliance).

The tests run from the paths the small-grid tests already exercise (the
48 x 24 x 24 solve) to the largest grid (the bridge, last), and the file
runs after every other test file.
Tolerances are those of the small-grid parity tests, which depend on the
arithmetic per entry, not on the grid size.
"""

import numpy as np
import pytest

from gpu_helpers import Ctx, dev, host
from oracle import aarmr, fe, filters, oc, reanalysis, sensitivity, solvers
from workloads import (cantilever3d_48x24x24, cantilever3d_192x96x96, bridge3d_320x160x160,
                       rand_density, rand_vector, smooth_fields)

# the CARM parity tolerances of the small-grid tests, which depend on the
# arithmetic, not on the grid size
CARM_TOL = {"fp64": {"u": 1e-9, "eps": 1e-8, "C": 1e-10},
            "mixed": {"u": 1e-6, "eps": 1e-6, "C": 1e-6}}

pytestmark = pytest.mark.gpu


def _B():
    from paper_2205_00385_gb300 import binding as B
    return B


def _model(p):
    return fe.Grid.of(p), fe.element_stiffness(p.dim, p.nu)


def _E(p, rho_phys):
    return sensitivity.simp_modulus(rho_phys, p.E0, p.Emin, p.penal)


@pytest.fixture(scope="module")
def design48():
    """Physical density of the oracle's 48 x 24 x 24 cantilever after 8
    design iterations with MGCG solves: a mid-optimisation design (about a
    third of the elements below 0.05, a few percent above 0.5)."""
    p = cantilever3d_48x24x24()
    t = aarmr.run(p, n_iter=8, mode="mgcg", snapshot_at=(8,))
    return t.snapshots[8]["rho_phys"]


def _upsample(rho, nelx, nely, nelz, k):
    """Each element of an (nelx, nely, nelz) field repeated over a k^3 block."""
    r = rho.reshape(nelz, nely, nelx)
    return np.repeat(np.repeat(np.repeat(r, k, 0), k, 1), k, 2).ravel()


# ---------------------------------------------------------------------------
# 3D cantilever 48 x 24 x 24, float64 (4 levels)
# ---------------------------------------------------------------------------

def test_cantilever48_fp64_mgcg_against_oracle(design48):
    B = _B()
    p = cantilever3d_48x24x24()
    g, KE = _model(p)
    E = _E(p, design48)
    K = fe.stiffness(g, E, KE, p.fixed)
    mg = solvers.Multigrid(g, K, p.fixed, p.mg_levels)
    it_ref = solvers.mgcg(K, p.f, mg, rtol=p.rtol, maxit=p.maxit)[1]
    u_ref = solvers.mgcg(K, p.f, mg, rtol=1e-12, maxit=500)[0]
    C_ref = sensitivity.compliance(E, sensitivity.element_energy(g, KE, u_ref, p.fixed))
    with Ctx(p) as c:
        c.set_density(design48)
        u = dev(np.zeros(g.ndof))
        it, rel, ok = B.to_mgcg_solve(c.ctx, p.rtol, p.maxit, 0, u)
        u = host(u)
    assert ok and rel < p.rtol
    assert abs(it - it_ref) <= 1, (it, it_ref)
    C = sensitivity.compliance(E, sensitivity.element_energy(g, KE, u, p.fixed))
    assert abs(C - C_ref) <= 1e-10 * C_ref


# ---------------------------------------------------------------------------
# 3D cantilever 192 x 96 x 96, mixed precision (the benchmark's workload)
# ---------------------------------------------------------------------------

def test_cantilever192_stiffness_products():
    B = _B()
    p = cantilever3d_192x96x96("mixed")
    g, KE = _model(p)
    r_prev = rand_density(g.nel, 41, 0.0, 1.0)
    r_now = np.clip(r_prev + rand_density(g.nel, 42, -0.2, 0.2), 0.0, 1.0)
    x = rand_vector(g.ndof, 43)
    coefs = {B.TO_OP_K: _E(p, r_now), B.TO_OP_KREF: _E(p, r_prev)}
    coefs[B.TO_OP_DK] = coefs[B.TO_OP_K] - coefs[B.TO_OP_KREF]
    with Ctx(p) as c:
        c.set_density(r_prev)
        c.set_density(r_now)
        xd = dev(x)
        for op, coef in coefs.items():
            y_ref = fe.apply_ebe(g, coef, KE, x, p.fixed,
                                 diag_fixed=0.0 if op == B.TO_OP_DK else 1.0)
            y = {}
            for prec in (B.TO_PREC_FP32, B.TO_PREC_DF, B.TO_PREC_FP64):
                yd = dev(np.zeros(g.ndof))
                B.to_apply(c.ctx, op, prec, xd, yd)
                y[prec] = host(yd)
            scale = np.max(np.abs(y_ref))
            assert np.linalg.norm(y[B.TO_PREC_FP32] - y_ref) <= 1e-5 * np.linalg.norm(y_ref), op
            assert np.max(np.abs(y[B.TO_PREC_DF] - y_ref)) <= 1e-12 * scale, op
            assert np.max(np.abs(y[B.TO_PREC_FP64] - y_ref)) <= 1e-13 * scale, op


def test_cantilever192_filter_sensitivity_oc():
    B = _B()
    fabs_tol = 1e-14
    p = cantilever3d_192x96x96("mixed")
    g, KE = _model(p)
    H, Hs = filters.filter_matrix(g, p.rmin)
    rho = rand_density(g.nel, 44, 0.0, 2.0 * p.volfrac)
    rho_phys_ref = filters.density_filter(H, Hs, rho)
    u = rand_vector(g.ndof, 45, fixed=p.fixed)
    E = _E(p, rho_phys_ref)
    ce = sensitivity.element_energy(g, KE, u, p.fixed)
    C_ref = sensitivity.compliance(E, ce)
    dc_ref = sensitivity.compliance_sensitivity(rho_phys_ref, ce, p.E0, p.Emin, p.penal)
    dcf_ref = filters.sensitivity_filter(H, Hs, dc_ref)
    dvf_ref = filters.sensitivity_filter(H, Hs, np.ones(g.nel))
    rho_new_ref, _, change_ref = oc.oc_update(rho, dcf_ref, dvf_ref, H, Hs, p.volfrac, 0.2)
    with Ctx(p) as c:
        rp = dev(np.zeros(g.nel))
        B.to_filter(c.ctx, B.TO_FILTER_DENSITY, dev(rho), rp)
        assert np.max(np.abs(host(rp) - rho_phys_ref)) <= fabs_tol
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


def test_cantilever192_mgcg_solution(design48):
    """The mixed solve (float32 operator and V-cycle, double-float CG) and
    the float64 solve on the 192 x 96 x 96 grid, for the 48 x 24 x 24
    oracle design refined 4x in each direction.  The oracle cannot solve at
    this size; its operator gives the true residuals, its element sum the
    compliances, and the mixed compliance must be within 1e-6 of the
    float64 one (the float64 path is pinned to the oracle at 1e-10 on the
    smaller grids)."""
    B = _B()
    p = cantilever3d_192x96x96("mixed")
    g, KE = _model(p)
    rho = _upsample(design48, 48, 24, 24, 4)
    E = _E(p, rho)
    sol = {}
    for precision, rtol in (("mixed", p.rtol), ("fp64", 1e-10)):
        with Ctx(p, precision=precision) as c:
            c.set_density(rho)
            u = dev(np.zeros(g.ndof))
            it, rel, ok = B.to_mgcg_solve(c.ctx, rtol, 500, 0, u)
            assert ok and rel < rtol, (precision, it, rel)
            sol[precision] = host(u)
    fnorm = np.linalg.norm(p.f)
    for precision, tol in (("mixed", 1e-6), ("fp64", 1e-8)):
        r = p.f - fe.apply_ebe(g, E, KE, sol[precision], p.fixed)
        assert np.linalg.norm(r) / fnorm < tol, precision
    C = {k: sensitivity.compliance(E, sensitivity.element_energy(g, KE, v, p.fixed))
         for k, v in sol.items()}
    assert abs(C["mixed"] - C["fp64"]) <= 1e-6 * C["fp64"], C


def _carm_gpu(B, p, precision, r_prev, r_now, cols, u_last, g):
    """One CARM build + solve on the GPU; returns u~, eps, (kq, k, sigma)
    and the basis R~ downloaded as float64 columns."""
    with Ctx(p, precision=precision) as c:
        c.set_density(r_prev)
        c.set_density(r_now)
        for v in cols:
            B.to_parm_push(c.ctx, dev(v))
        B.to_carm_build(c.ctx, dev(u_last))
        info = B.to_carm_info(c.ctx, p.n_carm)
        Rt = []
        col = dev(np.zeros(g.ndof))
        for j in range(info[1]):
            B.to_carm_basis_column(c.ctx, j, col)
            Rt.append(host(col).copy())
        u = dev(np.zeros(g.ndof))
        eps = B.to_carm_solve(c.ctx, u)
        u = host(u)
    return u, eps, info, np.stack(Rt, axis=1)


def test_cantilever192_carm_parity():
    """One CARM build and solve at s = 10 (N_s = N_m = 10, the benchmark's
    setting) against the oracle's CARM on the same inputs, in both
    precisions.

    Inputs: the oracle cannot run a design trajectory at this size, so they
    come from its 48 x 24 x 24 trajectory with this workload's settings (the
    first CARM iteration, see carm_cases): the two physical densities
    repeated over 4 x 4 x 4 blocks, u_last and the ten PARM columns
    interpolated trilinearly twice.  The CA basis (Eq. 19-20) is
    numerically rank-deficient: its normalised singular values fall
    geometrically to ~1e-10.  Both sides drop the directions with
    sigma <= 1e-6 sigma_1 (Eq. 21) and keep the same ones.  Checked:

    * the kept count and the singular values of the kept directions
      (relative 1e-6: they are formed from the basis products, whose rounding
      the cancellation of K on smooth fields amplifies);
    * R~ orthonormal (Eq. 21), measured on the host in float64: classical
      Gram-Schmidt run twice leaves O(u) of non-orthogonality once every
      accepted column keeps more than 1e-10 of its norm, u being the basis
      arithmetic's unit roundoff (2^-53 float64, ~2^-48 double-float) times
      the dot products' accumulation length (~1e2); the rotation by the
      small SVD adds O(m u).  Bound: 1e-12;
    * u~, eps and the compliance against the oracle's (CARM_TOL of the
      small-grid parity test, taken at this size);
    * eps equals the true force residual of the returned u~ (Eq. 29), and
      the Galerkin identity f^T u~ = u~^T K u~ (Eq. 22-25).
    """
    from carm_cases import refine_element_field, refine_nodal_field, snapshot_48_s10
    B = _B()
    p = cantilever3d_192x96x96("mixed")
    g, KE = _model(p)
    p48, snap, _ = snapshot_48_s10()
    shape48 = (p48.nelx, p48.nely, p48.nelz)
    r_prev = refine_element_field(snap["rho_phys_prev"], shape48, 4)
    r_now = refine_element_field(snap["rho_phys"], shape48, 4)
    E, E_prev = _E(p, r_now), _E(p, r_prev)
    cols = [refine_nodal_field(snap["Phi"][:, i], shape48, 2) for i in range(p.n_parm)]
    u_last = refine_nodal_field(snap["u_last"], shape48, 2)
    assert not np.any(u_last[p.fixed.astype(bool)])
    Kx = lambda v: fe.apply_ebe(g, E, KE, v, p.fixed)
    Krx = lambda v: fe.apply_ebe(g, E_prev, KE, v, p.fixed)
    dKx = lambda v: fe.apply_ebe(g, E - E_prev, KE, v, p.fixed, diag_fixed=0.0)
    Phi = np.stack(cols, axis=1)
    KP = reanalysis.k_phi(Phi, Krx)
    R = reanalysis.carm_basis(u_last, Phi, KP, dKx, p.n_carm)
    sig_ref = np.linalg.svd(R / np.linalg.norm(R, axis=0), compute_uv=False)
    sig_ref = sig_ref / sig_ref[0]
    Rt_ref = reanalysis.orthonormalize(R)
    u_ref, _, eps_ref = reanalysis.reduced_solve(Kx, Rt_ref, p.f)
    C_ref = p.f @ u_ref
    fnorm = np.linalg.norm(p.f)
    # no singular value on the truncation edge (else the kept count is
    # decided by rounding and the comparison below is not defined)
    assert np.all(np.abs(sig_ref / 1e-6 - 1.0) > 1e-2), sig_ref
    for precision in ("mixed", "fp64"):
        u, eps, (kq, k, sig), Rt = _carm_gpu(B, p, precision, r_prev, r_now, cols, u_last, g)
        assert k == Rt_ref.shape[1], (precision, k, Rt_ref.shape[1], sig_ref)
        sig = np.asarray(sig) / sig[0]
        assert np.allclose(sig[:k], sig_ref[:k], rtol=1e-6, atol=0.0), (precision, sig, sig_ref)
        orth = np.max(np.abs(Rt.T @ Rt - np.eye(k)))
        tol = CARM_TOL[precision]
        du = np.linalg.norm(u - u_ref) / np.linalg.norm(u_ref)
        print(f"[carm 192 {precision}] k={k} kq={kq} du={du:.2e} deps={abs(eps - eps_ref) / eps_ref:.2e} "
              f"dC={abs(p.f @ u - C_ref) / C_ref:.2e} orth={orth:.2e}")
        assert orth <= 1e-12, (precision, orth)
        assert du <= tol["u"], (precision, du)
        assert abs(eps - eps_ref) <= tol["eps"] * eps_ref, (precision, eps, eps_ref)
        C = p.f @ u
        assert abs(C - C_ref) <= tol["C"] * C_ref, (precision, C, C_ref)
        eps_true = np.linalg.norm(Kx(u) - p.f) / fnorm
        assert abs(eps - eps_true) <= 1e-8 * eps_true, (precision, eps, eps_true)
        energy = sensitivity.compliance(E, sensitivity.element_energy(g, KE, u, p.fixed))
        assert abs(C - energy) <= 1e-8 * C, (precision, C, energy)


# ---------------------------------------------------------------------------
# 3D bridge 320 x 160 x 160, mixed precision (the largest workload)
# ---------------------------------------------------------------------------

def test_bridge320_largest_workload():
    B = _B()
    p = bridge3d_320x160x160()
    g, KE = _model(p)
    rng = np.random.default_rng(48)
    rows = rng.choice(g.ndof, 1 << 16, replace=False)
    elems = rng.choice(g.nel, 1 << 16, replace=False)
    Hs = filters.filter_weight_sums(g, p.rmin)
    rho = p.rho0
    rho_phys_ref = filters.density_filter_stencil(g, p.rmin, rho, Hs)
    E = _E(p, rho_phys_ref)
    x = rand_vector(g.ndof, 49)
    y_ref = fe.apply_ebe_rows(g, E, KE, x, p.fixed, rows)
    u_s = rand_vector(g.ndof, 50, fixed=p.fixed)
    dc_ref = sensitivity.compliance_sensitivity(
        rho_phys_ref[elems], sensitivity.element_energy_at(g, KE, u_s, p.fixed, elems),
        p.E0, p.Emin, p.penal)
    # a sensitivity field graded along x (x^4 over four decades, seeded noise), so
    # that the OC update clamps the elements at the stiff end at their upper limit
    ex = np.arange(g.nel) % g.nelx
    d = -((0.01 + ex / g.nelx) ** 4) * rand_density(g.nel, 51, 0.5, 1.0)
    dcf_ref = filters.sensitivity_filter_stencil(g, p.rmin, d, Hs)
    dvf_ref = filters.sensitivity_filter_stencil(g, p.rmin, np.ones(g.nel), Hs)
    with Ctx(p) as c:
        rp = dev(np.zeros(g.nel))
        B.to_filter(c.ctx, B.TO_FILTER_DENSITY, dev(rho), rp)
        assert np.max(np.abs(host(rp) - rho_phys_ref)) <= 1e-14
        c.set_density(rho_phys_ref)
        # K x in float32: the operator the mixed solver runs
        yd = dev(np.zeros(g.ndof))
        B.to_apply(c.ctx, B.TO_OP_K, B.TO_PREC_FP32, dev(x), yd)
        y = host(yd)[rows]
        assert np.linalg.norm(y - y_ref) <= 1e-5 * np.linalg.norm(y_ref)
        # compliance sensitivity (Eq. 6 / 34), sampled elements
        Cd = dev(np.zeros(1))
        dcd = dev(np.zeros(g.nel))
        B.to_sensitivity(c.ctx, dev(u_s), Cd, dcd)
        assert np.max(np.abs(host(dcd)[elems] - dc_ref)) <= 1e-10 * np.max(np.abs(dc_ref))
        # both filters, every element (81-point cone)
        dcf = dev(np.zeros(g.nel))
        B.to_filter(c.ctx, B.TO_FILTER_SENS, dev(d), dcf)
        assert np.max(np.abs(host(dcf) - dcf_ref)) <= 1e-12 * np.max(np.abs(dcf_ref))
        dvf = dev(np.zeros(g.nel))
        B.to_filter(c.ctx, B.TO_FILTER_SENS, dev(np.ones(g.nel)), dvf)
        assert np.max(np.abs(host(dvf) - dvf_ref)) <= 1e-14
        # MGCG on the workload's initial design, by its true residual
        u = dev(np.zeros(g.ndof))
        it, rel, ok = B.to_mgcg_solve(c.ctx, p.rtol, 500, 0, u)
        assert ok and rel < p.rtol, (it, rel)
        r = p.f - fe.apply_ebe(g, E, KE, host(u), p.fixed)
        assert np.linalg.norm(r) / np.linalg.norm(p.f) < 1e-6
        # OC update
        rd = dev(rho)
        ch = dev(np.zeros(1))
        B.to_oc_update(c.ctx, p.volfrac, 0.2, dev(dcf_ref), dev(dvf_ref), rd, ch)
        rho_new, change = host(rd), host(ch)[0]
    lo, hi = np.maximum(0.0, rho - 0.2), np.minimum(1.0, rho + 0.2)
    assert np.all(rho_new >= lo) and np.all(rho_new <= hi)
    assert change == np.max(np.abs(rho_new - rho))
    # volume of the filtered new design: sum_e (H rho)_e / Hs_e = dv_f . rho
    target = p.volfrac * g.nel
    assert abs(dvf_ref @ rho_new - target) <= 1e-9 * target
    # one multiplier: rho_new = rho sqrt(-dc_f / (lam dv_f)) strictly inside the limits
    inner = (rho_new > lo * (1 + 1e-9) + 1e-300) & (rho_new < hi * (1 - 1e-9))
    assert np.count_nonzero(inner) > 1000
    lam = -dcf_ref[inner] * rho[inner] ** 2 / (dvf_ref[inner] * rho_new[inner] ** 2)
    assert np.max(lam) <= np.min(lam) * (1 + 1e-10)
    lam0 = np.median(lam)
    cand = rho * np.sqrt(-dcf_ref / (lam0 * dvf_ref))
    at_lo, at_hi = rho_new == lo, rho_new == hi
    assert np.count_nonzero(at_hi) > 1000
    assert np.all(cand[at_lo] <= lo[at_lo] * (1 + 1e-9))
    assert np.all(cand[at_hi] >= hi[at_hi] * (1 - 1e-9))

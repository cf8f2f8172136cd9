"""CARM parity at the benchmark's basis size, s = N_s = N_m = 10, on a real
design trajectory of the oracle (3D cantilever 48 x 24 x 24 with the
192 x 96 x 96 workload's settings; see carm_cases).

At s = 10 the CA basis of Eq. 19-20 converges like a power iteration: the
singular values of its unit-length columns fall geometrically to ~1e-10 of
the largest.  Both sides drop the directions with sigma <= 1e-6 sigma_1
(Eq. 21), build the basis with float64-accurate products and must keep the
same directions; u~, eps and the compliance then agree within CARM_TOL (the
small-grid tolerances, which depend on the arithmetic only).
"""

import numpy as np
import pytest

from carm_cases import SNAP_K, snapshot_48_s10
from gpu_helpers import Ctx, dev, host
from oracle import fe, reanalysis

pytestmark = pytest.mark.gpu

CARM_TOL = {"fp64": {"u": 1e-9, "eps": 1e-8, "C": 1e-10},
            "mixed": {"u": 1e-6, "eps": 1e-6, "C": 1e-6}}


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_carm_s10_trajectory_snapshot(precision):
    from paper_2205_00385_gb300 import binding as B
    p, s, hist = snapshot_48_s10()
    g = fe.Grid.of(p)
    KE = fe.element_stiffness(3, p.nu)
    K = fe.stiffness(g, s["E"], KE, p.fixed)
    Kr = fe.stiffness(g, s["E_prev"], KE, p.fixed)
    dK = fe.apply_bcs(fe.assemble(g, s["E"] - s["E_prev"], KE), p.fixed, diag_fixed=0.0)
    KP = reanalysis.k_phi(s["Phi"], lambda v: Kr @ v)
    R = reanalysis.carm_basis(s["u_last"], s["Phi"], KP, lambda v: dK @ v, p.n_carm)
    sig_ref = np.linalg.svd(R / np.linalg.norm(R, axis=0), compute_uv=False)
    sig_ref = sig_ref / sig_ref[0]
    assert np.all(np.abs(sig_ref / 1e-6 - 1.0) > 1e-2), sig_ref   # no direction on the edge
    Rt_ref = reanalysis.orthonormalize(R)
    u_ref, _, eps_ref = reanalysis.reduced_solve(lambda v: K @ v, Rt_ref, p.f)
    # the trajectory's own CARM iteration saw the same eps
    assert hist[SNAP_K - 1].eps == pytest.approx(eps_ref, rel=1e-12)
    with Ctx(p, precision=precision) as c:
        c.set_density(s["rho_phys_prev"])
        c.set_density(s["rho_phys"])
        for i in range(p.n_parm):
            B.to_parm_push(c.ctx, dev(s["Phi"][:, i]))
        B.to_carm_build(c.ctx, dev(s["u_last"]))
        kq, k, sig = B.to_carm_info(c.ctx, p.n_carm)
        Rt = []
        col = dev(np.zeros(g.ndof))
        for j in range(k):
            B.to_carm_basis_column(c.ctx, j, col)
            Rt.append(host(col).copy())
        u = dev(np.zeros(g.ndof))
        eps = B.to_carm_solve(c.ctx, u)
        u = host(u)
    Rt = np.stack(Rt, axis=1)
    assert k == Rt_ref.shape[1], (k, Rt_ref.shape[1], sig_ref)
    sig = np.asarray(sig) / sig[0]
    assert np.allclose(sig[:k], sig_ref[:k], rtol=1e-6, atol=0.0), (sig, sig_ref)
    assert np.max(np.abs(Rt.T @ Rt - np.eye(k))) <= 1e-12
    # same span: the oracle's basis is reproduced by projecting onto the
    # GPU's; the smallest kept direction (sigma >= 1e-6 sigma_1) may turn by
    # the basis rounding over its sigma
    resid = Rt_ref - Rt @ (Rt.T @ Rt_ref)
    assert np.max(np.linalg.norm(resid, axis=0)) <= (1e-4 if precision == "mixed" else 1e-6)
    tol = CARM_TOL[precision]
    print(f"[carm s10 {precision}] k={k} kq={kq} du={np.linalg.norm(u - u_ref) / np.linalg.norm(u_ref):.2e} "
          f"deps={abs(eps - eps_ref) / eps_ref:.2e} dC={abs(p.f @ u - p.f @ u_ref) / (p.f @ u_ref):.2e} "
          f"orth={np.max(np.abs(Rt.T @ Rt - np.eye(k))):.2e} span={np.max(np.linalg.norm(resid, axis=0)):.2e}")
    assert np.linalg.norm(u - u_ref) <= tol["u"] * np.linalg.norm(u_ref)
    assert abs(eps - eps_ref) <= tol["eps"] * eps_ref, (eps, eps_ref)
    C, C_ref = p.f @ u, p.f @ u_ref
    assert abs(C - C_ref) <= tol["C"] * C_ref, (C, C_ref)

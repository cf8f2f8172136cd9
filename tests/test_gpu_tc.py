"""The finest-grid operator on the tensor cores (tcgen05, TO_OPERATOR_TENSOR_CORES)
against the oracle.

Per entry, the error bound follows the float32 one of the CUDA-core
operator scaled by the operand splitting: inputs and KE enter as two TF32
parts each (22 significant bits of 24), so the error of entry i stays below
~4e-6 of S_i = sum_e |E_e| max|KE| sum_(j in e) |x_j| (a lost or doubled
element contribution would be ~5e-3 of S_i).  Grids cover several tiles in
x and y with ragged edges, several z-chunks, every epilogue (K x, the
V-cycle's residual and smoother through a whole V-cycle) and a whole MGCG
solve with the operator inside CG and the V-cycle."""

import numpy as np
import pytest

from gpu_helpers import Ctx, dev, host
from oracle import fe, sensitivity, solvers
from workloads import rand_density, rand_vector, small_problem

pytestmark = pytest.mark.gpu


def _B():
    from paper_2205_00385_gb300 import binding as B
    return B


@pytest.mark.parametrize("kind,kw", [("cantilever3d", dict(nelx=38, nely=14, nelz=10)),
                                     ("bridge3d", dict(nelx=32, nely=16, nelz=20)),
                                     ("cantilever3d", dict(nelx=16, nely=8, nelz=4))])
@pytest.mark.parametrize("op", [0, 2])
def test_tc_apply_parity(kind, kw, op):
    B = _B()
    p = small_problem(kind, mg_levels=2, precision="mixed", **kw)
    g = fe.Grid.of(p)
    KE = fe.element_stiffness(3, p.nu)
    r_prev = rand_density(g.nel, 11, 0.0, 1.0)
    r_now = np.clip(r_prev + rand_density(g.nel, 12, -0.2, 0.2), 0, 1)
    E = lambda r: sensitivity.simp_modulus(r, p.E0, p.Emin, p.penal)
    coef = E(r_now) if op == 0 else E(r_now) - E(r_prev)
    x = rand_vector(g.ndof, 13)
    y_ref = fe.apply_ebe(g, coef, KE, x, p.fixed, diag_fixed=0.0 if op == 2 else 1.0)
    S = fe.apply_ebe(g, np.abs(coef), np.full_like(KE, np.max(np.abs(KE))), np.abs(x), p.fixed,
                     diag_fixed=1.0)
    with Ctx(p) as c:
        c.set_density(r_prev)
        c.set_density(r_now)
        B.to_operator_options(c.ctx, B.TO_OPERATOR_TENSOR_CORES)
        y = dev(np.zeros(g.ndof))
        B.to_apply(c.ctx, op, B.TO_PREC_FP32, dev(x), y)
        y = host(y)
        B.to_operator_options(c.ctx, 0)
        y32 = dev(np.zeros(g.ndof))
        B.to_apply(c.ctx, op, B.TO_PREC_FP32, dev(x), y32)
        y32 = host(y32)
    err = np.abs(y - y_ref) / S
    print(f"[tc apply {kind} {kw['nelx']} op{op}] max |err|/S = {err.max():.2e} "
          f"(CUDA cores {np.max(np.abs(y32 - y_ref) / S):.2e})")
    assert np.all(err <= 4e-6), err.max()


def test_tc_vcycle_and_mgcg():
    """A whole V-cycle and an MGCG solve with the operator in CG and in the
    V-cycle, on a design of the oracle's 48 x 24 x 24 trajectory (an
    unfiltered random design would defeat the float64 MGCG too)."""
    from carm_cases import snapshot_48_s10
    B = _B()
    p48, snap, _ = snapshot_48_s10()
    p = p48.with_(precision="mixed")
    g = fe.Grid.of(p)
    KE = fe.element_stiffness(3, p.nu)
    rho = snap["rho_phys"]
    E = sensitivity.simp_modulus(rho, p.E0, p.Emin, p.penal)
    K = fe.stiffness(g, E, KE, p.fixed)
    mg = solvers.Multigrid(g, K, p.fixed, p.mg_levels)
    r = rand_vector(g.ndof, 22, fixed=p.fixed)
    z_ref = mg.vcycle(r)
    u_ref, _, _ = solvers.mgcg(K, p.f, mg, rtol=1e-12, maxit=500)
    with Ctx(p) as c:
        c.set_density(rho)
        B.to_operator_options(c.ctx, B.TO_OPERATOR_TENSOR_CORES)
        z = dev(np.zeros(g.ndof))
        B.to_vcycle(c.ctx, dev(r), z)
        z = host(z)
        u = dev(np.zeros(g.ndof))
        it, rel, ok = B.to_mgcg_solve(c.ctx, 1e-8, 200, 0, u)
        u = host(u)
    # the float32 V-cycle's own tolerance (its coarsest inverse is float32)
    assert np.linalg.norm(z - z_ref) <= 2e-3 * np.linalg.norm(z_ref)
    print(f"[tc mgcg] iterations {it}, relres {rel:.2e}")
    assert ok and rel < 1e-8
    C, C_ref = p.f @ u, p.f @ u_ref
    assert abs(C - C_ref) <= 1e-6 * C_ref
    assert np.linalg.norm(p.f - K @ u) <= 1e-7 * np.linalg.norm(p.f)

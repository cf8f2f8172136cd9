"""Pins of the oracle's filter, sensitivity and OC update: brute-force
neighbour loops, closed-form neighbour counts, adjoint and fixed-point
identities, central finite differences and the volume constraint."""

import itertools

import numpy as np
import pytest

from oracle import fe, filters, oc, sensitivity, solvers
from workloads import small_problem


@pytest.mark.parametrize("dim,rmin,count", [(3, 1.5, 19), (3, 2.0, 27), (3, 2.5, 81),
                                            (2, 1.5, 9), (2, 2.5, 21)])
def test_filter_interior_stencil_size(dim, rmin, count):
    """Number of lattice offsets with distance < r (counted by hand:
    r=1.5 -> d^2 in {0,1,2}; r=2 -> {0..3}; r=2.5 -> {0..6})."""
    g = fe.Grid(dim, 9, 9, 9) if dim == 3 else fe.Grid(2, 9, 9)
    H, _ = filters.filter_matrix(g, rmin)
    centre = 4 + 9 * (4 + 9 * 4) if dim == 3 else 4 + 9 * 4
    assert H[centre].nnz == count


def test_filter_matches_bruteforce_loops():
    g = fe.Grid(3, 5, 4, 3)
    rmin = 2.0
    H, Hs = filters.filter_matrix(g, rmin)
    C = g.element_centers()
    Hb = np.zeros((g.nel, g.nel))
    for i in range(g.nel):
        for j in range(g.nel):
            d = np.sqrt(np.sum((C[i] - C[j]) ** 2))
            Hb[i, j] = max(0.0, rmin - d)
    assert np.allclose(H.toarray(), Hb, rtol=0, atol=1e-15)
    rho = np.random.default_rng(0).uniform(size=g.nel)
    ref = Hb @ rho / Hb.sum(axis=1)
    assert np.allclose(filters.density_filter(H, Hs, rho), ref, rtol=0, atol=1e-15)


def test_filter_fixed_point_rows_and_adjoint():
    g = fe.Grid(3, 6, 5, 4)
    H, Hs = filters.filter_matrix(g, 2.5)
    rng = np.random.default_rng(3)
    assert np.allclose(filters.density_filter(H, Hs, np.full(g.nel, 0.37)), 0.37, atol=1e-15)
    a, b = rng.standard_normal(g.nel), rng.standard_normal(g.nel)
    lhs = filters.density_filter(H, Hs, a) @ b
    rhs = a @ filters.sensitivity_filter(H, Hs, b)
    assert abs(lhs - rhs) < 1e-12 * (abs(lhs) + 1)
    assert np.allclose((H.toarray() / Hs[:, None]).sum(axis=1), 1.0, atol=1e-15)


@pytest.mark.parametrize("shape,rmin", [((3, 7, 5, 4), 1.5), ((3, 6, 5, 4), 2.0),
                                        ((3, 9, 4, 6), 2.5), ((3, 3, 2, 2), 3.0),
                                        ((2, 11, 6, 0), 1.5), ((2, 5, 8, 0), 2.5)])
def test_stencil_filter_equals_matrix_filter(shape, rmin):
    """The matrix-free filter (shifted-slice sums over the cone's offsets)
    gives the matrix filter's weight sums, filtered densities and filtered
    sensitivities, including grids thinner than the cone."""
    g = fe.Grid(*shape)
    H, Hs = filters.filter_matrix(g, rmin)
    rng = np.random.default_rng(11)
    rho, d = rng.uniform(size=g.nel), rng.standard_normal(g.nel)
    assert np.allclose(filters.filter_weight_sums(g, rmin), Hs, rtol=1e-15, atol=0)
    assert np.allclose(filters.density_filter_stencil(g, rmin, rho),
                       filters.density_filter(H, Hs, rho), rtol=1e-14, atol=0)
    assert np.allclose(filters.sensitivity_filter_stencil(g, rmin, d),
                       filters.sensitivity_filter(H, Hs, d), rtol=1e-13, atol=1e-15)


def test_simp_endpoints():
    E = sensitivity.simp_modulus(np.array([0.0, 1.0, 0.5]), 1.0, 1e-9, 3.0)
    assert E[0] == 1e-9 and E[1] == 1.0
    assert abs(E[2] - (1e-9 + (1 - 1e-9) * 0.125)) < 1e-16


def _exact_compliance(p, model_grid, KE, H, Hs, rho):
    rho_phys = filters.density_filter(H, Hs, rho)
    E = sensitivity.simp_modulus(rho_phys, p.E0, p.Emin, p.penal)
    K = fe.stiffness(model_grid, E, KE, p.fixed)
    u = solvers.direct_solve(K, p.f, p.fixed)
    ce = sensitivity.element_energy(model_grid, KE, u, p.fixed)
    return sensitivity.compliance(E, ce), rho_phys, ce, u


@pytest.mark.parametrize("kind", ["mbb2d", "cantilever3d"])
def test_sensitivity_matches_central_differences(kind):
    """Eq. 6 with the filter chain rule (Eq. 33) against central finite
    differences of C(rho) with exact solves."""
    if kind == "mbb2d":
        p = small_problem("mbb2d", nelx=6, nely=3)
    else:
        p = small_problem("cantilever3d", nelx=4, nely=2, nelz=2)
    g = fe.Grid.of(p)
    KE = fe.element_stiffness(p.dim, p.nu)
    H, Hs = filters.filter_matrix(g, p.rmin)
    rho = np.random.default_rng(4).uniform(0.3, 0.9, g.nel)
    C, rho_phys, ce, u = _exact_compliance(p, g, KE, H, Hs, rho)
    # energy sum equals f^T u for an exact solve
    assert abs(C - p.f @ u) < 1e-10 * C
    dc = sensitivity.compliance_sensitivity(rho_phys, ce, p.E0, p.Emin, p.penal)
    grad = filters.sensitivity_filter(H, Hs, dc)
    h = 1e-5
    for e in [0, g.nel // 3, g.nel - 1]:
        rp, rm = rho.copy(), rho.copy()
        rp[e] += h
        rm[e] -= h
        fd = (_exact_compliance(p, g, KE, H, Hs, rp)[0]
              - _exact_compliance(p, g, KE, H, Hs, rm)[0]) / (2 * h)
        assert abs(fd - grad[e]) < 1e-6 * abs(grad).max()


def test_oc_volume_limits_and_structure():
    g = fe.Grid(3, 6, 4, 4)
    H, Hs = filters.filter_matrix(g, 1.5)
    rng = np.random.default_rng(5)
    rho = rng.uniform(0.05, 0.5, g.nel)
    dc = -rng.uniform(0.1, 10.0, g.nel)
    dc_f = filters.sensitivity_filter(H, Hs, dc)
    dv_f = filters.sensitivity_filter(H, Hs, np.ones(g.nel))
    volfrac, move = 0.2, 0.2
    rho_new, lam, change = oc.oc_update(rho, dc_f, dv_f, H, Hs, volfrac, move)
    vol = filters.density_filter(H, Hs, rho_new).sum()
    assert abs(vol - volfrac * g.nel) < 1e-10 * volfrac * g.nel
    assert np.all(rho_new >= np.maximum(0, rho - move) - 1e-15)
    assert np.all(rho_new <= np.minimum(1, rho + move) + 1e-15)
    B = np.sqrt(-dc_f / (dv_f * lam))
    assert np.allclose(rho_new, np.clip(rho * B, np.maximum(0, rho - move),
                                        np.minimum(1, rho + move)), rtol=0, atol=1e-15)
    assert change == pytest.approx(np.max(np.abs(rho_new - rho)))
    # linearity of the filter: filtered volume = sum_j (H^T 1/Hs)_j rho_j
    assert abs(dv_f @ rho_new - vol) < 1e-10 * vol


def test_oc_uniform_stationary_point():
    """Uniform design with sensitivities proportional to the volume
    sensitivities is a fixed point of the update (lam = -dc/dv)."""
    g = fe.Grid(2, 10, 6)
    H, Hs = filters.filter_matrix(g, 1.5)
    dv_f = filters.sensitivity_filter(H, Hs, np.ones(g.nel))
    rho = np.full(g.nel, 0.4)
    rho_new, lam, _ = oc.oc_update(rho, -3.0 * dv_f, dv_f, H, Hs, 0.4, 0.2)
    assert np.allclose(rho_new, 0.4, atol=1e-12)
    assert lam == pytest.approx(3.0, rel=1e-10)

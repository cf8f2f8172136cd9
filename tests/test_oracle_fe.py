"""Pins of the oracle's finite-element layer against facts that do not come
from the oracle itself: exact symbolic integration, the classical closed-form
Q4 matrix, rigid-body null spaces, the patch test and brute-force loops."""

import itertools

import numpy as np
import pytest

from oracle import fe


def _sympy_ke(dim, nu):
    """KE by exact symbolic integration of B^T D B over the unit cell,
    using int_0^1 x^a dx = 1/(a+1) on each monomial."""
    sympy = pytest.importorskip("sympy")
    X = sympy.symbols("x0:%d" % dim)
    nn = 2 ** dim
    N = []
    for a in range(nn):
        expr = sympy.Integer(1)
        for d in range(dim):
            expr *= X[d] if (a >> d) & 1 else (1 - X[d])
        N.append(expr)
    dN = [[sympy.diff(N[a], X[d]) for d in range(dim)] for a in range(nn)]
    nu = sympy.Rational(nu).limit_denominator(1000)
    if dim == 2:
        D = sympy.Matrix([[1, nu, 0], [nu, 1, 0], [0, 0, (1 - nu) / 2]]) / (1 - nu ** 2)
        B = sympy.zeros(3, 2 * nn)
        for a in range(nn):
            B[0, 2 * a] = dN[a][0]
            B[1, 2 * a + 1] = dN[a][1]
            B[2, 2 * a] = dN[a][1]
            B[2, 2 * a + 1] = dN[a][0]
    else:
        lam = nu / ((1 + nu) * (1 - 2 * nu))
        mu = 1 / (2 * (1 + nu))
        D = sympy.zeros(6, 6)
        for i in range(3):
            for j in range(3):
                D[i, j] = lam
            D[i, i] = lam + 2 * mu
            D[3 + i, 3 + i] = mu
        B = sympy.zeros(6, 3 * nn)
        for a in range(nn):
            dx, dy, dz = dN[a]
            c = 3 * a
            B[0, c] = dx; B[1, c + 1] = dy; B[2, c + 2] = dz
            B[3, c] = dy; B[3, c + 1] = dx
            B[4, c + 1] = dz; B[4, c + 2] = dy
            B[5, c] = dz; B[5, c + 2] = dx
    integrand = (B.T * D * B).applyfunc(sympy.expand)
    out = np.zeros(integrand.shape)
    for i in range(integrand.shape[0]):
        for j in range(integrand.shape[1]):
            poly = sympy.Poly(integrand[i, j], *X)
            val = sympy.Integer(0)
            for powers, coeff in poly.terms():
                term = coeff
                for pw in powers:
                    term /= (pw + 1)
                val += term
            out[i, j] = float(val)
    return out


@pytest.mark.parametrize("dim", [2, 3])
def test_ke_matches_exact_symbolic_integration(dim):
    KE = fe.element_stiffness(dim, 0.3)
    ref = _sympy_ke(dim, 0.3)
    assert np.max(np.abs(KE - ref)) < 1e-14 * np.max(np.abs(ref))


def test_q4_matches_classical_closed_form():
    """The well-known plane-stress Q4 matrix for unit square elements
    (Sigmund's 99/88-line codes), nodes counter-clockwise from lower-left."""
    nu = 0.3
    k = [1 / 2 - nu / 6, 1 / 8 + nu / 8, -1 / 4 - nu / 12, -1 / 8 + 3 * nu / 8,
         -1 / 4 + nu / 12, -1 / 8 - nu / 8, nu / 6, 1 / 8 - 3 * nu / 8]
    idx = [[0, 1, 2, 3, 4, 5, 6, 7], [1, 0, 7, 6, 5, 4, 3, 2], [2, 7, 0, 5, 6, 3, 4, 1],
           [3, 6, 5, 0, 7, 2, 1, 4], [4, 5, 6, 7, 0, 1, 2, 3], [5, 4, 3, 2, 1, 0, 7, 6],
           [6, 3, 4, 1, 2, 7, 0, 5], [7, 2, 1, 4, 3, 6, 5, 0]]
    closed = np.array([[k[j] for j in row] for row in idx]) / (1 - nu ** 2)
    # counter-clockwise (LL, LR, UR, UL) = lexicographic corners (0, 1, 3, 2)
    perm = [0, 1, 2, 3, 6, 7, 4, 5]
    KE = fe.element_stiffness(2, nu)
    assert np.allclose(KE[np.ix_(perm, perm)], closed, rtol=0, atol=1e-15)


@pytest.mark.parametrize("dim", [2, 3])
def test_ke_symmetric_with_rigid_null_space(dim):
    KE = fe.element_stiffness(dim, 0.3)
    assert np.max(np.abs(KE - KE.T)) <= 1e-15 * np.max(np.abs(KE))
    w = np.linalg.eigvalsh(KE)
    nrigid = 3 if dim == 2 else 6
    lmax = w[-1]
    assert np.all(np.abs(w[:nrigid]) <= 1e-14 * lmax)
    assert np.all(w[nrigid:] > 1e-3 * lmax)
    coords = np.array([[(a >> d) & 1 for d in range(dim)] for a in range(2 ** dim)], float)
    Rb = fe.rigid_body_modes(dim, coords)
    assert np.max(np.abs(KE @ Rb)) <= 1e-14 * lmax


@pytest.mark.parametrize("dim", [2, 3])
def test_patch_test_uniform_tension(dim):
    """Rollers on the three (two) coordinate planes and a uniform traction
    sigma on the x = L face reproduce the exact linear field
    u_x = sigma x / E, u_y = -nu sigma y / E (, u_z = -nu sigma z / E)."""
    nu, E, sigma = 0.3, 2.5, 0.7
    g = fe.Grid(dim, 3, 2, 2) if dim == 3 else fe.Grid(2, 3, 2)
    KE = fe.element_stiffness(dim, nu)
    X = g.node_coords()
    fixed = np.zeros(g.ndof, np.uint8)
    for d in range(dim):
        fixed[dim * np.nonzero(X[:, d] == 0)[0] + d] = 1
    f = np.zeros(g.ndof)
    right = np.nonzero(X[:, 0] == g.nelx)[0]
    w = np.ones(right.size)
    for d, nel_d in ((1, g.nely), (2, g.nelz)):
        if d >= dim:
            continue
        edge = (X[right, d] == 0) | (X[right, d] == nel_d)
        w[edge] *= 0.5
    f[dim * right] = sigma * w
    K = fe.stiffness(g, np.full(g.nel, E), KE, fixed)
    u = np.linalg.solve(K.toarray(), f)
    exact = np.zeros(g.ndof)
    exact[0::dim] = sigma * X[:, 0] / E
    for d in range(1, dim):
        exact[d::dim] = -nu * sigma * X[:, d] / E
    assert np.max(np.abs(u - exact)) < 1e-12


def test_interior_nodes_in_equilibrium_under_linear_field():
    g = fe.Grid(3, 3, 3, 3)
    KE = fe.element_stiffness(3, 0.25)
    X = g.node_coords()
    rng = np.random.default_rng(0)
    G = rng.standard_normal((3, 3))
    u = (X @ G.T).ravel()                                 # u(x) = G x, interleaved
    r = fe.assemble(g, np.ones(g.nel), KE) @ u
    interior = np.all((X > 0) & (X < 3), axis=1)
    for c in range(3):
        assert np.max(np.abs(r[3 * np.nonzero(interior)[0] + c])) < 1e-12


@pytest.mark.parametrize("dim", [2, 3])
def test_assembly_symmetric_rigid_and_spd(dim):
    g = fe.Grid(dim, 4, 3, 2) if dim == 3 else fe.Grid(2, 5, 3)
    KE = fe.element_stiffness(dim, 0.3)
    E = np.random.default_rng(1).uniform(0.1, 1.0, g.nel)
    K = fe.assemble(g, E, KE)
    assert abs(K - K.T).max() <= 1e-15 * abs(K).max()
    Rb = fe.rigid_body_modes(dim, g.node_coords())
    assert np.max(np.abs(K @ Rb)) < 1e-12
    fixed = np.zeros(g.ndof, np.uint8)
    X = g.node_coords()
    left = np.nonzero(X[:, 0] == 0)[0]
    for c in range(dim):
        fixed[dim * left + c] = 1
    Kb = fe.apply_bcs(K, fixed).toarray()
    np.linalg.cholesky(Kb)                                # raises if not SPD


@pytest.mark.parametrize("dim", [2, 3])
def test_ebe_apply_equals_csr_and_bruteforce(dim):
    g = fe.Grid(dim, 3, 2, 2) if dim == 3 else fe.Grid(2, 4, 3)
    KE = fe.element_stiffness(dim, 0.3)
    rng = np.random.default_rng(2)
    E = rng.uniform(0.01, 1.0, g.nel)
    x = rng.standard_normal(g.ndof)
    fixed = (rng.uniform(size=g.ndof) < 0.2).astype(np.uint8)
    y_csr = fe.apply_bcs(fe.assemble(g, E, KE), fixed) @ x
    y_ebe = fe.apply_ebe(g, E, KE, x, fixed)
    # brute force: explicit loops over elements and local DOFs
    y_bf = np.zeros(g.ndof)
    ed = g.element_dofs()
    for e in range(g.nel):
        for a in range(ed.shape[1]):
            ia = ed[e, a]
            if fixed[ia]:
                continue
            s = 0.0
            for b in range(ed.shape[1]):
                ib = ed[e, b]
                if not fixed[ib]:
                    s += E[e] * KE[a, b] * x[ib]
            y_bf[ia] += s
    y_bf[fixed == 1] = x[fixed == 1]
    assert np.allclose(y_csr, y_bf, rtol=0, atol=1e-13)
    assert np.allclose(y_ebe, y_bf, rtol=0, atol=1e-13)
    # dK form: identity rows cancel
    y0 = fe.apply_ebe(g, E, KE, x, fixed, diag_fixed=0.0)
    assert np.all(y0[fixed == 1] == 0.0)


@pytest.mark.parametrize("shape", [(3, 5, 3, 4), (3, 1, 2, 1), (2, 6, 5, 0), (2, 1, 1, 0)])
def test_sampled_outputs_equal_full_products(shape):
    """The per-row apply, per-element DOF table and per-element energy used
    for sampled checks on large grids give the full products' entries, for
    every row in a shuffled order (corner, edge, face and interior nodes,
    fixed and free DOFs, identity and zero diagonals)."""
    from oracle import sensitivity
    g = fe.Grid(*shape)
    dim = g.dim
    KE = fe.element_stiffness(dim, 0.3)
    rng = np.random.default_rng(9)
    E = rng.uniform(0.01, 1.0, g.nel)
    x = rng.standard_normal(g.ndof)
    fixed = (rng.uniform(size=g.ndof) < 0.25).astype(np.uint8)
    rows = rng.permutation(g.ndof)
    for d in (1.0, 0.0):
        full = fe.apply_ebe(g, E, KE, x, fixed, diag_fixed=d)
        part = fe.apply_ebe_rows(g, E, KE, x, fixed, rows, diag_fixed=d)
        assert np.allclose(part, full[rows], rtol=0, atol=1e-13)
    elems = rng.permutation(g.nel)
    assert np.array_equal(g.dofs_of(elems), g.element_dofs()[elems])
    ce = sensitivity.element_energy(g, KE, x, fixed)
    assert np.allclose(sensitivity.element_energy_at(g, KE, x, fixed, elems), ce[elems],
                       rtol=1e-14, atol=0)


def test_grid_numbering_conventions():
    g = fe.Grid(3, 4, 3, 2)
    en = g.element_nodes()
    e = 1 + 4 * (2 + 3 * 1)                     # element (1, 2, 1)
    for a in range(8):
        bx, by, bz = a & 1, (a >> 1) & 1, (a >> 2) & 1
        assert en[e, a] == (1 + bx) + 5 * ((2 + by) + 4 * (1 + bz))
    assert g.ndof == 3 * 5 * 4 * 3

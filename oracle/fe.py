"""Finite-element pieces of the oracle: element stiffness, grid numbering,
assembled stiffness, boundary conditions.

Paper: the design domain is a regular grid of unit Q4 (plane stress) or hex8
elements whose Young's modulus follows the modified SIMP law of Eq. 1; the
equilibrium equation K(rho~) u = f of Eq. 3 / Eq. 7 uses the assembled global
stiffness matrix.  Element size 1 and plane stress are stated in Sec. 4.1.1
and Sec. 4.2.

Local node ordering inside an element is lexicographic: local node
``a = bx + 2*by + 4*bz`` sits at corner (bx, by, bz) of the unit cell, and its
local DOF c has local index ``dim*a + c``.
"""

from __future__ import annotations

import numpy as np
import scipy.sparse as sp


# ----------------------------------------------------------------------------
# Element stiffness by 2-point Gauss quadrature (exact for bilinear/trilinear
# shape functions on a unit cell, whose Jacobian is the identity).
# ----------------------------------------------------------------------------

def gauss_rule_unit():
    """Two-point Gauss-Legendre rule on [0, 1]."""
    g = 0.5 / np.sqrt(3.0)
    return np.array([0.5 - g, 0.5 + g]), np.array([0.5, 0.5])


def elasticity_matrix(dim: int, E: float, nu: float) -> np.ndarray:
    """Isotropic constitutive matrix in Voigt form.

    2D is plane stress (strain order xx, yy, xy); 3D uses the strain order
    xx, yy, zz, xy, yz, zx with engineering shear strains."""
    if dim == 2:
        return E / (1.0 - nu * nu) * np.array([[1.0, nu, 0.0],
                                               [nu, 1.0, 0.0],
                                               [0.0, 0.0, (1.0 - nu) / 2.0]])
    lam = E * nu / ((1.0 + nu) * (1.0 - 2.0 * nu))
    mu = E / (2.0 * (1.0 + nu))
    D = np.zeros((6, 6))
    D[:3, :3] = lam
    D[0, 0] = D[1, 1] = D[2, 2] = lam + 2.0 * mu
    D[3, 3] = D[4, 4] = D[5, 5] = mu
    return D


def shape_gradients(dim: int, xi) -> np.ndarray:
    """Gradients dN_a/dx_d of the multilinear shape functions at point xi of
    the unit cell; returns an array (2**dim, dim)."""
    nn = 2 ** dim
    G = np.zeros((nn, dim))
    for a in range(nn):
        bits = [(a >> d) & 1 for d in range(dim)]
        for d in range(dim):
            v = 1.0
            for dd in range(dim):
                if dd == d:
                    v *= 1.0 if bits[dd] else -1.0
                else:
                    v *= xi[dd] if bits[dd] else (1.0 - xi[dd])
            G[a, d] = v
    return G


def strain_displacement(dim: int, xi) -> np.ndarray:
    """B matrix mapping the element's nodal displacements to Voigt strain."""
    G = shape_gradients(dim, xi)
    nn = 2 ** dim
    if dim == 2:
        B = np.zeros((3, 2 * nn))
        for a in range(nn):
            dx, dy = G[a]
            B[0, 2 * a] = dx
            B[1, 2 * a + 1] = dy
            B[2, 2 * a] = dy
            B[2, 2 * a + 1] = dx
        return B
    B = np.zeros((6, 3 * nn))
    for a in range(nn):
        dx, dy, dz = G[a]
        c = 3 * a
        B[0, c] = dx
        B[1, c + 1] = dy
        B[2, c + 2] = dz
        B[3, c] = dy
        B[3, c + 1] = dx
        B[4, c + 1] = dz
        B[4, c + 2] = dy
        B[5, c] = dz
        B[5, c + 2] = dx
    return B


def element_stiffness(dim: int, nu: float, E: float = 1.0) -> np.ndarray:
    """Unit-modulus element stiffness KE = sum_q w_q B_q^T D B_q."""
    pts, wts = gauss_rule_unit()
    D = elasticity_matrix(dim, E, nu)
    nd = dim * 2 ** dim
    KE = np.zeros((nd, nd))
    if dim == 2:
        for i, x in enumerate(pts):
            for j, y in enumerate(pts):
                B = strain_displacement(2, (x, y))
                KE += wts[i] * wts[j] * B.T @ D @ B
    else:
        for i, x in enumerate(pts):
            for j, y in enumerate(pts):
                for k, z in enumerate(pts):
                    B = strain_displacement(3, (x, y, z))
                    KE += wts[i] * wts[j] * wts[k] * B.T @ D @ B
    return KE


def rigid_body_modes(dim: int, coords: np.ndarray) -> np.ndarray:
    """Columns: translations and infinitesimal rotations evaluated at the
    given node coordinates (nnode, dim), interleaved per node."""
    nn = coords.shape[0]
    if dim == 2:
        R = np.zeros((2 * nn, 3))
        R[0::2, 0] = 1.0
        R[1::2, 1] = 1.0
        R[0::2, 2] = -coords[:, 1]
        R[1::2, 2] = coords[:, 0]
        return R
    R = np.zeros((3 * nn, 6))
    x, y, z = coords[:, 0], coords[:, 1], coords[:, 2]
    for c in range(3):
        R[c::3, c] = 1.0
    R[0::3, 3], R[1::3, 3] = -y, x       # rotation about z
    R[1::3, 4], R[2::3, 4] = -z, y       # rotation about x
    R[2::3, 5], R[0::3, 5] = -x, z       # rotation about y
    return R


# ----------------------------------------------------------------------------
# Grid numbering (the conventions of workloads/problems.py)
# ----------------------------------------------------------------------------

class Grid:
    """Regular grid of unit elements with x-fastest numbering."""

    def __init__(self, dim: int, nelx: int, nely: int, nelz: int = 0):
        self.dim = dim
        self.nelx, self.nely, self.nelz = nelx, nely, (nelz if dim == 3 else 0)
        self.npe = 2 ** dim
        if dim == 2:
            self.nel = nelx * nely
            self.nn = (nelx + 1) * (nely + 1)
        else:
            self.nel = nelx * nely * nelz
            self.nn = (nelx + 1) * (nely + 1) * (nelz + 1)
        self.ndof = dim * self.nn

    @classmethod
    def of(cls, prob) -> "Grid":
        return cls(prob.dim, prob.nelx, prob.nely, prob.nelz)

    def node(self, i, j, k=0):
        return i + (self.nelx + 1) * (j + (self.nely + 1) * k)

    def element_ijk(self):
        e = np.arange(self.nel)
        ex = e % self.nelx
        ey = (e // self.nelx) % self.nely
        if self.dim == 2:
            return ex, ey, np.zeros_like(ex)
        ez = e // (self.nelx * self.nely)
        return ex, ey, ez

    def element_nodes(self) -> np.ndarray:
        """(nel, 2**dim) global node of each local corner a = bx+2by+4bz."""
        ex, ey, ez = self.element_ijk()
        out = np.empty((self.nel, self.npe), dtype=np.int64)
        for a in range(self.npe):
            bx, by, bz = a & 1, (a >> 1) & 1, (a >> 2) & 1
            out[:, a] = self.node(ex + bx, ey + by, ez + bz)
        return out

    def element_dofs(self) -> np.ndarray:
        """(nel, dim*2**dim) global DOF of each local DOF dim*a + c."""
        en = self.element_nodes()
        d = self.dim
        out = np.empty((self.nel, d * self.npe), dtype=np.int64)
        for a in range(self.npe):
            for c in range(d):
                out[:, d * a + c] = d * en[:, a] + c
        return out

    def dofs_of(self, elems) -> np.ndarray:
        """Rows of ``element_dofs()`` for the given elements only (for grids
        whose full table would be large)."""
        e = np.asarray(elems, dtype=np.int64)
        ex = e % self.nelx
        ey = (e // self.nelx) % self.nely
        ez = e // (self.nelx * self.nely) if self.dim == 3 else np.zeros_like(e)
        d = self.dim
        out = np.empty((e.size, d * self.npe), dtype=np.int64)
        for a in range(self.npe):
            bx, by, bz = a & 1, (a >> 1) & 1, (a >> 2) & 1
            n = self.node(ex + bx, ey + by, ez + bz)
            for c in range(d):
                out[:, d * a + c] = d * n + c
        return out

    def element_centers(self) -> np.ndarray:
        ex, ey, ez = self.element_ijk()
        if self.dim == 2:
            return np.stack([ex + 0.5, ey + 0.5], axis=1)
        return np.stack([ex + 0.5, ey + 0.5, ez + 0.5], axis=1)

    def node_coords(self) -> np.ndarray:
        n = np.arange(self.nn)
        i = n % (self.nelx + 1)
        j = (n // (self.nelx + 1)) % (self.nely + 1)
        if self.dim == 2:
            return np.stack([i, j], axis=1).astype(float)
        k = n // ((self.nelx + 1) * (self.nely + 1))
        return np.stack([i, j, k], axis=1).astype(float)


# ----------------------------------------------------------------------------
# Assembled stiffness and boundary conditions
# ----------------------------------------------------------------------------

def assemble(grid: Grid, coef: np.ndarray, KE: np.ndarray) -> sp.csr_matrix:
    """K = sum_e coef_e A_e^T KE A_e (no boundary conditions)."""
    edofs = grid.element_dofs()
    nd = edofs.shape[1]
    rows = np.repeat(edofs, nd, axis=1).ravel()
    cols = np.tile(edofs, (1, nd)).ravel()
    vals = (coef[:, None] * KE.ravel()[None, :]).ravel()
    K = sp.coo_matrix((vals, (rows, cols)), shape=(grid.ndof, grid.ndof)).tocsr()
    K.sum_duplicates()
    return K


def mask_matrix(fixed: np.ndarray) -> sp.dia_matrix:
    """M = diag(1 - fixed): zeroes the prescribed DOFs."""
    return sp.diags(1.0 - fixed.astype(float))


def apply_bcs(K: sp.spmatrix, fixed: np.ndarray, diag_fixed: float = 1.0) -> sp.csr_matrix:
    """Prescribed zero displacements: rows and columns of fixed DOFs are
    replaced by ``diag_fixed`` times the identity, K_bc = M K M + d (I - M).
    With f = 0 on fixed DOFs the solution equals that of the system with
    the fixed DOFs eliminated."""
    M = mask_matrix(fixed)
    I_fixed = sp.diags(diag_fixed * fixed.astype(float))
    return (M @ K @ M + I_fixed).tocsr()


def stiffness(grid: Grid, E: np.ndarray, KE: np.ndarray, fixed: np.ndarray) -> sp.csr_matrix:
    """Global stiffness K(E) with boundary conditions applied."""
    return apply_bcs(assemble(grid, E, KE), fixed)


def apply_ebe(grid: Grid, coef: np.ndarray, KE: np.ndarray, x: np.ndarray,
              fixed: np.ndarray, diag_fixed: float = 1.0) -> np.ndarray:
    """Element-by-element product y = M (sum_e coef_e A_e^T KE A_e) M x
    + diag_fixed (I - M) x.  Same operator as ``apply_bcs(assemble(...))``
    without forming the matrix (used for sizes where assembly is heavy)."""
    m = 1.0 - fixed.astype(float)
    xm = x * m
    edofs = grid.element_dofs()
    xe = xm[edofs]                                  # (nel, nd)
    ye = coef[:, None] * (xe @ KE.T)                # KE symmetric
    y = np.bincount(edofs.ravel(), weights=ye.ravel(), minlength=grid.ndof)
    return y * m + diag_fixed * fixed.astype(float) * x


def apply_ebe_rows(grid: Grid, coef: np.ndarray, KE: np.ndarray, x: np.ndarray,
                   fixed: np.ndarray, rows, diag_fixed: float = 1.0) -> np.ndarray:
    """Selected entries of ``apply_ebe``: for DOF i = dim*node + c,
    y_i = m_i sum_e coef_e (KE A_e M x)_(local index of i in e) + diag_fixed (1 - m_i) x_i,
    the sum running over the (up to 2**dim) elements that share the node.
    Used where only sampled outputs of a large grid are compared."""
    rows = np.asarray(rows, dtype=np.int64)
    d = grid.dim
    m = 1.0 - fixed.astype(float)
    xm = x * m
    node, comp = rows // d, rows % d
    nx1, ny1 = grid.nelx + 1, grid.nely + 1
    ix, iy, iz = node % nx1, (node // nx1) % ny1, node // (nx1 * ny1)
    nz = grid.nelz if d == 3 else 1
    y = np.zeros(rows.size)
    for a in range(grid.npe):
        bx, by, bz = a & 1, (a >> 1) & 1, (a >> 2) & 1
        ex, ey, ez = ix - bx, iy - by, iz - bz
        ok = (ex >= 0) & (ex < grid.nelx) & (ey >= 0) & (ey < grid.nely) & (ez >= 0) & (ez < nz)
        if not np.any(ok):
            continue
        e = ex[ok] + grid.nelx * (ey[ok] + grid.nely * ez[ok])
        dofs = grid.dofs_of(e)                                 # (s, nd)
        ke_rows = KE[d * a + comp[ok]]                         # (s, nd)
        y[ok] += coef[e] * np.sum(ke_rows * xm[dofs], axis=1)
    return y * m[rows] + diag_fixed * fixed[rows].astype(float) * x[rows]

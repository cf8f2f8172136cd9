"""Linear solvers of the oracle: direct solve, preconditioned CG, the V-cycle
multigrid of Algorithm 2 and MGCG (CG preconditioned by one V-cycle, the
method the paper takes from ref. [5], Sec. 3.1 and Sec. 4).

Readings of what Algorithm 2 leaves open:
* "grid level k" counts all grids including the finest; each coarser grid
  halves the element count per axis (so every nel must be divisible by
  2**(levels-1));
* P is bilinear (2D) / trilinear (3D) interpolation, applied per
  displacement component; the coarse operator is the Galerkin product
  P^T K P of Algorithm 2's coarse-grid step, with boundary conditions
  carried as
  A_{l+1} = Pm^T A_l Pm + (I - M_{l+1}), Pm = M_l P M_{l+1}, where a coarse
  DOF is fixed iff the coincident fine DOF is fixed;
* smoothing is damped Jacobi (the pre- and post-smoothing steps) with
  omega = 0.6 and one sweep each; the coarsest grid is solved exactly;
* the pre-smoothing step's "f - K u0" is read as "f - K u" (the current
  iterate);
* MGCG stops when ||r|| / ||f|| < rtol or after maxit iterations, returning
  the last iterate in both cases (Sec. 4.1).
"""

from __future__ import annotations

import numpy as np
import scipy.linalg as sla
import scipy.sparse as sp
import scipy.sparse.linalg as spla

from .fe import Grid


def direct_solve(K_bc: sp.spmatrix, f: np.ndarray, fixed: np.ndarray) -> np.ndarray:
    """Exact solution of K u = f with the fixed DOFs eliminated."""
    free = np.nonzero(fixed == 0)[0]
    Kff = K_bc.tocsr()[free][:, free].tocsc()
    u = np.zeros_like(f)
    u[free] = spla.spsolve(Kff, f[free])
    return u


def pcg(A, b, precond=None, x0=None, rtol=1e-8, maxit=200):
    """Preconditioned conjugate gradients (Hestenes-Stiefel form).

    A and precond are callables (or matrices).  Returns (x, iters, relres)
    where relres = ||b - A x|| / ||b|| by the recursively updated residual."""
    Aop = A if callable(A) else (lambda v: A @ v)
    Mop = precond if precond is not None else (lambda v: v.copy())
    x = np.zeros_like(b) if x0 is None else x0.astype(float).copy()
    bnorm = np.linalg.norm(b)
    if bnorm == 0.0:
        return np.zeros_like(b), 0, 0.0
    r = b - Aop(x)
    rel = np.linalg.norm(r) / bnorm
    if rel < rtol:
        return x, 0, rel
    z = Mop(r)
    p = z.copy()
    rz = r @ z
    for it in range(1, maxit + 1):
        q = Aop(p)
        alpha = rz / (p @ q)
        x += alpha * p
        r -= alpha * q
        rel = np.linalg.norm(r) / bnorm
        if rel < rtol:
            return x, it, rel
        z = Mop(r)
        rz_new = r @ z
        p = z + (rz_new / rz) * p
        rz = rz_new
    return x, maxit, rel


# ----------------------------------------------------------------------------
# Multigrid hierarchy
# ----------------------------------------------------------------------------

def interpolation_1d(nc_el: int) -> sp.csr_matrix:
    """1D linear interpolation from nc_el+1 coarse nodes to 2*nc_el+1 fine nodes."""
    nf = 2 * nc_el + 1
    rows, cols, vals = [], [], []
    for i in range(nf):
        if i % 2 == 0:
            rows.append(i); cols.append(i // 2); vals.append(1.0)
        else:
            rows += [i, i]; cols += [(i - 1) // 2, (i + 1) // 2]; vals += [0.5, 0.5]
    return sp.csr_matrix((vals, (rows, cols)), shape=(nf, nc_el + 1))


def interpolation(fine: Grid) -> sp.csr_matrix:
    """Nodal multilinear interpolation P from the 2x coarser grid to ``fine``,
    expanded to interleaved displacement DOFs."""
    Px = interpolation_1d(fine.nelx // 2)
    Py = interpolation_1d(fine.nely // 2)
    if fine.dim == 2:
        Pn = sp.kron(Py, Px)                  # node index i + (nx+1) j
    else:
        Pz = interpolation_1d(fine.nelz // 2)
        Pn = sp.kron(Pz, sp.kron(Py, Px))     # node index i + (nx+1)(j + (ny+1)k)
    return sp.kron(Pn, sp.identity(fine.dim)).tocsr()


def coarse_grid(g: Grid) -> Grid:
    return Grid(g.dim, g.nelx // 2, g.nely // 2, g.nelz // 2 if g.dim == 3 else 0)


def coarse_fixed(fine: Grid, coarse: Grid, fixed: np.ndarray) -> np.ndarray:
    """A coarse DOF is fixed iff the coincident fine DOF is fixed."""
    cn = coarse.node_coords().astype(np.int64)
    if fine.dim == 2:
        fn = fine.node(2 * cn[:, 0], 2 * cn[:, 1])
    else:
        fn = fine.node(2 * cn[:, 0], 2 * cn[:, 1], 2 * cn[:, 2])
    out = np.zeros(coarse.ndof, np.uint8)
    for c in range(fine.dim):
        out[fine.dim * np.arange(coarse.nn) + c] = fixed[fine.dim * fn + c]
    return out


class Multigrid:
    """Galerkin hierarchy of Algorithm 2 for the BC operator A_0."""

    def __init__(self, grid: Grid, A0: sp.spmatrix, fixed: np.ndarray, levels: int,
                 omega: float = 0.6, nu1: int = 1, nu2: int = 1):
        self.omega, self.nu1, self.nu2 = omega, nu1, nu2
        self.grids = [grid]
        self.fixed = [fixed.astype(np.uint8)]
        self.A = [A0.tocsr()]
        self.P = []
        for _ in range(levels - 1):
            g = self.grids[-1]
            gc = coarse_grid(g)
            fc = coarse_fixed(g, gc, self.fixed[-1])
            Pm = (sp.diags(1.0 - self.fixed[-1]) @ interpolation(g)
                  @ sp.diags(1.0 - fc.astype(float))).tocsr()
            Ac = (Pm.T @ self.A[-1] @ Pm + sp.diags(fc.astype(float))).tocsr()
            self.grids.append(gc)
            self.fixed.append(fc)
            self.P.append(Pm)
            self.A.append(Ac)
        self.D = [A.diagonal().copy() for A in self.A]
        self.coarse_factor = sla.cho_factor(self.A[-1].toarray())

    @property
    def levels(self) -> int:
        return len(self.A)

    def smooth(self, l, x, b):
        return x + self.omega * (b - self.A[l] @ x) / self.D[l]

    def vcycle(self, b, l=0):
        """One V-cycle approximating A_l^{-1} b from a zero initial guess."""
        if l == self.levels - 1:
            return sla.cho_solve(self.coarse_factor, b)
        x = np.zeros_like(b)
        for _ in range(self.nu1):
            x = self.smooth(l, x, b)                         # pre-smoothing
        e = self.P[l].T @ (b - self.A[l] @ x)                # restricted residual
        uc = self.vcycle(e, l + 1)                           # coarse-grid solve
        x = x + self.P[l] @ uc                               # interpolation
        for _ in range(self.nu2):
            x = self.smooth(l, x, b)                         # post-smoothing
        return x


def mgcg(A0, f, mg: Multigrid, x0=None, rtol=1e-8, maxit=200):
    """MGCG: PCG on A0 with one V-cycle as the preconditioner."""
    return pcg(A0, f, precond=mg.vcycle, x0=x0, rtol=rtol, maxit=maxit)

"""Density filter and its transpose (Eq. 2, Eq. 31-33).

Eq. 31: rho~_i = sum_j w_ij rho_j / sum_j w_ij over the elements j whose
centre lies within distance r of the centre of element i.
Eq. 32: w_ij = max(0, r - |x_i - x_j|) (linear cone).
Eq. 33 (the weights print garbled): read as the transpose of the filter,
dC/drho_e = sum_i H_ie / Hs_i * dC/drho~_i, with H_ij = w_ij and
Hs_i = sum_j H_ij.  Neighbourhoods are truncated at the domain boundary.
"""

from __future__ import annotations

import itertools

import numpy as np
import scipy.sparse as sp

from .fe import Grid


def filter_matrix(grid: Grid, rmin: float):
    """Return (H, Hs): the sparse cone-weight matrix and its row sums."""
    R = int(np.ceil(rmin))          # superset of the support; w <= 0 is dropped below
    ex, ey, ez = grid.element_ijk()
    rows, cols, vals = [], [], []
    offs = range(-R, R + 1)
    if grid.dim == 2:
        offsets = [(dx, dy, 0) for dx in offs for dy in offs]
    else:
        offsets = list(itertools.product(offs, offs, offs))
    nx, ny, nz = grid.nelx, grid.nely, max(grid.nelz, 1)
    for dx, dy, dz in offsets:
        dist = np.sqrt(dx * dx + dy * dy + dz * dz)
        w = rmin - dist
        if w <= 0.0:
            continue
        jx, jy, jz = ex + dx, ey + dy, ez + dz
        ok = (jx >= 0) & (jx < nx) & (jy >= 0) & (jy < ny) & (jz >= 0) & (jz < nz)
        i = np.nonzero(ok)[0]
        j = jx[ok] + nx * (jy[ok] + ny * jz[ok])
        rows.append(i)
        cols.append(j)
        vals.append(np.full(i.size, w))
    H = sp.coo_matrix((np.concatenate(vals), (np.concatenate(rows), np.concatenate(cols))),
                      shape=(grid.nel, grid.nel)).tocsr()
    Hs = np.asarray(H.sum(axis=1)).ravel()
    return H, Hs


def density_filter(H, Hs, rho: np.ndarray) -> np.ndarray:
    """Eq. 31: physical densities rho~ = (H rho) / Hs."""
    return (H @ rho) / Hs


def sensitivity_filter(H, Hs, d: np.ndarray) -> np.ndarray:
    """Eq. 33 (transpose reading): chain rule through the density filter,
    returns H^T (d / Hs)."""
    return H.T @ (d / Hs)


# ----------------------------------------------------------------------------
# The same filter without forming H, for grids where the sparse matrix would
# not fit in host memory (8.19M elements x 81 neighbours for r = 2.5).  Each
# cone offset (dx, dy, dz) with weight w = r - |offset| > 0 adds w times the
# shifted field to every element whose neighbour lies inside the domain
# (Eq. 31-32, truncated at the boundary).  H is symmetric (the weight depends
# on |offset| only, and "both inside" is symmetric), so Eq. 33's transpose is
# the same stencil applied to d / Hs.
# ----------------------------------------------------------------------------

def _cone_offsets(dim: int, rmin: float):
    R = int(np.ceil(rmin))
    offs = range(-R, R + 1)
    cand = itertools.product(offs, offs, offs if dim == 3 else (0,))
    out = []
    for dx, dy, dz in cand:
        w = rmin - np.sqrt(dx * dx + dy * dy + dz * dz)
        if w > 0.0:
            out.append((dx, dy, dz, w))
    return out


def _block(grid: Grid, v: np.ndarray) -> np.ndarray:
    """Element field as an array indexed [ez, ey, ex] (x fastest)."""
    return v.reshape(max(grid.nelz, 1), grid.nely, grid.nelx)


def _stencil_sum(grid: Grid, rmin: float, v: np.ndarray) -> np.ndarray:
    """(H v)_i = sum over in-domain neighbours j of w_ij v_j."""
    nz, ny, nx = max(grid.nelz, 1), grid.nely, grid.nelx
    src = _block(grid, v)
    acc = np.zeros((nz, ny, nx))
    for dx, dy, dz, w in _cone_offsets(grid.dim, rmin):
        # element i = (x, y, z) receives v at j = (x+dx, y+dy, z+dz)
        xi, xj = slice(max(0, -dx), min(nx, nx - dx)), slice(max(0, dx), min(nx, nx + dx))
        yi, yj = slice(max(0, -dy), min(ny, ny - dy)), slice(max(0, dy), min(ny, ny + dy))
        zi, zj = slice(max(0, -dz), min(nz, nz - dz)), slice(max(0, dz), min(nz, nz + dz))
        acc[zi, yi, xi] += w * src[zj, yj, xj]
    return acc.ravel()


def filter_weight_sums(grid: Grid, rmin: float) -> np.ndarray:
    """Hs_i = sum_j w_ij over the truncated cone (Eq. 31's denominator)."""
    return _stencil_sum(grid, rmin, np.ones(grid.nel))


def density_filter_stencil(grid: Grid, rmin: float, rho: np.ndarray,
                           Hs: np.ndarray | None = None) -> np.ndarray:
    """Eq. 31 without the matrix: (H rho) / Hs."""
    if Hs is None:
        Hs = filter_weight_sums(grid, rmin)
    return _stencil_sum(grid, rmin, rho) / Hs


def sensitivity_filter_stencil(grid: Grid, rmin: float, d: np.ndarray,
                               Hs: np.ndarray | None = None) -> np.ndarray:
    """Eq. 33 (transpose reading) without the matrix: H^T (d / Hs) = H (d / Hs)."""
    if Hs is None:
        Hs = filter_weight_sums(grid, rmin)
    return _stencil_sum(grid, rmin, d / Hs)

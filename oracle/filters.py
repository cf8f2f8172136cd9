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

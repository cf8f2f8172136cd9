"""Oracle-side inputs of the CARM parity tests at the benchmark's basis size
(N_s = N_m = s = 10), shared by the test files that need them and computed
once per test process.

The snapshot is a real design trajectory of the oracle: the 3D cantilever
at 48 x 24 x 24 with the settings of the 192 x 96 x 96 workload (volume
fraction 0.12, filter radius 2.0, s = 10, eps_tol = 1e-3, MGCG rtol 1e-8),
except N_on = 11 instead of 15, which shortens the oracle run while still
filling the PARM (iterations 2-11) before the first CARM iteration (12).
"""

from __future__ import annotations

import functools

import numpy as np

from oracle import aarmr, fe, solvers
from workloads import cantilever3d

SNAP_K = 12


def problem_48_s10():
    return cantilever3d(48, 24, 24, volfrac=0.12, rmin=2.0, n_iter=SNAP_K, mg_levels=4,
                        precision="fp64", n_parm=10, n_carm=10, n_on=SNAP_K - 1, eps_tol=1e-3,
                        rtol=1e-8, maxit=200)


@functools.lru_cache(maxsize=None)
def snapshot_48_s10():
    """(problem, snapshot dict of iteration SNAP_K, oracle history): the
    snapshot holds rho_phys, rho_phys_prev, E, E_prev, u_last and Phi."""
    p = problem_48_s10()
    t = aarmr.run(p, n_iter=SNAP_K, mode="aarmr", snapshot_at=(SNAP_K,))
    return p, t.snapshots[SNAP_K], t.history


def refine_element_field(r: np.ndarray, shape, k: int) -> np.ndarray:
    """Each element of a (nelx, nely, nelz) field repeated over a k^3 block."""
    nx, ny, nz = shape
    r = r.reshape(nz, ny, nx)
    return np.repeat(np.repeat(np.repeat(r, k, 0), k, 1), k, 2).ravel()


def refine_nodal_field(v: np.ndarray, shape, times: int) -> np.ndarray:
    """A nodal displacement field interpolated trilinearly (the oracle's
    multigrid interpolation) onto the grid 2^times finer."""
    nx, ny, nz = shape
    for _ in range(times):
        nx, ny, nz = 2 * nx, 2 * ny, 2 * nz
        v = solvers.interpolation(fe.Grid(3, nx, ny, nz)) @ v
    return v

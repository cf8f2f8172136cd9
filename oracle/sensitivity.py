"""SIMP modulus, compliance and compliance sensitivity.

Eq. 1:  E_e = Emin + (E0 - Emin) rho~_e^p.
Eq. 3:  C = u^T K(rho~) u.  Written as the element sum
        C = sum_e E_e u_e^T KE u_e, which equals u^T K u for any u that is
        zero on the fixed DOFs (and is the quantity compared for iterative
        solutions, where u^T K u and f^T u differ by u^T r).
Eq. 6 / Eq. 34: dC/drho~_e = -u_e^T (dK/drho~_e) u_e
        = -p (E0 - Emin) rho~_e^(p-1) u_e^T KE u_e, with u the MGCG solution
        or the reduced-model solution R~ y.
"""

from __future__ import annotations

import numpy as np

from .fe import Grid


def simp_modulus(rho_phys: np.ndarray, E0: float, Emin: float, penal: float) -> np.ndarray:
    """Eq. 1."""
    return Emin + (E0 - Emin) * rho_phys ** penal


def element_energy(grid: Grid, KE: np.ndarray, u: np.ndarray, fixed: np.ndarray) -> np.ndarray:
    """ce_e = u_e^T KE u_e with prescribed DOFs taken as zero."""
    um = u * (1.0 - fixed.astype(float))
    ue = um[grid.element_dofs()]
    return np.einsum("ei,ij,ej->e", ue, KE, ue)


def element_energy_at(grid: Grid, KE: np.ndarray, u: np.ndarray, fixed: np.ndarray,
                      elems) -> np.ndarray:
    """``element_energy`` for the given elements only."""
    um = u * (1.0 - fixed.astype(float))
    ue = um[grid.dofs_of(elems)]
    return np.einsum("ei,ij,ej->e", ue, KE, ue)


def compliance(E: np.ndarray, ce: np.ndarray) -> float:
    """Eq. 3 as the element sum of E_e u_e^T KE u_e."""
    return float(np.sum(E * ce))


def compliance_sensitivity(rho_phys: np.ndarray, ce: np.ndarray, E0: float, Emin: float,
                           penal: float) -> np.ndarray:
    """Eq. 6 / Eq. 34: derivative of C with respect to the physical densities."""
    return -penal * (E0 - Emin) * rho_phys ** (penal - 1.0) * ce

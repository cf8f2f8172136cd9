"""Combined-approximation reanalysis with the projection auxiliary model
(Sec. 2.2, Eq. 8-29).

Notation: K_ref is the paper's reference stiffness K_0 (the stiffness of the
previous design iteration), dK = K - K_ref (Eq. 8), Phi the PARM (n x N_s),
R the CARM basis (n x N_m).

Readings of what the paper leaves open:
* Eq. 16-17 are not valid for a non-square Phi; the approximate inverse is
  taken as the result they arrive at, Eq. 18: Phi (Phi^T K_ref Phi)^{-1} Phi^T.
* K_Phi is inverted by Cholesky; if that fails, by the symmetric
  eigen-pseudo-inverse with relative cutoff 1e-14.
* Eq. 21 (PCA by SVD) gives no truncation rule: the columns of R are first
  scaled to unit length (the span, and hence the reduced solution, does not
  depend on column scaling) and singular directions with
  sigma_i <= 1e-6 sigma_1 are dropped.  The CA sequence converges like a
  power iteration, so these singular values fall geometrically (to 1e-10 of
  sigma_1 and below at s = 10); a direction below 1e-6 is set by rounding
  of the basis products (K applied to smooth fields cancels by 1e3-1e5)
  more than by the data, and dropping it leaves the reduced solution
  unchanged to well below the per-solve tolerances.
* Algorithm 1's reduced right-hand side "R f" is read as R~^T f (Eq. 23).
"""

from __future__ import annotations

from typing import Callable, List

import numpy as np
import scipy.linalg as sla

SVD_DROP_TOL = 1e-6


def normalized(u: np.ndarray) -> np.ndarray:
    """Eq. 28: phi(u) = u / ||u||."""
    return u / np.linalg.norm(u)


class Parm:
    """Projection auxiliary reduced model Phi (Eq. 27-28) with the update of
    Sec. 3.1 / Fig. 1: columns are normalised MGCG solutions; when full, the
    earliest column is removed and the newest appended."""

    def __init__(self, capacity: int):
        self.capacity = capacity
        self.cols: List[np.ndarray] = []

    def push(self, u: np.ndarray) -> None:
        if len(self.cols) == self.capacity:
            self.cols.pop(0)
        self.cols.append(normalized(u))

    @property
    def full(self) -> bool:
        return len(self.cols) == self.capacity

    def matrix(self) -> np.ndarray:
        return np.stack(self.cols, axis=1)


def k_phi(Phi: np.ndarray, K_ref_apply: Callable) -> np.ndarray:
    """Eq. 15: K_Phi = Phi^T K_ref Phi."""
    KP = np.stack([K_ref_apply(Phi[:, i]) for i in range(Phi.shape[1])], axis=1)
    return Phi.T @ KP


def small_spd_inverse(A: np.ndarray) -> np.ndarray:
    """Inverse of the small SPD matrix K_Phi (Cholesky, else pseudo-inverse)."""
    A = 0.5 * (A + A.T)
    try:
        c = sla.cho_factor(A)
        return sla.cho_solve(c, np.eye(A.shape[0]))
    except np.linalg.LinAlgError:
        w, V = np.linalg.eigh(A)
        keep = w > 1e-14 * np.max(np.abs(w))
        return (V[:, keep] / w[keep]) @ V[:, keep].T


def approx_inverse(Phi: np.ndarray, K_Phi: np.ndarray) -> Callable:
    """Eq. 18: v -> Phi K_Phi^{-1} Phi^T v."""
    Kinv = small_spd_inverse(K_Phi)
    return lambda v: Phi @ (Kinv @ (Phi.T @ v))


def carm_basis(r1: np.ndarray, Phi: np.ndarray, K_Phi: np.ndarray, dK_apply: Callable,
               m: int) -> np.ndarray:
    """Eq. 19-20 / Eq. 26: R = [r1, C r1, ..., C^{m-1} r1] with
    C = -Phi K_Phi^{-1} Phi^T dK."""
    Kt_inv = approx_inverse(Phi, K_Phi)
    cols = [r1.copy()]
    for _ in range(1, m):
        cols.append(-Kt_inv(dK_apply(cols[-1])))
    return np.stack(cols, axis=1)


def ca_exact_basis(r1: np.ndarray, K_ref_solve: Callable, dK_apply: Callable,
                   m: int) -> np.ndarray:
    """Eq. 11-13: classical CA basis with the exact inverse,
    r_i = B r_{i-1}, B = -K_ref^{-1} dK (Eq. 12)."""
    cols = [r1.copy()]
    for _ in range(1, m):
        cols.append(-K_ref_solve(dK_apply(cols[-1])))
    return np.stack(cols, axis=1)


def orthonormalize(R: np.ndarray, drop_tol: float = SVD_DROP_TOL) -> np.ndarray:
    """Eq. 21: R = R~ Sigma V^T; returns R~ restricted to the retained
    singular directions (columns of R scaled to unit length first)."""
    norms = np.linalg.norm(R, axis=0)
    keep_cols = norms > 0.0
    Rn = R[:, keep_cols] / norms[keep_cols]
    if Rn.shape[1] == 0:
        return Rn
    U, s, _ = np.linalg.svd(Rn, full_matrices=False)
    return U[:, s > drop_tol * s[0]]


def reduced_solve(K_apply: Callable, Rt: np.ndarray, f: np.ndarray):
    """Eq. 22-25 and Eq. 29.

    Returns (u~, y, eps) with K_R = R~^T K R~, f_R = R~^T f, y = K_R^{-1} f_R,
    u~ = R~ y and eps = ||K R~ y - f|| / ||f||."""
    KR = np.stack([K_apply(Rt[:, i]) for i in range(Rt.shape[1])], axis=1)
    K_R = Rt.T @ KR
    f_R = Rt.T @ f
    y = np.linalg.solve(0.5 * (K_R + K_R.T), f_R)
    u = Rt @ y
    eps = np.linalg.norm(KR @ y - f) / np.linalg.norm(f)
    return u, y, eps


def aarmr_solve(K_apply: Callable, K_ref_apply: Callable, dK_apply: Callable,
                f: np.ndarray, u_last: np.ndarray, Phi: np.ndarray, m: int,
                r1: str = "u_last"):
    """One CARM build and solve as in Algorithm 1's else-branch:
    K_Phi (Eq. 15), basis from r_1 (Eq. 26), SVD (Eq. 21), reduced solve
    (Eq. 23-25) and force residual (Eq. 29).  Returns (u~, eps, R~).

    r_1 is u_last (Sec. 3.1, the choice the paper uses), or with
    r1="projected_load" the load multiplied by the approximate inverse of
    Eq. 18, Phi K_Phi^-1 Phi^T f, the alternative Fig. 2 compares."""
    KP = k_phi(Phi, K_ref_apply)
    r_first = u_last if r1 == "u_last" else approx_inverse(Phi, KP)(f)
    R = carm_basis(r_first, Phi, KP, dK_apply, m)
    Rt = orthonormalize(R)
    u, _, eps = reduced_solve(K_apply, Rt, f)
    return u, eps, Rt

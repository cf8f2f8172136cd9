"""Optimality-criteria design update (Eq. 3 constraint; the paper defers the
update rule to refs. [31, 32]).

Reading of the rule (the heuristic of the cited 88-line code): with move
limit m = 0.2 and damping exponent 1/2,

    rho_new_e(lam) = clamp(rho_e * sqrt(max(0, -dc_e / (lam * dv_e))),
                           max(0, rho_e - m), min(1, rho_e + m)),

and the Lagrange multiplier lam is the root of the volume constraint
sum_e rho~_new_e = volfrac * N (Eq. 3 with unit element volumes), where
rho~_new is the density filter (Eq. 31) applied to rho_new.  lam is found by
bisection on [0, 1e9], narrowed to a relative bracket of 1e-13 (tighter than
the cited code, so the root does not depend on summation order).  The
max(0, .) guards against tiny positive sensitivities produced by rounding.

The mechanism problem of Sec. 4.3 uses the same rule with the damping
exponent eta = 0.3 in place of 1/2 (max(0, .)^eta; reading recorded in
oracle.mechanism).
"""

from __future__ import annotations

import numpy as np

from .filters import density_filter


def oc_candidate(rho, dc_f, dv_f, lam, move, eta=0.5):
    """rho_new for a given multiplier lam (damping exponent eta)."""
    x = np.maximum(0.0, -dc_f / (dv_f * lam))
    B = np.sqrt(x) if eta == 0.5 else x ** eta
    return np.clip(rho * B, np.maximum(0.0, rho - move), np.minimum(1.0, rho + move))


def oc_update(rho, dc_f, dv_f, H, Hs, volfrac, move=0.2, l1=0.0, l2=1e9, rel_tol=1e-13,
              max_steps=400, eta=0.5):
    """Return (rho_new, lam, change) with change = max |rho_new - rho|."""
    target = volfrac * rho.size
    steps = 0
    while (l2 - l1) > rel_tol * (l1 + l2) and steps < max_steps:
        lmid = 0.5 * (l1 + l2)
        cand = oc_candidate(rho, dc_f, dv_f, lmid, move, eta)
        if np.sum(density_filter(H, Hs, cand)) > target:
            l1 = lmid
        else:
            l2 = lmid
        steps += 1
    lam = 0.5 * (l1 + l2)
    rho_new = oc_candidate(rho, dc_f, dv_f, lam, move, eta)
    return rho_new, lam, float(np.max(np.abs(rho_new - rho)))

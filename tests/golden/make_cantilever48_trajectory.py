"""Writes cantilever48_trajectory.json: the oracle's design trajectory of the 3D
cantilever 48 x 24 x 24 workload (91,875 DOFs, float64, 4 MG levels,
N_s = N_m = 8, N_on = 20, eps_tol = 1e-3, 40 iterations of Algorithm 1).

Calls only the oracle (``oracle.aarmr.run``) on the seeded problem
definition; the GPU trajectory test compares against what it stores: per
iteration the branch taken, the compliance, the CARM force residual eps
(Eq. 29) where a CARM was built, the MGCG iteration count and the design
change, and the final design's volume and compliance.

Run from the repository root:  python tests/golden/make_cantilever48_trajectory.py
"""

import json
import os
import sys
import time

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

from oracle import aarmr  # noqa: E402
from workloads import cantilever3d_48x24x24  # noqa: E402


def main():
    p = cantilever3d_48x24x24()
    t0 = time.time()
    tr = aarmr.run(p, mode="aarmr")
    out = {
        "workload": "3D cantilever 48x24x24 hex8, float64, 4 levels, N_s = N_m = 8, N_on = 20, "
                    "eps_tol 1e-3, rtol 1e-8, 40 iterations",
        "generator": "oracle.aarmr.run(cantilever3d_48x24x24(), mode='aarmr')",
        "history": [dict(k=h.k, branch=h.branch, compliance=h.compliance, eps=h.eps,
                         cg_iters=h.cg_iters, change=h.change) for h in tr.history],
        "final_volume_mean": float(np.mean(tr.rho)),
        "oracle_seconds": round(time.time() - t0, 1),
    }
    path = os.path.join(os.path.dirname(os.path.abspath(__file__)), "cantilever48_trajectory.json")
    with open(path, "w") as f:
        json.dump(out, f, indent=1)
    print(path, out["oracle_seconds"], "s")


if __name__ == "__main__":
    main()

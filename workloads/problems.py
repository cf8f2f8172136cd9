"""Problem definitions for the minimum-compliance examples (Sec. 4 of the paper
and the five benchmark workloads built on it).

Conventions fixed here and used by both the CUDA library and the oracle:

* Unit square (Q4) or unit cube (hex8) elements on a regular grid of
  ``nelx x nely (x nelz)`` elements; x is the length, y the height (y = 0 is
  the bottom) and z the depth.
* Node (i, j, k) has index ``i + (nelx+1) * (j + (nely+1) * k)``; degree of
  freedom c (0 = x, 1 = y, 2 = z) of that node has index ``dim*node + c``.
* Element (ex, ey, ez) has index ``ex + nelx * (ey + nely * ez)``.

Readings of what the paper leaves open (load normalisation, supports, seeds)
are the ones listed for the workloads: point loads of magnitude 1, line and
surface loads of total magnitude 1 with consistent (trapezoidal) nodal
weights, loads pointing in -y.
"""

from __future__ import annotations

from dataclasses import dataclass, field, replace
from typing import List, Tuple

import numpy as np


def grid_counts(dim: int, nelx: int, nely: int, nelz: int = 0) -> Tuple[int, int, int]:
    """Return (n_elements, n_nodes, n_dofs) of a regular grid."""
    if dim == 2:
        nel = nelx * nely
        nn = (nelx + 1) * (nely + 1)
    else:
        nel = nelx * nely * nelz
        nn = (nelx + 1) * (nely + 1) * (nelz + 1)
    return nel, nn, dim * nn


@dataclass
class Problem:
    name: str
    dim: int
    nelx: int
    nely: int
    nelz: int
    fixed: np.ndarray          # uint8 per DOF, 1 = prescribed zero displacement
    f: np.ndarray              # float64 nodal load vector, per DOF
    rho0: np.ndarray           # float64 initial design field, per element
    volfrac: float
    rmin: float
    E0: float = 1.0
    Emin: float = 1e-9
    nu: float = 0.3
    penal: float = 3.0
    move: float = 0.2
    n_iter: int = 30
    mg_levels: int = 3
    precision: str = "fp64"   # "fp64" or "mixed"
    n_parm: int = 2           # N_s, columns of the PARM
    n_carm: int = 2           # N_m, columns of the CARM
    n_on: int = 20            # activation parameter N_on
    eps_tol: float = 1e-3     # force-residual criterion of Eq. 29
    rtol: float = 1e-8        # MGCG convergence tolerance
    maxit: int = 200          # MGCG iteration cap
    carm_r1: str = "u_last"   # first CA basis vector: "u_last" or "projected_load" (Phi K_Phi^-1 Phi^T f)
    volfrac_ramp: tuple = ()  # (k0, v_end, step): from iteration k0 the volume fraction
                              # falls by `step` per iteration down to v_end
    springs: tuple = ()       # ((dof, k), ...): linear springs to ground (Sec. 4.3)
    out_dof: int = -1         # mechanism objective u_out = u[out_dof] (Sec. 4.3); -1: compliance
    oc_eta: float = 0.5       # damping exponent of the OC update
    meta: dict = field(default_factory=dict)

    def volfrac_at(self, k: int) -> float:
        """Volume fraction of design iteration k (constant unless ramped)."""
        if not self.volfrac_ramp:
            return self.volfrac
        k0, v_end, step = self.volfrac_ramp
        return max(v_end, self.volfrac - step * max(0, k - k0))

    @property
    def nel(self) -> int:
        return grid_counts(self.dim, self.nelx, self.nely, self.nelz)[0]

    @property
    def n_nodes(self) -> int:
        return grid_counts(self.dim, self.nelx, self.nely, self.nelz)[1]

    @property
    def ndof(self) -> int:
        return grid_counts(self.dim, self.nelx, self.nely, self.nelz)[2]

    def with_(self, **kw) -> "Problem":
        return replace(self, **kw)


def _node(nelx, nely, i, j, k=0):
    return i + (nelx + 1) * (j + (nely + 1) * k)


def _trapezoid_weights(n_el: int) -> np.ndarray:
    """Nodal weights of a unit total load spread evenly over n_el segments."""
    w = np.full(n_el + 1, 1.0 / n_el)
    w[0] = w[-1] = 0.5 / n_el
    return w


def mbb2d(nelx: int, nely: int, volfrac: float = 0.5, rmin: float = 1.5, **kw) -> Problem:
    """2D MBB half-beam: unit downward point load at the top-left node,
    symmetry (u_x = 0) along the left edge, roller (u_y = 0) at the
    bottom-right node."""
    dim = 2
    _, nn, ndof = grid_counts(dim, nelx, nely)
    fixed = np.zeros(ndof, np.uint8)
    for j in range(nely + 1):
        fixed[dim * _node(nelx, nely, 0, j) + 0] = 1
    fixed[dim * _node(nelx, nely, nelx, 0) + 1] = 1
    f = np.zeros(ndof)
    f[dim * _node(nelx, nely, 0, nely) + 1] = -1.0
    nel = nelx * nely
    p = Problem("mbb2d", dim, nelx, nely, 0, fixed, f, np.full(nel, volfrac), volfrac, rmin)
    return p.with_(**kw)


def cantilever2d(nelx: int, nely: int, volfrac: float = 0.5, rmin: float = 1.5, **kw) -> Problem:
    """2D cantilever: left edge clamped, unit downward point load at the
    middle of the right edge (the setting of Sec. 4.1.1)."""
    dim = 2
    _, nn, ndof = grid_counts(dim, nelx, nely)
    fixed = np.zeros(ndof, np.uint8)
    for j in range(nely + 1):
        n = _node(nelx, nely, 0, j)
        fixed[dim * n] = fixed[dim * n + 1] = 1
    f = np.zeros(ndof)
    if nely % 2 == 0:
        f[dim * _node(nelx, nely, nelx, nely // 2) + 1] = -1.0
    else:
        f[dim * _node(nelx, nely, nelx, nely // 2) + 1] = -0.5
        f[dim * _node(nelx, nely, nelx, nely // 2 + 1) + 1] = -0.5
    nel = nelx * nely
    p = Problem("cantilever2d", dim, nelx, nely, 0, fixed, f, np.full(nel, volfrac), volfrac, rmin)
    return p.with_(**kw)


def cantilever3d(nelx: int, nely: int, nelz: int, volfrac: float = 0.12, rmin: float = 1.5,
                 **kw) -> Problem:
    """3D cantilever: the x = 0 face clamped, a downward line load of total
    magnitude 1 along the bottom edge (y = 0) of the right face (x = nelx)."""
    dim = 3
    _, nn, ndof = grid_counts(dim, nelx, nely, nelz)
    fixed = np.zeros(ndof, np.uint8)
    j, k = np.meshgrid(np.arange(nely + 1), np.arange(nelz + 1), indexing="ij")
    nodes = _node(nelx, nely, 0, j.ravel(), k.ravel())
    for c in range(3):
        fixed[dim * nodes + c] = 1
    f = np.zeros(ndof)
    w = _trapezoid_weights(nelz)
    for kk in range(nelz + 1):
        f[dim * _node(nelx, nely, nelx, 0, kk) + 1] = -w[kk]
    nel = nelx * nely * nelz
    p = Problem("cantilever3d", dim, nelx, nely, nelz, fixed, f, np.full(nel, volfrac),
                volfrac, rmin)
    return p.with_(**kw)


def bridge3d(nelx: int, nely: int, nelz: int, volfrac: float = 0.10, rmin: float = 2.5,
             noise: float = 0.0, seed: int = 2205, **kw) -> Problem:
    """3D MBB bridge: all DOFs fixed at the four bottom corner nodes, a
    downward distributed load of total magnitude 1 on the top face (y = nely)
    with bilinear area weights.  With ``noise > 0`` the initial field is
    volfrac + U(-noise, noise), drawn with ``numpy.random.default_rng(seed)``
    in element order."""
    dim = 3
    _, nn, ndof = grid_counts(dim, nelx, nely, nelz)
    fixed = np.zeros(ndof, np.uint8)
    for i in (0, nelx):
        for k in (0, nelz):
            n = _node(nelx, nely, i, 0, k)
            fixed[dim * n:dim * n + 3] = 1
    f = np.zeros(ndof)
    wx = _trapezoid_weights(nelx)
    wz = _trapezoid_weights(nelz)
    ii, kk = np.meshgrid(np.arange(nelx + 1), np.arange(nelz + 1), indexing="ij")
    nodes = _node(nelx, nely, ii.ravel(), nely, kk.ravel())
    f[dim * nodes + 1] = -(wx[ii.ravel()] * wz[kk.ravel()])
    nel = nelx * nely * nelz
    if noise > 0.0:
        rng = np.random.default_rng(seed)
        rho0 = volfrac + rng.uniform(-noise, noise, nel)
    else:
        rho0 = np.full(nel, volfrac)
    p = Problem("bridge3d", dim, nelx, nely, nelz, fixed, f, rho0, volfrac, rmin)
    return p.with_(**kw)


def halfwheel2d(nelx: int, nely: int, volfrac: float = 0.5, rmin: float = 2.5, **kw) -> Problem:
    """2D half-wheel of Sec. 4.2.1: a rectangle (aspect ratio 2 in the paper),
    the lower-left node fully constrained, the lower-right node constrained in
    the load direction (y), a unit downward point load at the midpoint of the
    bottom edge."""
    dim = 2
    _, nn, ndof = grid_counts(dim, nelx, nely)
    fixed = np.zeros(ndof, np.uint8)
    fixed[dim * _node(nelx, nely, 0, 0) + 0] = 1
    fixed[dim * _node(nelx, nely, 0, 0) + 1] = 1
    fixed[dim * _node(nelx, nely, nelx, 0) + 1] = 1
    f = np.zeros(ndof)
    f[dim * _node(nelx, nely, nelx // 2, 0) + 1] = -1.0
    nel = nelx * nely
    p = Problem("halfwheel2d", dim, nelx, nely, 0, fixed, f, np.full(nel, volfrac), volfrac, rmin)
    return p.with_(**kw)


def beam3d(nelx: int, nely: int, nelz: int, volfrac: float = 0.2, rmin: float = 2.5,
           **kw) -> Problem:
    """3D simply supported beam of Sec. 4.2.2: a cuboid (x length, y height,
    z depth), all DOFs of the four bottom corner nodes fixed, a unit downward
    point load at the midpoint of the bottom face."""
    dim = 3
    _, nn, ndof = grid_counts(dim, nelx, nely, nelz)
    fixed = np.zeros(ndof, np.uint8)
    for i in (0, nelx):
        for k in (0, nelz):
            n = _node(nelx, nely, i, 0, k)
            fixed[dim * n:dim * n + 3] = 1
    f = np.zeros(ndof)
    f[dim * _node(nelx, nely, nelx // 2, 0, nelz // 2) + 1] = -1.0
    nel = nelx * nely * nelz
    p = Problem("beam3d", dim, nelx, nely, nelz, fixed, f, np.full(nel, volfrac), volfrac, rmin)
    return p.with_(**kw)


def inverter2d(nelx: int, nely: int, volfrac: float = 0.3, rmin: float = 2.5,
               k_in: float = 1.0, k_out: float = 0.1, **kw) -> Problem:
    """2D displacement inverter of Sec. 4.3 (half model): the bottom edge is
    the symmetry axis (y-displacements fixed), the input A is the bottom-left
    node with a unit force in +x and a spring k_in, the output B the
    bottom-right node with a spring k_out; the top end of the left edge is
    clamped: nely/16 of it, rounded up to whole elements of the coarsest
    multigrid level (so that the supports stay closed under the coarse-grid
    interpolation).  The objective is u_out = u_x(B), minimised (B moves
    against the input); OC damping 0.3, move limit 0.05."""
    dim = 2
    _, nn, ndof = grid_counts(dim, nelx, nely)
    fixed = np.zeros(ndof, np.uint8)
    for i in range(nelx + 1):
        fixed[dim * _node(nelx, nely, i, 0) + 1] = 1
    unit = 2 ** (kw.get("mg_levels", 3) - 1)
    clamp = -(-max(1, nely // 16) // unit) * unit
    for j in range(nely - clamp, nely + 1):
        n = _node(nelx, nely, 0, j)
        fixed[dim * n:dim * n + 2] = 1
    a = dim * _node(nelx, nely, 0, 0)
    b = dim * _node(nelx, nely, nelx, 0)
    f = np.zeros(ndof)
    f[a] = 1.0
    nel = nelx * nely
    p = Problem("inverter2d", dim, nelx, nely, 0, fixed, f, np.full(nel, volfrac), volfrac, rmin,
                move=0.05, springs=((a, k_in), (b, k_out)), out_dof=b, oc_eta=0.3)
    return p.with_(**kw)


# Sec. 4.3 (Table 1): the inverter at 320 x 160 and 640 x 320, 200 design
# iterations, N_on = 20, N_s = N_m = 2, MGCG rtol 1e-6 and maxit 200, the
# force-residual criterion 0.01 % and 0.1 %.  The paper uses 3 grid levels;
# here the hierarchy goes down to a 40 x 20 coarsest grid (4 and 5 levels),
# which the dense coarsest solve handles.
INVERTER_MODELS = [(320, 160), (640, 320)]


def study_inverter(nelx: int, nely: int, eps_tol: float, n_iter: int = 200,
                   mg_levels: int = 0, **kw) -> Problem:
    levels = mg_levels or 1 + max(1, (nelx // 40).bit_length() - 1)
    return inverter2d(nelx, nely, n_iter=n_iter, mg_levels=levels, n_parm=2, n_carm=2,
                      n_on=20, eps_tol=eps_tol, rtol=1e-6, maxit=200, **kw)


# The reproduction studies of Sec. 4.2: MGCG and AARMR on the same problem
# (N_on = 20, N_s = N_m = 2, MGCG rtol 1e-6; MGCG maxit 200 in 2D, 50 in
# 3D), the force-residual criterion eps_tol varied.  The paper uses 3 grid
# levels; here the hierarchy is the deepest the grid allows (the coarsest
# grid is solved densely), the same for both methods.
HALFWHEEL_MODELS = [(320, 160), (640, 320), (840, 420), (960, 480)]
BEAM_MODELS = [(72, 24, 48), (84, 28, 56), (96, 32, 64), (120, 40, 80)]


def deepest_levels(*nel: int) -> int:
    """Grid levels of the deepest 2x-coarsened hierarchy of a grid: halve
    while every axis stays even and the halved axes keep at least 2
    elements."""
    levels, dims = 1, [n for n in nel if n > 0]
    while all(n % 2 == 0 and n // 2 >= 2 for n in dims):
        dims = [n // 2 for n in dims]
        levels += 1
    return levels


def study_halfwheel(nelx: int, nely: int, eps_tol: float, n_iter: int = 100,
                    mg_levels: int = 0, **kw) -> Problem:
    return halfwheel2d(nelx, nely, n_iter=n_iter, mg_levels=mg_levels or deepest_levels(nelx, nely),
                       n_parm=2, n_carm=2, n_on=20, eps_tol=eps_tol, rtol=1e-6, maxit=200, **kw)


def study_beam(nelx: int, nely: int, nelz: int, eps_tol: float, n_iter: int = 100,
               mg_levels: int = 0, **kw) -> Problem:
    return beam3d(nelx, nely, nelz, n_iter=n_iter,
                  mg_levels=mg_levels or deepest_levels(nelx, nely, nelz), n_parm=2, n_carm=2,
                  n_on=20, eps_tol=eps_tol, rtol=1e-6, maxit=50, **kw)


# --------------------------------------------------------------------------
# The five benchmark workloads.  Parameters the paper leaves open take the
# readings recorded with the design notes (N_s = N_m = s, N_on per workload,
# levels limited by 2x coarsening).
# --------------------------------------------------------------------------

def mbb2d_60x20() -> Problem:
    """2D MBB half-beam, 60 x 20 Q4 (2,562 DOFs), FP64, s = 6."""
    return mbb2d(60, 20, volfrac=0.5, rmin=1.5, n_iter=50, mg_levels=3, precision="fp64",
                 n_parm=6, n_carm=6, n_on=20, eps_tol=1e-3, rtol=1e-8, maxit=200)


def cantilever3d_48x24x24() -> Problem:
    """3D cantilever, 48 x 24 x 24 hex8 (91,875 DOFs), FP64, 4 levels, s = 8."""
    return cantilever3d(48, 24, 24, volfrac=0.12, rmin=1.5, n_iter=40, mg_levels=4,
                        precision="fp64", n_parm=8, n_carm=8, n_on=20, eps_tol=1e-3,
                        rtol=1e-8, maxit=200)


def cantilever3d_192x96x96(precision: str = "mixed") -> Problem:
    """3D cantilever, 192 x 96 x 96 hex8 (5,447,811 DOFs), 6 levels, s = 10."""
    return cantilever3d(192, 96, 96, volfrac=0.12, rmin=2.0, n_iter=30, mg_levels=6,
                        precision=precision, n_parm=10, n_carm=10, n_on=15, eps_tol=1e-3,
                        rtol=1e-8, maxit=200)


def bridge3d_320x160x160() -> Problem:
    """3D MBB bridge, 320 x 160 x 160 hex8 (24,961,923 DOFs), mixed, s = 10,
    6 levels (2x coarsening allows no more), seeded +-0.05 initial noise."""
    return bridge3d(320, 160, 160, volfrac=0.10, rmin=2.5, noise=0.05, seed=2205, n_iter=20,
                    mg_levels=6, precision="mixed", n_parm=10, n_carm=10, n_on=11,
                    eps_tol=1e-3, rtol=1e-8, maxit=200)


SERVE_MESHES = [(32, 16, 16, 4), (64, 32, 32, 5), (96, 48, 48, 5), (128, 64, 64, 6)]


@dataclass
class Job:
    job_id: int
    arrival_s: float
    problem: Problem


def served_job_stream(n_jobs: int = 256, rate_per_s: float = 4.0, seed: int = 385,
                 n_iter: int = 30) -> List[Job]:
    """Served stream: Poisson arrivals (mean rate 4 jobs/s), cantilever or
    bridge 50/50, mesh uniform over four sizes, volfrac U[0.08, 0.3],
    rmin 1.5, mixed precision, s = 8, all drawn from default_rng(385)."""
    rng = np.random.default_rng(seed)
    gaps = rng.exponential(1.0 / rate_per_s, n_jobs)
    kinds = rng.integers(0, 2, n_jobs)
    sizes = rng.integers(0, len(SERVE_MESHES), n_jobs)
    vfs = rng.uniform(0.08, 0.3, n_jobs)
    t = np.cumsum(gaps)
    jobs = []
    for q in range(n_jobs):
        nx, ny, nz, lv = SERVE_MESHES[int(sizes[q])]
        common = dict(volfrac=float(vfs[q]), rmin=1.5, n_iter=n_iter, mg_levels=lv,
                      precision="mixed", n_parm=8, n_carm=8, n_on=15, eps_tol=1e-3,
                      rtol=1e-6, maxit=200)
        if kinds[q] == 0:
            p = cantilever3d(nx, ny, nz, **common)
        else:
            p = bridge3d(nx, ny, nz, **common)
        jobs.append(Job(q, float(t[q]), p))
    return jobs


def small_problem(kind: str = "cantilever3d", **kw) -> Problem:
    """Tiny meshes for unit tests."""
    if kind == "cantilever3d":
        base = dict(nelx=8, nely=4, nelz=4)
        base.update({k: kw.pop(k) for k in list(kw) if k in ("nelx", "nely", "nelz")})
        return cantilever3d(base["nelx"], base["nely"], base["nelz"], **kw)
    if kind == "bridge3d":
        base = dict(nelx=8, nely=4, nelz=4)
        base.update({k: kw.pop(k) for k in list(kw) if k in ("nelx", "nely", "nelz")})
        return bridge3d(base["nelx"], base["nely"], base["nelz"], **kw)
    if kind == "mbb2d":
        base = dict(nelx=12, nely=4)
        base.update({k: kw.pop(k) for k in list(kw) if k in ("nelx", "nely")})
        return mbb2d(base["nelx"], base["nely"], **kw)
    if kind == "cantilever2d":
        base = dict(nelx=12, nely=8)
        base.update({k: kw.pop(k) for k in list(kw) if k in ("nelx", "nely")})
        return cantilever2d(base["nelx"], base["nely"], **kw)
    if kind == "inverter2d":
        base = dict(nelx=16, nely=8)
        base.update({k: kw.pop(k) for k in list(kw) if k in ("nelx", "nely")})
        return inverter2d(base["nelx"], base["nely"], **kw)
    raise ValueError(kind)


def rand_vector(n: int, seed: int, fixed: np.ndarray | None = None) -> np.ndarray:
    """Standard-normal float64 vector; zero at fixed DOFs when a mask is given."""
    x = np.random.default_rng(seed).standard_normal(n)
    if fixed is not None:
        x[fixed.astype(bool)] = 0.0
    return x


def rand_density(nel: int, seed: int, lo: float = 0.0, hi: float = 1.0) -> np.ndarray:
    """Uniform float64 density field in [lo, hi]."""
    return np.random.default_rng(seed).uniform(lo, hi, nel)


def smooth_fields(nelx: int, nely: int, nelz: int, fixed: np.ndarray, count: int) -> List[np.ndarray]:
    """Smooth displacement-like 3D nodal fields (interleaved x, y, z
    components), zero on the fixed DOFs: component c of field i is
    x^(1 + (i + c) mod 3) cos((i + 1) y + c) cos(i z / 2) in coordinates
    scaled to [0, 1].  Linearly independent for distinct i; a stand-in for
    stored displacement solutions where none can be computed."""
    nn = (nelx + 1) * (nely + 1) * (nelz + 1)
    n = np.arange(nn)
    x = (n % (nelx + 1)) / nelx
    y = ((n // (nelx + 1)) % (nely + 1)) / nely
    z = (n // ((nelx + 1) * (nely + 1))) / nelz
    out = []
    for i in range(count):
        v = np.zeros(3 * nn)
        for c in range(3):
            v[c::3] = x ** (1 + (i + c) % 3) * np.cos((i + 1) * y + c) * np.cos(0.5 * i * z)
        v[fixed.astype(bool)] = 0.0
        out.append(v)
    return out

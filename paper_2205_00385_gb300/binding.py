"""ctypes binding of libtopo.so (include/topo.h).

Argument marshalling only: every function forwards to the C entry point of
the same name.  Device arrays are torch CUDA tensors (their data pointers
are passed); PyTorch provides device memory and the stream, the library does
all of the arithmetic.  There is no fallback: if the library cannot be
loaded, every call raises.
"""

from __future__ import annotations

import ctypes as C
import os
from typing import Optional

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libtopo.so")

TO_OK, TO_E_INVALID, TO_E_STATE, TO_E_OOM, TO_E_CUDA, TO_E_NOT_CONVERGED, TO_E_SINGULAR, \
    TO_E_TIMEOUT = range(8)
TO_FP64, TO_MIXED = 0, 1
TO_FILTER_DENSITY, TO_FILTER_SENS = 0, 1
TO_SOLVE_WARM_START, TO_SOLVE_PUSH_PARM = 1, 2
TO_OP_K, TO_OP_KREF, TO_OP_DK = 0, 1, 2
TO_PREC_NATIVE, TO_PREC_FP64, TO_PREC_FP32, TO_PREC_DF = 0, 1, 2, 3

STATUS_NAMES = {0: "TO_OK", 1: "TO_E_INVALID", 2: "TO_E_STATE", 3: "TO_E_OOM", 4: "TO_E_CUDA",
                5: "TO_E_NOT_CONVERGED", 6: "TO_E_SINGULAR", 7: "TO_E_TIMEOUT"}


class TopoError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"{STATUS_NAMES.get(status, status)}: {msg}")
        self.status = status


class to_mesh_desc(C.Structure):
    _fields_ = [("dim", C.c_int32), ("nel", C.c_int32 * 3), ("E0", C.c_double),
                ("Emin", C.c_double), ("nu", C.c_double), ("penal", C.c_double),
                ("rmin", C.c_double), ("mg_levels", C.c_int32), ("precision", C.c_int32),
                ("n_parm", C.c_int32), ("n_carm", C.c_int32)]


_VP = C.c_void_p
_SIGS = {
    "to_workspace_bytes": [C.POINTER(to_mesh_desc), C.POINTER(C.c_int64)],
    "to_mesh_init": [C.POINTER(to_mesh_desc), _VP, _VP, _VP, C.c_int64, _VP, C.POINTER(_VP)],
    "to_carm_basis_error": [_VP, C.POINTER(C.c_double)],
    "to_carm_info": [_VP, C.POINTER(C.c_int32), C.POINTER(C.c_int32), _VP],
    "to_autotune": [_VP, C.c_int32, _VP, C.c_int32, C.POINTER(C.c_int32)],
    "to_batch_step": [_VP, C.c_int32, C.c_int32, _VP],
    "to_carm_options": [_VP, C.c_int32],
    "to_operator_options": [_VP, C.c_int32],
    "to_carm_basis_column": [_VP, C.c_int32, _VP],
    "to_set_density": [_VP, _VP],
    "to_mgcg_solve": [_VP, C.c_double, C.c_int32, C.c_int32, _VP, C.POINTER(C.c_int32),
                      C.POINTER(C.c_double)],
    "to_parm_push": [_VP, _VP],
    "to_parm_count": [_VP, C.POINTER(C.c_int32)],
    "to_parm_reset": [_VP],
    "to_carm_build": [_VP, _VP],
    "to_carm_solve": [_VP, _VP, C.POINTER(C.c_double), _VP],
    "to_sensitivity": [_VP, _VP, _VP, _VP],
    "to_mesh_springs": [_VP, C.c_int32, _VP, _VP],
    "to_sensitivity_adjoint": [_VP, _VP, _VP, _VP, _VP],
    "to_oc_options": [_VP, C.c_double],
    "to_filter": [_VP, C.c_int32, _VP, _VP],
    "to_oc_update": [_VP, C.c_double, C.c_double, _VP, _VP, _VP, _VP],
    "to_oc_update_noalloc": [C.c_int64, C.c_double, C.c_double, _VP, _VP, _VP, _VP, _VP],
    "to_apply": [_VP, C.c_int32, C.c_int32, _VP, _VP],
    "to_vcycle": [_VP, _VP, _VP],
    "to_level_apply": [_VP, C.c_int32, _VP, _VP],
    "to_level_info": [_VP, C.c_int32, C.POINTER(C.c_int32), C.POINTER(C.c_int64)],
    "to_profile_enable": [_VP, C.c_int32],
    "to_profile_read": [_VP, C.c_int32, C.POINTER(C.c_int64), C.POINTER(C.c_double),
                        C.POINTER(C.c_double)],
    "to_launch_count": [_VP, C.POINTER(C.c_int64), C.c_int32],
    "to_last_error": [_VP],
    "to_destroy": [_VP],
}

_lib = None


def load(path: str = LIB_PATH):
    """Load libtopo.so (raises if it is missing: there is no CPU path)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise RuntimeError(f"libtopo.so not built ({path}); run __graft_entry__.build()")
    lib = C.CDLL(path)
    for name, args in _SIGS.items():
        fn = getattr(lib, name)
        fn.argtypes = args
        fn.restype = C.c_int32
    lib.to_last_error.restype = C.c_char_p
    lib.to_destroy.restype = None
    _lib = lib
    return lib


def exported_symbols():
    return list(_SIGS)


def _ptr(t) -> Optional[int]:
    if t is None:
        return None
    return t.data_ptr()


def _check(st: int, ctx=None, allow=()):
    if st == TO_OK or st in allow:
        return st
    msg = load().to_last_error(ctx).decode(errors="replace")
    raise TopoError(st, msg)


def make_desc(dim, nel, E0=1.0, Emin=1e-9, nu=0.3, penal=3.0, rmin=1.5, mg_levels=3,
              precision=TO_FP64, n_parm=2, n_carm=2) -> to_mesh_desc:
    d = to_mesh_desc()
    d.dim = dim
    for i in range(3):
        d.nel[i] = int(nel[i]) if i < len(nel) else 0
    d.E0, d.Emin, d.nu, d.penal, d.rmin = E0, Emin, nu, penal, rmin
    d.mg_levels, d.precision, d.n_parm, d.n_carm = mg_levels, precision, n_parm, n_carm
    return d


# ---------------------------------------------------------------------------
# One Python function per C entry point (same names).
# ---------------------------------------------------------------------------

def to_workspace_bytes(desc: to_mesh_desc) -> int:
    b = C.c_int64()
    _check(load().to_workspace_bytes(C.byref(desc), C.byref(b)))
    return b.value


def to_mesh_init(desc, fixed_mask, f, workspace, stream_handle: int):
    ctx = C.c_void_p()
    _check(load().to_mesh_init(C.byref(desc), _ptr(fixed_mask), _ptr(f), _ptr(workspace),
                               workspace.numel() * workspace.element_size(), stream_handle,
                               C.byref(ctx)))
    return ctx


def to_set_density(ctx, rho_phys):
    _check(load().to_set_density(ctx, _ptr(rho_phys)), ctx)


def to_mgcg_solve(ctx, rtol, maxit, flags, u, allow_not_converged=True):
    it, rel = C.c_int32(), C.c_double()
    st = load().to_mgcg_solve(ctx, rtol, maxit, flags, _ptr(u), C.byref(it), C.byref(rel))
    _check(st, ctx, allow=(TO_E_NOT_CONVERGED,) if allow_not_converged else ())
    return it.value, rel.value, st == TO_OK


def to_parm_push(ctx, u):
    _check(load().to_parm_push(ctx, _ptr(u)), ctx)


def to_parm_count(ctx) -> int:
    n = C.c_int32()
    _check(load().to_parm_count(ctx, C.byref(n)), ctx)
    return n.value


def to_parm_reset(ctx):
    _check(load().to_parm_reset(ctx), ctx)


def to_carm_build(ctx, u_last):
    _check(load().to_carm_build(ctx, _ptr(u_last)), ctx)


def to_carm_solve(ctx, u, eps_dev=None, read_eps=True):
    e = C.c_double()
    _check(load().to_carm_solve(ctx, _ptr(u), C.byref(e) if read_eps else None, _ptr(eps_dev)),
           ctx)
    return e.value if read_eps else None


def to_carm_basis_error(ctx) -> float:
    """max |R~^T R~ - I| of the last CARM basis (test hook)."""
    e = C.c_double()
    _check(load().to_carm_basis_error(ctx, C.byref(e)), ctx)
    return e.value


def to_carm_info(ctx, n_carm=None):
    """(kq, k, sigma) of the last CARM basis (test hook): QR columns, kept
    directions and, when n_carm is given, the singular values (descending)."""
    kq, k = C.c_int32(), C.c_int32()
    sig = (C.c_double * n_carm)() if n_carm else None
    _check(load().to_carm_info(ctx, C.byref(kq), C.byref(k),
                               C.cast(sig, _VP) if sig is not None else None), ctx)
    return kq.value, k.value, (list(sig) if sig is not None else None)


TUNE_KERNELS = ("op_apply", "op_resid", "op_smooth", "gal1_resid", "gal1_smooth", "acc_apply",
                "acc_resid")


class to_tune_result(C.Structure):
    _fields_ = [("kernel", C.c_int32), ("candidates", C.c_int32), ("chunk_layers", C.c_int32),
                ("chosen_us", C.c_double), ("heuristic_us", C.c_double), ("variant", C.c_int32)]


def to_autotune(ctx, reps=10):
    """Times the launch shapes of the context's column-streaming operators and
    keeps the fastest (see include/topo.h); returns one dict per kernel."""
    res = (to_tune_result * len(TUNE_KERNELS))()
    n = C.c_int32()
    _check(load().to_autotune(ctx, reps, C.cast(res, _VP), len(TUNE_KERNELS), C.byref(n)), ctx)
    return [dict(kernel=TUNE_KERNELS[r.kernel], candidates=r.candidates,
                 chunk_layers=r.chunk_layers, chosen_us=r.chosen_us, heuristic_us=r.heuristic_us,
                 variant=r.variant)
            for r in res[:n.value]]


TO_PHASE_DENSITY, TO_PHASE_UPDATE = 0, 1
TO_CARM_R1_PROJECTED_LOAD = 1


TO_OPERATOR_TENSOR_CORES = 1
TO_OPERATOR_FUSED_COARSE = 2
TO_OPERATOR_TALL_TILES = 4
TO_OPERATOR_WORK_LIST = 8


def to_operator_options(ctx, flags):
    _check(load().to_operator_options(ctx, flags), ctx)


def to_carm_options(ctx, flags):
    _check(load().to_carm_options(ctx, flags), ctx)


class to_batch_job(C.Structure):
    _fields_ = [("ctx", _VP), ("rho", _VP), ("rho_phys", _VP), ("u", _VP), ("dc", _VP),
                ("dc_f", _VP), ("dv_f", _VP), ("compliance_dev", _VP), ("change_dev", _VP),
                ("volfrac", C.c_double), ("move", C.c_double)]


def to_batch_step(jobs, phase, stream_handle):
    """One design-loop phase of several jobs as one graph launch; jobs are
    dicts with the to_batch_job fields (device arrays as tensors)."""
    arr = (to_batch_job * len(jobs))()
    for q, j in enumerate(jobs):
        arr[q] = to_batch_job(j["ctx"], _ptr(j["rho"]), _ptr(j.get("rho_phys")), _ptr(j.get("u")),
                              _ptr(j.get("dc")), _ptr(j.get("dc_f")), _ptr(j.get("dv_f")),
                              _ptr(j.get("compliance_dev")), _ptr(j.get("change_dev")),
                              float(j.get("volfrac", 0.0)), float(j.get("move", 0.0)))
    _check(load().to_batch_step(C.cast(arr, _VP), len(jobs), phase, stream_handle))


def to_carm_basis_column(ctx, j, out):
    _check(load().to_carm_basis_column(ctx, j, _ptr(out)), ctx)


def to_sensitivity(ctx, u, compliance_dev, dc):
    _check(load().to_sensitivity(ctx, _ptr(u), _ptr(compliance_dev), _ptr(dc)), ctx)


TO_MAX_SPRINGS = 4


def to_mesh_springs(ctx, dofs, ks):
    """Springs to ground on free DOFs (2D): lists of DOF indices and
    stiffnesses, copied by the library."""
    n = len(dofs)
    d = (C.c_int64 * max(n, 1))(*[int(x) for x in dofs])
    k = (C.c_double * max(n, 1))(*[float(x) for x in ks])
    _check(load().to_mesh_springs(ctx, n, C.cast(d, _VP), C.cast(k, _VP)), ctx)


def to_sensitivity_adjoint(ctx, u, lam, mutual_dev, dc):
    _check(load().to_sensitivity_adjoint(ctx, _ptr(u), _ptr(lam), _ptr(mutual_dev), _ptr(dc)),
           ctx)


def to_oc_options(ctx, eta):
    _check(load().to_oc_options(ctx, float(eta)), ctx)


def to_filter(ctx, mode, x, out):
    _check(load().to_filter(ctx, mode, _ptr(x), _ptr(out)), ctx)


def to_oc_update(ctx, volfrac, move, dc_f, dv_f, rho, change_dev=None):
    _check(load().to_oc_update(ctx, volfrac, move, _ptr(dc_f), _ptr(dv_f), _ptr(rho),
                               _ptr(change_dev)), ctx)


def to_oc_update_noalloc(nel, volfrac, move, dc_f, dv_f, rho, change_dev, stream_handle):
    """OC update without a context or workspace (scratch is a static device
    array of the library); errors read from to_last_error(None)."""
    _check(load().to_oc_update_noalloc(nel, volfrac, move, _ptr(dc_f), _ptr(dv_f), _ptr(rho),
                                       _ptr(change_dev), stream_handle))


def to_apply(ctx, op, prec, x, y):
    _check(load().to_apply(ctx, op, prec, _ptr(x), _ptr(y)), ctx)


def to_vcycle(ctx, r, z):
    _check(load().to_vcycle(ctx, _ptr(r), _ptr(z)), ctx)


def to_level_apply(ctx, level, x, y):
    _check(load().to_level_apply(ctx, level, _ptr(x), _ptr(y)), ctx)


def to_level_info(ctx, level):
    nel = (C.c_int32 * 3)()
    n = C.c_int64()
    _check(load().to_level_info(ctx, level, nel, C.byref(n)), ctx)
    return tuple(nel), n.value


# profiling kinds (to_profile_read) and their bits in to_profile_enable
PK_FINE32, PK_COARSE, PK_VCYCLE, PK_FINE_OTHER = 0, 1, 2, 3


def to_profile_enable(ctx, kinds):
    """kinds: bit mask of profiling kinds (bit k = kind k); True = all, False = off."""
    if isinstance(kinds, bool):
        kinds = 0xF if kinds else 0
    _check(load().to_profile_enable(ctx, int(kinds)), ctx)


def to_profile_read(ctx, kind: int):
    """Returns (launches, milliseconds, algorithmic bytes)."""
    cnt, ms, by = C.c_int64(), C.c_double(), C.c_double()
    _check(load().to_profile_read(ctx, kind, C.byref(cnt), C.byref(ms), C.byref(by)), ctx)
    return cnt.value, ms.value, by.value


def to_launch_count(ctx, reset=False) -> int:
    cnt = C.c_int64()
    _check(load().to_launch_count(ctx, C.byref(cnt), int(reset)), ctx)
    return cnt.value


def to_last_error(ctx=None) -> str:
    return load().to_last_error(ctx).decode(errors="replace")


def to_destroy(ctx):
    load().to_destroy(ctx)

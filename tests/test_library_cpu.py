"""Host-only checks of the C-ABI library (no GPU needed): it builds, loads,
exports every entry point declared in include/topo.h, and its host-side
validation and workspace sizing behave as documented."""

import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "topo.h")


def _lib():
    from paper_2205_00385_gb300 import binding as B
    from paper_2205_00385_gb300 import build
    if not os.path.exists(B.LIB_PATH):
        build.build()
    return B, B.load()


def _declared():
    src = open(HEADER).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(to_[a-z_0-9]+)\s*\(", src)))


def test_header_declares_the_boundary():
    names = _declared()
    for required in ("to_mesh_init", "to_set_density", "to_mgcg_solve", "to_carm_build",
                     "to_carm_solve", "to_sensitivity", "to_filter", "to_oc_update",
                     "to_workspace_bytes", "to_destroy"):
        assert required in names


def test_library_exports_every_declared_symbol():
    B, lib = _lib()
    for name in _declared():
        assert hasattr(lib, name), name
    # the binding covers the same names
    assert sorted(B.exported_symbols()) == _declared()


def _header_constants():
    """Integer constants of include/topo.h: #define TO_X <int> and the
    TO_X = <int> entries of its enums."""
    src = re.sub(r"/\*.*?\*/", "", open(HEADER).read(), flags=re.S)
    vals = {k: int(v) for k, v in re.findall(r"#define\s+(TO_[A-Z_0-9]+)\s+(-?\d+)\s*$", src,
                                             flags=re.M)}
    for body in re.findall(r"enum\s*\{(.*?)\}", src, flags=re.S):
        for k, v in re.findall(r"(TO_[A-Z_0-9]+)\s*=\s*(-?\d+)", body):
            vals[k] = int(v)
    return vals


def test_binding_constants_match_the_header():
    """Every TO_* integer the Python binding defines has the header's value
    (option bits, enums, limits, status codes)."""
    from paper_2205_00385_gb300 import binding as B
    hdr = _header_constants()
    assert len(hdr) >= 30
    shared = [k for k in hdr if hasattr(B, k)]
    assert "TO_OPERATOR_WORK_LIST" in shared and "TO_PREC_DF" in shared
    for k in shared:
        assert getattr(B, k) == hdr[k], k


def test_workspace_bytes_and_validation():
    B, _ = _lib()
    d = B.make_desc(3, (192, 96, 96), rmin=2.0, mg_levels=6, precision=B.TO_MIXED,
                    n_parm=10, n_carm=10)
    nbytes = B.to_workspace_bytes(d)
    n = 3 * 193 * 97 * 97
    # at least the float64 PARM/CARM blocks (4 x 10 columns) and CG vectors
    assert nbytes > (40 + 5) * n * 8
    assert nbytes < 6 * 2 ** 30
    bad = [
        B.make_desc(4, (8, 8, 8)),
        B.make_desc(3, (0, 8, 8)),       # empty meshes
        B.make_desc(3, (8, 8, 0)),
        B.make_desc(2, (0, 8, 0)),
        B.make_desc(3, (-2, 8, 8)),
        B.make_desc(3, (9, 8, 8), mg_levels=2),
        B.make_desc(3, (8, 8, 8), mg_levels=1),
        B.make_desc(3, (8, 8, 8), precision=7),
        B.make_desc(3, (8, 8, 8), n_parm=0),
        B.make_desc(3, (8, 8, 8), n_carm=17),
        B.make_desc(3, (8, 8, 8), Emin=0.0),
        B.make_desc(3, (8, 8, 8), nu=0.5),
        B.make_desc(3, (8, 8, 8), rmin=-1.0),
    ]
    for d in bad:
        with pytest.raises(B.TopoError) as e:
            B.to_workspace_bytes(d)
        assert e.value.status == B.TO_E_INVALID


def test_mixed_workspace_smaller_than_fp64():
    B, _ = _lib()
    a = B.to_workspace_bytes(B.make_desc(3, (48, 24, 24), mg_levels=4, precision=B.TO_MIXED))
    b = B.to_workspace_bytes(B.make_desc(3, (48, 24, 24), mg_levels=4, precision=B.TO_FP64))
    assert a < b

"""Host-side checks of the C ABI that need no GPU: the library loads, exports every
function include/*.h declares, and rejects invalid grids before touching the device."""
import ctypes as C
import glob
import os
import re

import numpy as np
import pytest

import paper_1806_06623_gb300 as S
from paper_1806_06623_gb300 import _binding as B

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    names = set()
    for h in glob.glob(os.path.join(ROOT, "include", "*.h")):
        text = open(h).read()
        text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
        for m in re.finditer(r"^\s*[A-Za-z_][\w\s\*]*?\b(sp_\w+)\s*\(", text, flags=re.M):
            names.add(m.group(1))
    return sorted(names)


def test_header_declares_the_boundary():
    names = declared_functions()
    for need in ("sp_plan_create", "sp_solve", "sp_apply_laplacian", "sp_plan_destroy"):
        assert need in names


def test_library_exports_every_declared_symbol():
    L = S.lib()
    for name in declared_functions():
        assert hasattr(L, name), name
    assert set(declared_functions()) <= set(B.declared_symbols()) | set(declared_functions())


def test_status_strings():
    assert S.sp_status_string(S.SP_OK) == "SP_OK"
    assert S.sp_status_string(S.SP_ERR_GRID) == "SP_ERR_GRID"
    assert S.sp_status_string(99) == "SP_ERR_UNKNOWN"


def _create(r, th, nphi, **kw):
    out = C.c_void_p()
    r = np.ascontiguousarray(r, dtype=np.float64)
    thp = None if th is None else np.ascontiguousarray(th, dtype=np.float64)
    nth = kw.pop("nth", None) or (len(thp) - 1)
    st = S.lib().sp_plan_create(r.ctypes.data_as(C.c_void_p), len(r) - 1,
                                None if thp is None else thp.ctypes.data_as(C.c_void_p), nth, nphi,
                                kw.get("bc", 0), 1.0, kw.get("prec", 0), 1e-10, 8, None, C.byref(out))
    return st, out


@pytest.mark.parametrize("r,th,nphi,expect", [
    ([0.0, 0.5, 0.4, 1.0], np.linspace(0, np.pi, 5), 8, S.SP_ERR_GRID),          # not increasing
    ([-0.1, 0.5, 1.0], np.linspace(0, np.pi, 5), 8, S.SP_ERR_GRID),              # negative radius
    ([0.0, 0.5, 1.0], np.linspace(0, 3.0, 5), 8, S.SP_ERR_GRID),                  # theta not to pi
    ([0.0, 0.5, 1.0], np.array([0.0, 1.0, 0.9, np.pi]), 8, S.SP_ERR_GRID),       # theta not increasing
    ([0.0, 0.5, 1.0], np.linspace(0, np.pi, 5), 14, S.SP_ERR_UNSUPPORTED),       # radix 7
    ([0.0, 0.5, 1.0], np.linspace(0, np.pi, 200), 8, S.SP_ERR_UNSUPPORTED),      # Ntheta > 160
    ([0.0, 0.5, 1.0], np.linspace(0, np.pi, 5), 0, S.SP_ERR_GRID),               # no phi zones
])
def test_invalid_grids_are_rejected_on_the_host(r, th, nphi, expect):
    st, out = _create(r, th, nphi)
    assert st == expect and not out.value


def test_invalid_enums_and_null_output():
    r = np.array([0.0, 0.5, 1.0])
    th = np.linspace(0, np.pi, 5)
    assert _create(r, th, 8, bc=7)[0] == S.SP_ERR_INVALID_ARG
    assert _create(r, th, 8, prec=9)[0] == S.SP_ERR_INVALID_ARG
    assert S.lib().sp_plan_create(r.ctypes.data_as(C.c_void_p), 2, None, 4, 8, 0, 1.0, 0, 1e-10, 8, None,
                                  None) == S.SP_ERR_INVALID_ARG
    assert S.lib().sp_plan_destroy(None) == S.SP_OK


def test_pipelined_host_solve_rejects_null_arguments():
    """Argument checks of sp_solve_host_pipelined run on the host before any copy or solve."""
    L = S.lib()
    one = (C.c_void_p * 1)(None)
    assert L.sp_solve_host_pipelined(None, 1, one, one, None, None) == S.SP_ERR_INVALID_ARG
    assert L.sp_solve_host_pipelined(None, -1, None, None, None, None) == S.SP_ERR_INVALID_ARG

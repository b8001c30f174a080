"""The C-ABI library builds, loads and exports every entry point include/rfcmp.h declares.

No compute calls: these run without a GPU.
"""

import ctypes
import os
import re

import pytest

import paper_1803_08333_gb300 as rf
from paper_1803_08333_gb300 import build

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    txt = open(os.path.join(ROOT, "include", "rfcmp.h")).read()
    txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
    return sorted(set(re.findall(r"\b(rfcmp_[a-z0-9_]+)\s*\(", txt)))


@pytest.fixture(scope="module")
def libpath():
    return build.build()


def test_header_declarations_match_binding_list():
    assert _declared() == sorted(rf.EXPORTED_SYMBOLS)


def test_library_exports_every_declared_symbol(libpath):
    L = ctypes.CDLL(libpath)
    for name in _declared():
        assert hasattr(L, name), name


def test_status_strings_and_defaults(libpath):
    L = rf.lib()
    for code in (0, -1, -2, -3, -4, -5, -6, -7, -8):
        assert L.rfcmp_strerror(code)
    o = rf.OpOpts()
    L.rfcmp_op_opts_default(ctypes.byref(o))
    assert o.power_steps == 30 and o.scaling == 0 and o.factor_tol == 1e-13 and o.power_rtol == 1e-3
    s = rf.SolveOpts()
    L.rfcmp_solve_opts_default(ctypes.byref(s))
    assert s.tol == 1e-6 and s.precision == 0 and s.max_refine == 24


def test_phase_range_bound_matches_header():
    txt = open(os.path.join(ROOT, "include", "rfcmp.h")).read()
    (val,) = re.findall(r"#define RFCMP_MAX_K_EXTENT\s+([0-9.eE+-]+)", txt)
    assert float(val) == rf.MAX_K_EXTENT
    # the reduction's leading part of pi/2 has 8 significant bits (1.5703125 = 201 / 128), so q
    # times it is exact in FP32 while q < 2^16; the bound keeps q = rint(k R 2/pi) below that
    assert 1.5703125 * 128 == 201 and 201 < 2**8
    assert rf.MAX_K_EXTENT * 2 / 3.141592653589793 + 0.5 < 2**16


def test_struct_layouts_match_header(libpath):
    # sizes implied by include/rfcmp.h on LP64
    assert ctypes.sizeof(rf.OpOpts) == 4 + 4 + 8 * 5 + 8 + 4 * 8
    assert ctypes.sizeof(rf.SolveOpts) == 8 + 4 + 4 + 8 + 4 + 4 + 4 * 8
    assert ctypes.sizeof(rf.SolveReport) == 4 * 4 + 8
    assert ctypes.sizeof(rf.OpInfo) == 3 * 8 + 2 * 4 + 4 * 8 + 8 + 3 * 8 + 2 * 4
    assert ctypes.sizeof(rf.Plan) == 8 * 4


def test_plan_defaults_and_argument_checks(libpath):
    L = rf.lib()
    p = rf.Plan()
    p.mrhs_min, p.gemm_bn = 7, 64
    L.rfcmp_plan_default(ctypes.byref(p))
    assert p.as_dict() == {k: 0 for k in rf.Plan.KEYS}
    assert L.rfcmp_op_set_plan(None, ctypes.byref(p)) == -1
    assert L.rfcmp_ctx_set_plan(None, ctypes.byref(p)) == -1
    assert L.rfcmp_op_get_plan(None, ctypes.byref(p)) == -1
    assert rf.Plan.of({"gemm_bn": 32}).gemm_bn == 32
    with pytest.raises(KeyError):
        rf.Plan.of({"tile": 3})


def test_no_device_is_an_error_not_a_fallback(libpath):
    import torch

    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    h = ctypes.c_void_p()
    st = rf.lib().rfcmp_ctx_create(0, 0, ctypes.byref(h))
    assert st == -8  # RFCMP_ERR_NO_DEVICE
    assert not h.value

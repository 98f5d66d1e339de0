"""Host-side checks of the C ABI that need no GPU: the library loads, exports
every entry point include/*.h declares, and rejects invalid parameters before
touching the device."""
from __future__ import annotations

import ctypes
import glob
import os
import re

import pytest

from paper_2601_02540_b300 import build, sgn

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_symbols() -> set[str]:
    names = set()
    for hdr in glob.glob(os.path.join(ROOT, "include", "*.h")):
        text = open(hdr).read()
        names |= set(re.findall(r"SGN_API\s+[\w\s\*]+?\b(sgn_\w+)\s*\(", text))
    return names


@pytest.fixture(scope="module")
def lib():
    build.build()
    return sgn.lib()


def test_header_declares_the_boundary():
    names = declared_symbols()
    for required in ("sgn_create", "sgn_destroy", "sgn_rhs", "sgn_step", "sgn_mass_energy",
                     "sgn_init_aux", "sgn_status_str", "sgn_last_error"):
        assert required in names


def test_library_exports_every_declared_symbol(lib):
    missing = [n for n in sorted(declared_symbols()) if not hasattr(lib, n)]
    assert missing == []
    # the binding knows every declared entry point
    assert declared_symbols() <= set(sgn._SIGNATURES)


def test_status_strings(lib):
    for code, name in sgn.STATUS.items():
        assert lib.sgn_status_str(code).decode() == name


@pytest.mark.parametrize("field,value", [("nx", 2), ("ny", 0), ("xmax", -1.0), ("bc", 7),
                                         ("prec", 9), ("g", 0.0), ("lam", -1.0),
                                         ("xmin", float("nan"))])
def test_create_rejects_bad_params_without_device(lib, field, value):
    p = sgn.Params(8, 8, 0.0, 1.0, 0.0, 1.0, 0, 9.81, 500.0, 0)
    setattr(p, field, value)
    ctx = ctypes.c_void_p(1234)
    st = lib.sgn_create(ctypes.byref(p), None, ctypes.byref(ctx))
    assert st == 1  # SGN_E_INVAL
    assert ctx.value is None
    assert lib.sgn_last_error().decode() != ""


@pytest.mark.parametrize("prec", [0, 1, 2, 3])
def test_create_rejects_grids_beyond_the_launch_limit_without_device(lib, prec):
    p = sgn.Params(8, 65535 * 8 + 1, 0.0, 1.0, 0.0, 1.0, 0, 9.81, 500.0, prec)
    ctx = ctypes.c_void_p(1234)
    assert lib.sgn_create(ctypes.byref(p), None, ctypes.byref(ctx)) == 1
    assert ctx.value is None
    assert "launch-grid limit" in lib.sgn_last_error().decode()


@pytest.mark.parametrize("prec,rejected", [(0, False), (1, True), (2, True), (3, True)])
def test_create_rejects_float_grids_of_2_32_nodes_without_device(lib, prec, rejected):
    p = sgn.Params(65536, 65537, 0.0, 1.0, 0.0, 1.0, 0, 9.81, 500.0, prec)
    ctx = ctypes.c_void_p(1234)
    assert lib.sgn_create(ctypes.byref(p), None, ctypes.byref(ctx)) == 1     # FP64: no b_dev
    assert ctx.value is None
    assert ("2^32" in lib.sgn_last_error().decode()) == rejected


def test_null_context_is_rejected(lib):
    assert lib.sgn_rhs(None, None, None, None) == 1
    assert lib.sgn_step(None, None, 0.1, 1, None) == 1
    assert lib.sgn_mass_energy(None, None, None, None) == 1
    assert lib.sgn_step_host(None, None, 0.1, 1, None, None) == 1
    assert lib.sgn_step_record_tape(None, None, 0.1, 1, None, None, None) == 1
    assert lib.sgn_step_vjp_tape(None, None, None, None, None, 0.1, None) == 1
    assert lib.sgn_set_tile_rows(None, 1) == 1
    assert lib.sgn_tile_rows(None, None) == 1
    assert lib.sgn_set_stage_fusion(None, 1) == 1
    assert lib.sgn_batch_set_stage_fusion(None, 1) == 1
    assert lib.sgn_batch_stage_fusion(None, None) == 1
    assert lib.sgn_destroy(None) == 0


def test_fma_rate_rejects_bad_arguments_without_device(lib):
    n, sec = ctypes.c_double(), ctypes.c_double()
    for iters in (0, 3, 1 << 21):
        assert lib.sgn_measure_fp64_fma(iters, ctypes.byref(n), ctypes.byref(sec), None) == 1
    assert lib.sgn_measure_fp64_fma(64, None, ctypes.byref(sec), None) == 1

"""The C-ABI library builds, loads and exports every declared symbol (no GPU).

No compute call is made here: without a GPU only loading and symbol lookup
are checked, plus the argument validation that fails before touching the
device.
"""
import ctypes
import os
import re
import subprocess

import pytest

from paper_2011_07099_gb300 import binding, build

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    names = set()
    for h in os.listdir(os.path.join(ROOT, "include")):
        if not h.endswith(".h"):
            continue
        text = open(os.path.join(ROOT, "include", h)).read()
        text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
        text = re.sub(r"//[^\n]*", "", text)
        for m in re.finditer(r"\b(fmm_[a-z0-9_]+)\s*\(", text):
            names.add(m.group(1))
    return names


@pytest.fixture(scope="module")
def lib():
    build.build()
    return binding.lib()


def test_library_exports_every_declared_symbol(lib):
    declared = _declared()
    assert declared, "no declarations found"
    for name in declared:
        assert hasattr(lib, name), name
    out = subprocess.run(["nm", "-D", "--defined-only", binding.LIB_PATH], capture_output=True, text=True).stdout
    exported = set(re.findall(r" T (fmm_[a-z0-9_]+)", out))
    assert declared <= exported
    assert declared == set(binding.SIGNATURES), "binding and header disagree"


def test_error_strings(lib):
    for code in range(7):
        assert binding.lib().fmm_error_string(code)
    assert binding.lib().fmm_error_string(99) == b"unknown error code"


@pytest.mark.parametrize("args", [(32, 1, 2), (32, 9, 2), (30, 3, 2), (32, 3, 0), (32, 3, 9), (512, 3, 4), (0, 2, 2), (40, 3, 2), (80, 2, 3)])
def test_plan_create_rejects_bad_shapes_before_touching_the_device(lib, args):
    # sizes are validated on the host first: S in {1, 2, 3, 4, 6, 8}, 2 <= L <= 8, 1 <= order <= 8
    assert binding.lib().fmm_plan_create(*args) is None
    assert binding.lib().fmm_last_error() == binding.FMM_ERR_ARG


def test_null_plan_calls_fail_cleanly(lib):
    L = binding.lib()
    assert L.fmm_solve(None, None, None, None, None) == binding.FMM_ERR_ARG
    assert L.fmm_plan_set_precision(None, 0) == binding.FMM_ERR_ARG
    L.fmm_plan_destroy(None)


def test_setters_validate_before_touching_the_device(lib):
    # null plans and out-of-range knobs are refused on the host
    L = binding.lib()
    for call in (lambda: L.fmm_plan_set_m2l_group(None, 2), lambda: L.fmm_plan_set_tc_min_level(None, 4),
                 lambda: L.fmm_plan_set_timeout_ms(None, 100),
                 lambda: L.fmm_plan_inject_fault(None, 0), lambda: L.fmm_plan_set_correction_inference(None, 0),
                 lambda: L.fmm_plan_error_stats(None, None, None, None, 16, 0, None, None),
                 lambda: L.fmm_probe_fma(None, 1, 1, None)):
        assert call() == binding.FMM_ERR_ARG
        assert L.fmm_last_error() == binding.FMM_ERR_ARG


def test_batch_and_autotuner_validate_before_touching_the_device(lib):
    import ctypes
    L = binding.lib()
    ints = lambda *v: (ctypes.c_int * len(v))(*v)
    assert not L.fmm_batch_create(0, ints(32), ints(3), ints(4))
    assert L.fmm_last_error() == binding.FMM_ERR_ARG
    assert not L.fmm_batch_create(1, None, ints(3), ints(4))
    assert L.fmm_last_error() == binding.FMM_ERR_ARG
    # the first field's shape is invalid (30 is not a multiple of 2^3)
    assert not L.fmm_batch_create(1, ints(30), ints(3), ints(4))
    assert L.fmm_last_error() == binding.FMM_ERR_ARG
    for call in (lambda: L.fmm_batch_set_precision(None, 0), lambda: L.fmm_batch_get_levels(None, None),
                 lambda: L.fmm_batch_solve(None, None, None, None, None), lambda: L.fmm_batch_check(None)):
        assert call() == binding.FMM_ERR_ARG
    out_L, out_ms = ctypes.c_int(), ctypes.c_float()
    assert L.fmm_autotune_levels(2, 4, 0, None, ctypes.byref(out_L), ctypes.byref(out_ms)) == binding.FMM_ERR_ARG
    assert L.fmm_autotune_levels(64, 0, 0, None, ctypes.byref(out_L), ctypes.byref(out_ms)) == binding.FMM_ERR_ARG
    assert L.fmm_autotune_levels(64, 4, 0, None, None, ctypes.byref(out_ms)) == binding.FMM_ERR_ARG
    L.fmm_batch_destroy(None)


def test_fma_probe_counts_its_flops(lib):
    # 1024 threads x 8 chains x 16 FMAs per trip x 2 flop
    assert binding.lib().fmm_probe_fma_flops(3, 5) == 2.0 * 3 * 1024 * 5 * 16 * 8

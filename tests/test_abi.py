"""The C-ABI library builds, loads and exports every declared entry point.

No GPU needed: only host-side functions and argument checks are called."""
import ctypes
import glob
import os
import re
import subprocess

import pytest

from paper_1505_04086_gb300 import _build, gc

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    _build.build()
    return gc.load()


def declared_functions():
    names = set()
    for h in glob.glob(os.path.join(ROOT, "include", "*.h")):
        text = open(h).read()
        text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
        for m in re.finditer(r"\b(gc_[a-z0-9_]+)\s*\(", text):
            names.add(m.group(1))
    return names


def test_exports_every_declared_symbol(lib):
    names = declared_functions()
    assert {"gc_color", "gc_color_async", "gc_ctx_stats", "gc_color_batch"} <= names
    out = subprocess.run(["nm", "-D", "--defined-only", _build.LIB], capture_output=True,
                         text=True, check=True).stdout
    exported = {l.split()[-1] for l in out.splitlines() if " T " in l}
    missing = names - exported
    assert not missing, missing
    for n in names:
        assert hasattr(lib, n)
    # the binding declares a signature for each one
    assert names <= set(gc._SIGS)


def test_host_only_calls(lib):
    assert gc.gc_version() >= 100
    assert gc.gc_strerror(gc.GC_OK) == "ok"
    assert "cap" in gc.gc_strerror(gc.GC_ERR_NO_CONVERGENCE)
    assert gc.gc_strerror(12345) == "unknown status"


def test_argument_errors_need_no_device(lib):
    # A null context or bad sizes are rejected before any CUDA call.
    csr = gc.gc_csr(0, 0)
    assert lib.gc_color_async(None, ctypes.byref(csr), 4, 0, 0, None, None, None) == gc.GC_ERR_ARG
    assert lib.gc_color_async(None, None, 4, 0, 0, None, None, None) == gc.GC_ERR_ARG
    assert lib.gc_ctx_stats(None, None) == gc.GC_ERR_ARG
    assert lib.gc_color(ctypes.byref(csr), -1, 0, 0, None, None) == gc.GC_ERR_ARG
    assert lib.gc_color(ctypes.byref(csr), 4, 0, 0, None, None) == gc.GC_ERR_ARG  # null arrays
    b = gc.gc_batch(-1, 0, 0, 0, 0, 0, 0)
    assert lib.gc_color_batch(None, ctypes.byref(b), 0, None, None, None, None, None) == gc.GC_ERR_ARG
    h = ctypes.c_void_p()
    assert lib.gc_ctx_create(None, 0) == gc.GC_ERR_ARG
    r = ctypes.c_double()
    assert lib.gc_measure_gather_rate(0, 100, 2, 0, ctypes.byref(r)) == gc.GC_ERR_ARG     # array too small
    assert lib.gc_measure_gather_rate(0, 2 << 30, 2, 0, ctypes.byref(r)) == gc.GC_ERR_ARG  # too large
    assert lib.gc_measure_gather_rate(0, 8 << 20, 9, 0, ctypes.byref(r)) == gc.GC_ERR_ARG  # blocks per SM
    assert lib.gc_measure_gather_rate(0, 8 << 20, 2, 2, ctypes.byref(r)) == gc.GC_ERR_ARG  # kind
    assert lib.gc_measure_gather_rate(0, 8 << 20, 2, 0, None) == gc.GC_ERR_ARG


def test_binding_refuses_missing_library(monkeypatch, tmp_path):
    monkeypatch.setattr(gc, "_lib", None)
    monkeypatch.setattr(_build, "LIB", str(tmp_path / "nope.so"))
    with pytest.raises(RuntimeError, match="not built"):
        gc.load()


def test_mode_combinations_are_checked_on_the_host(lib):
    # GC_FF_KEEPERS needs asynchronous RSOC with lower-keeps ties and in-place
    # repairs; unknown bits are refused.  An empty batch keeps every other
    # argument valid, and the check comes before any device work.
    b = gc.gc_batch(0, 0, 0, 0, 0, 0, 0)
    h = ctypes.c_void_p()
    K, A, D2 = gc.GC_FF_KEEPERS, gc.GC_SCHED_ASYNC, gc.GC_DIST2
    # distance-2 colouring is a single-graph mode: never a batch or plan
    for mode in (K, K | A | gc.GC_ALG_TWO_PHASE, K | A | gc.GC_TIE_HIGHER_KEEPS,
                 K | A | gc.GC_REPAIR_SNAPSHOT, K | A | gc.GC_DEBUG_NO_TIEBREAK, D2, D2 | A, 1 << 11, 1 << 31):
        assert lib.gc_plan_create(ctypes.byref(b), 0, mode, None, None, None, None,
                                  ctypes.byref(h)) == gc.GC_ERR_ARG, mode
        assert not h.value
    r = gc.gc_tune_result()
    assert lib.gc_autotune_batch(None, ctypes.byref(b), A | K, 3, None, ctypes.byref(r)) == gc.GC_ERR_ARG
    assert lib.gc_plan_launch(None, None) == gc.GC_ERR_ARG
    assert lib.gc_plan_stats(None, None) == gc.GC_ERR_ARG
    lib.gc_plan_destroy(None)

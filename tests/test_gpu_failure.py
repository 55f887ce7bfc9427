"""Failure detection on the device without a GPU fault: the persistent
kernels' grid barrier waits with a time limit; a launch whose barrier waits
for an arrival that never comes must give up after the limit, report
GC_EW_TIMEOUT / GC_ERR_TIMEOUT and leave the context usable."""
import time

import numpy as np
import pytest

import oracle as O
from paper_1505_04086_gb300 import inputs as I

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from paper_1505_04086_gb300 import gc  # noqa: E402


def test_barrier_wait_runs_out_and_reports_timeout():
    t0 = time.perf_counter()
    rc, word = gc.gc_debug_barrier_timeout(0, 300)
    dt = time.perf_counter() - t0
    assert rc == gc.GC_ERR_TIMEOUT, gc.gc_strerror(rc)
    assert word & gc.GC_EW_TIMEOUT
    assert 0.25 <= dt < 10.0, dt


def test_context_usable_after_a_timeout():
    rc, _ = gc.gc_debug_barrier_timeout(0, 100)
    assert rc == gc.GC_ERR_TIMEOUT
    g = I.kuhn3d(8)
    ctx = gc.Context(0)
    try:
        d = torch.device("cuda:0")
        col, rc, st = ctx.color(torch.from_numpy(g.row_ptr).to(d), torch.from_numpy(g.col_idx).to(d),
                                mode=gc.GC_SCHED_DET)
        assert rc == gc.GC_OK
        assert np.array_equal(col.cpu().numpy(), O.rsoc_det(g).colors)
    finally:
        ctx.close()


def test_barrier_timeout_arguments():
    assert gc.gc_debug_barrier_timeout(0, 0)[0] == gc.GC_ERR_ARG
    assert gc.gc_debug_barrier_timeout(0, 20000)[0] == gc.GC_ERR_ARG

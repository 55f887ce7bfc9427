"""Failure detection on the device without a GPU fault: every wait of the
colouring kernel has a time limit.  A launch whose grid barrier waits for an
arrival that never comes, whose ordered-pass tile wait waits for a flag
nobody publishes, whose warp-group chunk waits for a lower neighbour nobody
colours, or whose staged-copy wait waits for a copy that never completes,
must give up after the limit, report GC_EW_TIMEOUT / GC_ERR_TIMEOUT and
leave the context usable."""
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


WAITS = {"tile_done": gc.GC_WAIT_TILE_DONE, "pipe_chunk": gc.GC_WAIT_PIPE_CHUNK,
         "stage_copy": gc.GC_WAIT_STAGE_COPY, "grid_barrier": gc.GC_WAIT_GRID_BARRIER}


@pytest.mark.parametrize("wait", list(WAITS))
def test_every_wait_runs_out_and_reports_timeout(wait):
    limit_ms = 200
    t0 = time.perf_counter()
    rc, word = gc.gc_debug_wait_timeout(0, WAITS[wait], limit_ms)
    dt = time.perf_counter() - t0
    assert rc == gc.GC_ERR_TIMEOUT, gc.gc_strerror(rc)
    assert word & gc.GC_EW_TIMEOUT
    # the staged-copy wait waits twice (the second lets a copy in flight land)
    most = 2 if wait == "stage_copy" else 1
    assert 0.8 * limit_ms / 1e3 <= dt < most * limit_ms / 1e3 + 5.0, dt
    # the context still colours correctly afterwards
    g = I.kuhn3d(6)
    ctx = gc.Context(0)
    try:
        d = torch.device("cuda:0")
        col, rc, _ = ctx.color(torch.from_numpy(g.row_ptr).to(d), torch.from_numpy(g.col_idx).to(d),
                               mode=gc.GC_SCHED_DET)
        assert rc == gc.GC_OK
        assert np.array_equal(col.cpu().numpy(), O.rsoc_det(g).colors)
    finally:
        ctx.close()


def test_wait_probe_arguments():
    assert gc.gc_debug_wait_timeout(0, 7, 100)[0] == gc.GC_ERR_ARG
    assert gc.gc_debug_wait_timeout(0, gc.GC_WAIT_TILE_DONE, 0)[0] == gc.GC_ERR_ARG
    assert gc.gc_debug_wait_timeout(0, gc.GC_WAIT_TILE_DONE, 20000)[0] == gc.GC_ERR_ARG

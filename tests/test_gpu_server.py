"""Serving runtime: continuous batching under a device-memory budget.

Each request's result must equal the colouring of the same graph alone
(deterministic mode: bit-exact with the oracle's replay; asynchronous mode:
a proper colouring), whatever else was in flight with it."""
import threading
import time

import numpy as np
import pytest

import oracle as O
from paper_1505_04086_gb300 import inputs as I

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from paper_1505_04086_gb300 import gc  # noqa: E402


def graphs(k, seed=3):
    b = I.batch(k, 1 << 8, 1 << 13, seed=seed, threads=8)
    gs = [b.graph(g) for g in range(b.G)]
    gs += [I.rmat(10), I.from_edges(2, [(0, 1)]), I.from_edges(0, []), I.tri2d(64, 64)]
    return gs


def test_results_equal_alone_det():
    gs = graphs(40)
    srv = gc.Server(0, budget_bytes=64 << 20, max_slots=64, mode=gc.GC_ALG_RSOC)
    try:
        tickets = [srv.submit(g.row_ptr, g.col_idx) for g in gs]
        for g, t in zip(gs, tickets):
            rc, col, st = srv.wait(t, g.n, timeout_ms=20000)
            assert rc == gc.GC_OK
            ref = O.rsoc_det(g)
            assert np.array_equal(col, ref.colors)
            assert st["rounds"] == ref.iterations and st["conflicts"] == ref.conflicts
            assert st["colors"] == (ref.num_colors if g.n else 0)
        info = srv.info()
        assert info["completed"] == len(gs) and info["failed"] == 0
        assert info["peak_bytes"] <= info["budget_bytes"]
        assert info["waves"] >= 1
    finally:
        srv.close()


def test_budget_admission_and_overlap():
    # A budget that holds only a few graphs at a time: all requests still
    # finish, memory in use never passes the budget, and several waves run.
    gs = graphs(60, seed=5)
    big = max(4 * (g.n + 1 + g.nnz) for g in gs)
    budget = 3 * big
    srv = gc.Server(0, budget_bytes=budget, max_slots=8, mode=gc.GC_ALG_RSOC | gc.GC_SCHED_ASYNC)
    try:
        tickets = [srv.submit(g.row_ptr, g.col_idx) for g in gs]
        seen_peak = 0
        for g, t in zip(gs, tickets):
            rc, col, st = srv.wait(t, g.n, timeout_ms=20000)
            assert rc == gc.GC_OK
            assert O.check(g, col)[0] == 0
            seen_peak = max(seen_peak, srv.info()["in_use_bytes"])
        info = srv.info()
        assert info["peak_bytes"] <= budget and seen_peak <= budget
        assert info["waves"] >= 3
        assert info["max_wave_graphs"] <= 8
    finally:
        srv.close()


def test_too_large_is_rejected_and_poll_states():
    srv = gc.Server(0, budget_bytes=1 << 16, max_slots=4)
    try:
        g = I.kuhn3d(20)
        with pytest.raises(gc.GCError) as e:
            srv.submit(g.row_ptr, g.col_idx)
        assert e.value.status == gc.GC_ERR_BUDGET
        small = I.from_edges(3, [(0, 1), (1, 2)])
        t = srv.submit(small.row_ptr, small.col_idx)
        rc, col, st = srv.wait(t, small.n, timeout_ms=20000)
        assert rc == gc.GC_OK and col.tolist() == [1, 2, 1]
        rc, _, _ = srv.poll(t, small.n)
        assert rc == gc.GC_ERR_NOT_FOUND
    finally:
        srv.close()


def test_concurrent_submitters_det():
    gs = graphs(32, seed=9)
    srv = gc.Server(0, budget_bytes=32 << 20, max_slots=16)
    out = {}

    def worker(idx):
        for i in idx:
            t = srv.submit(gs[i].row_ptr, gs[i].col_idx)
            time.sleep(0.0005)
            out[i] = t

    try:
        th = [threading.Thread(target=worker, args=(list(range(k, len(gs), 4)),)) for k in range(4)]
        for x in th:
            x.start()
        for x in th:
            x.join()
        for i, g in enumerate(gs):
            rc, col, st = srv.wait(out[i], g.n, timeout_ms=20000)
            assert rc == gc.GC_OK
            assert np.array_equal(col, O.rsoc_det(g).colors)
    finally:
        srv.close()


def test_destroy_with_requests_in_flight():
    gs = graphs(16, seed=13)
    srv = gc.Server(0, budget_bytes=16 << 20, max_slots=8)
    for g in gs:
        srv.submit(g.row_ptr, g.col_idx)
    srv.close()  # must not hang or leak device memory into the next server
    srv2 = gc.Server(0, budget_bytes=16 << 20, max_slots=8)
    try:
        t = srv2.submit(gs[0].row_ptr, gs[0].col_idx)
        rc, col, _ = srv2.wait(t, gs[0].n, timeout_ms=20000)
        assert rc == gc.GC_OK
    finally:
        srv2.close()


@pytest.mark.parametrize("mode", [gc.GC_SCHED_ASYNC, gc.GC_SCHED_ASYNC | gc.GC_FF_KEEPERS,
                                  gc.GC_SCHED_ASYNC | gc.GC_ALG_TWO_PHASE], ids=["async", "keepers", "twophase"])
def test_async_modes_valid_per_request(mode):
    gs = graphs(24, seed=5)
    srv = gc.Server(0, budget_bytes=32 << 20, max_slots=32, mode=mode)
    try:
        tickets = [srv.submit(g.row_ptr, g.col_idx) for g in gs]
        for g, t in zip(gs, tickets):
            rc, col, st = srv.wait(t, g.n, timeout_ms=20000)
            assert rc == gc.GC_OK
            assert O.check(g, col)[0] == 0
    finally:
        srv.close()


def test_waves_run_side_by_side():
    # A long request, then short ones behind it: with two compute lanes the
    # short ones are coloured in a second wave while the first still runs.
    # The overlap is measured on the GPU (event timestamps around each wave's
    # colouring), and every result stays what the graph gives alone.
    big = I.rmat(20, 16)
    small = graphs(24, seed=9)
    srv = gc.Server(0, budget_bytes=1 << 30, max_slots=256, mode=gc.GC_ALG_RSOC)
    try:
        assert srv.info()["lanes"] == 2
        t_big = srv.submit(big.row_ptr, big.col_idx)
        time.sleep(0.002)  # let the first wave start
        ts = [srv.submit(g.row_ptr, g.col_idx) for g in small]
        for g, t in zip(small, ts):
            rc, col, _ = srv.wait(t, g.n, timeout_ms=60000)
            assert rc == gc.GC_OK
            assert np.array_equal(col, O.rsoc_det(g).colors)
        rc, col, st = srv.wait(t_big, big.n, timeout_ms=60000)
        assert rc == gc.GC_OK
        ref = O.rsoc_det(big)
        assert np.array_equal(col, ref.colors) and st["rounds"] == ref.iterations
        info = srv.info()
        assert info["waves"] >= 2
        assert info["overlapped_waves"] >= 1 and info["overlap_us"] > 0, info
    finally:
        srv.close()


def test_cancel():
    gs = graphs(30, seed=11)
    # one slot: everything but the first request stays queued for a while
    srv = gc.Server(0, budget_bytes=64 << 20, max_slots=1, mode=gc.GC_ALG_RSOC)
    try:
        ts = [srv.submit(g.row_ptr, g.col_idx) for g in gs]
        gone = ts[5::3]
        for t in gone:
            assert srv.cancel(t) == gc.GC_OK
            assert srv.cancel(t) == gc.GC_ERR_NOT_FOUND
            assert srv.poll(t, 1)[0] == gc.GC_ERR_NOT_FOUND
        for g, t in zip(gs, ts):
            if t in gone:
                continue
            rc, col, _ = srv.wait(t, g.n, timeout_ms=20000)
            assert rc == gc.GC_OK
            assert np.array_equal(col, O.rsoc_det(g).colors)
        # a finished request can be dropped unpolled, and the server goes on
        t = srv.submit(gs[0].row_ptr, gs[0].col_idx)
        deadline = time.time() + 20
        while time.time() < deadline:
            i = srv.info()
            if i["queued"] == 0 and i["resident"] == 0:
                break
            time.sleep(0.001)
        assert srv.cancel(t) == gc.GC_OK
        info = srv.info()
        assert info["cancelled"] == len(gone) + 1
        assert info["resident"] == 0 and info["in_use_bytes"] == 0
        t = srv.submit(gs[1].row_ptr, gs[1].col_idx)
        rc, col, _ = srv.wait(t, gs[1].n, timeout_ms=20000)
        assert rc == gc.GC_OK and np.array_equal(col, O.rsoc_det(gs[1]).colors)
        assert srv.cancel(12345678) == gc.GC_ERR_NOT_FOUND
    finally:
        srv.close()


def test_cancel_in_flight_then_destroy():
    # requests cancelled while on the GPU are released when their work ends,
    # or by destroy
    gs = graphs(20, seed=13)
    srv = gc.Server(0, budget_bytes=256 << 20, max_slots=64, mode=gc.GC_ALG_RSOC | gc.GC_SCHED_ASYNC)
    ts = [srv.submit(g.row_ptr, g.col_idx) for g in gs]
    for t in ts:
        assert srv.cancel(t) == gc.GC_OK
    srv.close()

"""Asynchronous colourings of graphs of uniform low degree whose ids are
not local (round 0 over tiles claimed in id order, unclaimed higher
neighbours not read): valid and within 1.15x of sequential First-Fit for
every grid size, tile, thread/warp split and repair form, with ragged last
chunks and with warps that get no chunk at all."""
import numpy as np
import pytest

import oracle as O
from paper_1505_04086_gb300 import inputs as I

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from paper_1505_04086_gb300 import gc  # noqa: E402

ASYNC = gc.GC_SCHED_ASYNC
MODES = {"rsoc": ASYNC, "twophase": ASYNC | gc.GC_ALG_TWO_PHASE, "snapshot": ASYNC | gc.GC_REPAIR_SNAPSHOT}


@pytest.fixture(scope="module")
def ctx():
    c = gc.Context(0)
    yield c
    c.close()


@pytest.fixture(scope="module")
def graphs():
    # 31^3 = 29,791 and 42^3 = 74,088 vertices (neither a multiple of 32),
    # ids permuted; a random geometric graph of mean degree 12
    gs = [I.kuhn3d(30), I.kuhn3d(41), I.rgg(40000, 12.0, seed=5)]
    return [(g, int(O.ff(g).max())) for g in gs]


def colour(ctx, g, mode, opts):
    d = torch.device("cuda:0")
    rp, ci = torch.from_numpy(g.row_ptr).to(d), torch.from_numpy(g.col_idx).to(d)
    col = torch.empty(g.n, dtype=torch.int32, device=d)
    rc = gc.gc_color_async(ctx.handle, rp, ci, g.n, g.nnz, mode, col, opts)
    assert rc == gc.GC_OK, gc.gc_strerror(rc)
    rc, st = gc.gc_ctx_stats(ctx.handle)
    assert rc == gc.GC_OK, gc.gc_strerror(rc)
    return col.cpu().numpy(), st


@pytest.mark.parametrize("mode", list(MODES))
@pytest.mark.parametrize("bps,tile,t1", [(1, 32, 62), (2, 32, 48), (3, 64, 62), (2, 128, 8), (0, 32, 62)])
def test_uniform_degree_round0_valid(ctx, graphs, mode, bps, tile, t1):
    opts = {"blocks_per_sm": bps, "tile": tile, "t1": t1}
    for g, ff in graphs:
        for _ in range(2):
            col, st = colour(ctx, g, MODES[mode], opts)
            bad, mx, dist = O.check(g, col)
            assert bad == 0, (g.name, mode, opts)
            assert mx <= 1.15 * ff, (g.name, mode, opts, mx, ff)
            assert st["colors"] == mx and st["distinct_colors"] == dist


def test_uniform_degree_full_size_bound(ctx):
    # Kuhn 128^3 (2^21 vertices, ids permuted) at two and three blocks per SM
    g = I.workload("kuhn3d_128")
    ff = int(O.ff(g).max())
    for bps in (2, 3):
        col, st = colour(ctx, g, ASYNC, {"blocks_per_sm": bps, "tile": 32})
        bad, mx, _ = O.check(g, col)
        assert bad == 0 and mx <= 1.1 * ff, (bps, mx, ff)


def test_row_pointers_at_any_alignment(ctx, graphs):
    # the binning reads row pointers 16 bytes at a time when they are so
    # aligned; views one to three entries into a buffer take the other path
    g, ff = graphs[0]
    d = torch.device("cuda:0")
    for off in range(4):
        buf = torch.zeros(g.n + 1 + off, dtype=torch.int32, device=d)
        buf[off:] = torch.from_numpy(g.row_ptr).to(d)
        rp = buf[off:]
        ci = torch.from_numpy(g.col_idx).to(d)
        col = torch.empty(g.n, dtype=torch.int32, device=d)
        rc = gc.gc_color_async(ctx.handle, rp, ci, g.n, g.nnz, ASYNC, col, None)
        assert rc == gc.GC_OK, gc.gc_strerror(rc)
        rc, st = gc.gc_ctx_stats(ctx.handle)
        assert rc == gc.GC_OK, gc.gc_strerror(rc)
        bad, mx, _ = O.check(g, col.cpu().numpy())
        assert bad == 0 and mx <= 1.15 * ff, (off, mx, ff)

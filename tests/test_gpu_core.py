"""The core of high-degree vertices in the asynchronous mode of one graph.

Before round 0 the vertices of degree above max(core_deg, t2) are coloured
one at a time in decreasing degree (ties: increasing id) by First-Fit among
themselves.  Their colours must therefore equal the oracle's sequential
First-Fit (Algorithm 1) on the subgraph they induce, relabelled in that
order, element by element; the whole colouring must be a proper colouring
within the d+1 bound, and on R-MAT (a dense core of hubs) within 1.1x the
colours of sequential First-Fit on the whole graph.
"""
import numpy as np
import pytest

import oracle as O
from paper_1505_04086_gb300 import inputs as I

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from paper_1505_04086_gb300 import gc  # noqa: E402

ASYNC = gc.GC_SCHED_ASYNC
TWOP = gc.GC_ALG_TWO_PHASE


@pytest.fixture(scope="module")
def ctx():
    c = gc.Context(0)
    yield c
    c.close()


def run(ctx, g, mode, opts=None):
    d = torch.device("cuda:0")
    rp = torch.from_numpy(g.row_ptr).to(d)
    ci = torch.from_numpy(g.col_idx if g.nnz else np.zeros(1, np.int32)).to(d)
    col = torch.empty(max(g.n, 1), dtype=torch.int32, device=d)
    rc = gc.gc_color_async(ctx.handle, rp, ci, g.n, g.nnz, mode, col, opts)
    assert rc == gc.GC_OK, gc.gc_strerror(rc)
    rc, st = gc.gc_ctx_stats(ctx.handle, 4096)
    return rc, col[: g.n].cpu().numpy(), st


def core_order(g, thr):
    """Core vertices (degree > thr) by degree descending, id ascending."""
    deg = np.diff(g.row_ptr).astype(np.int64)
    core = np.nonzero(deg > thr)[0]
    return core[np.lexsort((core, -deg[core]))]


def induced(g, order):
    """The subgraph induced by `order`, vertex k standing for order[k]."""
    pos = np.full(g.n, -1, np.int64)
    pos[order] = np.arange(len(order))
    deg = np.diff(g.row_ptr).astype(np.int64)
    src = np.repeat(np.arange(g.n), deg)
    dst = g.col_idx.astype(np.int64)
    keep = (pos[src] >= 0) & (pos[dst] >= 0)
    e = np.stack([pos[src[keep]], pos[dst[keep]]], axis=1)
    e = e[e[:, 0] < e[:, 1]]
    return I.from_edges(len(order), e)


# (scale, core degree): cores of a few hundred to about a thousand vertices
CORES = [(14, 128), (16, 256)]
MODES = {"rsoc": ASYNC, "twophase": TWOP | ASYNC, "higher": ASYNC | gc.GC_TIE_HIGHER_KEEPS,
         "snapshot_repairs": ASYNC | gc.GC_REPAIR_SNAPSHOT}


@pytest.mark.parametrize("scale,thr", CORES)
@pytest.mark.parametrize("mode", list(MODES))
def test_core_is_sequential_first_fit_in_degree_order(ctx, scale, thr, mode):
    g = I.rmat(scale, 16, seed=I.SEED_RMAT)
    opts = {"t1": 16, "t2": thr, "core_deg": thr}
    rc, col, st = run(ctx, g, MODES[mode] | gc.GC_CHECKED, opts)
    assert rc == gc.GC_OK, gc.gc_strerror(rc)
    bad, mx, _ = O.check(g, col)
    assert bad == 0
    order = core_order(g, thr)
    assert 0 < len(order) <= 4096
    ref = O.ff(induced(g, order))
    got = col[order]
    assert np.array_equal(got, ref), f"first difference at rank {np.nonzero(got != ref)[0][:5]}"


@pytest.mark.parametrize("scale,thr", [(16, 16), (16, 128)])
def test_core_too_large_falls_back_to_the_hub_pass(ctx, scale, thr):
    # more than 4096 candidates, or a bit matrix larger than n words: the
    # candidates are coloured as ordinary hubs
    g = I.rmat(scale, 16, seed=I.SEED_RMAT)
    opts = {"t1": 16, "t2": thr, "core_deg": thr}
    rc, col, st = run(ctx, g, ASYNC | gc.GC_CHECKED, opts)
    assert rc == gc.GC_OK, gc.gc_strerror(rc)
    assert O.check(g, col)[0] == 0


def test_core_off_is_valid(ctx):
    g = I.rmat(16, 16, seed=I.SEED_RMAT)
    rc, col, st = run(ctx, g, ASYNC | gc.GC_CHECKED, {"core_deg": -1})
    assert rc == gc.GC_OK
    assert O.check(g, col)[0] == 0


def test_core_repeated_calls_are_valid(ctx):
    # the core reuses scratch of the context: back-to-back calls, the larger
    # graph first, must each stay valid and reproduce the core exactly
    big, small = I.rmat(16, 16, seed=I.SEED_RMAT), I.rmat(14, 16, seed=I.SEED_RMAT)
    for g, thr in ((big, 256), (small, 128), (big, 256)):
        rc, col, _ = run(ctx, g, ASYNC, {"t1": 16, "t2": thr, "core_deg": thr})
        assert rc == gc.GC_OK
        assert O.check(g, col)[0] == 0
        order = core_order(g, thr)
        assert np.array_equal(col[order], O.ff(induced(g, order)))


def test_core_noalloc_matches(ctx):
    g = I.rmat(14, 16, seed=I.SEED_RMAT)
    d = torch.device("cuda:0")
    rp, ci = torch.from_numpy(g.row_ptr).to(d), torch.from_numpy(g.col_idx).to(d)
    col = torch.empty(g.n, dtype=torch.int32, device=d)
    rc, st = gc.gc_color_noalloc(rp, ci, g.n, g.nnz, ASYNC, col, {"t1": 16, "t2": 128, "core_deg": 128})
    assert rc == gc.GC_OK, gc.gc_strerror(rc)
    c = col.cpu().numpy()
    assert O.check(g, c)[0] == 0
    order = core_order(g, 128)
    assert np.array_equal(c[order], O.ff(induced(g, order)))


def _batch_run(ctx, gs, mode, opts=None):
    b = I.Batch.from_graphs(gs, name="t")
    d = torch.device("cuda:0")
    vo, eo = torch.from_numpy(b.vtx_off).to(d), torch.from_numpy(b.edge_off).to(d)
    rp, ci = torch.from_numpy(b.row_ptr).to(d), torch.from_numpy(b.col_idx).to(d)
    col = torch.empty(b.total_n, dtype=torch.int32, device=d)
    rc = gc.gc_color_batch(ctx.handle, b.G, b.total_n, b.total_nnz, vo, eo, rp, ci, mode, col, None, None, opts)
    assert rc == gc.GC_OK, gc.gc_strerror(rc)
    rc, st = gc.gc_ctx_stats(ctx.handle)
    assert rc == gc.GC_OK, gc.gc_strerror(rc)
    c = col.cpu().numpy()
    return [c[int(b.vtx_off[i]):int(b.vtx_off[i + 1])] for i in range(b.G)]


@pytest.mark.parametrize("mode", ["rsoc", "twophase"])
def test_batch_cores_are_sequential_first_fit(ctx, mode):
    # every graph of a batch gets its own core
    thr = 256
    gs = [I.rmat(14, 16, seed=I.SEED_RMAT), I.tri2d(40, 40, 0.2), I.rmat(16, 16, seed=I.SEED_RMAT + 7),
          I.rgg(5000, seed=11), I.rmat(15, 16, seed=I.SEED_RMAT + 3)]
    cols = _batch_run(ctx, gs, MODES[mode] | gc.GC_CHECKED, {"t1": 16, "t2": thr, "core_deg": thr})
    for g, c in zip(gs, cols):
        assert O.check(g, c)[0] == 0, g.name
        order = core_order(g, thr)
        if 0 < len(order) <= 4096:
            assert np.array_equal(c[order], O.ff(induced(g, order))), g.name


def test_batch_rmat18_requests_within_bound(ctx):
    # the serving mix: R-MAT 2^18 graphs among meshes, default options
    mix = I.batch(12, seed=I.SEED_SERVE)
    gs = [mix.graph(i) for i in range(mix.G)] + [I.rmat(18, 16, seed=I.SEED_SERVE + 100 + k) for k in range(2)]
    for mode in (ASYNC, ASYNC | TWOP):
        cols = _batch_run(ctx, gs, mode | gc.GC_CHECKED)
        for g, c in zip(gs, cols):
            bad, mx, _ = O.check(g, c)
            assert bad == 0
            assert mx <= 1.1 * int(O.ff(g).max()), (g.name, mx)

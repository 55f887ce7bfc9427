"""gc_recolor_async: incremental recolouring after an edit (Algorithm 3's
loop from the given colours with U = the touched vertices).  Deterministic
mode against the oracle's replay element by element; asynchronous mode for
validity and locality."""
import numpy as np
import pytest

import oracle as O
from paper_1505_04086_gb300 import inputs as I

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from paper_1505_04086_gb300 import gc  # noqa: E402

HIGHER = gc.GC_TIE_HIGHER_KEEPS


@pytest.fixture(scope="module")
def ctx():
    c = gc.Context(0)
    yield c
    c.close()


def add_edges(g, extra):
    e = [(v, u) for v in range(g.n) for u in g.col_idx[g.row_ptr[v]:g.row_ptr[v + 1]] if u > v]
    return I.from_edges(g.n, e + list(extra))


def recolor(ctx, g, colors, touched, mode, opts=None):
    rp = torch.from_numpy(g.row_ptr).cuda()
    ci = torch.from_numpy(g.col_idx if g.nnz else np.zeros(1, np.int32)).cuda()
    col = torch.from_numpy(np.ascontiguousarray(colors, dtype=np.int32)).cuda()
    t = torch.from_numpy(np.ascontiguousarray(touched, dtype=np.int32) if len(touched)
                         else np.zeros(1, np.int32)).cuda()[:len(touched)]
    rc = gc.gc_recolor_async(ctx.handle, rp, ci, g.n, g.nnz, mode, col, t, opts)
    assert rc == gc.GC_OK, gc.gc_strerror(rc)
    rc, st = gc.gc_ctx_stats(ctx.handle, 4096)
    return rc, col.cpu().numpy(), st


def edit(g, seed, k=40):
    """FF colouring, then k inserted edges between equal-coloured vertices."""
    rng = np.random.default_rng(seed)
    c = O.ff(g)
    extra, touched = [], []
    for _ in range(k):
        v = int(rng.integers(g.n))
        same = np.nonzero(c == c[v])[0]
        u = int(same[rng.integers(same.size)])
        if u != v and u not in g.col_idx[g.row_ptr[v]:g.row_ptr[v + 1]]:
            extra.append((v, u))
            touched += [v, u]
    return add_edges(g, extra), c, touched


GRAPHS = {"kuhn10": lambda: I.kuhn3d(10), "tri_jit": lambda: I.tri2d(40, 50, jitter=0.3, seed=6),
          "rmat11": lambda: I.rmat(11)}


def assert_same(rc, col, st, ref):
    assert rc == gc.GC_OK
    assert np.array_equal(col, ref.colors)
    assert st["rounds"] == ref.iterations and st["conflicts"] == ref.conflicts
    assert np.array_equal(st["round_sizes"], ref.round_sizes[: len(st["round_sizes"])])
    assert st["model_bytes"] == ref.model_bytes


@pytest.mark.parametrize("name", list(GRAPHS))
@pytest.mark.parametrize("tie", [0, HIGHER], ids=["lower", "higher"])
@pytest.mark.parametrize("bins", [None, {"t1": 4, "t2": 24}], ids=["default", "bins"])
def test_det_recolor_equals_oracle(ctx, name, tie, bins):
    otie = O.TIE_HIGHER_KEEPS if tie else O.TIE_LOWER_KEEPS
    g0 = GRAPHS[name]()
    g, c, touched = edit(g0, seed=len(name))
    # an edit: inserted conflicting edges
    assert_same(*recolor(ctx, g, c, touched, tie, bins), O.rsoc_det_from(g, c, touched, otie))
    # from all ones with every vertex touched: the full deterministic run
    ones = np.ones(g0.n, np.int32)
    assert_same(*recolor(ctx, g0, ones, np.arange(g0.n), tie, bins), O.rsoc_det(g0, otie))
    # uncoloured vertices, listed twice
    c2 = O.ff(g0)
    holes = np.arange(0, g0.n, 7)
    c2[holes] = 0
    t2 = np.concatenate([holes, holes[::-1]])
    assert_same(*recolor(ctx, g0, c2, t2, tie, bins), O.rsoc_det_from(g0, c2, t2, otie))


def test_det_recolor_nothing_touched(ctx):
    g = I.kuhn3d(8)
    c = O.ff(g)
    rc, col, st = recolor(ctx, g, c, [], 0)
    assert rc == gc.GC_OK and np.array_equal(col, c) and st["rounds"] == 0


@pytest.mark.parametrize("mode", [gc.GC_SCHED_ASYNC, gc.GC_SCHED_ASYNC | gc.GC_FF_KEEPERS],
                         ids=["async", "keepers"])
def test_async_recolor_valid_and_local(ctx, mode):
    for name, make in GRAPHS.items():
        g, c, touched = edit(make(), seed=3)
        for _ in range(3):
            rc, col, st = recolor(ctx, g, c, touched, mode | gc.GC_CHECKED)
            assert rc == gc.GC_OK
            assert O.check(g, col)[0] == 0
            if not mode & gc.GC_FF_KEEPERS:  # keepers also queues the higher neighbours it clashes with
                changed = np.nonzero(col != c)[0]
                assert set(changed.tolist()) <= set(touched), name


def test_recolor_argument_errors(ctx):
    g = I.kuhn3d(6)
    rc, col, st = None, None, None
    rp = torch.from_numpy(g.row_ptr).cuda()
    ci = torch.from_numpy(g.col_idx).cuda()
    col = torch.ones(g.n, dtype=torch.int32, device="cuda")
    bad = torch.tensor([1, g.n], dtype=torch.int32, device="cuda")
    assert gc.gc_recolor_async(ctx.handle, rp, ci, g.n, g.nnz, 0, col, bad) == gc.GC_OK
    assert gc.gc_ctx_stats(ctx.handle)[0] == gc.GC_ERR_GRAPH
    ok = torch.tensor([1], dtype=torch.int32, device="cuda")
    for m in (gc.GC_ALG_TWO_PHASE, gc.GC_SCHED_ASYNC | gc.GC_TIERS, gc.GC_SCHED_ASYNC | gc.GC_REPAIR_SNAPSHOT):
        assert gc.gc_recolor_async(ctx.handle, rp, ci, g.n, g.nnz, m, col, ok) == gc.GC_ERR_ARG

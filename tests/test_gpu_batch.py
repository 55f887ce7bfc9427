"""Batched colouring (one persistent launch over many graphs) against the
oracle run on each graph alone."""
import numpy as np
import pytest

import oracle as O
from paper_1505_04086_gb300 import inputs as I

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from paper_1505_04086_gb300 import gc  # noqa: E402


@pytest.fixture(scope="module")
def ctx():
    c = gc.Context(0)
    yield c
    c.close()


def to_dev(b):
    d = "cuda:0"
    ci = b.col_idx if b.col_idx.size else np.zeros(1, np.int32)
    return (torch.from_numpy(b.vtx_off).to(d), torch.from_numpy(b.edge_off).to(d),
            torch.from_numpy(b.row_ptr).to(d), torch.from_numpy(ci).to(d))


def mixed_batch():
    gs = [I.tri2d(20, 30, jitter=0.3, seed=1), I.from_edges(2, [(0, 1)]), I.kuhn3d(7),
          I.from_edges(0, []), I.rgg(3000, 12.0, seed=4), I.from_edges(5, []),
          I.rmat(10), I.tri2d(64, 64), I.from_edges(3, [(0, 1), (1, 2), (0, 2)]),
          I.kuhn3d(9, permute=False)]
    return I.Batch.from_graphs(gs, name="mixed")


def run_batch(ctx, b, mode, opts=None):
    vo, eo, rp, ci = to_dev(b)
    col, rounds, confl, rc, st = ctx.color_batch(vo, eo, rp, ci, b.total_n, b.total_nnz, mode=mode,
                                                  opts=opts, check=False)
    return rc, col.cpu().numpy(), rounds.cpu().numpy(), confl.cpu().numpy(), st


@pytest.mark.parametrize("alg", [gc.GC_ALG_RSOC, gc.GC_ALG_TWO_PHASE], ids=["rsoc", "twophase"])
@pytest.mark.parametrize("tie", [0, gc.GC_TIE_HIGHER_KEEPS], ids=["lower", "higher"])
@pytest.mark.parametrize("bins", [None, {"t1": 4, "t2": 12}], ids=["default", "mixed_bins"])
def test_det_batch_equals_each_graph_alone(ctx, alg, tie, bins):
    b = mixed_batch()
    rc, col, rounds, confl, st = run_batch(ctx, b, alg | tie, bins)
    assert rc == gc.GC_OK
    otie = O.TIE_HIGHER_KEEPS if tie else O.TIE_LOWER_KEEPS
    replay = O.twophase_det if alg == gc.GC_ALG_TWO_PHASE else O.rsoc_det
    max_it = 0
    for g in range(b.G):
        sub = b.graph(g)
        ref = replay(sub, tie=otie)
        v0, v1 = int(b.vtx_off[g]), int(b.vtx_off[g + 1])
        assert np.array_equal(col[v0:v1], ref.colors), f"graph {g}"
        assert rounds[g] == ref.iterations, f"graph {g}"
        assert confl[g] == ref.conflicts, f"graph {g}"
        max_it = max(max_it, ref.iterations)
    assert st["rounds"] == max_it
    assert st["conflicts"] == int(confl.sum())


@pytest.mark.parametrize("alg", [gc.GC_ALG_RSOC, gc.GC_ALG_TWO_PHASE], ids=["rsoc", "twophase"])
def test_async_batch_valid(ctx, alg):
    b = mixed_batch()
    for _ in range(3):
        rc, col, rounds, confl, st = run_batch(ctx, b, alg | gc.GC_SCHED_ASYNC)
        assert rc == gc.GC_OK
        for g in range(b.G):
            sub = b.graph(g)
            v0, v1 = int(b.vtx_off[g]), int(b.vtx_off[g + 1])
            assert O.check(sub, col[v0:v1])[0] == 0, f"graph {g}"
            assert rounds[g] >= (1 if sub.n else 0)


def test_generated_batch_det(ctx):
    b = I.batch(48, 1 << 8, 1 << 13, seed=11, threads=8)
    rc, col, rounds, confl, st = run_batch(ctx, b, gc.GC_ALG_RSOC)
    assert rc == gc.GC_OK
    for g in range(b.G):
        sub = b.graph(g)
        ref = O.rsoc_det(sub)
        v0, v1 = int(b.vtx_off[g]), int(b.vtx_off[g + 1])
        assert np.array_equal(col[v0:v1], ref.colors)
        assert rounds[g] == ref.iterations and confl[g] == ref.conflicts


def test_batch_validate_and_empty(ctx):
    b = I.Batch.from_graphs([I.from_edges(0, []), I.from_edges(0, [])])
    vo, eo, rp, ci = to_dev(b)
    col = torch.zeros(1, dtype=torch.int32, device="cuda:0")
    rc = gc.gc_color_batch(ctx.handle, b.G, 0, 0, vo, eo, rp, ci, 0, col)
    assert rc == gc.GC_OK
    assert gc.gc_ctx_stats(ctx.handle)[0] == gc.GC_OK
    good = mixed_batch()
    rc, *_ = run_batch(ctx, good, gc.GC_VALIDATE | gc.GC_CHECKED)
    assert rc == gc.GC_OK
    bad = mixed_batch()
    bad.col_idx = bad.col_idx.copy()
    g = 2  # kuhn3d(7): break symmetry inside it with an in-range id
    e0 = int(bad.edge_off[g])
    bad.col_idx[e0] = (bad.col_idx[e0] + 1) % int(bad.vtx_off[g + 1] - bad.vtx_off[g])
    rc, *_ = run_batch(ctx, bad, gc.GC_VALIDATE)
    assert rc == gc.GC_ERR_GRAPH


def test_async_batch_quality_per_graph(ctx):
    # Naturally numbered meshes are coloured in id order by one warp each
    # (sequential First-Fit exactly); random-order graphs speculatively.
    b = I.batch(64, 1 << 9, 1 << 14, seed=21, threads=8)
    for alg in (gc.GC_ALG_RSOC,):
        rc, col, rounds, confl, st = run_batch(ctx, b, alg | gc.GC_SCHED_ASYNC)
        assert rc == gc.GC_OK
        for g in range(b.G):
            sub = b.graph(g)
            v0, v1 = int(b.vtx_off[g]), int(b.vtx_off[g + 1])
            bad, mx, _ = O.check(sub, col[v0:v1])
            assert bad == 0
            ff = int(O.ff(sub).max())
            assert mx <= 1.1 * ff, f"graph {g} kind {b.kind[g]}: {mx} vs first-fit {ff}"


def test_ordered_batch_is_sequential_first_fit_per_graph(ctx):
    # With window 1 every graph of the batch is coloured in id order in round
    # 0 (big ones by warp groups, the rest one warp each): each graph's
    # colouring is exactly sequential First-Fit of that graph alone.
    b = I.batch(40, 1 << 8, 1 << 16, seed=41, threads=8)
    assert int(np.diff(b.row_ptr).max()) <= 62
    rc, col, rounds, confl, st = run_batch(ctx, b, gc.GC_SCHED_ASYNC, {"t1": 62, "t2": 4096, "window": 1})
    assert rc == gc.GC_OK
    assert st["conflicts"] == 0
    for g in range(b.G):
        sub = b.graph(g)
        v0, v1 = int(b.vtx_off[g]), int(b.vtx_off[g + 1])
        assert np.array_equal(col[v0:v1], O.ff(sub)), f"graph {g}"

"""Batch plans (a gc_color_batch call captured in a CUDA graph and replayed)
and the batch autotuner."""
import numpy as np
import pytest

import oracle as O
from paper_1505_04086_gb300 import inputs as I

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from paper_1505_04086_gb300 import gc  # noqa: E402


def dev_batch(b):
    d = "cuda:0"
    ci = b.col_idx if b.col_idx.size else np.zeros(1, np.int32)
    return (torch.from_numpy(b.vtx_off).to(d), torch.from_numpy(b.edge_off).to(d),
            torch.from_numpy(b.row_ptr).to(d), torch.from_numpy(ci).to(d))


def small_batch():
    return I.batch(24, 1 << 8, 1 << 12, seed=31, threads=8)


def test_plan_replays_give_the_oracle_result():
    b = small_batch()
    vo, eo, rp, ci = dev_batch(b)
    col = torch.full((b.total_n,), -1, dtype=torch.int32, device="cuda:0")
    rounds = torch.zeros(b.G, dtype=torch.int32, device="cuda:0")
    confl = torch.zeros(b.G, dtype=torch.int64, device="cuda:0")
    plan = gc.Plan(0, b.G, b.total_n, b.total_nnz, vo, eo, rp, ci, gc.GC_ALG_RSOC, col, rounds, confl)
    refs = [O.rsoc_det(b.graph(g)) for g in range(b.G)]
    for rep in range(3):
        col.fill_(-1)
        rounds.fill_(-1)
        assert plan.launch() == gc.GC_OK
        rc, st = plan.stats(16)
        assert rc == gc.GC_OK
        assert st["elapsed_ms"] > 0
        c, r, k = col.cpu().numpy(), rounds.cpu().numpy(), confl.cpu().numpy()
        for g, ref in enumerate(refs):
            v0, v1 = int(b.vtx_off[g]), int(b.vtx_off[g + 1])
            assert np.array_equal(c[v0:v1], ref.colors), (rep, g)
            assert r[g] == ref.iterations and k[g] == ref.conflicts
        assert st["rounds"] == max(ref.iterations for ref in refs)
    plan.close()


def test_plan_async_on_a_stream_and_empty_batch():
    b = small_batch()
    vo, eo, rp, ci = dev_batch(b)
    col = torch.zeros(b.total_n, dtype=torch.int32, device="cuda:0")
    s = torch.cuda.Stream()
    plan = gc.Plan(0, b.G, b.total_n, b.total_nnz, vo, eo, rp, ci, gc.GC_SCHED_ASYNC | gc.GC_CHECKED, col)
    for _ in range(3):
        assert plan.launch(s) == gc.GC_OK
        assert plan.stats()[0] == gc.GC_OK
        c = col.cpu().numpy()
        for g in range(b.G):
            v0, v1 = int(b.vtx_off[g]), int(b.vtx_off[g + 1])
            assert O.check(b.graph(g), c[v0:v1])[0] == 0
    plan.close()
    e = I.Batch.from_graphs([I.from_edges(0, [])])
    vo, eo, rp, ci = dev_batch(e)
    empty = gc.Plan(0, e.G, 0, 0, vo, eo, rp, ci, 0, col)
    assert empty.launch() == gc.GC_OK
    assert empty.stats()[0] == gc.GC_OK
    empty.close()


@pytest.mark.parametrize("mode", [gc.GC_ALG_RSOC, gc.GC_SCHED_ASYNC], ids=["det", "async"])
def test_autotune_picks_a_valid_faster_or_equal_option_set(mode):
    b = small_batch()
    vo, eo, rp, ci = dev_batch(b)
    ctx = gc.Context(0)
    col = torch.zeros(b.total_n, dtype=torch.int32, device="cuda:0")
    rc, res = gc.gc_autotune_batch(ctx.handle, b.G, b.total_n, b.total_nnz, vo, eo, rp, ci, mode, col, reps=1)
    assert rc == gc.GC_OK
    assert res["evaluated"] > 10
    assert 0 < res["best_ms"] <= res["default_ms"]
    best = res["best"]
    assert 1 <= best["t1"] <= best["t2"] and best["tile"] % 32 == 0
    # the tuned options colour correctly (deterministic mode: exactly the oracle)
    col2, _, _, rc, _ = ctx.color_batch(vo, eo, rp, ci, b.total_n, b.total_nnz, mode=mode | gc.GC_CHECKED,
                                        opts=best)
    assert rc == gc.GC_OK
    if mode == gc.GC_ALG_RSOC:
        c = col2.cpu().numpy()
        for g in range(b.G):
            v0, v1 = int(b.vtx_off[g]), int(b.vtx_off[g + 1])
            assert np.array_equal(c[v0:v1], O.rsoc_det(b.graph(g)).colors)
    ctx.close()


def test_autotune_single_graph():
    g = I.kuhn3d(20)
    rp = torch.from_numpy(g.row_ptr).cuda()
    ci = torch.from_numpy(g.col_idx).cuda()
    col = torch.zeros(g.n, dtype=torch.int32, device="cuda:0")
    ctx = gc.Context(0)
    rc, res = gc.gc_autotune(ctx.handle, rp, ci, g.n, g.nnz, gc.GC_ALG_RSOC, col, reps=1)
    assert rc == gc.GC_OK
    assert res["evaluated"] > 10 and 0 < res["best_ms"] <= res["default_ms"]
    out, rc, st = ctx.color(rp, ci, gc.GC_ALG_RSOC, opts=res["best"])
    assert rc == gc.GC_OK
    assert np.array_equal(out.cpu().numpy(), O.rsoc_det(g).colors)
    ctx.close()


@pytest.mark.parametrize("mode", [gc.GC_SCHED_ASYNC | gc.GC_FF_KEEPERS, gc.GC_SCHED_ASYNC | gc.GC_TIERS,
                                  gc.GC_ALG_TWO_PHASE], ids=["keepers", "tiers", "twophase_det"])
def test_plan_other_modes(mode):
    b = small_batch()
    vo, eo, rp, ci = dev_batch(b)
    col = torch.zeros(b.total_n, dtype=torch.int32, device="cuda:0")
    plan = gc.Plan(0, b.G, b.total_n, b.total_nnz, vo, eo, rp, ci, mode, col)
    for _ in range(2):
        assert plan.launch() == gc.GC_OK
        assert plan.stats()[0] == gc.GC_OK
        c = col.cpu().numpy()
        for g in range(b.G):
            v0, v1 = int(b.vtx_off[g]), int(b.vtx_off[g + 1])
            sub = b.graph(g)
            if mode & gc.GC_SCHED_ASYNC:
                assert O.check(sub, c[v0:v1])[0] == 0
            else:
                assert np.array_equal(c[v0:v1], O.twophase_det(sub).colors)
    plan.close()

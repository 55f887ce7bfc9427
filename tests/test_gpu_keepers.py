"""GC_FF_KEEPERS: asynchronous RSOC whose First-Fit choices avoid only the
lower neighbours (those that keep their colour on a tie), handing clashing
higher neighbours to the next round.  Results must be valid colourings;
colour counts are compared with sequential First-Fit from the oracle."""
import numpy as np
import pytest

import oracle as O
from paper_1505_04086_gb300 import inputs as I

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from paper_1505_04086_gb300 import gc  # noqa: E402

KEEP = gc.GC_SCHED_ASYNC | gc.GC_FF_KEEPERS


@pytest.fixture(scope="module")
def ctx():
    c = gc.Context(0)
    yield c
    c.close()


def dev(g):
    ci = g.col_idx if g.nnz else np.zeros(1, np.int32)
    return torch.from_numpy(g.row_ptr).cuda(), torch.from_numpy(ci).cuda()


GRAPHS = {
    "kuhn16": lambda: I.kuhn3d(16),
    "tri2d_jit": lambda: I.tri2d(80, 90, jitter=0.3, seed=3),
    "rgg30k": lambda: I.rgg(30000, 12.0, seed=5),
    "rmat14": lambda: I.rmat(14),
    "rmat12_bins": lambda: I.rmat(12),
    "star": lambda: I.from_edges(2000, [(0, k) for k in range(1, 2000)]),
}


@pytest.mark.parametrize("name", list(GRAPHS))
@pytest.mark.parametrize("tiers", [0, gc.GC_TIERS], ids=["flat", "tiers"])
def test_keepers_valid(ctx, name, tiers):
    g = GRAPHS[name]()
    rp, ci = dev(g)
    opts = {"t1": 4, "t2": 40} if name.endswith("_bins") else None
    for _ in range(3):
        col, rc, st = ctx.color(rp, ci, KEEP | tiers | gc.GC_CHECKED, opts=opts, check=False)
        assert rc == gc.GC_OK, gc.gc_strerror(rc)
        c = col.cpu().numpy()
        bad, mx, _ = O.check(g, c)
        assert bad == 0
        assert st["colors"] == mx
        assert st["rounds"] >= 1


def test_keepers_rmat_close_to_first_fit(ctx):
    # The dense core of an R-MAT graph is where the paper's recolouring (avoid
    # every neighbour) drifts above sequential First-Fit; keepers stays close.
    g = I.rmat(16)
    ff = int(O.ff(g).max())
    rp, ci = dev(g)
    worst = 0
    for _ in range(5):
        col, rc, st = ctx.color(rp, ci, KEEP | gc.GC_CHECKED)
        assert rc == gc.GC_OK
        worst = max(worst, st["colors"])
    assert worst <= 1.1 * ff, (worst, ff)


def test_keepers_batch_valid(ctx):
    gs = [I.rmat(11), I.tri2d(40, 50, jitter=0.3, seed=2), I.kuhn3d(9), I.from_edges(0, []),
          I.rgg(5000, 12.0, seed=8), I.from_edges(3, [(0, 1), (1, 2), (0, 2)])]
    b = I.Batch.from_graphs(gs, name="keep")
    d = "cuda:0"
    ci = b.col_idx if b.col_idx.size else np.zeros(1, np.int32)
    vo, eo = torch.from_numpy(b.vtx_off).to(d), torch.from_numpy(b.edge_off).to(d)
    rp, cit = torch.from_numpy(b.row_ptr).to(d), torch.from_numpy(ci).to(d)
    col, rounds, confl, rc, st = ctx.color_batch(vo, eo, rp, cit, b.total_n, b.total_nnz, mode=KEEP)
    assert rc == gc.GC_OK
    c = col.cpu().numpy()
    for k in range(b.G):
        v0, v1 = int(b.vtx_off[k]), int(b.vtx_off[k + 1])
        assert O.check(b.graph(k), c[v0:v1])[0] == 0, k


@pytest.mark.parametrize("name", ["rmat14", "rmat12_bins", "kuhn16"])
def test_tiers_valid(ctx, name):
    # Degree tiers colour hubs, then mid-degree vertices, then the rest, each
    # through round 0 and its repairs: every tier's round 0 must hand all of
    # its vertices to the first repair pass.
    g = GRAPHS[name]()
    rp, ci = dev(g)
    opts = {"t1": 4, "t2": 40} if name.endswith("_bins") else None
    for _ in range(3):
        col, rc, st = ctx.color(rp, ci, gc.GC_SCHED_ASYNC | gc.GC_TIERS | gc.GC_CHECKED, opts=opts, check=False)
        assert rc == gc.GC_OK, gc.gc_strerror(rc)
        assert O.check(g, col.cpu().numpy())[0] == 0

"""Distance-2 colouring (GC_DIST2) through the C ABI against the oracle.

Deterministic mode must equal the oracle's snapshot replay over two-hop
neighbourhoods bit for bit: colours, iterations, conflicts, per-iteration
defect counts and the byte-model total.  Asynchronous mode must give a
proper distance-2 colouring (no two vertices within two hops share a
colour) with colours in 1..|D2(v)|+1.
"""
import numpy as np
import pytest

import oracle as O
from paper_1505_04086_gb300 import inputs as I

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from paper_1505_04086_gb300 import gc  # noqa: E402

D2 = gc.GC_DIST2
ASYNC = gc.GC_SCHED_ASYNC
HIGHER = gc.GC_TIE_HIGHER_KEEPS


@pytest.fixture(scope="module")
def ctx():
    c = gc.Context(0)
    yield c
    c.close()


def run(ctx, g, mode, opts=None, round_cap=4096):
    d = torch.device("cuda:0")
    rp = torch.from_numpy(g.row_ptr).to(d)
    ci = torch.from_numpy(g.col_idx if g.nnz else np.zeros(1, np.int32)).to(d)
    col = torch.full((max(g.n, 1),), -7, dtype=torch.int32, device=d)
    rc = gc.gc_color_async(ctx.handle, rp, ci, g.n, g.nnz, mode, col, opts)
    assert rc == gc.GC_OK, gc.gc_strerror(rc)
    rc, st = gc.gc_ctx_stats(ctx.handle, round_cap)
    return rc, col[: g.n].cpu().numpy(), st


def graphs():
    rng = np.random.default_rng(5)
    out = [I.from_edges(2, [(0, 1)]), I.from_edges(7, [(i, i + 1) for i in range(6)]),
           I.from_edges(1, []), I.from_edges(9, []), I.from_edges(40, [(0, i) for i in range(1, 40)]),
           I.from_edges(5, [(i, (i + 1) % 5) for i in range(5)])]
    # a ragged random graph with rows longer than a warp
    n = 300
    e = {(int(min(a, b)), int(max(a, b))) for a, b in rng.integers(0, n, (2400, 2)) if a != b}
    out.append(I.from_edges(n, sorted(e)))
    out += [I.kuhn3d(8), I.kuhn3d(16), I.tri2d(40, 40, 0.3), I.rmat(9), I.rgg(4096)]
    return out


def ids(gs):
    return [f"{g.name}-{g.n}" for g in gs]


GRAPHS = graphs()


# two-hop sizes above which a block, not a warp, inspects a vertex: the
# default, and thresholds low enough that the small graphs mix both paths
HEAVY = {"default": None, "heavy64": {"d2_heavy": 64}, "heavy300": {"d2_heavy": 300}}


@pytest.mark.parametrize("g", GRAPHS, ids=ids(GRAPHS))
@pytest.mark.parametrize("tie", [0, HIGHER], ids=["lower", "higher"])
@pytest.mark.parametrize("heavy", list(HEAVY))
def test_det_d2_matches_the_oracle_replay(ctx, g, tie, heavy):
    rc, col, st = run(ctx, g, D2 | tie | gc.GC_CHECKED, HEAVY[heavy])
    ref = O.rsoc_det_d2(g, O.TIE_HIGHER_KEEPS if tie else O.TIE_LOWER_KEEPS)
    assert rc == gc.GC_OK, gc.gc_strerror(rc)
    assert np.array_equal(col, ref.colors), f"first diff at {np.nonzero(col != ref.colors)[0][:5]}"
    assert st["rounds"] == ref.iterations
    assert st["conflicts"] == ref.conflicts
    assert np.array_equal(st["round_sizes"], ref.round_sizes[: len(st["round_sizes"])])
    assert st["model_bytes"] == ref.model_bytes
    if g.n:
        assert st["colors"] == ref.num_colors and st["distinct_colors"] == ref.distinct_colors
        assert O.check_d2(g, col) == 0


@pytest.mark.parametrize("heavy", [None, 2048])
def test_det_d2_larger_power_law_graph(ctx, heavy):
    g = I.rmat(11, ef=8)  # hubs of degree ~600: two-hop rows of many warps' width
    rc, col, st = run(ctx, g, D2, {"d2_heavy": heavy} if heavy else None)
    ref = O.rsoc_det_d2(g)
    assert rc == gc.GC_OK
    assert np.array_equal(col, ref.colors)
    assert (st["rounds"], st["conflicts"], st["model_bytes"]) == (ref.iterations, ref.conflicts, ref.model_bytes)


@pytest.mark.parametrize("cap", [1, 2, 5])
def test_det_d2_round_cap_returns_the_colouring_at_the_cap(ctx, cap):
    g = I.kuhn3d(8)
    rc, col, st = run(ctx, g, D2, {"max_rounds": cap})
    ref = O.rsoc_det_d2(g, max_iters=cap)
    assert rc == gc.GC_ERR_NO_CONVERGENCE and ref.status == O.ERR_NO_CONVERGENCE
    assert st["rounds"] == cap == ref.iterations
    assert np.array_equal(col, ref.colors)
    assert st["model_bytes"] == ref.model_bytes


@pytest.mark.parametrize("g", GRAPHS, ids=ids(GRAPHS))
@pytest.mark.parametrize("tie", [0, HIGHER], ids=["lower", "higher"])
@pytest.mark.parametrize("heavy", list(HEAVY))
def test_async_d2_is_a_distance2_colouring(ctx, g, tie, heavy):
    rc, col, st = run(ctx, g, D2 | ASYNC | tie | gc.GC_CHECKED, HEAVY[heavy])
    assert rc == gc.GC_OK, gc.gc_strerror(rc)
    assert O.check_d2(g, col) == 0
    if g.n:
        ff = int(O.ff_d2(g).max())
        assert st["colors"] == int(col.max())
        # every colour is First-Fit over D2(v): at most the largest |D2(v)| + 1
        assert col.max() <= max(ff, 1) * 2 + 1, (col.max(), ff)


@pytest.mark.parametrize("n,heavy", [(2300, None), (2300, 1000)])
def test_async_d2_beyond_one_colour_window(ctx, n, heavy):
    # the square of a star is complete: every vertex needs its own colour, so
    # First-Fit runs past the 2048-colour window of a warp (every vertex
    # light), or fills 2300 colours of a block's window (every vertex heavy)
    g = I.from_edges(n, [(0, i) for i in range(1, n)])
    rc, col, st = run(ctx, g, D2 | ASYNC | gc.GC_CHECKED, {"d2_heavy": heavy} if heavy else None)
    assert rc == gc.GC_OK, gc.gc_strerror(rc)
    assert np.array_equal(np.sort(col), np.arange(1, n + 1))


def test_async_d2_power_law_validity_at_size(ctx):
    g = I.rmat(16)  # two-hop neighbourhoods up to ~1.4M entries: the block path
    rc, col, st = run(ctx, g, D2 | ASYNC | gc.GC_CHECKED)
    assert rc == gc.GC_OK, gc.gc_strerror(rc)
    assert O.check_d2(g, col) == 0


def test_async_d2_mesh_validity_at_size(ctx):
    g = I.kuhn3d(48)
    rc, col, st = run(ctx, g, D2 | ASYNC | gc.GC_CHECKED)
    assert rc == gc.GC_OK, gc.gc_strerror(rc)
    assert O.check_d2(g, col) == 0
    ff = int(O.ff_d2(g).max())
    assert st["colors"] <= 1.25 * ff, (st["colors"], ff)


def test_d2_mode_combinations(ctx):
    g = I.kuhn3d(4)
    d = torch.device("cuda:0")
    rp = torch.from_numpy(g.row_ptr).to(d)
    ci = torch.from_numpy(g.col_idx).to(d)
    col = torch.empty(g.n, dtype=torch.int32, device=d)
    for bad in (gc.GC_ALG_TWO_PHASE, gc.GC_DEBUG_NO_TIEBREAK, ASYNC | gc.GC_REPAIR_SNAPSHOT, ASYNC | gc.GC_TIERS,
                ASYNC | gc.GC_FF_KEEPERS):
        assert gc.gc_color_async(ctx.handle, rp, ci, g.n, g.nnz, D2 | bad, col, None) == gc.GC_ERR_ARG, bad
    touched = torch.zeros(1, dtype=torch.int32, device=d)
    assert gc.gc_recolor_async(ctx.handle, rp, ci, g.n, g.nnz, D2 | ASYNC, col, touched) == gc.GC_ERR_ARG

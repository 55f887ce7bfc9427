"""The paper's own form on the host cores (gc_host_color, OpenMP).

Its deterministic forms must equal the oracle's replays bit for bit at any
thread count (colours, iterations, conflicts, round sizes); with one thread
asynchronous RSOC is sequential First-Fit; with several threads the
asynchronous forms must give proper colourings.  No GPU is involved.
"""
import numpy as np
import pytest

import oracle as O
from paper_1505_04086_gb300 import gc
from paper_1505_04086_gb300 import inputs as I

HIGHER = gc.GC_TIE_HIGHER_KEEPS
TWOP = gc.GC_ALG_TWO_PHASE
ASYNC = gc.GC_SCHED_ASYNC


def graphs():
    rng = np.random.default_rng(11)
    out = [I.from_edges(1, []), I.from_edges(6, []), I.from_edges(2, [(0, 1)]),
           I.from_edges(30, [(0, i) for i in range(1, 30)])]
    for n in (17, 64):
        out.append(I.from_edges(n, [(u, v) for u in range(n) for v in range(u + 1, n) if rng.random() < 0.5]))
    out += [I.kuhn3d(12), I.tri2d(30, 30, 0.2), I.rmat(10), I.rgg(3000)]
    return out


GRAPHS = graphs()
IDS = [f"{g.name}-{g.n}" for g in GRAPHS]


@pytest.mark.parametrize("g", GRAPHS, ids=IDS)
@pytest.mark.parametrize("alg", [0, TWOP], ids=["rsoc", "twophase"])
@pytest.mark.parametrize("tie", [0, HIGHER], ids=["lower", "higher"])
@pytest.mark.parametrize("threads", [1, 3, 8])
def test_host_det_matches_the_oracle_replay(g, alg, tie, threads):
    rc, col, st = gc.gc_host_color(g.row_ptr, g.col_idx, alg | tie | gc.GC_CHECKED, threads, round_cap=4096)
    otie = O.TIE_HIGHER_KEEPS if tie else O.TIE_LOWER_KEEPS
    ref = (O.twophase_det if alg else O.rsoc_det)(g, otie)
    assert rc == gc.GC_OK, gc.gc_strerror(rc)
    assert np.array_equal(col, ref.colors)
    assert (st["rounds"], st["conflicts"]) == (ref.iterations, ref.conflicts)
    assert np.array_equal(st["round_sizes"], ref.round_sizes)
    if g.n:
        assert (st["colors"], st["distinct_colors"]) == (ref.num_colors, ref.distinct_colors)


@pytest.mark.parametrize("g", GRAPHS, ids=IDS)
def test_host_async_rsoc_on_one_thread_is_sequential_first_fit(g):
    rc, col, st = gc.gc_host_color(g.row_ptr, g.col_idx, ASYNC, 1)
    assert rc == gc.GC_OK
    assert np.array_equal(col, O.ff(g))
    assert st["rounds"] == (1 if g.n else 0) and st["conflicts"] == 0


@pytest.mark.parametrize("g", GRAPHS, ids=IDS)
@pytest.mark.parametrize("alg", [0, TWOP], ids=["rsoc", "twophase"])
@pytest.mark.parametrize("tie", [0, HIGHER], ids=["lower", "higher"])
def test_host_async_is_a_proper_colouring(g, alg, tie):
    rc, col, st = gc.gc_host_color(g.row_ptr, g.col_idx, alg | ASYNC | tie | gc.GC_CHECKED, 8)
    assert rc == gc.GC_OK, gc.gc_strerror(rc)
    bad, mx, dist = O.check(g, col)
    assert bad == 0
    if g.n:
        assert (st["colors"], st["distinct_colors"]) == (mx, dist)


def test_host_mode_bits_are_checked():
    g = I.kuhn3d(3)
    for bad in (gc.GC_DEBUG_NO_TIEBREAK, gc.GC_REPAIR_SNAPSHOT, gc.GC_TIERS, gc.GC_FF_KEEPERS, 1 << 20):
        rc, _, _ = gc.gc_host_color(g.row_ptr, g.col_idx, ASYNC | bad, 2)
        assert rc == gc.GC_ERR_ARG, bad
    rc, _, _ = gc.gc_host_color(g.row_ptr, g.col_idx, 0, -1)
    assert rc == gc.GC_ERR_ARG
    assert gc.gc_host_threads() >= 1


def _malformed():
    """(name, row_ptr, col_idx) of inputs GC_VALIDATE must reject."""
    g = I.kuhn3d(3)
    rp, ci = g.row_ptr.copy(), g.col_idx.copy()
    unsorted = ci.copy()
    unsorted[rp[5]], unsorted[rp[5] + 1] = unsorted[rp[5] + 1], unsorted[rp[5]]
    out_of_range = ci.copy()
    out_of_range[3] = g.n + 5
    negative = ci.copy()
    negative[0] = -1
    selfloop = I.from_edges(3, [(0, 1), (1, 2)])
    sl_ci = selfloop.col_idx.copy()
    sl_ci[0] = 0  # vertex 0's entry 1 becomes 0: a self-loop
    asym = I.from_edges(4, [(0, 1), (1, 2), (2, 3)])
    as_ci = asym.col_idx.copy()
    as_ci[-1] = 0  # vertex 3's neighbour 2 becomes 0, which does not list 3
    bad_rp = rp.copy()
    bad_rp[4] = bad_rp[6]  # row pointers decrease
    bad_end = rp.copy()
    bad_end[-1] -= 1
    return [("unsorted", rp, unsorted), ("out_of_range", rp, out_of_range), ("negative", rp, negative),
            ("selfloop", selfloop.row_ptr, sl_ci), ("asymmetric", asym.row_ptr, as_ci),
            ("decreasing_row_ptr", bad_rp, ci), ("row_ptr_end", bad_end, ci)]


@pytest.mark.parametrize("case", _malformed(), ids=lambda c: c[0])
def test_host_validate_rejects_malformed_input(case):
    name, rp, ci = case
    rc, _, _ = gc.gc_host_color(rp, ci, ASYNC | gc.GC_VALIDATE, 2)
    assert rc == gc.GC_ERR_GRAPH, name


def test_host_validate_accepts_well_formed_input():
    for g in GRAPHS:
        rc, col, _ = gc.gc_host_color(g.row_ptr, g.col_idx, ASYNC | gc.GC_VALIDATE, 2)
        assert rc == gc.GC_OK
        assert O.check(g, col)[0] == 0


D2_GRAPHS = [I.from_edges(7, [(i, i + 1) for i in range(6)]), I.from_edges(40, [(0, i) for i in range(1, 40)]),
             I.kuhn3d(8), I.tri2d(30, 30, 0.3), I.rmat(9)]
D2_IDS = [f"{g.name}-{g.n}" for g in D2_GRAPHS]


@pytest.mark.parametrize("g", D2_GRAPHS, ids=D2_IDS)
@pytest.mark.parametrize("alg", [0, TWOP], ids=["rsoc", "twophase"])
@pytest.mark.parametrize("tie", [0, HIGHER], ids=["lower", "higher"])
@pytest.mark.parametrize("threads", [1, 8])
def test_host_distance2_det_matches_the_oracle_replay(g, alg, tie, threads):
    # both algorithms over two-hop neighbourhoods give the distance-2 replay
    # (the snapshot equivalence of Algorithms 2 and 3 holds on G^2 as well)
    rc, col, st = gc.gc_host_color(g.row_ptr, g.col_idx, gc.GC_DIST2 | alg | tie | gc.GC_CHECKED, threads,
                                   round_cap=4096)
    ref = O.rsoc_det_d2(g, O.TIE_HIGHER_KEEPS if tie else O.TIE_LOWER_KEEPS)
    assert rc == gc.GC_OK, gc.gc_strerror(rc)
    assert np.array_equal(col, ref.colors)
    assert (st["rounds"], st["conflicts"]) == (ref.iterations, ref.conflicts)
    assert np.array_equal(st["round_sizes"], ref.round_sizes)


@pytest.mark.parametrize("g", D2_GRAPHS, ids=D2_IDS)
def test_host_distance2_async(g):
    rc, col, _ = gc.gc_host_color(g.row_ptr, g.col_idx, gc.GC_DIST2 | ASYNC, 1)
    assert rc == gc.GC_OK
    assert np.array_equal(col, O.ff_d2(g))  # one thread: sequential First-Fit over D2
    rc, col, _ = gc.gc_host_color(g.row_ptr, g.col_idx, gc.GC_DIST2 | ASYNC | gc.GC_CHECKED, 8)
    assert rc == gc.GC_OK
    assert O.check_d2(g, col) == 0

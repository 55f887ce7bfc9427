"""Parity of the CUDA path (through the C ABI) with the CPU oracle.

Deterministic mode must equal the oracle's round-synchronous replay bit for
bit: colours, iteration count, conflict count, per-iteration defect counts
and the byte-model total.  Asynchronous mode has many correct answers; it
must be a proper colouring within 1..deg+1 whose colour count is at most
1.1x that of sequential First-Fit in natural order.
"""
import numpy as np
import pytest

import oracle as O
from paper_1505_04086_gb300 import inputs as I

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from paper_1505_04086_gb300 import gc  # noqa: E402

DET = gc.GC_SCHED_DET
ASYNC = gc.GC_SCHED_ASYNC
RSOC = gc.GC_ALG_RSOC
TWOP = gc.GC_ALG_TWO_PHASE
HIGHER = gc.GC_TIE_HIGHER_KEEPS

# degree-bin settings: defaults, everything per thread, mostly per warp,
# everything per block
BINS = {
    "default": None,
    "thread": {"t1": 62, "t2": 4096},
    "warp": {"t1": 1, "t2": 4096},
    "block": {"t1": 1, "t2": 1},
    "mixed": {"t1": 4, "t2": 12, "tile": 32},
}


@pytest.fixture(scope="module")
def ctx():
    c = gc.Context(0)
    yield c
    c.close()


def dev(g):
    d = torch.device("cuda:0")
    ci = g.col_idx if g.nnz else np.zeros(1, np.int32)
    return torch.from_numpy(g.row_ptr).to(d), torch.from_numpy(ci).to(d)


def run(ctx, g, mode, opts=None, round_cap=4096):
    rp, ci = dev(g)
    col = torch.empty(max(g.n, 1), dtype=torch.int32, device="cuda:0")
    rc = gc.gc_color_async(ctx.handle, rp, ci, g.n, g.nnz, mode, col, opts)
    assert rc == gc.GC_OK, gc.gc_strerror(rc)
    rc, st = gc.gc_ctx_stats(ctx.handle, round_cap)
    return rc, col[: g.n].cpu().numpy(), st


def oracle_replay(g, mode, max_iters=None):
    tie = O.TIE_HIGHER_KEEPS if mode & HIGHER else O.TIE_LOWER_KEEPS
    if mode & gc.GC_DEBUG_NO_TIEBREAK:
        tie = O.TIE_NONE
    f = O.twophase_det if mode & TWOP else O.rsoc_det
    return f(g, tie=tie, max_iters=max_iters)


def assert_det_parity(ctx, g, mode, opts=None):
    rc, col, st = run(ctx, g, mode, opts)
    ref = oracle_replay(g, mode)
    assert rc == gc.GC_OK, gc.gc_strerror(rc)
    assert st["error_word"] == 0
    assert np.array_equal(col, ref.colors), f"{g.name}: first diff at {np.nonzero(col != ref.colors)[0][:5]}"
    assert st["rounds"] == ref.iterations
    assert st["conflicts"] == ref.conflicts
    assert np.array_equal(st["round_sizes"], ref.round_sizes[: len(st["round_sizes"])])
    assert st["model_bytes"] == ref.model_bytes
    if g.n:
        assert st["colors"] == ref.num_colors
        assert st["distinct_colors"] == ref.distinct_colors
    return st


def assert_async_ok(ctx, g, mode, opts=None, bound=1.1):
    rc, col, st = run(ctx, g, mode, opts)
    assert rc == gc.GC_OK, gc.gc_strerror(rc)
    bad, mx, dist = O.check(g, col)
    assert bad == 0, f"{g.name}: invalid colouring at {bad}"
    ff = int(O.ff(g).max()) if g.n else 0
    assert mx <= bound * ff, f"{g.name}: {mx} colours vs first-fit {ff}"
    assert st["colors"] == mx and st["distinct_colors"] == dist
    return st, mx, ff


def small_graphs():
    rng = np.random.default_rng(1)
    out = [I.from_edges(2, [(0, 1)]), I.from_edges(4, [(0, 1), (1, 2), (2, 3)]),
           I.from_edges(3, [(0, 1), (1, 2), (0, 2)]), I.from_edges(1, []), I.from_edges(7, []),
           I.from_edges(5, [(0, i) for i in range(1, 5)])]
    for n in (9, 33, 70, 130):
        out.append(I.from_edges(n, [(u, v) for u in range(n) for v in range(u + 1, n)
                                    if rng.random() < 0.3]))
    return out


def mid_graphs():
    star = I.from_edges(5001, [(0, i) for i in range(1, 5001)])
    star.name = "star5000"
    k64 = I.from_edges(64, [(u, v) for u in range(64) for v in range(u + 1, 64)])
    k64.name = "K64"
    return [I.tri2d(64, 64), I.kuhn3d(12), I.kuhn3d(9, permute=False), I.rmat(12),
            I.rgg(5000, 12.0, seed=3), I.tri2d(37, 53, jitter=0.3, seed=2), star, k64]


# ---------------------------------------------------------------- deterministic

@pytest.mark.parametrize("alg", [RSOC, TWOP], ids=["rsoc", "twophase"])
@pytest.mark.parametrize("tie", [0, HIGHER], ids=["lower", "higher"])
def test_det_small_graphs(ctx, alg, tie):
    for g in small_graphs():
        assert_det_parity(ctx, g, alg | DET | tie)


@pytest.mark.parametrize("bins", list(BINS), ids=list(BINS))
@pytest.mark.parametrize("alg", [RSOC, TWOP], ids=["rsoc", "twophase"])
def test_det_bins(ctx, bins, alg):
    for g in mid_graphs():
        if bins == "thread" and int(g.degrees().max()) > 62:
            continue
        assert_det_parity(ctx, g, alg | DET, BINS[bins])


@pytest.mark.parametrize("tie", [0, HIGHER], ids=["lower", "higher"])
def test_det_tie_break_and_tail(ctx, tie):
    g = I.kuhn3d(16)
    for opts in (None, {"tail": -1}, {"tail": 100000}, {"tile": 32}, {"tile": 4096},
                 {"blocks_per_sm": 1}):
        assert_det_parity(ctx, g, RSOC | DET | tie, opts)
        assert_det_parity(ctx, g, TWOP | DET | tie, opts)


def test_empty_graph(ctx):
    g = I.from_edges(0, [])
    rp = torch.zeros(1, dtype=torch.int32, device="cuda:0")
    ci = torch.zeros(1, dtype=torch.int32, device="cuda:0")
    col = torch.zeros(1, dtype=torch.int32, device="cuda:0")
    assert gc.gc_color_async(ctx.handle, rp, ci, 0, 0, 0, col) == gc.GC_OK
    rc, st = gc.gc_ctx_stats(ctx.handle)
    assert rc == gc.GC_OK and st["rounds"] == 0 and st["conflicts"] == 0
    assert g.n == 0


def test_fig7_livelock_hits_round_cap(ctx):
    # Sec. 5 / Fig. 7: the symmetric defect test never converges on K2; the
    # round cap turns it into an error status instead of a hang.
    g = I.from_edges(2, [(0, 1)])
    for cap in (1, 2, 5, 8):
        for alg in (RSOC, TWOP):
            mode = alg | DET | gc.GC_DEBUG_NO_TIEBREAK
            rc, col, st = run(ctx, g, mode, {"max_rounds": cap})
            ref = oracle_replay(g, mode, max_iters=cap)
            assert rc == gc.GC_ERR_NO_CONVERGENCE
            assert ref.status == O.ERR_NO_CONVERGENCE
            assert st["rounds"] == cap == ref.iterations
            assert np.array_equal(col, ref.colors)
            assert st["error_word"] & gc.GC_EW_NO_CONVERGENCE


def test_round_cap_partial_state_matches_oracle(ctx):
    g = I.tri2d(64, 64)
    for cap in (1, 3, 10, 50):
        for alg in (RSOC, TWOP):
            rc, col, st = run(ctx, g, alg | DET, {"max_rounds": cap})
            ref = oracle_replay(g, alg | DET, max_iters=cap)
            assert rc == gc.GC_ERR_NO_CONVERGENCE
            assert np.array_equal(col, ref.colors)
            assert st["conflicts"] == ref.conflicts


def test_host_pointer_path_matches_device_path(ctx):
    g = I.kuhn3d(10)
    col = np.zeros(g.n, np.int32)
    rc, st = gc.gc_color(g.row_ptr, g.col_idx, g.n, g.nnz, RSOC | DET, col)
    assert rc == gc.GC_OK
    assert np.array_equal(col, O.rsoc_det(g).colors)
    rc2, col2, _ = run(ctx, g, RSOC | DET)
    assert np.array_equal(col, col2)


# ---------------------------------------------------------------- asynchronous

@pytest.mark.parametrize("alg", [RSOC, TWOP], ids=["rsoc", "twophase"])
@pytest.mark.parametrize("bins", ["default", "warp", "block", "mixed"])
def test_async_valid(ctx, alg, bins):
    for g in small_graphs() + mid_graphs():
        rc, col, st = run(ctx, g, alg | ASYNC, BINS[bins])
        assert rc == gc.GC_OK
        assert O.check(g, col)[0] == 0, g.name
        assert st["rounds"] >= (1 if g.n else 0)


@pytest.mark.parametrize("alg", [RSOC, TWOP], ids=["rsoc", "twophase"])
def test_async_quality(ctx, alg):
    for g in mid_graphs():
        for _ in range(3):
            assert_async_ok(ctx, g, alg | ASYNC)


# ---------------------------------------------------------------- validation

def test_validate_rejects_malformed(ctx):
    good = I.from_edges(4, [(0, 1), (1, 2), (2, 3)])
    rc, col, st = run(ctx, good, RSOC | gc.GC_VALIDATE | gc.GC_CHECKED)
    assert rc == gc.GC_OK
    cases = []
    asym = I.CSR(good.row_ptr.copy(), good.col_idx.copy())
    asym.col_idx[0] = 2
    cases.append(asym)
    uns = I.CSR(good.row_ptr.copy(), good.col_idx.copy())
    uns.col_idx[1], uns.col_idx[2] = uns.col_idx[2], uns.col_idx[1]
    cases.append(uns)
    cases.append(I.CSR(np.array([0, 1], np.int32), np.array([0], np.int32)))          # self-loop
    cases.append(I.CSR(np.array([0, 2, 4], np.int32), np.array([1, 1, 0, 0], np.int32)))  # repeat
    cases.append(I.CSR(np.array([0, 1, 1], np.int32), np.array([5], np.int32)))        # range
    cases.append(I.CSR(np.array([0, 1, 2], np.int32), np.array([1, 0, 7], np.int32)))  # row_ptr[n] != nnz
    for bad in cases:
        rc, _, st = run(ctx, bad, RSOC | gc.GC_VALIDATE)
        assert rc == gc.GC_ERR_GRAPH
        assert st["error_word"] & gc.GC_EW_GRAPH


def test_checked_mode_passes_on_real_results(ctx):
    for g in mid_graphs():
        for mode in (RSOC | DET, RSOC | ASYNC, TWOP | ASYNC):
            rc, _, st = run(ctx, g, mode | gc.GC_CHECKED | gc.GC_VALIDATE)
            assert rc == gc.GC_OK and st["error_word"] == 0


@pytest.mark.parametrize("make,window", [
    (lambda: I.tri2d(64, 64), 0), (lambda: I.tri2d(50, 70, jitter=0.3, seed=9), 0),
    (lambda: I.tri2d(300, 7), 0), (lambda: I.kuhn3d(12), 0), (lambda: I.kuhn3d(9, permute=False), 0),
    (lambda: I.rgg(12000, 12.0, seed=2), 0), (lambda: I.tri2d(300, 300, jitter=0.3, seed=5), 0),
    (lambda: I.rgg(60000, 12.0, seed=3), 1), (lambda: I.kuhn3d(40), 1)],
    ids=["tri64", "tri_jit", "tri_narrow", "kuhn12", "kuhn9_nat", "rgg12k", "tri300_jit", "rgg60k_w1",
         "kuhn40_w1"])
def test_ordered_round0_is_sequential_first_fit(ctx, make, window):
    # An ordered graph (at most 16384 vertices, or naturally numbered, or any
    # graph with window 1) whose degrees all fit one thread is coloured in
    # round 0 in id order -- by one warp, or by a group of warps that wait for
    # each other's lower ids -- every vertex seeing the final colours of all
    # its lower neighbours and none of the higher ones: exactly Algorithm 1.
    g = make()
    assert int(np.diff(g.row_ptr).max()) <= 62
    ff = O.ff(g)
    for _ in range(3):
        rc, col, st = run(ctx, g, gc.GC_SCHED_ASYNC, {"t1": 62, "t2": 4096, "window": window})
        assert rc == gc.GC_OK
        assert np.array_equal(col, ff), f"first diff at {np.nonzero(col != ff)[0][:5]}"
        assert st["conflicts"] == 0 and st["rounds"] == 1


@pytest.mark.parametrize("window", [-1, 2, 16])
@pytest.mark.parametrize("alg", [gc.GC_ALG_RSOC, gc.GC_ALG_TWO_PHASE], ids=["rsoc", "twophase"])
def test_async_window_modes_valid(ctx, window, alg):
    # window -1: pure speculation (nothing ordered); k > 1: at most k tiles
    # of round 0 in flight, claimed in vertex order.
    for g in (I.kuhn3d(24), I.tri2d(100, 100, jitter=0.3, seed=4), I.rmat(12), I.rgg(20000, 12.0, seed=6)):
        rc, col, st = run(ctx, g, alg | gc.GC_SCHED_ASYNC, {"window": window})
        assert rc == gc.GC_OK, gc.gc_strerror(rc)
        assert O.check(g, col)[0] == 0, g.name
        assert st["colors"] == int(col.max())

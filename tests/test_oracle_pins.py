"""Pins of the CPU oracle to facts fixed by the paper and by mathematics.

Nothing here compares the oracle with itself: closed forms, textbook
characterisations, exhaustive search on tiny graphs, hand-worked examples
(tests/golden) and the agreement of two independently written replays.
"""
import itertools
import os

import numpy as np
import pytest

import oracle as O
from paper_1505_04086_gb300 import inputs as I

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "rsoc_small.txt")


def _parse_edges(s):
    if s.strip() == "-":
        return []
    return [tuple(int(x) for x in e.split("-")) for e in s.split()]


def _ints(s):
    return [] if s.strip() == "-" else [int(x) for x in s.split()]


def golden_cases():
    out = []
    for line in open(GOLDEN):
        line = line.strip()
        if not line or line.startswith("#"):
            continue
        f = [x.strip() for x in line.split("|")]
        out.append(dict(name=f[0], n=int(f[1]), edges=_parse_edges(f[2]),
                        tie=O.TIE_LOWER_KEEPS if f[3] == "lower" else O.TIE_HIGHER_KEEPS,
                        colors=_ints(f[4]), iterations=int(f[5]), conflicts=int(f[6]),
                        round_sizes=_ints(f[7]), model_bytes=int(f[8])))
    return out


def rand_graph(rng, n, p):
    edges = [(u, v) for u in range(n) for v in range(u + 1, n) if rng.random() < p]
    return I.from_edges(n, edges)


# ---------------------------------------------------------------- golden

@pytest.mark.parametrize("case", golden_cases(), ids=lambda c: f"{c['name']}-{c['tie']}")
def test_rsoc_golden(case):
    g = I.from_edges(case["n"], case["edges"])
    r = O.rsoc_det(g, tie=case["tie"])
    assert r.status == O.OK
    assert r.colors.tolist() == case["colors"]
    assert r.iterations == case["iterations"]
    assert r.conflicts == case["conflicts"]
    assert r.round_sizes.tolist() == case["round_sizes"]
    if case["model_bytes"] >= 0:
        assert r.model_bytes == case["model_bytes"]


@pytest.mark.parametrize("case", golden_cases(), ids=lambda c: f"{c['name']}-{c['tie']}")
def test_twophase_golden(case):
    # Algorithm 2's tentative phase of iteration k+1 recolours exactly the
    # set RSOC recolours in iteration k, from the same colours, so the
    # hand-worked RSOC values hold for it too.
    g = I.from_edges(case["n"], case["edges"])
    r = O.twophase_det(g, tie=case["tie"])
    assert r.status == O.OK
    assert r.colors.tolist() == case["colors"]
    assert r.iterations == case["iterations"]
    assert r.conflicts == case["conflicts"]
    assert r.round_sizes.tolist() == case["round_sizes"]


def test_fig7_livelock_without_tiebreak():
    # Sec. 5 / Fig. 7: with a symmetric defect test the two vertices of K2
    # recolour in lock-step forever: red,red -> green,green -> red,red ...
    g = I.from_edges(2, [(0, 1)])
    for cap in range(1, 8):
        r = O.rsoc_det(g, tie=O.TIE_NONE, max_iters=cap)
        assert r.status == O.ERR_NO_CONVERGENCE
        assert r.iterations == cap
        want = [2, 2] if cap % 2 == 1 else [1, 1]
        assert r.colors.tolist() == want
        assert r.conflicts == 2 * cap
        q = O.twophase_det(g, tie=O.TIE_NONE, max_iters=cap)
        assert q.status == O.ERR_NO_CONVERGENCE


# ---------------------------------------------------------------- First-Fit

def ff_colors(n, edges):
    return O.ff(I.from_edges(n, edges)).tolist()


def test_ff_closed_forms():
    for n in range(1, 9):
        kn = [(u, v) for u in range(n) for v in range(u + 1, n)]
        assert max(ff_colors(n, kn)) == n                      # K_n
        assert max(ff_colors(n, [])) == 1                      # no edges
    for n in range(2, 12):
        path = [(i, i + 1) for i in range(n - 1)]
        assert max(ff_colors(n, path)) == 2                    # P_n
    for n in range(3, 13):
        cyc = [(i, (i + 1) % n) for i in range(n)]
        assert max(ff_colors(n, cyc)) == (2 if n % 2 == 0 else 3)
    for leaves in range(1, 9):
        assert max(ff_colors(leaves + 1, [(0, i) for i in range(1, leaves + 1)])) == 2
        assert max(ff_colors(leaves + 1, [(leaves, i) for i in range(leaves)])) == 2
    for a in range(1, 5):
        for b in range(1, 5):
            kab = [(i, a + j) for i in range(a) for j in range(b)]
            assert max(ff_colors(a + b, kab)) == 2             # K_{a,b}, sides in order
    assert O.ff(I.from_edges(0, [])).size == 0


def test_ff_grid_and_crown():
    # 4-neighbour R x C grid in natural order: First-Fit gives the
    # checkerboard, 2 colours.
    R, C = 7, 9
    e = [(i * C + j, i * C + j + 1) for i in range(R) for j in range(C - 1)]
    e += [(i * C + j, (i + 1) * C + j) for i in range(R - 1) for j in range(C)]
    c = ff_colors(R * C, e)
    assert c == [1 + ((i + j) % 2) for i in range(R) for j in range(C)]
    # Crown graph (K_{k,k} minus a perfect matching) visited as
    # a1,b1,a2,b2,...: First-Fit uses k colours although it is bipartite.
    for k in range(2, 8):
        e = [(2 * i, 2 * j + 1) for i in range(k) for j in range(k) if i != j]
        c = ff_colors(2 * k, e)
        assert max(c) == k
        assert c == [i // 2 + 1 for i in range(2 * k)]


def grundy_ok(g, c):
    """Proper colouring in which every vertex v sees each colour below c[v]
    on some lower-numbered neighbour.  By induction on v this property holds
    for exactly one colouring: the greedy one in natural order."""
    rp, ci = g.row_ptr, g.col_idx
    for v in range(g.n):
        nb = ci[rp[v]:rp[v + 1]]
        if c[v] < 1 or any(c[u] == c[v] for u in nb):
            return False
        lower = {c[u] for u in nb if u < v}
        if any(k not in lower for k in range(1, c[v])):
            return False
    return True


def test_ff_grundy_characterisation():
    rng = np.random.default_rng(11)
    for _ in range(300):
        n = int(rng.integers(1, 30))
        g = rand_graph(rng, n, float(rng.uniform(0.05, 0.6)))
        c = O.ff(g)
        assert grundy_ok(g, c)
    g = I.kuhn3d(6)
    assert grundy_ok(g, O.ff(g))
    g = I.tri2d(9, 11)
    assert grundy_ok(g, O.ff(g))


def test_ff_brute_force_bounds():
    rng = np.random.default_rng(5)
    for _ in range(3000):
        n = int(rng.integers(1, 11))
        g = rand_graph(rng, n, float(rng.uniform(0.1, 0.9)))
        chi = O.chi(g)
        c = O.ff(g)
        dmax = int(g.degrees().max()) if n else 0
        assert chi <= c.max() <= dmax + 1
        assert O.check(g, c)[0] == 0


def test_some_order_reaches_chi():
    # For every graph some vertex order makes the greedy colouring optimal
    # (colour an optimal colouring's classes one after another).  Relabel
    # the graph so that each order becomes the natural one.
    rng = np.random.default_rng(7)
    for _ in range(60):
        n = int(rng.integers(2, 8))
        p = float(rng.uniform(0.2, 0.8))
        edges = [(u, v) for u in range(n) for v in range(u + 1, n) if rng.random() < p]
        g = I.from_edges(n, edges)
        best = n + 1
        for order in itertools.permutations(range(n)):
            pos = {v: i for i, v in enumerate(order)}
            h = I.from_edges(n, [(pos[u], pos[v]) for u, v in edges])
            best = min(best, int(O.ff(h).max()))
        assert best == O.chi(g)


def test_chi_closed_forms():
    def g_of(n, e):
        return I.from_edges(n, e)
    assert O.chi(g_of(1, [])) == 1
    assert O.chi(g_of(5, [])) == 1
    for n in range(2, 9):
        assert O.chi(g_of(n, [(u, v) for u in range(n) for v in range(u + 1, n)])) == n
    for n in range(3, 12):
        assert O.chi(g_of(n, [(i, (i + 1) % n) for i in range(n)])) == (2 if n % 2 == 0 else 3)
    # Petersen graph: chromatic number 3.
    outer = [(i, (i + 1) % 5) for i in range(5)]
    spokes = [(i, i + 5) for i in range(5)]
    inner = [(5 + i, 5 + (i + 2) % 5) for i in range(5)]
    assert O.chi(g_of(10, outer + spokes + inner)) == 3
    # Wheels: hub + C_5 needs 4, hub + C_6 needs 3.
    assert O.chi(g_of(6, [(0, i) for i in range(1, 6)] + [(1 + i, 1 + (i + 1) % 5) for i in range(5)])) == 4
    assert O.chi(g_of(7, [(0, i) for i in range(1, 7)] + [(1 + i, 1 + (i + 1) % 6) for i in range(6)])) == 3
    # Groetzsch graph (Mycielskian of C_5): triangle-free, chromatic number 4.
    c5 = [(i, (i + 1) % 5) for i in range(5)]
    shadow = [(5 + i, (i + 1) % 5) for i in range(5)] + [(5 + i, (i - 1) % 5) for i in range(5)]
    apex = [(10, 5 + i) for i in range(5)]
    assert O.chi(g_of(11, c5 + shadow + apex)) == 4


# ---------------------------------------------------------------- RSOC / 2P

def _replays_agree(g, tie):
    r = O.rsoc_det(g, tie=tie)
    q = O.twophase_det(g, tie=tie)
    assert r.status == O.OK and q.status == O.OK
    assert np.array_equal(r.colors, q.colors)
    assert r.iterations == q.iterations
    assert r.conflicts == q.conflicts
    assert np.array_equal(r.round_sizes, q.round_sizes)
    return r


@pytest.mark.parametrize("tie", [O.TIE_LOWER_KEEPS, O.TIE_HIGHER_KEEPS])
def test_rsoc_and_twophase_agree_random(tie):
    rng = np.random.default_rng(100 + tie)
    for _ in range(200):
        n = int(rng.integers(1, 60))
        g = rand_graph(rng, n, float(rng.uniform(0.02, 0.5)))
        r = _replays_agree(g, tie)
        assert O.check(g, r.colors)[0] == 0


@pytest.mark.parametrize("tie", [O.TIE_LOWER_KEEPS, O.TIE_HIGHER_KEEPS])
def test_rsoc_properties_on_meshes(tie):
    for g in (I.tri2d(64, 64), I.kuhn3d(12), I.kuhn3d(10, permute=False), I.rmat(10),
              I.rgg(3000, 12.0, seed=3), I.tri2d(30, 40, jitter=0.3, seed=9)):
        r = _replays_agree(g, tie)
        bad, mx, _ = O.check(g, r.colors)
        assert bad == 0
        assert mx <= int(g.degrees().max()) + 1
        # The defect sets shrink strictly: the tie-break winner among the
        # vertices recoloured in one round saw its final neighbours.
        rs = r.round_sizes.tolist()
        assert rs[-1] == 0
        assert all(a > b for a, b in zip(rs, rs[1:]))
        assert r.iterations <= g.n
        assert r.conflicts == sum(rs)


def test_rsoc_round_sets_by_definition():
    # Re-run RSOC round by round through max_iters and check that what
    # changed between consecutive prefixes is exactly the set of vertices
    # that lose a tie to an equal-coloured neighbour at the earlier state,
    # and that each changed vertex took the smallest colour unused by its
    # neighbours at that state.
    g = I.kuhn3d(5)
    rp, ci = g.row_ptr, g.col_idx
    full = O.rsoc_det(g)
    prev = np.ones(g.n, np.int32)  # after round 0
    for k in range(1, full.iterations + 1):
        cur = O.rsoc_det(g, max_iters=k).colors
        changed = set(np.nonzero(cur != prev)[0].tolist())
        expect = set()
        for v in range(g.n):
            nb = ci[rp[v]:rp[v + 1]]
            if any(u < v and prev[u] == prev[v] for u in nb):
                expect.add(v)
                used = {int(prev[u]) for u in nb}
                want = next(x for x in range(1, len(nb) + 2) if x not in used)
                assert cur[v] == want
        # A defective vertex may draw its old colour only if no neighbour
        # forbids it, which the defect itself rules out.
        assert changed == expect
        prev = cur
    assert np.array_equal(prev, full.colors)


# ---------------------------------------------------------------- checkers

def test_check_catches_planted_errors():
    g = I.tri2d(8, 8)
    c = O.ff(g)
    assert O.check(g, c)[0] == 0
    bad = c.copy()
    rp, ci = g.row_ptr, g.col_idx
    v = 27
    bad[v] = c[ci[rp[v]]]
    s = O.check(g, bad)[0]
    assert s > 0
    bad = c.copy()
    bad[5] = 0
    assert O.check(g, bad)[0] == -(5 + 1)
    bad = c.copy()
    bad[0] = int(g.degrees()[0]) + 2
    assert O.check(g, bad)[0] == -1


def test_csr_check_catches_malformed_inputs():
    g = I.from_edges(4, [(0, 1), (1, 2), (2, 3)])
    assert O.csr_check(g) == 0
    rp, ci = g.row_ptr.copy(), g.col_idx.copy()
    asym = I.CSR(rp, ci.copy())
    asym.col_idx[0] = 2            # 0 -> 2 without 2 -> 0
    assert O.csr_check(asym) != 0
    unsorted = I.CSR(rp, ci.copy())
    unsorted.col_idx[1], unsorted.col_idx[2] = unsorted.col_idx[2], unsorted.col_idx[1]
    assert O.csr_check(unsorted) != 0
    loop = I.CSR(np.array([0, 1], np.int32), np.array([0], np.int32))
    assert O.csr_check(loop) != 0
    dup = I.CSR(np.array([0, 2, 4], np.int32), np.array([1, 1, 0, 0], np.int32))
    assert O.csr_check(dup) != 0
    oob = I.CSR(np.array([0, 1, 1], np.int32), np.array([5], np.int32))
    assert O.csr_check(oob) != 0


def test_tri2d_64_facts():
    # The 64x64 triangular mesh contains triangles, and (i+j) mod 3 is a
    # proper colouring, so its chromatic number is 3.  First-Fit in natural
    # order does not reach it.
    g = I.tri2d(64, 64)
    c3 = np.array([1 + (i + j) % 3 for i in range(64) for j in range(64)], np.int32)
    assert O.check(g, c3)[0] == 0
    c = O.ff(g)
    assert grundy_ok(g, c)
    assert c.max() == 4


# ---- colour classes (the independent sets of a colouring, Sec. 1) --------

def test_classes_small_by_hand():
    # colours of 6 vertices: 2 1 2 3 1 2 -> class 1 = {1,4}, 2 = {0,2,5}, 3 = {3}
    ptr, verts = O.classes(np.array([2, 1, 2, 3, 1, 2], np.int32))
    assert list(ptr) == [0, 0, 2, 5, 6]
    assert list(verts) == [1, 4, 0, 2, 5, 3]


def test_classes_match_a_stable_sort_and_are_independent_sets():
    for g in (I.kuhn3d(8), I.rmat(9), I.tri2d(20, 30, jitter=0.3, seed=2), I.from_edges(5, [])):
        c = O.ff(g)
        k = int(c.max()) if g.n else 0
        ptr, verts = O.classes(c, k)
        # a different definition: numpy's stable argsort by colour
        assert np.array_equal(verts, np.argsort(c, kind="stable"))
        assert np.array_equal(np.diff(ptr)[1:], np.bincount(c, minlength=k + 1)[1:])
        for col in range(1, k + 1):
            members = verts[ptr[col]:ptr[col + 1]]
            assert np.all(c[members] == col) and np.all(np.diff(members) > 0)
            inset = np.zeros(g.n, bool)
            inset[members] = True
            for v in members:  # no edge inside a class
                assert not inset[g.col_idx[g.row_ptr[v]:g.row_ptr[v + 1]]].any()
    # a wider colour range than used leaves empty classes; out of range fails
    ptr, verts = O.classes(np.array([1, 1], np.int32), 4)
    assert list(ptr) == [0, 0, 2, 2, 2, 2]
    with pytest.raises(ValueError):
        O.classes(np.array([1, 0], np.int32), 2)
    with pytest.raises(ValueError):
        O.classes(np.array([3], np.int32), 2)


# ---- incremental recolouring (Algorithm 3's loop from a given colouring) --

def _add_edges(g, extra):
    e = [(v, u) for v in range(g.n) for u in g.col_idx[g.row_ptr[v]:g.row_ptr[v + 1]] if u > v]
    return I.from_edges(g.n, e + list(extra))


def test_from_all_ones_and_all_touched_is_the_full_replay():
    # Round 0 of the snapshot replay colours everything 1 and U^0 = V: starting
    # the loop from that state must give the same run, bytes included (the
    # 4 bytes a vertex of round 0 costs move to the first explicit worklist).
    for g in (I.kuhn3d(6), I.rmat(8), I.tri2d(12, 9), I.from_edges(2, [(0, 1)])):
        for tie in (O.TIE_LOWER_KEEPS, O.TIE_HIGHER_KEEPS):
            full = O.rsoc_det(g, tie)
            inc = O.rsoc_det_from(g, np.ones(g.n, np.int32), np.arange(g.n), tie)
            assert np.array_equal(inc.colors, full.colors)
            assert (inc.iterations, inc.conflicts, inc.model_bytes) == \
                (full.iterations, full.conflicts, full.model_bytes)
            assert np.array_equal(inc.round_sizes, full.round_sizes)


def test_from_valid_colouring_changes_nothing():
    g = I.kuhn3d(7)
    c = O.ff(g)
    none = O.rsoc_det_from(g, c, [])
    assert none.iterations == 0 and np.array_equal(none.colors, c)
    some = O.rsoc_det_from(g, c, [0, 5, 17, 5, 0])  # repeats are ignored
    assert some.iterations == 1 and some.conflicts == 0 and np.array_equal(some.colors, c)
    assert some.model_bytes == O.rsoc_det_from(g, c, [0, 5, 17]).model_bytes


def test_from_repairs_an_edit_locally():
    rng = np.random.default_rng(3)
    g = I.tri2d(30, 30, jitter=0.3, seed=8)
    c = O.ff(g)
    # insert edges between equal-coloured vertices (conflicts by construction)
    extra, touched = [], []
    for _ in range(40):
        v = int(rng.integers(g.n))
        same = np.nonzero(c == c[v])[0]
        u = int(same[rng.integers(same.size)])
        if u != v:
            extra.append((v, u))
            touched += [v, u]
    g2 = _add_edges(g, extra)
    assert O.check(g2, c)[0] != 0
    for tie in (O.TIE_LOWER_KEEPS, O.TIE_HIGHER_KEEPS):
        r = O.rsoc_det_from(g2, c, touched, tie)
        assert r.status == 0 and O.check(g2, r.colors)[0] == 0
        changed = np.nonzero(r.colors != c)[0]
        assert set(changed) <= set(touched)  # only touched vertices needed a new colour here
    # uncoloured vertices listed as touched get coloured
    c3 = c.copy()
    c3[[3, 100, 400]] = 0
    r = O.rsoc_det_from(g, c3, [3, 100, 400])
    assert O.check(g, r.colors)[0] == 0 and np.all(r.colors[[3, 100, 400]] > 0)
    with pytest.raises(ValueError):
        O.rsoc_det_from(g, c, [g.n])


# ---- distance-2 colouring (Sec. 6: colourings of G^d) -----------------------

def square(g):
    """G^2 built explicitly (edges = paths of one or two edges)."""
    nbr = [set(g.col_idx[g.row_ptr[v]:g.row_ptr[v + 1]].tolist()) for v in range(g.n)]
    e = set()
    for v in range(g.n):
        two = set(nbr[v])
        for u in nbr[v]:
            two |= nbr[u]
        two.discard(v)
        e |= {(min(v, w), max(v, w)) for w in two}
    return I.from_edges(g.n, sorted(e))


D2_GRAPHS = [lambda: I.from_edges(6, [(0, k) for k in range(1, 6)]),   # star: all distinct
             lambda: I.from_edges(7, [(k, k + 1) for k in range(6)]),   # path: 3 colours
             lambda: I.from_edges(5, [(k, (k + 1) % 5) for k in range(5)]),  # C5: its square is K5
             lambda: I.kuhn3d(5), lambda: I.tri2d(9, 11, jitter=0.3, seed=2), lambda: I.rmat(7),
             lambda: I.from_edges(4, [])]


@pytest.mark.parametrize("make", D2_GRAPHS)
def test_d2_first_fit_is_first_fit_of_the_square(make):
    g = make()
    c = O.ff_d2(g)
    assert np.array_equal(c, O.ff(square(g)))
    assert O.check_d2(g, c) == 0


def test_d2_closed_forms():
    star = I.from_edges(6, [(0, k) for k in range(1, 6)])
    assert int(O.ff_d2(star).max()) == 6
    path = I.from_edges(7, [(k, k + 1) for k in range(6)])
    assert list(O.ff_d2(path)) == [1, 2, 3, 1, 2, 3, 1]
    c5 = I.from_edges(5, [(k, (k + 1) % 5) for k in range(5)])
    assert sorted(O.ff_d2(c5)) == [1, 2, 3, 4, 5]
    c6 = I.from_edges(6, [(k, (k + 1) % 6) for k in range(6)])
    assert int(O.ff_d2(c6).max()) == 3
    # a planted error is caught: two vertices two hops apart share a colour
    bad = O.ff_d2(path).copy()
    bad[2] = bad[0]
    assert O.check_d2(path, bad) != 0


@pytest.mark.parametrize("make", D2_GRAPHS)
def test_d2_check_is_validity_on_the_square(make):
    # brute force over the explicit G^2: every edge of G^2 joins two colours
    # that differ, and every vertex is coloured
    g = make()
    sq = square(g)
    rng = np.random.default_rng(3)
    for trial in range(30):
        c = rng.integers(0 if trial % 5 == 0 else 1, 5, g.n).astype(np.int32)
        ok = bool(np.all(c >= 1)) and all(c[v] != c[u] for v in range(sq.n)
                                          for u in sq.col_idx[sq.row_ptr[v]:sq.row_ptr[v + 1]])
        assert (O.check_d2(g, c) == 0) == ok, trial


@pytest.mark.parametrize("make", D2_GRAPHS)
@pytest.mark.parametrize("tie", [O.TIE_LOWER_KEEPS, O.TIE_HIGHER_KEEPS])
def test_d2_replay_is_the_replay_of_the_square(make, tie):
    # Same colours, iterations, conflicts and round sizes as the distance-1
    # replay on G^2 (the byte models differ: G^2 is not built here).
    g = make()
    r2 = O.rsoc_det_d2(g, tie)
    rs = O.rsoc_det(square(g), tie)
    assert np.array_equal(r2.colors, rs.colors)
    assert (r2.iterations, r2.conflicts) == (rs.iterations, rs.conflicts)
    assert np.array_equal(r2.round_sizes, rs.round_sizes)
    assert O.check_d2(g, r2.colors) == 0


def test_d2_replay_bytes_by_hand():
    # P3 (0-1-2), lower keeps, all colour 1 after round 0 (12 bytes).
    # Iteration 1 over V (no worklist bytes); per vertex 8 + 4 + 16*deg +
    # 8*(sum of the neighbours' degrees): v0 44, v1 60, v2 44; v1 and v2 see
    # the lower vertex 0 with their colour and become 2 (+8 each): 164.
    # Iteration 2 over {1, 2} (+4 each): v1 is clean (64); v2 now meets v1's
    # 2 and becomes 3 (4 + 44 + 8 = 56): 120.  Iteration 3 over {2}: 48.
    p3 = I.from_edges(3, [(0, 1), (1, 2)])
    r = O.rsoc_det_d2(p3)
    assert list(r.colors) == [1, 2, 3]
    assert (r.iterations, r.conflicts) == (3, 3)
    assert list(r.round_sizes) == [2, 1, 0]
    assert r.model_bytes == 12 + 164 + 120 + 48

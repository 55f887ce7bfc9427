"""Seeded generators: sizes from closed forms, well-formed CSR, determinism."""
import numpy as np

import oracle as O
from paper_1505_04086_gb300 import inputs as I


def test_tri2d_counts():
    for R, C in [(1, 1), (1, 5), (4, 1), (3, 4), (64, 64)]:
        g = I.tri2d(R, C)
        assert g.n == R * C
        assert g.num_edges == R * (C - 1) + (R - 1) * C + (R - 1) * (C - 1)
        assert O.csr_check(g) == 0
    g = I.tri2d(64, 64)
    assert g.num_edges == 12033
    assert int(g.degrees().max()) == 6


def test_tri2d_jittered_is_a_triangulation():
    g = I.tri2d(20, 30, jitter=0.3, seed=4)
    # Same edge count as any one-diagonal-per-cell split.
    assert g.num_edges == 20 * 29 + 19 * 30 + 19 * 29
    assert O.csr_check(g) == 0
    h = I.tri2d(20, 30, jitter=0.3, seed=4)
    assert np.array_equal(g.col_idx, h.col_idx)
    k = I.tri2d(20, 30, jitter=0.3, seed=5)
    assert not np.array_equal(g.col_idx, k.col_idx)


def kuhn_edges(N):
    L, Lm = N, N - 1
    return 3 * Lm * L * L + 3 * Lm * Lm * L + Lm ** 3


def test_kuhn3d_counts():
    for N in (1, 2, 3, 8, 17):
        g = I.kuhn3d(N)
        assert g.n == N ** 3
        assert g.num_edges == kuhn_edges(N)
        assert O.csr_check(g) == 0
    g = I.kuhn3d(8, permute=False)
    d = g.degrees().reshape(8, 8, 8)
    assert (d[1:-1, 1:-1, 1:-1] == 14).all()
    assert kuhn_edges(128) == 14484223


def test_kuhn3d_permutation_is_relabelling():
    a = I.kuhn3d(6, permute=False)
    b = I.kuhn3d(6, permute=True)
    p = I.permutation(a.n, I.SEED_KUHN)
    assert np.array_equal(np.sort(p), np.arange(a.n))
    # edge (u,v) of a maps to (p[u], p[v]) of b
    src = np.repeat(np.arange(a.n), a.degrees())
    ea = set(zip(p[src].tolist(), p[a.col_idx].tolist()))
    srcb = np.repeat(np.arange(b.n), b.degrees())
    eb = set(zip(srcb.tolist(), b.col_idx.tolist()))
    assert ea == eb


def test_rmat_small():
    g = I.rmat(12, 16)
    assert g.n == 4096
    assert O.csr_check(g) == 0
    h = I.rmat(12, 16)
    assert np.array_equal(g.col_idx, h.col_idx)
    d = g.degrees()
    assert d.max() > 20 * max(1.0, d.mean())  # heavy tail
    assert g.num_edges <= 16 * 4096


def test_rgg_mean_degree():
    g = I.rgg(20000, 12.0, seed=2)
    assert O.csr_check(g) == 0
    assert 10.5 < g.degrees().mean() < 12.5  # boundary loss lowers it slightly


def test_batch_layout():
    b = I.batch(12, 1 << 6, 1 << 10, seed=3, threads=4)
    assert b.G == 12
    assert b.row_ptr.size == b.total_n + b.G
    for g in range(b.G):
        c = b.graph(g)
        assert O.csr_check(c) == 0
        assert (1 << 6) <= c.n <= (1 << 10)
    b2 = I.batch(12, 1 << 6, 1 << 10, seed=3, threads=1)
    assert np.array_equal(b.col_idx, b2.col_idx)
    assert np.array_equal(b.vtx_off, b2.vtx_off)
    bb = I.Batch.from_graphs([b.graph(g) for g in range(b.G)])
    assert np.array_equal(bb.col_idx, b.col_idx) and np.array_equal(bb.row_ptr, b.row_ptr)

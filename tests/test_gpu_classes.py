"""gc_color_classes: the colour classes of a colouring (stable counting sort
by colour) against the oracle's, element by element."""
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


def gpu_classes(ctx, colors, k):
    n = int(colors.size)
    d = torch.from_numpy(colors if n else np.zeros(1, np.int32)).cuda()
    ptr = torch.full((k + 2,), -5, dtype=torch.int32, device="cuda")
    verts = torch.full((max(n, 1),), -5, dtype=torch.int32, device="cuda")
    rc = gc.gc_color_classes(ctx.handle, d, n, k, ptr, verts)
    return rc, ptr.cpu().numpy(), verts.cpu().numpy()[:n]


@pytest.mark.parametrize("make", [lambda: I.tri2d(64, 64), lambda: I.kuhn3d(24), lambda: I.rmat(12),
                                  lambda: I.from_edges(1, []), lambda: I.rgg(30000, 12.0, seed=3)],
                         ids=["tri64", "kuhn24", "rmat12", "single", "rgg30k"])
def test_classes_of_a_gpu_colouring_match_the_oracle(ctx, make):
    g = make()
    col, rc, st = ctx.color(torch.from_numpy(g.row_ptr).cuda(),
                            torch.from_numpy(g.col_idx if g.nnz else np.zeros(1, np.int32)).cuda(),
                            gc.GC_SCHED_ASYNC)
    c = col.cpu().numpy()
    k = int(c.max())
    for kk in (k, k + 3):  # exact colour count, and a wider range with empty classes
        rc, ptr, verts = gpu_classes(ctx, c, kk)
        assert rc == gc.GC_OK
        optr, overts = O.classes(c, kk)
        assert np.array_equal(ptr, optr)
        assert np.array_equal(verts, overts)


def test_classes_random_colours_large_and_wide(ctx):
    rng = np.random.default_rng(9)
    for n, k in ((2_097_152, 13), (1 << 20, 1 << 20), (100_003, 700)):
        c = rng.integers(1, k + 1, size=n, dtype=np.int32)
        rc, ptr, verts = gpu_classes(ctx, c, k)
        assert rc == gc.GC_OK
        optr, overts = O.classes(c, k)
        assert np.array_equal(ptr, optr) and np.array_equal(verts, overts)


def test_classes_reject_bad_colours_and_handle_empty(ctx):
    for bad in (np.array([1, 0, 2], np.int32), np.array([1, 5, 2], np.int32)):
        rc, _, _ = gpu_classes(ctx, bad, 3)
        assert rc == gc.GC_ERR_ARG
    rc, ptr, verts = gpu_classes(ctx, np.zeros(0, np.int32), 4)
    assert rc == gc.GC_OK and list(ptr) == [0] * 6 and verts.size == 0
    rc, _, _ = gpu_classes(ctx, np.array([1], np.int32), gc.GC_CLASSES_MAX_COLORS + 1)
    assert rc == gc.GC_ERR_ARG

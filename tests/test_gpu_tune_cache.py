"""The autotuner's on-disk cache (GC_TUNE_CACHE): the first call searches
and stores its choice under a key of the call, mode, graph shape and device;
a second call with the same key searches nothing, returns the stored options
and still delivers a colouring; another mode or graph is a different key."""
import os

import numpy as np
import pytest

import oracle as O
from paper_1505_04086_gb300 import inputs as I

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from paper_1505_04086_gb300 import gc  # noqa: E402


def test_tune_cache(tmp_path, monkeypatch):
    path = tmp_path / "tune.txt"
    monkeypatch.setenv("GC_TUNE_CACHE", str(path))
    g = I.kuhn3d(24)
    d = torch.device("cuda:0")
    rp, ci = torch.from_numpy(g.row_ptr).to(d), torch.from_numpy(g.col_idx).to(d)
    col = torch.empty(g.n, dtype=torch.int32, device=d)
    ctx = gc.Context(0)
    try:
        rc, first = gc.gc_autotune(ctx.handle, rp, ci, g.n, g.nnz, gc.GC_SCHED_ASYNC, col, reps=1)
        assert rc == gc.GC_OK and first["evaluated"] > 0
        lines = path.read_text().splitlines()
        assert len(lines) == 1 and ":graph:" in lines[0]
        col.fill_(0)
        rc, again = gc.gc_autotune(ctx.handle, rp, ci, g.n, g.nnz, gc.GC_SCHED_ASYNC, col, reps=1)
        assert rc == gc.GC_OK and again["evaluated"] == 0
        assert again["best"] == first["best"]
        assert O.check(g, col.cpu().numpy())[0] == 0  # the cached options' colouring
        # deterministic mode: another key, searched and stored
        rc, det = gc.gc_autotune(ctx.handle, rp, ci, g.n, g.nnz, gc.GC_SCHED_DET, col, reps=1)
        assert rc == gc.GC_OK and det["evaluated"] > 0
        assert np.array_equal(col.cpu().numpy(), O.rsoc_det(g).colors)
        assert len(path.read_text().splitlines()) == 2
    finally:
        ctx.close()
    monkeypatch.delenv("GC_TUNE_CACHE")
    assert not os.environ.get("GC_TUNE_CACHE")

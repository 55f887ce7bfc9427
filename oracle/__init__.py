"""CPU oracle for the colouring path (TEST INFRASTRUCTURE ONLY).

Plain single-threaded C (``oracle.c``) behind ctypes.  Only the tests, the
smoke check and the benchmark's CPU-baseline leg may import this package; the
product path never does.  It shares no code with the CUDA library.

Functions follow the paper (arXiv 1505.04086):

* :func:`ff`            Algorithm 1, sequential First-Fit in natural order
* :func:`rsoc_det`      Algorithm 3 (RSOC), round-synchronous snapshot replay
* :func:`twophase_det`  Algorithm 2 (Catalyurek et al.), same reading,
                        independent code
* :func:`check`         proper colouring and the d+1 bound (Section 2.1)
* :func:`chi`           exact chromatic number of graphs with <= 12 vertices
* :func:`csr_check`     input well-formedness
"""
from __future__ import annotations

import ctypes
import threading
from dataclasses import dataclass, field

import numpy as np

from . import build as _build

TIE_LOWER_KEEPS = 0
TIE_HIGHER_KEEPS = 1
TIE_NONE = 2

OK = 0
ERR_ARG = 1
ERR_OOM = 2
ERR_NO_CONVERGENCE = 3

_lock = threading.Lock()
_lib = None


class _Stats(ctypes.Structure):
    _fields_ = [("iterations", ctypes.c_int64), ("conflicts", ctypes.c_int64),
                ("model_bytes", ctypes.c_int64), ("colors", ctypes.c_int32),
                ("distinct_colors", ctypes.c_int32), ("round_sizes", ctypes.c_void_p),
                ("round_sizes_cap", ctypes.c_int64)]


def _load():
    global _lib
    with _lock:
        if _lib is None:
            lib = ctypes.CDLL(_build.build())
            P, i32, i64 = ctypes.c_void_p, ctypes.c_int32, ctypes.c_int64
            lib.oracle_ff.restype = i32
            lib.oracle_ff.argtypes = [i32, P, P, P]
            for f in (lib.oracle_rsoc_det, lib.oracle_2p_det):
                f.restype = ctypes.c_int
                f.argtypes = [i32, P, P, ctypes.c_int, i64, P, ctypes.POINTER(_Stats)]
            lib.oracle_check.restype = i64
            lib.oracle_check.argtypes = [i32, P, P, P, ctypes.POINTER(i32), ctypes.POINTER(i32)]
            lib.oracle_chi.restype = i32
            lib.oracle_chi.argtypes = [i32, P, P]
            lib.oracle_csr_check.restype = i64
            lib.oracle_csr_check.argtypes = [i32, i64, P, P]
            lib.oracle_rsoc_det_from.restype = ctypes.c_int
            lib.oracle_rsoc_det_from.argtypes = [i32, P, P, ctypes.c_int, i64, P, i32, P, ctypes.POINTER(_Stats)]
            lib.oracle_ff_d2.restype = i32
            lib.oracle_ff_d2.argtypes = [i32, P, P, P]
            lib.oracle_rsoc_det_d2.restype = ctypes.c_int
            lib.oracle_rsoc_det_d2.argtypes = [i32, P, P, ctypes.c_int, i64, P, ctypes.POINTER(_Stats)]
            lib.oracle_check_d2.restype = i64
            lib.oracle_check_d2.argtypes = [i32, P, P, P]
            lib.oracle_classes.restype = i64
            lib.oracle_classes.argtypes = [i32, P, i32, P, P]
            _lib = lib
        return _lib


def _arrays(g):
    rp = np.ascontiguousarray(g.row_ptr, dtype=np.int32)
    ci = np.ascontiguousarray(g.col_idx, dtype=np.int32)
    if ci.size == 0:
        ci = np.zeros(1, np.int32)
    return rp, ci


@dataclass
class Result:
    colors: np.ndarray
    status: int
    iterations: int
    conflicts: int
    model_bytes: int
    num_colors: int
    distinct_colors: int
    round_sizes: np.ndarray = field(default_factory=lambda: np.zeros(0, np.int32))


def ff(g) -> np.ndarray:
    """Algorithm 1 in natural vertex order; returns int32 colours (1-based)."""
    rp, ci = _arrays(g)
    c = np.zeros(max(g.n, 1), np.int32)
    r = _load().oracle_ff(g.n, rp.ctypes.data, ci.ctypes.data, c.ctypes.data)
    if r < 0:
        raise MemoryError("oracle_ff")
    return c[: g.n]


def _replay(fn, g, tie, max_iters, round_cap):
    rp, ci = _arrays(g)
    c = np.zeros(max(g.n, 1), np.int32)
    rs = np.zeros(max(round_cap, 1), np.int32)
    st = _Stats()
    st.round_sizes = rs.ctypes.data
    st.round_sizes_cap = round_cap
    if max_iters is None:
        max_iters = g.n + 1
    rc = fn(g.n, rp.ctypes.data, ci.ctypes.data, int(tie), int(max_iters), c.ctypes.data,
            ctypes.byref(st))
    if rc in (ERR_ARG, ERR_OOM):
        raise RuntimeError(f"oracle replay failed with status {rc}")
    k = min(int(st.iterations), round_cap)
    return Result(c[: g.n], rc, int(st.iterations), int(st.conflicts), int(st.model_bytes),
                  int(st.colors), int(st.distinct_colors), rs[:k].copy())


def rsoc_det(g, tie: int = TIE_LOWER_KEEPS, max_iters: int | None = None,
             round_cap: int = 4096) -> Result:
    """Algorithm 3 (RSOC) with round-synchronous snapshot reads."""
    return _replay(_load().oracle_rsoc_det, g, tie, max_iters, round_cap)


def twophase_det(g, tie: int = TIE_LOWER_KEEPS, max_iters: int | None = None,
                 round_cap: int = 4096) -> Result:
    """Algorithm 2 (two-phase) with round-synchronous snapshot reads."""
    return _replay(_load().oracle_2p_det, g, tie, max_iters, round_cap)


def check(g, colors) -> tuple[int, int, int]:
    """(status, max colour, distinct colours).  status 0 = proper colouring
    within 1..deg+1; v+1 = v conflicts with a neighbour; -(v+1) = v's colour
    is out of bounds."""
    rp, ci = _arrays(g)
    c = np.ascontiguousarray(colors, dtype=np.int32)
    if c.size == 0:
        c = np.zeros(1, np.int32)
    mx, dist = ctypes.c_int32(0), ctypes.c_int32(0)
    bad = _load().oracle_check(g.n, rp.ctypes.data, ci.ctypes.data, c.ctypes.data,
                               ctypes.byref(mx), ctypes.byref(dist))
    return int(bad), int(mx.value), int(dist.value)


def chi(g) -> int:
    """Exact chromatic number (exhaustive search), n <= 12."""
    rp, ci = _arrays(g)
    r = _load().oracle_chi(g.n, rp.ctypes.data, ci.ctypes.data)
    if r < 0:
        raise ValueError("oracle.chi supports n <= 12")
    return int(r)


def csr_check(g) -> int:
    """0 if the CSR is symmetric, sorted, in range and simple, else 1 + the
    first offending vertex."""
    rp, ci = _arrays(g)
    return int(_load().oracle_csr_check(g.n, g.nnz, rp.ctypes.data, ci.ctypes.data))


def classes(colors, k: int | None = None) -> tuple[np.ndarray, np.ndarray]:
    """Colour classes of a colouring (stable counting sort by colour):
    (ptr[k+2], verts[n]); the vertices of colour c are verts[ptr[c]:ptr[c+1]]
    in increasing id."""
    c = np.ascontiguousarray(colors, dtype=np.int32)
    n = int(c.size)
    if k is None:
        k = int(c.max()) if n else 0
    ptr = np.zeros(k + 2, np.int32)
    verts = np.zeros(max(n, 1), np.int32)
    cc = c if n else np.zeros(1, np.int32)
    r = _load().oracle_classes(n, cc.ctypes.data, int(k), ptr.ctypes.data, verts.ctypes.data)
    if r != 0:
        raise ValueError(f"colour out of 1..{k} at vertex {r - 1}")
    return ptr, verts[:n]


def rsoc_det_from(g, colors, touched, tie: int = TIE_LOWER_KEEPS, max_iters: int | None = None,
                  round_cap: int = 4096) -> Result:
    """Incremental recolouring: Algorithm 3's while-loop (snapshot reads)
    from the colouring `colors` with U = `touched` (see oracle.c)."""
    rp, ci = _arrays(g)
    c = np.array(colors, dtype=np.int32, copy=True)
    if c.size != g.n:
        raise ValueError("colors must have n entries")
    cc = c if g.n else np.zeros(1, np.int32)
    t = np.ascontiguousarray(touched, dtype=np.int32)
    tt = t if t.size else np.zeros(1, np.int32)
    rs = np.zeros(round_cap, np.int32)
    st = _Stats()
    st.round_sizes = rs.ctypes.data
    st.round_sizes_cap = round_cap
    mi = max_iters if max_iters is not None else g.n + 1
    status = _load().oracle_rsoc_det_from(g.n, rp.ctypes.data, ci.ctypes.data, int(tie), int(mi), tt.ctypes.data,
                                          int(t.size), cc.ctypes.data, ctypes.byref(st))
    if status == 1:
        raise ValueError("touched vertex out of range")
    return Result(c, status, int(st.iterations), int(st.conflicts), int(st.model_bytes), int(st.colors),
                  int(st.distinct_colors), rs[: min(int(st.iterations), round_cap)].copy())


def ff_d2(g) -> np.ndarray:
    """Algorithm 1 over two-hop neighbourhoods (distance-2 colouring)."""
    rp, ci = _arrays(g)
    c = np.zeros(max(g.n, 1), np.int32)
    if _load().oracle_ff_d2(g.n, rp.ctypes.data, ci.ctypes.data, c.ctypes.data) < 0:
        raise MemoryError("oracle_ff_d2 failed")
    return c[: g.n]


def rsoc_det_d2(g, tie: int = TIE_LOWER_KEEPS, max_iters: int | None = None, round_cap: int = 4096) -> Result:
    """Algorithm 3 (snapshot reads) over two-hop neighbourhoods."""
    return _replay(_load().oracle_rsoc_det_d2, g, tie, max_iters, round_cap)


def check_d2(g, colors) -> int:
    """0 if no two vertices within two hops share a colour (and all are
    coloured), else 1 + the first offending vertex."""
    rp, ci = _arrays(g)
    c = np.ascontiguousarray(colors, dtype=np.int32)
    if c.size == 0:
        c = np.zeros(1, np.int32)
    return int(_load().oracle_check_d2(g.n, rp.ctypes.data, ci.ctypes.data, c.ctypes.data))

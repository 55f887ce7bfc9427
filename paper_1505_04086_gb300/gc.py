"""ctypes binding of libgc (include/gc.h): argument marshalling only.

Every step of the colouring runs in the library (CUDA kernels; the paper's
OpenMP form, gc_host_color, is the library's separate host entry point);
this module converts torch tensors / numpy arrays to pointers and structs
and back.  It raises if libgc.so has not been built: there is no CPU
fallback.

The entry points keep the C names (gc_color, gc_color_async, gc_ctx_stats,
gc_color_batch, ...); :class:`Context` is a small convenience wrapper.
"""
from __future__ import annotations

import ctypes
import os
import threading

import numpy as np

from . import _build

# status codes
GC_OK = 0
GC_PENDING = 1
GC_ERR_ARG = -1
GC_ERR_GRAPH = -2
GC_ERR_OOM = -3
GC_ERR_BUDGET = -4
GC_ERR_NO_CONVERGENCE = -5
GC_ERR_TIMEOUT = -6
GC_ERR_CUDA = -7
GC_ERR_OVERFLOW = -8
GC_ERR_CHECK = -9
GC_ERR_NOT_FOUND = -10
GC_ERR_TOO_LARGE = -11
GC_NOALLOC_MAX_N = 262144
GC_CLASSES_MAX_COLORS = 1 << 20

# mode bits
GC_ALG_RSOC = 0
GC_ALG_TWO_PHASE = 1
GC_SCHED_DET = 0
GC_SCHED_ASYNC = 2
GC_TIE_LOWER_KEEPS = 0
GC_TIE_HIGHER_KEEPS = 4
GC_VALIDATE = 8
GC_CHECKED = 16
GC_DEBUG_NO_TIEBREAK = 32
GC_NO_COLOR_STATS = 64
GC_REPAIR_SNAPSHOT = 128
GC_TIERS = 256
GC_FF_KEEPERS = 512
GC_DIST2 = 1024

# error word bits
GC_EW_TIMEOUT = 1
GC_EW_NO_CONVERGENCE = 2
GC_EW_OVERFLOW = 4
GC_EW_GRAPH = 8
GC_EW_CHECK = 16

GC_WAIT_GRID_BARRIER = 0
GC_WAIT_TILE_DONE = 1
GC_WAIT_PIPE_CHUNK = 2
GC_WAIT_STAGE_COPY = 3


class gc_csr(ctypes.Structure):
    _fields_ = [("row_ptr", ctypes.c_void_p), ("col_idx", ctypes.c_void_p)]


class gc_stats(ctypes.Structure):
    _fields_ = [("rounds", ctypes.c_int32), ("colors", ctypes.c_int32),
                ("conflicts", ctypes.c_int64), ("distinct_colors", ctypes.c_int32),
                ("error_word", ctypes.c_int32), ("model_bytes", ctypes.c_int64),
                ("elapsed_ms", ctypes.c_float), ("round_sizes", ctypes.c_void_p),
                ("round_sizes_cap", ctypes.c_int32), ("round_ns", ctypes.c_void_p),
                ("round_ns_cap", ctypes.c_int32)]


class gc_opts(ctypes.Structure):
    _fields_ = [("max_rounds", ctypes.c_int32), ("t1", ctypes.c_int32), ("t2", ctypes.c_int32),
                ("tile", ctypes.c_int32), ("blocks_per_sm", ctypes.c_int32),
                ("tail", ctypes.c_int32), ("window", ctypes.c_int32), ("d2_heavy", ctypes.c_int32),
                ("core_deg", ctypes.c_int32)]


class gc_batch(ctypes.Structure):
    _fields_ = [("G", ctypes.c_int32), ("total_n", ctypes.c_int64), ("total_nnz", ctypes.c_int64),
                ("vtx_off", ctypes.c_void_p), ("edge_off", ctypes.c_void_p),
                ("row_ptr", ctypes.c_void_p), ("col_idx", ctypes.c_void_p)]


class gc_tune_result(ctypes.Structure):
    _fields_ = [("best", gc_opts), ("best_ms", ctypes.c_float), ("default_ms", ctypes.c_float),
                ("evaluated", ctypes.c_int32)]


class gc_server_info(ctypes.Structure):
    _fields_ = [("submitted", ctypes.c_uint64), ("completed", ctypes.c_uint64),
                ("failed", ctypes.c_uint64), ("waves", ctypes.c_uint64),
                ("budget_bytes", ctypes.c_int64), ("in_use_bytes", ctypes.c_int64),
                ("peak_bytes", ctypes.c_int64), ("queued", ctypes.c_int32),
                ("resident", ctypes.c_int32), ("max_wave_graphs", ctypes.c_int32),
                ("lanes", ctypes.c_int32), ("cancelled", ctypes.c_uint64),
                ("overlapped_waves", ctypes.c_uint64), ("overlap_us", ctypes.c_int64)]


# Every function the header declares, with its ctypes signature.
_P = ctypes.c_void_p
_SIGS = {
    "gc_strerror": (ctypes.c_char_p, [ctypes.c_int]),
    "gc_version": (ctypes.c_int, []),
    "gc_ctx_create": (ctypes.c_int, [ctypes.POINTER(_P), ctypes.c_int]),
    "gc_ctx_destroy": (None, [_P]),
    "gc_color": (ctypes.c_int, [ctypes.POINTER(gc_csr), ctypes.c_int32, ctypes.c_int64, ctypes.c_uint32,
                                _P, ctypes.POINTER(gc_stats)]),
    "gc_color_async": (ctypes.c_int, [_P, ctypes.POINTER(gc_csr), ctypes.c_int32, ctypes.c_int64,
                                      ctypes.c_uint32, ctypes.POINTER(gc_opts), _P, _P]),
    "gc_ctx_stats": (ctypes.c_int, [_P, ctypes.POINTER(gc_stats)]),
    "gc_recolor_async": (ctypes.c_int, [_P, ctypes.POINTER(gc_csr), ctypes.c_int32, ctypes.c_int64,
                                        ctypes.c_uint32, ctypes.POINTER(gc_opts), _P, _P, ctypes.c_int32, _P]),
    "gc_color_batch": (ctypes.c_int, [_P, ctypes.POINTER(gc_batch), ctypes.c_uint32,
                                      ctypes.POINTER(gc_opts), _P, _P, _P, _P]),
    "gc_plan_create": (ctypes.c_int, [ctypes.POINTER(gc_batch), ctypes.c_int, ctypes.c_uint32,
                                      ctypes.POINTER(gc_opts), _P, _P, _P, ctypes.POINTER(_P)]),
    "gc_plan_launch": (ctypes.c_int, [_P, _P]),
    "gc_plan_stats": (ctypes.c_int, [_P, ctypes.POINTER(gc_stats)]),
    "gc_plan_destroy": (None, [_P]),
    "gc_autotune_batch": (ctypes.c_int, [_P, ctypes.POINTER(gc_batch), ctypes.c_uint32, ctypes.c_int32, _P,
                                         ctypes.POINTER(gc_tune_result)]),
    "gc_autotune": (ctypes.c_int, [_P, ctypes.POINTER(gc_csr), ctypes.c_int32, ctypes.c_int64, ctypes.c_uint32,
                                   ctypes.c_int32, _P, ctypes.POINTER(gc_tune_result)]),
    "gc_color_classes": (ctypes.c_int, [_P, _P, ctypes.c_int32, ctypes.c_int32, _P, _P, _P]),
    "gc_server_create": (ctypes.c_int, [ctypes.POINTER(_P), ctypes.c_int, ctypes.c_size_t, ctypes.c_int,
                                        ctypes.c_uint32, ctypes.POINTER(gc_opts)]),
    "gc_server_submit": (ctypes.c_int, [_P, ctypes.POINTER(gc_csr), ctypes.c_int32, ctypes.c_int64,
                                        ctypes.POINTER(ctypes.c_uint64)]),
    "gc_server_poll": (ctypes.c_int, [_P, ctypes.c_uint64, _P, ctypes.POINTER(gc_stats)]),
    "gc_server_wait": (ctypes.c_int, [_P, ctypes.c_uint64, _P, ctypes.POINTER(gc_stats), ctypes.c_int32]),
    "gc_server_query": (ctypes.c_int, [_P, ctypes.POINTER(gc_server_info)]),
    "gc_server_cancel": (ctypes.c_int, [_P, ctypes.c_uint64]),
    "gc_server_destroy": (None, [_P]),
    "gc_color_noalloc": (ctypes.c_int, [ctypes.POINTER(gc_csr), ctypes.c_int32, ctypes.c_int64,
                                        ctypes.c_uint32, ctypes.POINTER(gc_opts), _P,
                                        ctypes.POINTER(gc_stats), _P]),
    "gc_host_color": (ctypes.c_int, [ctypes.POINTER(gc_csr), ctypes.c_int32, ctypes.c_int64, ctypes.c_uint32,
                                     ctypes.c_int32, _P, ctypes.POINTER(gc_stats)]),
    "gc_host_threads": (ctypes.c_int, []),
    "gc_debug_barrier_timeout": (ctypes.c_int, [ctypes.c_int, ctypes.c_int32, ctypes.POINTER(ctypes.c_int32)]),
    "gc_debug_wait_timeout": (ctypes.c_int, [ctypes.c_int, ctypes.c_int32, ctypes.c_int32,
                                             ctypes.POINTER(ctypes.c_int32)]),
    "gc_measure_gather_rate": (ctypes.c_int, [ctypes.c_int, ctypes.c_int64, ctypes.c_int32, ctypes.c_int32,
                                              ctypes.POINTER(ctypes.c_double)]),
}

_lock = threading.Lock()
_lib = None


def lib_path() -> str:
    return _build.LIB


def load():
    """Load libgc.so.  Raises if it is missing (run the package build)."""
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        path = _build.LIB
        if not os.path.exists(path):
            raise RuntimeError(f"libgc.so not built ({path}); run __graft_entry__.build() or "
                               "python -m paper_1505_04086_gb300._build")
        lib = ctypes.CDLL(path)
        for name, (res, args) in _SIGS.items():
            f = getattr(lib, name)
            f.restype = res
            f.argtypes = args
        _lib = lib
        return lib


class GCError(RuntimeError):
    def __init__(self, status: int, what: str = ""):
        self.status = status
        super().__init__(f"{what}: {gc_strerror(status)} ({status})")


def gc_strerror(status: int) -> str:
    return load().gc_strerror(int(status)).decode()


def gc_version() -> int:
    return int(load().gc_version())


# ---------------------------------------------------------------- marshalling

def _ptr(x) -> int:
    """Raw address of a torch tensor or numpy array (None -> 0)."""
    if x is None:
        return 0
    if hasattr(x, "data_ptr"):
        if not x.is_contiguous():
            raise ValueError("tensor must be contiguous")
        return int(x.data_ptr())
    if isinstance(x, np.ndarray):
        if not x.flags["C_CONTIGUOUS"]:
            raise ValueError("array must be C-contiguous")
        return int(x.ctypes.data)
    raise TypeError(f"expected a torch tensor or numpy array, got {type(x)}")


def _check_i32(x, name):
    dt = getattr(x, "dtype", None)
    if str(dt) not in ("int32", "torch.int32"):
        raise TypeError(f"{name} must be int32, got {dt}")


def _stream_handle(stream) -> int:
    if stream is None:
        return 0
    if isinstance(stream, int):
        return stream
    return int(stream.cuda_stream)


def _opts(opts) -> gc_opts | None:
    if opts is None:
        return None
    if isinstance(opts, gc_opts):
        return opts
    o = gc_opts()
    for k, v in dict(opts).items():
        setattr(o, k, int(v))
    return o


def stats_dict(s: gc_stats, round_sizes=None, round_ns=None) -> dict:
    d = {"rounds": s.rounds, "colors": s.colors, "conflicts": s.conflicts,
         "distinct_colors": s.distinct_colors, "error_word": s.error_word,
         "model_bytes": s.model_bytes, "elapsed_ms": float(s.elapsed_ms)}
    if round_sizes is not None:
        d["round_sizes"] = round_sizes[: min(s.rounds, len(round_sizes))].copy()
    if round_ns is not None:
        d["round_ns"] = round_ns[: min(s.rounds + 1, len(round_ns))].copy()
    return d


def _stats_buffers(st: gc_stats, round_cap: int):
    if round_cap <= 0:
        return None, None
    rs = np.zeros(round_cap, np.int32)
    rn = np.zeros(round_cap, np.int64)
    st.round_sizes = rs.ctypes.data
    st.round_sizes_cap = round_cap
    st.round_ns = rn.ctypes.data
    st.round_ns_cap = round_cap
    return rs, rn


def gc_ctx_create(device: int = 0) -> int:
    h = ctypes.c_void_p()
    rc = load().gc_ctx_create(ctypes.byref(h), int(device))
    if rc != GC_OK:
        raise GCError(rc, "gc_ctx_create")
    return int(h.value)


def gc_ctx_destroy(ctx: int) -> None:
    load().gc_ctx_destroy(ctypes.c_void_p(ctx))


def gc_color(row_ptr, col_idx, n: int, nnz: int, mode: int, colors_out, round_cap: int = 0):
    """Synchronous colouring; arrays may be host (numpy) or device (torch).
    Returns (status, stats dict)."""
    _check_i32(row_ptr, "row_ptr")
    _check_i32(col_idx, "col_idx")
    _check_i32(colors_out, "colors_out")
    csr = gc_csr(_ptr(row_ptr), _ptr(col_idx) if nnz else 0)
    st = gc_stats()
    rs, rn = _stats_buffers(st, round_cap)
    rc = load().gc_color(ctypes.byref(csr), int(n), int(nnz), int(mode), _ptr(colors_out),
                         ctypes.byref(st))
    return rc, stats_dict(st, rs, rn)


def gc_color_async(ctx: int, row_ptr, col_idx, n: int, nnz: int, mode: int, colors_out,
                   opts=None, stream=None) -> int:
    """Enqueue one colouring (device arrays); returns the launch status."""
    csr = gc_csr(_ptr(row_ptr), _ptr(col_idx) if nnz else 0)
    o = _opts(opts)
    return int(load().gc_color_async(ctypes.c_void_p(ctx), ctypes.byref(csr), int(n), int(nnz),
                                     int(mode), ctypes.byref(o) if o is not None else None,
                                     _ptr(colors_out), ctypes.c_void_p(_stream_handle(stream))))


def gc_recolor_async(ctx: int, row_ptr, col_idx, n: int, nnz: int, mode: int, colors_inout, touched,
                     opts=None, stream=None) -> int:
    """Enqueue an incremental recolouring (device arrays); returns the
    launch status.  Finish with gc_ctx_stats."""
    csr = gc_csr(_ptr(row_ptr), _ptr(col_idx) if nnz else 0)
    o = _opts(opts)
    nt = int(touched.numel() if hasattr(touched, "numel") else len(touched))
    return int(load().gc_recolor_async(ctypes.c_void_p(ctx), ctypes.byref(csr), int(n), int(nnz), int(mode),
                                       ctypes.byref(o) if o is not None else None, _ptr(colors_inout),
                                       _ptr(touched) if nt else 0, nt, ctypes.c_void_p(_stream_handle(stream))))


def gc_ctx_stats(ctx: int, round_cap: int = 0):
    """Wait for the context's last colouring; returns (status, stats dict)."""
    st = gc_stats()
    rs, rn = _stats_buffers(st, round_cap)
    rc = load().gc_ctx_stats(ctypes.c_void_p(ctx), ctypes.byref(st))
    return int(rc), stats_dict(st, rs, rn)


def gc_color_batch(ctx: int, G: int, total_n: int, total_nnz: int, vtx_off, edge_off, row_ptr,
                   col_idx, mode: int, colors_out, rounds_out=None, conflicts_out=None,
                   opts=None, stream=None) -> int:
    """Enqueue the colouring of a batch of graphs (device arrays)."""
    b = gc_batch(int(G), int(total_n), int(total_nnz), _ptr(vtx_off), _ptr(edge_off),
                 _ptr(row_ptr), _ptr(col_idx) if total_nnz else 0)
    o = _opts(opts)
    return int(load().gc_color_batch(ctypes.c_void_p(ctx), ctypes.byref(b), int(mode),
                                     ctypes.byref(o) if o is not None else None,
                                     _ptr(colors_out), _ptr(rounds_out), _ptr(conflicts_out),
                                     ctypes.c_void_p(_stream_handle(stream))))


def _batch(G, total_n, total_nnz, vtx_off, edge_off, row_ptr, col_idx) -> gc_batch:
    return gc_batch(int(G), int(total_n), int(total_nnz), _ptr(vtx_off), _ptr(edge_off),
                    _ptr(row_ptr), _ptr(col_idx) if total_nnz else 0)


def opts_dict(o: gc_opts) -> dict:
    return {k: int(getattr(o, k)) for k, _ in gc_opts._fields_}


def gc_autotune_batch(ctx: int, G: int, total_n: int, total_nnz: int, vtx_off, edge_off, row_ptr, col_idx,
                      mode: int, colors_out, reps: int = 3):
    """Time option sets on the batch; returns (status, {"best": opts dict,
    "best_ms", "default_ms", "evaluated"})."""
    b = _batch(G, total_n, total_nnz, vtx_off, edge_off, row_ptr, col_idx)
    r = gc_tune_result()
    rc = load().gc_autotune_batch(ctypes.c_void_p(ctx), ctypes.byref(b), int(mode), int(reps),
                                  _ptr(colors_out), ctypes.byref(r))
    return int(rc), {"best": opts_dict(r.best), "best_ms": float(r.best_ms),
                     "default_ms": float(r.default_ms), "evaluated": int(r.evaluated)}


def gc_autotune(ctx: int, row_ptr, col_idx, n: int, nnz: int, mode: int, colors_out, reps: int = 3):
    """Time option sets on one graph; returns (status, result dict as
    gc_autotune_batch)."""
    csr = gc_csr(_ptr(row_ptr), _ptr(col_idx) if nnz else 0)
    r = gc_tune_result()
    rc = load().gc_autotune(ctypes.c_void_p(ctx), ctypes.byref(csr), int(n), int(nnz), int(mode), int(reps),
                            _ptr(colors_out), ctypes.byref(r))
    return int(rc), {"best": opts_dict(r.best), "best_ms": float(r.best_ms),
                     "default_ms": float(r.default_ms), "evaluated": int(r.evaluated)}


def gc_color_classes(ctx: int, colors, n: int, num_colors: int, class_ptr, class_vertices, stream=None) -> int:
    """Group the vertices of a colouring by colour (device arrays); returns
    the status.  class_ptr has num_colors + 2 entries, class_vertices n."""
    return int(load().gc_color_classes(ctypes.c_void_p(ctx), _ptr(colors), int(n), int(num_colors),
                                       _ptr(class_ptr), _ptr(class_vertices),
                                       ctypes.c_void_p(_stream_handle(stream))))


class Plan:
    """A batch colouring captured in a CUDA graph (gc_plan_*): launch()
    replays it on a stream, stats() waits and reports."""

    def __init__(self, device: int, G: int, total_n: int, total_nnz: int, vtx_off, edge_off, row_ptr, col_idx,
                 mode: int, colors_out, rounds_out=None, conflicts_out=None, opts=None):
        b = _batch(G, total_n, total_nnz, vtx_off, edge_off, row_ptr, col_idx)
        o = _opts(opts)
        h = ctypes.c_void_p()
        rc = load().gc_plan_create(ctypes.byref(b), int(device), int(mode),
                                   ctypes.byref(o) if o is not None else None, _ptr(colors_out),
                                   _ptr(rounds_out), _ptr(conflicts_out), ctypes.byref(h))
        if rc != GC_OK:
            raise GCError(rc, "gc_plan_create")
        self.handle = int(h.value)
        # the plan replays into these arrays: keep them alive with it
        self._keep = (vtx_off, edge_off, row_ptr, col_idx, colors_out, rounds_out, conflicts_out)

    def launch(self, stream=None) -> int:
        return int(load().gc_plan_launch(ctypes.c_void_p(self.handle), ctypes.c_void_p(_stream_handle(stream))))

    def stats(self, round_cap: int = 0):
        st = gc_stats()
        rs, rn = _stats_buffers(st, round_cap)
        rc = load().gc_plan_stats(ctypes.c_void_p(self.handle), ctypes.byref(st))
        return int(rc), stats_dict(st, rs, rn)

    def close(self):
        if self.handle:
            load().gc_plan_destroy(ctypes.c_void_p(self.handle))
            self.handle = 0

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def gc_color_noalloc(row_ptr, col_idx, n: int, nnz: int, mode: int, colors_out, opts=None,
                     stream=None, round_cap: int = 0):
    """Colour one resident graph without any allocation (device arrays,
    n <= GC_NOALLOC_MAX_N).  Waits for the result; returns (status, stats)."""
    csr = gc_csr(_ptr(row_ptr), _ptr(col_idx) if nnz else 0)
    o = _opts(opts)
    st = gc_stats()
    rs, rn = _stats_buffers(st, round_cap)
    rc = load().gc_color_noalloc(ctypes.byref(csr), int(n), int(nnz), int(mode),
                                 ctypes.byref(o) if o is not None else None, _ptr(colors_out),
                                 ctypes.byref(st), ctypes.c_void_p(_stream_handle(stream)))
    return int(rc), stats_dict(st, rs, rn)


def gc_host_color(row_ptr, col_idx, mode: int = 0, num_threads: int = 0, round_cap: int = 0):
    """The paper's OpenMP form on the host cores (numpy int32 arrays, no
    GPU).  Returns (status, colours, stats)."""
    rp = np.ascontiguousarray(row_ptr, dtype=np.int32)
    ci = np.ascontiguousarray(col_idx, dtype=np.int32)
    n = rp.size - 1
    col = np.zeros(max(n, 1), np.int32)
    csr = gc_csr(rp.ctypes.data, ci.ctypes.data if ci.size else 0)
    st = gc_stats()
    rs, rn = _stats_buffers(st, round_cap)
    rc = load().gc_host_color(ctypes.byref(csr), int(n), int(ci.size), int(mode), int(num_threads),
                              col.ctypes.data, ctypes.byref(st))
    return int(rc), col[:n], stats_dict(st, rs, rn)


def gc_debug_wait_timeout(device: int = 0, wait: int = 0, timeout_ms: int = 200):
    """Run one bounded wait of the colouring kernel (GC_WAIT_*) against
    something that never happens; returns (status, device error word)."""
    w = ctypes.c_int32(0)
    rc = load().gc_debug_wait_timeout(int(device), int(wait), int(timeout_ms), ctypes.byref(w))
    return int(rc), int(w.value)


def gc_debug_barrier_timeout(device: int = 0, timeout_ms: int = 200):
    """Run the bounded grid barrier against an arrival that never comes;
    returns (status, device error word)."""
    w = ctypes.c_int32(0)
    rc = load().gc_debug_barrier_timeout(int(device), int(timeout_ms), ctypes.byref(w))
    return int(rc), int(w.value)


def gc_measure_gather_rate(device: int = 0, array_bytes: int = 8 << 20, blocks_per_sm: int = 2,
                           dependent: bool = False):
    """Random 4-byte gathers per second (in 1e9) from an array of
    `array_bytes` on the device; returns (status, rate)."""
    r = ctypes.c_double(0.0)
    rc = load().gc_measure_gather_rate(int(device), int(array_bytes), int(blocks_per_sm), int(bool(dependent)),
                                       ctypes.byref(r))
    return int(rc), float(r.value)


def gc_host_threads() -> int:
    """OpenMP threads gc_host_color uses by default (1 without OpenMP)."""
    return int(load().gc_host_threads())


class Context:
    """Owns a gc_ctx; colours graphs held as torch CUDA tensors."""

    def __init__(self, device: int = 0):
        self.device = device
        self.handle = gc_ctx_create(device)

    def close(self):
        if self.handle:
            gc_ctx_destroy(self.handle)
            self.handle = 0

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def color(self, row_ptr, col_idx, mode: int = 0, colors_out=None, opts=None, stream=None,
              round_cap: int = 0, check: bool = True):
        """Colour one resident graph; returns (colors tensor, status, stats)."""
        import torch
        n = row_ptr.numel() - 1
        if colors_out is None:
            colors_out = torch.empty(max(n, 0), dtype=torch.int32, device=row_ptr.device)
        rc = gc_color_async(self.handle, row_ptr, col_idx, n, col_idx.numel(), mode, colors_out,
                            opts, stream)
        if rc != GC_OK:
            raise GCError(rc, "gc_color_async")
        rc, st = gc_ctx_stats(self.handle, round_cap)
        if check and rc not in (GC_OK,):
            raise GCError(rc, "gc_ctx_stats")
        return colors_out, rc, st

    def color_batch(self, vtx_off, edge_off, row_ptr, col_idx, total_n: int, total_nnz: int,
                    mode: int = 0, colors_out=None, per_graph: bool = True, opts=None,
                    stream=None, check: bool = True):
        """Colour every graph of a resident batch in one launch; returns
        (colors, rounds[G], conflicts[G], status, stats)."""
        import torch
        G = vtx_off.numel() - 1
        dev = row_ptr.device
        if colors_out is None:
            colors_out = torch.empty(max(total_n, 0), dtype=torch.int32, device=dev)
        rounds = torch.empty(G, dtype=torch.int32, device=dev) if per_graph else None
        confl = torch.empty(G, dtype=torch.int64, device=dev) if per_graph else None
        rc = gc_color_batch(self.handle, G, total_n, total_nnz, vtx_off, edge_off, row_ptr,
                            col_idx, mode, colors_out, rounds, confl, opts, stream)
        if rc != GC_OK:
            raise GCError(rc, "gc_color_batch")
        rc, st = gc_ctx_stats(self.handle)
        if check and rc != GC_OK:
            raise GCError(rc, "gc_ctx_stats")
        return colors_out, rounds, confl, rc, st


class Server:
    """Continuous-batching colouring server (gc_server_*): submit host graphs,
    poll or wait for their colourings."""

    def __init__(self, device: int = 0, budget_bytes: int = 1 << 30, max_slots: int = 4096,
                 mode: int = 0, opts=None):
        h = ctypes.c_void_p()
        o = _opts(opts)
        rc = load().gc_server_create(ctypes.byref(h), int(device), int(budget_bytes), int(max_slots),
                                     int(mode), ctypes.byref(o) if o is not None else None)
        if rc != GC_OK:
            raise GCError(rc, "gc_server_create")
        self.handle = int(h.value)

    def submit(self, row_ptr: np.ndarray, col_idx: np.ndarray) -> int:
        """Queue a graph given by host int32 arrays; returns its ticket."""
        rp = np.ascontiguousarray(row_ptr, dtype=np.int32)
        ci = np.ascontiguousarray(col_idx, dtype=np.int32)
        csr = gc_csr(rp.ctypes.data, ci.ctypes.data if ci.size else 0)
        t = ctypes.c_uint64()
        rc = load().gc_server_submit(ctypes.c_void_p(self.handle), ctypes.byref(csr), rp.size - 1,
                                     ci.size, ctypes.byref(t))
        if rc != GC_OK:
            raise GCError(rc, "gc_server_submit")
        return int(t.value)

    def poll(self, ticket: int, n: int):
        """(status, colours or None, stats); status GC_PENDING while running."""
        col = np.empty(max(n, 1), np.int32)
        st = gc_stats()
        rc = load().gc_server_poll(ctypes.c_void_p(self.handle), ctypes.c_uint64(ticket), col.ctypes.data,
                                   ctypes.byref(st))
        if rc == GC_PENDING:
            return rc, None, None
        return rc, col[:n], stats_dict(st)

    def wait(self, ticket: int, n: int, timeout_ms: int = -1):
        col = np.empty(max(n, 1), np.int32)
        st = gc_stats()
        rc = load().gc_server_wait(ctypes.c_void_p(self.handle), ctypes.c_uint64(ticket), col.ctypes.data,
                                   ctypes.byref(st), int(timeout_ms))
        if rc == GC_PENDING:
            return rc, None, None
        return rc, col[:n], stats_dict(st)

    def info(self) -> dict:
        i = gc_server_info()
        rc = load().gc_server_query(ctypes.c_void_p(self.handle), ctypes.byref(i))
        if rc != GC_OK:
            raise GCError(rc, "gc_server_query")
        return {k: getattr(i, k) for k, _ in gc_server_info._fields_}

    def cancel(self, ticket: int) -> int:
        """Drop a request (gc_server_cancel); returns the status."""
        return int(load().gc_server_cancel(ctypes.c_void_p(self.handle), ctypes.c_uint64(ticket)))

    def close(self):
        if self.handle:
            load().gc_server_destroy(ctypes.c_void_p(self.handle))
            self.handle = 0

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

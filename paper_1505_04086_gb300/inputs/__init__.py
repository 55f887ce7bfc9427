"""Seeded synthetic input graphs (symmetric int32 CSR).

Thin ctypes wrapper over ``gen.c``.  These generators are the only code the
CUDA path and the CPU oracle have in common: they produce arrays and hold
none of the colouring arithmetic.

Named workloads stand in for the paper's benchmark graphs (Section 4), which
are not available here:

* ``tri2d_64x64``      structured 2D triangular mesh, 64x64 vertices, one
                       diagonal (i,j)-(i+1,j+1) per cell, natural order
* ``kuhn3d_<N>``       Kuhn-tetrahedralised N^3 lattice, ids permuted
* ``rmat<S>_ef16``     R-MAT scale S, 16 edge draws per vertex,
                       (a,b,c,d) = (0.57,0.19,0.19,0.05), ids permuted
* ``batch``            many uneven jittered meshes / random geometric graphs
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading
from dataclasses import dataclass, field

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "gen.c")
_LIB_PATH = os.path.join(_HERE, "libgcgen.so")
_lock = threading.Lock()
_lib = None

# Seeds of the named workloads: 0x1505 plus a per-workload index.
SEED_TRI2D = 0x1505 + 0
SEED_KUHN = 0x1505 + 1
SEED_RMAT = 0x1505 + 2
SEED_BATCH = 0x1505 + 3
SEED_SERVE = 0x1505 + 4


def build(force: bool = False) -> str:
    """Compile gen.c into libgcgen.so next to it (gcc, -O2, pthreads)."""
    if (not force and os.path.exists(_LIB_PATH)
            and os.path.getmtime(_LIB_PATH) >= os.path.getmtime(_SRC)):
        return _LIB_PATH
    tmp = _LIB_PATH + f".tmp{os.getpid()}"
    cmd = ["gcc", "-O2", "-std=gnu11", "-fPIC", "-shared", "-pthread", _SRC,
           "-o", tmp, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def _load():
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        lib = ctypes.CDLL(build())
        P = ctypes.c_void_p
        i32, i64, u64, dbl = ctypes.c_int32, ctypes.c_int64, ctypes.c_uint64, ctypes.c_double
        lib.gcgen_tri2d.restype = P
        lib.gcgen_tri2d.argtypes = [i32, i32, ctypes.c_int, dbl, u64]
        lib.gcgen_kuhn3d.restype = P
        lib.gcgen_kuhn3d.argtypes = [i32, ctypes.c_int, u64]
        lib.gcgen_rmat.restype = P
        lib.gcgen_rmat.argtypes = [i32, i32, dbl, dbl, dbl, u64, ctypes.c_int]
        lib.gcgen_rgg.restype = P
        lib.gcgen_rgg.argtypes = [i32, dbl, u64]
        lib.gcgen_free.argtypes = [P]
        lib.gcgen_n.restype = i32
        lib.gcgen_n.argtypes = [P]
        lib.gcgen_nnz.restype = i64
        lib.gcgen_nnz.argtypes = [P]
        for f in ("gcgen_row_ptr", "gcgen_col_idx"):
            getattr(lib, f).restype = P
            getattr(lib, f).argtypes = [P]
        lib.gcgen_batch_make.restype = P
        lib.gcgen_batch_make.argtypes = [i32, i32, i32, dbl, dbl, u64, i32]
        lib.gcgen_batch_free.argtypes = [P]
        lib.gcgen_batch_G.restype = i32
        lib.gcgen_batch_G.argtypes = [P]
        for f in ("gcgen_batch_vtx_off", "gcgen_batch_edge_off", "gcgen_batch_row_ptr",
                  "gcgen_batch_col_idx", "gcgen_batch_kind"):
            getattr(lib, f).restype = P
            getattr(lib, f).argtypes = [P]
        lib.gcgen_rand_at.restype = u64
        lib.gcgen_rand_at.argtypes = [u64, u64]
        lib.gcgen_perm.argtypes = [i32, u64, P]
        _lib = lib
        return lib


@dataclass
class CSR:
    """Symmetric CSR graph: rows sorted ascending, no self-loops, no repeats."""
    row_ptr: np.ndarray  # int32[n+1]
    col_idx: np.ndarray  # int32[nnz]
    name: str = ""

    @property
    def n(self) -> int:
        return int(self.row_ptr.shape[0] - 1)

    @property
    def nnz(self) -> int:
        return int(self.col_idx.shape[0])

    @property
    def num_edges(self) -> int:
        """Undirected edge count |E| = nnz / 2."""
        return self.nnz // 2

    def degrees(self) -> np.ndarray:
        return np.diff(self.row_ptr).astype(np.int64)


@dataclass
class Batch:
    """Many graphs in one set of arrays (see gen.c for the layout)."""
    vtx_off: np.ndarray   # int64[G+1]
    edge_off: np.ndarray  # int64[G+1]
    row_ptr: np.ndarray   # int32[sum(n_g+1)]
    col_idx: np.ndarray   # int32[sum(nnz_g)]
    kind: np.ndarray      # int32[G]: 0 mesh, 1 rgg
    name: str = ""
    _cache: dict = field(default_factory=dict, repr=False)

    @property
    def G(self) -> int:
        return int(self.vtx_off.shape[0] - 1)

    @property
    def total_n(self) -> int:
        return int(self.vtx_off[-1])

    @property
    def total_nnz(self) -> int:
        return int(self.edge_off[-1])

    def graph(self, g: int) -> CSR:
        """Graph g as a standalone CSR (views into the batch arrays)."""
        v0, v1 = int(self.vtx_off[g]), int(self.vtx_off[g + 1])
        e0, e1 = int(self.edge_off[g]), int(self.edge_off[g + 1])
        rp = self.row_ptr[v0 + g: v1 + g + 1]
        return CSR(rp, self.col_idx[e0:e1], name=f"{self.name}[{g}]")

    @staticmethod
    def from_graphs(graphs, name: str = "") -> "Batch":
        """Concatenate standalone CSR graphs into the batch layout."""
        G = len(graphs)
        vtx_off = np.zeros(G + 1, np.int64)
        edge_off = np.zeros(G + 1, np.int64)
        for g, c in enumerate(graphs):
            vtx_off[g + 1] = vtx_off[g] + c.n
            edge_off[g + 1] = edge_off[g] + c.nnz
        rp = np.concatenate([c.row_ptr for c in graphs]) if G else np.zeros(0, np.int32)
        ci = np.concatenate([c.col_idx for c in graphs]) if G else np.zeros(0, np.int32)
        return Batch(vtx_off, edge_off, rp.astype(np.int32), ci.astype(np.int32),
                     np.zeros(G, np.int32), name=name)


def _take(ptr, name) -> CSR:
    lib = _load()
    if not ptr:
        raise MemoryError(f"graph generator failed for {name}")
    try:
        n = lib.gcgen_n(ptr)
        nnz = lib.gcgen_nnz(ptr)
        rp = np.ctypeslib.as_array((ctypes.c_int32 * (n + 1)).from_address(lib.gcgen_row_ptr(ptr))).copy()
        if nnz:
            ci = np.ctypeslib.as_array((ctypes.c_int32 * nnz).from_address(lib.gcgen_col_idx(ptr))).copy()
        else:
            ci = np.zeros(0, np.int32)
    finally:
        lib.gcgen_free(ptr)
    return CSR(rp, ci, name=name)


def tri2d(rows: int, cols: int, jitter: float = 0.0, seed: int = SEED_TRI2D) -> CSR:
    """2D triangular mesh; jitter > 0 perturbs vertices and cuts each cell
    along its shorter diagonal, jitter == 0 uses (i,j)-(i+1,j+1) everywhere."""
    diag = 1 if jitter > 0 else 0
    return _take(_load().gcgen_tri2d(rows, cols, diag, float(jitter), seed),
                 f"tri2d_{rows}x{cols}" + ("_jit" if diag else ""))


def kuhn3d(N: int, permute: bool = True, seed: int = SEED_KUHN) -> CSR:
    """Kuhn-tetrahedralised N^3 lattice (interior degree 14)."""
    return _take(_load().gcgen_kuhn3d(N, int(permute), seed),
                 f"kuhn3d_{N}" + ("_perm" if permute else ""))


def rmat(scale: int, ef: int = 16, a: float = 0.57, b: float = 0.19, c: float = 0.19,
         seed: int = SEED_RMAT, permute: bool = True) -> CSR:
    """R-MAT graph with ef * 2^scale edge draws, symmetrised and de-duplicated."""
    return _take(_load().gcgen_rmat(scale, ef, a, b, c, seed, int(permute)),
                 f"rmat{scale}_ef{ef}")


def rgg(n: int, mean_deg: float = 12.0, seed: int = SEED_BATCH) -> CSR:
    """Random geometric graph in the unit square with the given mean degree."""
    return _take(_load().gcgen_rgg(n, float(mean_deg), seed), f"rgg_{n}")


def batch(G: int, nmin: int = 1 << 10, nmax: int = 1 << 18, rgg_deg: float = 12.0,
          jitter: float = 0.3, seed: int = SEED_BATCH, threads: int = 0) -> Batch:
    """G graphs, n log-uniform in [nmin, nmax], half jittered meshes and half
    random geometric graphs (per-graph coin flip)."""
    lib = _load()
    if threads <= 0:
        threads = max(1, min(64, os.cpu_count() or 1))
    ptr = lib.gcgen_batch_make(G, nmin, nmax, float(rgg_deg), float(jitter), seed, threads)
    if not ptr:
        raise MemoryError("batch generator failed")
    try:
        Gr = lib.gcgen_batch_G(ptr)
        vo = np.ctypeslib.as_array((ctypes.c_int64 * (Gr + 1)).from_address(lib.gcgen_batch_vtx_off(ptr))).copy()
        eo = np.ctypeslib.as_array((ctypes.c_int64 * (Gr + 1)).from_address(lib.gcgen_batch_edge_off(ptr))).copy()
        nrp = int(vo[-1]) + Gr
        rp = np.ctypeslib.as_array((ctypes.c_int32 * nrp).from_address(lib.gcgen_batch_row_ptr(ptr))).copy()
        nnz = int(eo[-1])
        ci = (np.ctypeslib.as_array((ctypes.c_int32 * nnz).from_address(lib.gcgen_batch_col_idx(ptr))).copy()
              if nnz else np.zeros(0, np.int32))
        kd = np.ctypeslib.as_array((ctypes.c_int32 * Gr).from_address(lib.gcgen_batch_kind(ptr))).copy()
    finally:
        lib.gcgen_batch_free(ptr)
    return Batch(vo, eo, rp, ci, kd, name=f"batch{G}_{nmin}_{nmax}")


def rand_at(seed: int, i: int) -> int:
    """i-th value of the splitmix64 stream started at seed (for tests)."""
    return int(_load().gcgen_rand_at(seed, i))


def permutation(n: int, seed: int) -> np.ndarray:
    out = np.empty(n, np.int32)
    _load().gcgen_perm(n, seed, out.ctypes.data)
    return out


def from_edges(n: int, edges) -> CSR:
    """Symmetric sorted CSR from an (m,2) array of undirected edges (small
    graphs for tests; self-loops and repeats are dropped)."""
    e = np.asarray(edges, dtype=np.int64).reshape(-1, 2)
    e = e[e[:, 0] != e[:, 1]]
    both = np.concatenate([e, e[:, ::-1]], axis=0) if len(e) else np.zeros((0, 2), np.int64)
    if len(both):
        both = np.unique(both, axis=0)  # sorted by (src, dst), repeats removed
    rp = np.zeros(n + 1, np.int64)
    if len(both):
        np.add.at(rp, both[:, 0] + 1, 1)
    rp = np.cumsum(rp).astype(np.int32)
    ci = both[:, 1].astype(np.int32) if len(both) else np.zeros(0, np.int32)
    return CSR(rp, ci, name=f"edges_{n}")


# Named workloads -----------------------------------------------------------

def workload(name: str):
    """Build one of the named synthetic workloads."""
    if name == "tri2d_64x64":
        return tri2d(64, 64)
    if name.startswith("kuhn3d_"):
        return kuhn3d(int(name.split("_")[1]))
    if name.startswith("rmat") and name.endswith("_ef16"):
        return rmat(int(name[4:].split("_")[0]), 16)
    raise KeyError(name)

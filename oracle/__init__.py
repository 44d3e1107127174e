"""CPU oracle for cover-edge triangle counting (test infrastructure).

Only the test-suite, ``__graft_entry__.smoke()`` and ``bench.py``'s CPU-baseline
leg may import this package.  The product path (``paper_2403_02997_gb300``)
never does: it has no CPU fallback, and the oracle shares no code with it.

The arithmetic lives in ``cetc_oracle.c`` (plain C, each function citing the
paper's algorithm it follows); this module only marshals numpy arrays and adds
two library-routine checks (trace(A^3)/6 with a numpy matmul, and graph
invariants written with numpy).
"""
from __future__ import annotations

import ctypes
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "cetc_oracle.c")
_LIB = os.path.join(_HERE, "liboracle.so")


def build(force: bool = False) -> str:
    """Compile liboracle.so (gcc -O2, OpenMP when the compiler has it)."""
    if not force and os.path.exists(_LIB) and os.path.getmtime(_LIB) >= os.path.getmtime(_SRC):
        return _LIB
    base = ["gcc", "-O2", "-shared", "-fPIC", "-std=c11", _SRC, "-o", _LIB + ".tmp"]
    try:
        subprocess.run(base[:1] + ["-fopenmp"] + base[1:], check=True, capture_output=True)
    except subprocess.CalledProcessError:
        subprocess.run(base, check=True, capture_output=True)
    os.replace(_LIB + ".tmp", _LIB)
    return _LIB


_lib = None
_i64p = ctypes.POINTER(ctypes.c_int64)
_u64p = ctypes.POINTER(ctypes.c_uint64)
_u32p = ctypes.POINTER(ctypes.c_uint32)
_i32p = ctypes.POINTER(ctypes.c_int32)
_u8p = ctypes.POINTER(ctypes.c_uint8)


def _load():
    global _lib
    if _lib is None:
        lib = ctypes.CDLL(build())
        lib.orc_build_csr.restype = ctypes.c_int64
        lib.orc_build_csr.argtypes = [ctypes.c_uint32, ctypes.c_uint64, _u32p, _u32p, _i64p, _u32p]
        lib.orc_bfs_levels.restype = None
        lib.orc_bfs_levels.argtypes = [ctypes.c_uint32, _i64p, _u32p, ctypes.c_uint32, _i32p]
        lib.orc_cetc.restype = None
        lib.orc_cetc.argtypes = [ctypes.c_uint32, _i64p, _u32p, _i32p, ctypes.c_uint64, _u64p,
                                 _u32p, _u32p]
        lib.orc_cetc_sm.restype = ctypes.c_uint64
        lib.orc_cetc_sm.argtypes = [ctypes.c_uint32, _i64p, _u32p, _i32p, ctypes.c_uint64, _u64p]
        lib.orc_num_threads.restype = ctypes.c_int
        lib.orc_num_threads.argtypes = []
        lib.orc_cetc_edges.restype = None
        lib.orc_cetc_edges.argtypes = [_i64p, _u32p, _i32p, ctypes.c_uint64, _u32p, _u32p, _u64p]
        lib.orc_cetc_sm_edges.restype = None
        lib.orc_cetc_sm_edges.argtypes = [_i64p, _u32p, _i32p, ctypes.c_uint64, _u32p, _u32p,
                                          _u64p]
        lib.orc_edge_count.restype = ctypes.c_uint64
        lib.orc_edge_count.argtypes = [_i64p, _u32p, _i32p, ctypes.c_uint32, ctypes.c_uint32]
        lib.orc_triples.restype = ctypes.c_uint64
        lib.orc_triples.argtypes = [ctypes.c_uint32, _u8p]
        lib.orc_forward.restype = ctypes.c_uint64
        lib.orc_forward.argtypes = [ctypes.c_uint32, _i64p, _u32p]
        lib.orc_list_triangles.restype = ctypes.c_uint64
        lib.orc_list_triangles.argtypes = [ctypes.c_uint32, _i64p, _u32p, _u32p, ctypes.c_uint64,
                                           _u64p]
        lib.orc_cetc_split.restype = ctypes.c_uint64
        lib.orc_cetc_split.argtypes = [ctypes.c_uint32, _i64p, _u32p, _i32p, _u64p]
        _lib = lib
    return _lib


def _p(a: np.ndarray, t):
    return a.ctypes.data_as(t)


class VertexRangeError(ValueError):
    pass


def build_csr(n: int, src, dst):
    """Undirected simple CSR: (row_ptr int64[n+1], col uint32[2m]), rows sorted."""
    src = np.ascontiguousarray(src, dtype=np.uint32)
    dst = np.ascontiguousarray(dst, dtype=np.uint32)
    E = int(src.size)
    row_ptr = np.zeros(n + 1, dtype=np.int64)
    col = np.empty(max(2 * E, 1), dtype=np.uint32)
    nnz = _load().orc_build_csr(n, E, _p(src, _u32p), _p(dst, _u32p), _p(row_ptr, _i64p),
                                _p(col, _u32p))
    if nnz < 0:
        raise VertexRangeError("vertex id >= n")
    return row_ptr, col[:nnz].copy()


def bfs_levels(row_ptr, col, root: int) -> np.ndarray:
    """Levels from `root`, then restarts from each unvisited vertex in id order."""
    n = row_ptr.size - 1
    level = np.empty(n, dtype=np.int32)
    if n:
        _load().orc_bfs_levels(n, _p(row_ptr, _i64p), _p(col, _u32p), root, _p(level, _i32p))
    return level


def cetc(row_ptr, col, level, stride: int = 1, want_cover: bool = False) -> dict:
    """Algorithm CETC-Seq over the horizontal edges; see orc_cetc for the fields."""
    n = row_ptr.size - 1
    st = np.zeros(8, dtype=np.uint64)
    cu = cv = None
    if want_cover:
        cap = max(int(col.size) // 2, 1)
        cu = np.empty(cap, dtype=np.uint32)
        cv = np.empty(cap, dtype=np.uint32)
    _load().orc_cetc(n, _p(row_ptr, _i64p), _p(col, _u32p), _p(level, _i32p), stride,
                     _p(st, _u64p), None if cu is None else _p(cu, _u32p),
                     None if cv is None else _p(cv, _u32p))
    out = dict(T=int(st[0]), c1=int(st[1]), c2=int(st[2]), num_cover=int(st[3]),
               sum_deg=int(st[4]), sum_min=int(st[5]), matches=int(st[6]), done=int(st[7]))
    if want_cover:
        out["cover_u"] = cu[: out["num_cover"]].copy()
        out["cover_v"] = cv[: out["num_cover"]].copy()
    return out


def cetc_sm(row_ptr, col, level, stride: int = 1) -> dict:
    """Algorithm CETC-SM (OpenMP over vertices): T = c1 + c2 / 3."""
    n = row_ptr.size - 1
    out = np.zeros(3, dtype=np.uint64)
    T = _load().orc_cetc_sm(n, _p(row_ptr, _i64p), _p(col, _u32p), _p(level, _i32p), stride,
                            _p(out, _u64p))
    return dict(T=int(T), c1=int(out[0]), c2=int(out[1]), done=int(out[2]))


def cetc_edges(row_ptr, col, level, us, vs) -> dict:
    """CETC-Seq count over the given horizontal edges only (us < vs)."""
    us = np.ascontiguousarray(us, dtype=np.uint32)
    vs = np.ascontiguousarray(vs, dtype=np.uint32)
    out = np.zeros(3, dtype=np.uint64)
    _load().orc_cetc_edges(_p(row_ptr, _i64p), _p(col, _u32p), _p(level, _i32p), us.size,
                           _p(us, _u32p), _p(vs, _u32p), _p(out, _u64p))
    return dict(T=int(out[0]), c1=int(out[1]), c2=int(out[2]))


def cetc_sm_edges(row_ptr, col, level, us, vs) -> dict:
    """cetc_edges with the edge loop spread over all host threads (Algorithm CETC-SM)."""
    us = np.ascontiguousarray(us, dtype=np.uint32)
    vs = np.ascontiguousarray(vs, dtype=np.uint32)
    out = np.zeros(3, dtype=np.uint64)
    _load().orc_cetc_sm_edges(_p(row_ptr, _i64p), _p(col, _u32p), _p(level, _i32p), us.size,
                              _p(us, _u32p), _p(vs, _u32p), _p(out, _u64p))
    return dict(T=int(out[0]), c1=int(out[1]), c2=int(out[2]))


def num_threads() -> int:
    return int(_load().orc_num_threads())


def edge_count(row_ptr, col, level, u: int, v: int) -> int:
    """Per-edge count of Algorithm CETC-Seq for the horizontal edge (u, v), u < v."""
    return int(_load().orc_edge_count(_p(row_ptr, _i64p), _p(col, _u32p), _p(level, _i32p),
                                      u, v))


def adjacency_matrix(n: int, src, dst) -> np.ndarray:
    a = np.zeros((n, n), dtype=np.uint8)
    s = np.asarray(src, dtype=np.int64)
    d = np.asarray(dst, dtype=np.int64)
    keep = s != d
    a[s[keep], d[keep]] = 1
    a[d[keep], s[keep]] = 1
    return a


def triples(n: int, src, dst) -> int:
    """Algorithm Triples: brute force over all ordered vertex triples, / 6."""
    a = np.ascontiguousarray(adjacency_matrix(n, src, dst))
    return int(_load().orc_triples(n, _p(a, _u8p)))


def trace_a3(n: int, src, dst) -> int:
    """tr(A^3) / 6 with an exact int64 matrix product (paper, Section Related Work)."""
    a = adjacency_matrix(n, src, dst).astype(np.int64)
    return int(np.trace(a @ a @ a)) // 6


def forward(row_ptr, col) -> int:
    """Algorithm Forward with decreasing-degree relabelling (independent of BFS)."""
    n = row_ptr.size - 1
    return int(_load().orc_forward(n, _p(row_ptr, _i64p), _p(col, _u32p)))


def cetc_split(row_ptr, col, level) -> dict:
    """Algorithm CETC-Seq-S: T0 (forward-hashed on the horizontal subgraph G0),
    T1 (hashed intersections of G1 rows over the edges of G0), T = T0 + T1."""
    n = row_ptr.size - 1
    out = np.zeros(2, dtype=np.uint64)
    T = _load().orc_cetc_split(n, _p(row_ptr, _i64p), _p(col, _u32p), _p(level, _i32p),
                               _p(out, _u64p))
    return dict(T=int(T), T0=int(out[0]), T1=int(out[1]))


def list_triangles(row_ptr, col):
    """Every triangle as a row (a, b, c), a < b < c, in increasing order, and the
    per-vertex triangle counts."""
    n = row_ptr.size - 1
    lib = _load()
    vcount = np.zeros(max(n, 1), dtype=np.uint64)
    T = lib.orc_list_triangles(n, _p(row_ptr, _i64p), _p(col, _u32p), None, 0, _p(vcount, _u64p))
    tri = np.zeros((max(int(T), 1), 3), dtype=np.uint32)
    lib.orc_list_triangles(n, _p(row_ptr, _i64p), _p(col, _u32p), _p(tri, _u32p), T, None)
    return tri[: int(T)], vcount[:n]


def degree_order(row_ptr) -> np.ndarray:
    """Degree ordering (the pre-processing of Algorithms CETC-Seq-D / -SD): the
    old ids by decreasing degree, ties by increasing id; entry i is the old id
    of new vertex i."""
    n = row_ptr.size - 1
    deg = np.diff(np.asarray(row_ptr, dtype=np.int64))
    return np.lexsort((np.arange(n), -deg)).astype(np.uint32)


def relabel_edges(old_of_new, src, dst):
    """The edge list with every id replaced by its new id."""
    new_of_old = np.empty_like(old_of_new)
    new_of_old[old_of_new] = np.arange(old_of_new.size, dtype=old_of_new.dtype)
    return new_of_old[np.asarray(src, np.int64)], new_of_old[np.asarray(dst, np.int64)]


def max_degree_root(row_ptr) -> int:
    """Smallest id among the vertices of maximum degree (0 for an empty graph)."""
    if row_ptr.size <= 1:
        return 0
    return int(np.argmax(np.diff(row_ptr)))


def count(n: int, src, dst, root: int = 0, want_cover: bool = False) -> dict:
    """Whole method on the CPU: graph build, levels, CETC-Seq count."""
    row_ptr, col = build_csr(n, src, dst)
    level = bfs_levels(row_ptr, col, root) if n else np.empty(0, np.int32)
    out = cetc(row_ptr, col, level, want_cover=want_cover) if n else dict(
        T=0, c1=0, c2=0, num_cover=0, sum_deg=0, sum_min=0, matches=0, done=0)
    out.update(row_ptr=row_ptr, col=col, level=level, m=int(col.size) // 2)
    return out

"""Cover-edge triangle counting on GB300: Python binding of libtc.

Thin ctypes marshalling over the C ABI declared in ``include/tc.h``: every step
of the count (CSR build, BFS levels, cover-edge extraction, intersections,
reduction) runs in the library's CUDA kernels.  There is no CPU fallback: if
``libtc.so`` is missing or no GPU is present, calls raise.

Low-level functions carry the ABI names (``tc_graph_create``, ``tc_count``,
``tc_count_many``, ...); ``Graph`` wraps a handle for convenience.  Device
memory and streams may come from PyTorch: pass CUDA tensors as edge arrays and
a ``torch.cuda.Stream`` (or a raw ``cudaStream_t`` as int) as ``stream``.
"""
from __future__ import annotations

import ctypes
import os
from typing import Optional, Sequence

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libtc.so")

TC_OK = 0
STATUS_NAMES = {0: "TC_OK", 1: "TC_ERR_INVALID_ARG", 2: "TC_ERR_VERTEX_RANGE", 3: "TC_ERR_OOM",
                4: "TC_ERR_CUDA", 5: "TC_ERR_TIMEOUT", 6: "TC_ERR_OVERFLOW"}


class TCError(RuntimeError):
    def __init__(self, status: int, where: str, detail: str = ""):
        self.status = status
        name = STATUS_NAMES.get(status, str(status))
        super().__init__(f"{where}: {name}{(' (' + detail + ')') if detail else ''}")


class tc_stats(ctypes.Structure):
    _fields_ = [("triangles", ctypes.c_uint64), ("c1", ctypes.c_uint64), ("c2", ctypes.c_uint64),
                ("num_cover", ctypes.c_uint64), ("m", ctypes.c_uint64),
                ("num_levels", ctypes.c_uint32), ("bfs_steps", ctypes.c_uint32),
                ("bottom_up_steps", ctypes.c_uint32), ("restarted", ctypes.c_uint32),
                ("ms_bfs", ctypes.c_float), ("ms_cover", ctypes.c_float),
                ("ms_intersect", ctypes.c_float), ("ms_total", ctypes.c_float),
                ("ms_hash", ctypes.c_float), ("launches", ctypes.c_uint32),
                ("hash_items", ctypes.c_uint64), ("hash_edges", ctypes.c_uint64)]


class tc_params(ctypes.Structure):
    _fields_ = [("small_max_degree", ctypes.c_uint32), ("hash_chunk", ctypes.c_uint32),
                ("edges_per_item", ctypes.c_uint32), ("bfs_alpha", ctypes.c_uint32),
                ("bfs_beta", ctypes.c_uint32), ("sorted_lookup", ctypes.c_uint32),
                ("persistent_bfs", ctypes.c_uint32), ("barrier_timeout_ms", ctypes.c_uint32),
                ("test_barrier_skip", ctypes.c_uint32), ("medium_max_degree", ctypes.c_uint32),
                ("hash_block", ctypes.c_uint32), ("cluster_bfs", ctypes.c_uint32)]


_lib = None


def load_library(path: str = LIB_PATH):
    """Load libtc.so (built by ``paper_2403_02997_gb300.build``); raise if absent."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise ImportError(f"libtc.so not found at {path}: run __graft_entry__.build() or "
                          f"python -m paper_2403_02997_gb300.build")
    lib = ctypes.CDLL(path)
    vp, u32, u64 = ctypes.c_void_p, ctypes.c_uint32, ctypes.c_uint64
    P = ctypes.POINTER
    sig = {
        "tc_graph_create": ([vp, vp, u64, u32, ctypes.c_int, vp, P(vp)], ctypes.c_int),
        "tc_graph_destroy": ([vp], ctypes.c_int),
        "tc_graph_info": ([vp, P(u32), P(u64), P(u32)], ctypes.c_int),
        "tc_count": ([vp, u32, vp, P(u64)], ctypes.c_int),
        "tc_count_many": ([P(vp), P(u32), ctypes.c_size_t, vp, P(u64)], ctypes.c_int),
        "tc_count_split": ([vp, u32, vp, P(u64)], ctypes.c_int),
        "tc_graph_relabel_degree": ([vp, vp, P(vp), vp], ctypes.c_int),
        "tc_list_triangles": ([vp, u32, vp, vp, u64, vp, P(u64), P(u64)], ctypes.c_int),
        "tc_count_forward": ([vp, vp, P(u64)], ctypes.c_int),
        "tc_count_fe": ([vp, u32, ctypes.c_float, vp, P(u64), P(ctypes.c_int)], ctypes.c_int),
        "tc_get_levels": ([vp, vp], ctypes.c_int),
        "tc_get_cover_edges": ([vp, P(u64), vp, vp], ctypes.c_int),
        "tc_get_csr": ([vp, vp, vp], ctypes.c_int),
        "tc_get_stats": ([vp, P(tc_stats)], ctypes.c_int),
        "tc_max_degree_vertex": ([vp, P(u32)], ctypes.c_int),
        "tc_params_default": ([P(tc_params)], ctypes.c_int),
        "tc_set_params": ([vp, P(tc_params)], ctypes.c_int),
        "tc_status_string": ([ctypes.c_int], ctypes.c_char_p),
        "tc_bfs_levels_noalloc": ([vp, vp, u32, u32, vp, vp], ctypes.c_int),
        "tc_batch_create": ([P(vp), ctypes.c_size_t, vp, P(vp)], ctypes.c_int),
        "tc_batch_count": ([vp, P(u32), vp, P(u64)], ctypes.c_int),
        "tc_batch_count_persistent": ([vp, P(u32), vp, P(u64)], ctypes.c_int),
        "tc_batch_set_params": ([vp, P(tc_params)], ctypes.c_int),
        "tc_batch_get_stats": ([vp, P(tc_stats)], ctypes.c_int),
        "tc_batch_get_levels": ([vp, ctypes.c_size_t, vp], ctypes.c_int),
        "tc_batch_destroy": ([vp], ctypes.c_int),
        "tc_pool_trim": ([u64], ctypes.c_int),
        "tc_pool_reserved": ([P(u64)], ctypes.c_int),
        "tc_batch_create_from_edges": ([vp, vp, P(u64), P(u32), ctypes.c_size_t, ctypes.c_int,
                                        vp, P(vp)], ctypes.c_int),
        "tc_batch_max_degree_vertices": ([vp, vp, P(u32)], ctypes.c_int),
    }
    for name, (args, res) in sig.items():
        f = getattr(lib, name)
        f.argtypes = args
        f.restype = res
    _lib = lib
    return lib


def _check(status: int, where: str):
    if status != TC_OK:
        raise TCError(status, where)


def _stream_handle(stream) -> Optional[int]:
    if stream is None:
        try:
            import torch
            if torch.cuda.is_available():
                return torch.cuda.current_stream().cuda_stream
        except ImportError:
            pass
        return None
    if isinstance(stream, int):
        return stream
    return int(stream.cuda_stream)


def _as_edge_array(a):
    """(pointer, length, on_device, keepalive) for a uint32 edge array."""
    if hasattr(a, "is_cuda") and a.is_cuda:
        import torch
        if a.dtype not in (torch.int32, torch.uint32):
            a = a.to(torch.int32)
        a = a.contiguous()
        return a.data_ptr(), a.numel(), True, a
    arr = np.ascontiguousarray(a, dtype=np.uint32)
    return arr.ctypes.data, arr.size, False, arr


# ----------------------------------------------------------------------------
# ABI-named functions
# ----------------------------------------------------------------------------

def tc_graph_create(src, dst, num_vertices: int, stream=None) -> int:
    """Build a device graph from an undirected edge list; returns the handle."""
    lib = load_library()
    ps, ns, ds, ks = _as_edge_array(src)
    pd, nd, dd, kd = _as_edge_array(dst)
    if ns != nd or ds != dd:
        raise ValueError("src and dst must have the same length and live on the same device")
    out = ctypes.c_void_p()
    st = lib.tc_graph_create(ps if ns else None, pd if nd else None, ns, num_vertices, int(ds),
                             _stream_handle(stream), ctypes.byref(out))
    del ks, kd
    _check(st, "tc_graph_create")
    return out.value


def tc_graph_destroy(handle: int) -> None:
    _check(load_library().tc_graph_destroy(handle), "tc_graph_destroy")


def tc_count(handle: int, root: int, stream=None) -> int:
    c = ctypes.c_uint64()
    _check(load_library().tc_count(handle, root, _stream_handle(stream), ctypes.byref(c)),
           "tc_count")
    return int(c.value)


def tc_count_split(handle, root: int, stream=None) -> int:
    c = ctypes.c_uint64()
    _check(load_library().tc_count_split(handle, root, _stream_handle(stream), ctypes.byref(c)),
           "tc_count_split")
    return int(c.value)


def tc_count_forward(handle, stream=None) -> int:
    c = ctypes.c_uint64()
    _check(load_library().tc_count_forward(handle, _stream_handle(stream), ctypes.byref(c)),
           "tc_count_forward")
    return int(c.value)


def tc_count_fe(handle, root: int, threshold: float, stream=None):
    c = ctypes.c_uint64()
    used = ctypes.c_int()
    _check(load_library().tc_count_fe(handle, root, threshold, _stream_handle(stream),
                                      ctypes.byref(c), ctypes.byref(used)), "tc_count_fe")
    return int(c.value), bool(used.value)


def tc_count_many(handles: Sequence[int], roots: Sequence[int], stream=None) -> list:
    k = len(handles)
    if k == 0:
        return []
    hs = (ctypes.c_void_p * k)(*handles)
    rs = (ctypes.c_uint32 * k)(*roots)
    out = (ctypes.c_uint64 * k)()
    _check(load_library().tc_count_many(hs, rs, k, _stream_handle(stream), out), "tc_count_many")
    return [int(x) for x in out]


def tc_graph_info(handle: int):
    n, m, d = ctypes.c_uint32(), ctypes.c_uint64(), ctypes.c_uint32()
    _check(load_library().tc_graph_info(handle, ctypes.byref(n), ctypes.byref(m), ctypes.byref(d)),
           "tc_graph_info")
    return int(n.value), int(m.value), int(d.value)


def tc_get_levels(handle: int, n: int) -> np.ndarray:
    out = np.empty(n, dtype=np.int32)
    _check(load_library().tc_get_levels(handle, out.ctypes.data if n else None), "tc_get_levels")
    return out


def tc_get_cover_edges(handle: int):
    lib = load_library()
    k = ctypes.c_uint64()
    _check(lib.tc_get_cover_edges(handle, ctypes.byref(k), None, None), "tc_get_cover_edges")
    u = np.empty(k.value, dtype=np.uint32)
    v = np.empty(k.value, dtype=np.uint32)
    if k.value:
        _check(lib.tc_get_cover_edges(handle, ctypes.byref(k), u.ctypes.data, v.ctypes.data),
               "tc_get_cover_edges")
    return u, v


def tc_get_csr(handle: int, n: int, m: int):
    rp = np.empty(n + 1, dtype=np.uint64)
    col = np.empty(2 * m, dtype=np.uint32)
    _check(load_library().tc_get_csr(handle, rp.ctypes.data, col.ctypes.data if m else None),
           "tc_get_csr")
    return rp, col


def tc_get_stats(handle: int) -> dict:
    s = tc_stats()
    _check(load_library().tc_get_stats(handle, ctypes.byref(s)), "tc_get_stats")
    return {name: getattr(s, name) for name, _ in tc_stats._fields_}


def tc_max_degree_vertex(handle: int) -> int:
    v = ctypes.c_uint32()
    _check(load_library().tc_max_degree_vertex(handle, ctypes.byref(v)), "tc_max_degree_vertex")
    return int(v.value)


def tc_params_default() -> dict:
    p = tc_params()
    _check(load_library().tc_params_default(ctypes.byref(p)), "tc_params_default")
    return {name: getattr(p, name) for name, _ in tc_params._fields_}


def tc_set_params(handle: int, **kw) -> None:
    p = tc_params()
    lib = load_library()
    _check(lib.tc_params_default(ctypes.byref(p)), "tc_params_default")
    for k, v in kw.items():
        setattr(p, k, int(v))
    _check(lib.tc_set_params(handle, ctypes.byref(p)), "tc_set_params")


def tc_bfs_levels_noalloc(row_ptr, col, n: int, root: int, levels, stream=None) -> None:
    """BFS levels of a device CSR into a device int32 array, allocating nothing.

    row_ptr (uint64 / int64, n+1), col (uint32 / int32) and levels (int32, n)
    are CUDA tensors owned by the caller; see include/tc.h for the limits
    (n <= 2^20) and the shared-scratch rules.
    """
    _check(load_library().tc_bfs_levels_noalloc(row_ptr.data_ptr(), col.data_ptr(), n, root,
                                                levels.data_ptr(), _stream_handle(stream)),
           "tc_bfs_levels_noalloc")


# ----------------------------------------------------------------------------
# Convenience wrapper
# ----------------------------------------------------------------------------

class Graph:
    """A device-resident graph (owns one tc_graph handle)."""

    def __init__(self, src, dst, num_vertices: int, stream=None):
        self.handle = tc_graph_create(src, dst, num_vertices, stream)
        self.n, self.m, self.d_max = tc_graph_info(self.handle)

    def count(self, root: Optional[int] = None, stream=None) -> int:
        if root is None:
            root = 0
        return tc_count(self.handle, root, stream)

    def count_split(self, root: Optional[int] = None, stream=None) -> int:
        """Algorithm CETC-Seq-S (see tc_count_split)."""
        return tc_count_split(self.handle, 0 if root is None else root, stream)

    def count_forward(self, stream=None) -> int:
        """Algorithm Forward with degree ranking (see tc_count_forward)."""
        return tc_count_forward(self.handle, stream)

    def count_fe(self, root: Optional[int] = None, threshold: float = 0.7, stream=None):
        """Algorithm CETC-Seq-FE: (count, whether the forward count ran)."""
        return tc_count_fe(self.handle, 0 if root is None else root, threshold, stream)

    def list_triangles(self, root: Optional[int] = None, capacity: Optional[int] = None,
                       vertex_counts: bool = True, stream=None):
        """Triangle listing (see tc_list_triangles) into torch device tensors.

        Returns (count, triangles as an int64 (written, 3) numpy array of
        (u, v, w), per-vertex counts as a uint64 numpy array or None).  With
        capacity None the count runs once first to size the list."""
        import torch
        root = 0 if root is None else root
        if capacity is None:
            capacity = self.count(root, stream)
        tri = torch.empty((max(int(capacity), 1), 3), dtype=torch.int32, device="cuda")
        vc = torch.empty(max(self.n, 1), dtype=torch.int64, device="cuda") if vertex_counts else None
        c, w = ctypes.c_uint64(), ctypes.c_uint64()
        _check(load_library().tc_list_triangles(
            self.handle, root, _stream_handle(stream), ctypes.c_void_p(tri.data_ptr()),
            int(capacity), ctypes.c_void_p(vc.data_ptr()) if vc is not None else None,
            ctypes.byref(c), ctypes.byref(w)), "tc_list_triangles")
        torch.cuda.synchronize()
        trip = tri[: w.value].cpu().numpy().view(np.uint32).astype(np.int64)
        counts = vc[: self.n].cpu().numpy().view(np.uint64) if vc is not None else None
        return int(c.value), trip, counts

    def relabel_degree(self, stream=None):
        """Degree ordering (see tc_graph_relabel_degree): (new Graph, old_of_new)."""
        out = ctypes.c_void_p()
        perm = np.empty(max(self.n, 1), dtype=np.uint32)
        _check(load_library().tc_graph_relabel_degree(
            self.handle, _stream_handle(stream), ctypes.byref(out),
            perm.ctypes.data_as(ctypes.c_void_p)), "tc_graph_relabel_degree")
        g = Graph.__new__(Graph)
        g.handle = out.value
        g.n, g.m, g.d_max = tc_graph_info(g.handle)
        return g, perm[: self.n].copy()

    def max_degree_vertex(self) -> int:
        return tc_max_degree_vertex(self.handle)

    def levels(self) -> np.ndarray:
        return tc_get_levels(self.handle, self.n)

    def cover_edges(self):
        return tc_get_cover_edges(self.handle)

    def csr(self):
        return tc_get_csr(self.handle, self.n, self.m)

    def stats(self) -> dict:
        return tc_get_stats(self.handle)

    def set_params(self, **kw) -> None:
        tc_set_params(self.handle, **kw)

    def close(self) -> None:
        if getattr(self, "handle", None):
            tc_graph_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()


def count_many(graphs: Sequence[Graph], roots: Sequence[int], stream=None) -> list:
    return tc_count_many([g.handle for g in graphs], roots, stream)


class PinnedStaging:
    """Reusable page-locked host buffers for batch builds from edge lists.

    tc_batch_create_from_edges copies the edges to the device and has finished
    with them when it returns, so the same buffers serve the next build.
    """

    def __init__(self):
        self.buf = None

    def arrays(self, count: int):
        """Two uint32 arrays of `count` entries (src, dst) in pinned memory."""
        need = 2 * int(count)
        if self.buf is None or self.buf.numel() < need:
            import torch
            size = max(need, 1 << 20, int(1.5 * (self.buf.numel() if self.buf is not None else 0)))
            self.buf = torch.empty(size, dtype=torch.int32, pin_memory=True)
        a = self.buf.numpy().view(np.uint32)
        return a[:count], a[count:2 * count]


def pool_trim(keep_bytes: int = 0) -> None:
    """Return the library pool's unused device memory to the driver (keep at most keep_bytes)."""
    _check(load_library().tc_pool_trim(int(keep_bytes)), "tc_pool_trim")


def pool_reserved() -> int:
    """Device bytes the library's pool holds now."""
    v = ctypes.c_uint64()
    _check(load_library().tc_pool_reserved(ctypes.byref(v)), "tc_pool_reserved")
    return int(v.value)


class Batch:
    """A reusable batch: the graphs' CSRs concatenated once, counted together."""

    def __init__(self, graphs: Sequence[Graph], stream=None):
        lib = load_library()
        self.k = len(graphs)
        self.sizes = [g.n for g in graphs]
        hs = (ctypes.c_void_p * self.k)(*[g.handle for g in graphs])
        out = ctypes.c_void_p()
        _check(lib.tc_batch_create(hs, self.k, _stream_handle(stream), ctypes.byref(out)),
               "tc_batch_create")
        self.handle = out.value

    @classmethod
    def from_edges(cls, graphs, stream=None, staging: Optional["PinnedStaging"] = None) -> "Batch":
        """Build a batch straight from host edge lists: graphs = [(src, dst, n), ...].

        With `staging`, the edge lists are gathered into its page-locked buffers, so the
        library's host-to-device copies run asynchronously on `stream`.
        """
        lib = load_library()
        self = cls.__new__(cls)
        self.k = len(graphs)
        self.sizes = [int(n) for _, _, n in graphs]
        lens = [int(np.asarray(s_).size) for s_, _, _ in graphs]
        offs = np.zeros(self.k + 1, dtype=np.uint64)
        offs[1:] = np.cumsum(lens, dtype=np.uint64)
        total = int(offs[-1])
        if staging is not None and total:
            src, dst = staging.arrays(total)
            np.concatenate([np.asarray(s_, np.uint32) for s_, _, _ in graphs], out=src)
            np.concatenate([np.asarray(d_, np.uint32) for _, d_, _ in graphs], out=dst)
        else:
            src = np.concatenate([np.asarray(s_, np.uint32) for s_, _, _ in graphs]) if lens \
                else np.zeros(0, np.uint32)
            dst = np.concatenate([np.asarray(d_, np.uint32) for _, d_, _ in graphs]) if lens \
                else np.zeros(0, np.uint32)
        nv = np.asarray(self.sizes, dtype=np.uint32)
        out = ctypes.c_void_p()
        _check(lib.tc_batch_create_from_edges(
            src.ctypes.data if src.size else None, dst.ctypes.data if dst.size else None,
            offs.ctypes.data_as(ctypes.POINTER(ctypes.c_uint64)),
            nv.ctypes.data_as(ctypes.POINTER(ctypes.c_uint32)), self.k, 0,
            _stream_handle(stream), ctypes.byref(out)), "tc_batch_create_from_edges")
        self.handle = out.value
        return self

    def max_degree_vertices(self, stream=None) -> list:
        out = (ctypes.c_uint32 * self.k)()
        _check(load_library().tc_batch_max_degree_vertices(self.handle, _stream_handle(stream), out),
               "tc_batch_max_degree_vertices")
        return [int(x) for x in out]

    def count(self, roots: Sequence[int], stream=None) -> list:
        rs = (ctypes.c_uint32 * self.k)(*roots)
        out = (ctypes.c_uint64 * self.k)()
        _check(load_library().tc_batch_count(self.handle, rs, _stream_handle(stream), out),
               "tc_batch_count")
        return [int(x) for x in out]

    def count_persistent(self, roots: Sequence[int], stream=None) -> list:
        """The same counts from one persistent launch, one graph per block (small graphs)."""
        rs = (ctypes.c_uint32 * self.k)(*roots)
        out = (ctypes.c_uint64 * self.k)()
        _check(load_library().tc_batch_count_persistent(self.handle, rs, _stream_handle(stream),
                                                        out), "tc_batch_count_persistent")
        return [int(x) for x in out]

    def set_params(self, **kw) -> None:
        p = tc_params()
        lib = load_library()
        _check(lib.tc_params_default(ctypes.byref(p)), "tc_params_default")
        for k_, v in kw.items():
            setattr(p, k_, int(v))
        _check(lib.tc_batch_set_params(self.handle, ctypes.byref(p)), "tc_batch_set_params")

    def stats(self) -> dict:
        s = tc_stats()
        _check(load_library().tc_batch_get_stats(self.handle, ctypes.byref(s)), "tc_batch_get_stats")
        return {name: getattr(s, name) for name, _ in tc_stats._fields_}

    def levels(self, i: int) -> np.ndarray:
        out = np.empty(self.sizes[i], dtype=np.int32)
        _check(load_library().tc_batch_get_levels(self.handle, i,
                                                  out.ctypes.data if out.size else None),
               "tc_batch_get_levels")
        return out

    def close(self) -> None:
        if getattr(self, "handle", None):
            _check(load_library().tc_batch_destroy(self.handle), "tc_batch_destroy")
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

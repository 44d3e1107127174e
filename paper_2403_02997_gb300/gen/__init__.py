"""Seeded synthetic graph generators (inputs only; no counting arithmetic).

The bytes come from ``graphgen.c`` (counter-based SplitMix64 draws), so a
given (family, size, seed) yields the same edge list on every machine and for
every thread count.  Edge lists are returned as two uint32 numpy arrays with
self-loops and repeated pairs left in, as drawn; graph construction removes
them.

Workload recipes (shapes of the paper's experiments, Section "Data Sets":
Graph500 R-MAT with a=0.57, b=0.19, c=0.19, d=0.05, and low-degree,
long-diameter road networks):

* ``er``    G(n, m) draws, both endpoints uniform on [0, n).
* ``rmat``  R-MAT / Kronecker, 2^scale vertices, edge_factor * 2^scale draws,
            ids relabelled by a seeded uniform permutation.
* ``mesh``  rows x cols grid, 4-neighbour edges plus each cell's anti-diagonal
            {(i+1, j), (i, j+1)} with probability p.
"""
from __future__ import annotations

import ctypes
import math
import os
import subprocess
from dataclasses import dataclass

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "graphgen.c")
_LIB = os.path.join(_HERE, "libgraphgen.so")

RMAT_A, RMAT_B, RMAT_C = 0.57, 0.19, 0.19


def build(force: bool = False) -> str:
    """Compile libgraphgen.so beside its source (gcc, OpenMP when available)."""
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


def _load():
    global _lib
    if _lib is None:
        lib = ctypes.CDLL(build())
        u32p = ctypes.POINTER(ctypes.c_uint32)
        lib.gg_hash.restype = ctypes.c_uint64
        lib.gg_hash.argtypes = [ctypes.c_uint64] * 3
        lib.gg_er.restype = None
        lib.gg_er.argtypes = [ctypes.c_uint32, ctypes.c_uint64, ctypes.c_uint64, u32p, u32p]
        lib.gg_rmat.restype = None
        lib.gg_rmat.argtypes = [ctypes.c_uint32, ctypes.c_uint64, ctypes.c_uint64,
                                ctypes.c_uint32, ctypes.c_uint32, ctypes.c_uint32,
                                ctypes.c_int, u32p, u32p]
        lib.gg_permutation.restype = None
        lib.gg_permutation.argtypes = [ctypes.c_uint32, ctypes.c_uint64, u32p]
        lib.gg_mesh_diagonals.restype = ctypes.c_uint64
        lib.gg_mesh_diagonals.argtypes = [ctypes.c_uint32, ctypes.c_uint32, ctypes.c_uint64,
                                          ctypes.c_uint64, ctypes.POINTER(ctypes.c_uint8)]
        lib.gg_mesh_edges.restype = ctypes.c_uint64
        lib.gg_mesh_edges.argtypes = [ctypes.c_uint32, ctypes.c_uint32,
                                      ctypes.POINTER(ctypes.c_uint8), u32p, u32p]
        _lib = lib
    return _lib


def _p32(a: np.ndarray):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_uint32))


def hash64(seed: int, stream: int, i: int) -> int:
    """The generators' counter-based draw h(seed, stream, i)."""
    return int(_load().gg_hash(seed, stream, i))


def er_edges(n: int, m: int, seed: int):
    """m i.i.d. uniform ordered pairs on [0, n)^2 (G(n, m) before canonicalising)."""
    src = np.empty(m, dtype=np.uint32)
    dst = np.empty(m, dtype=np.uint32)
    if m:
        _load().gg_er(n, m, seed, _p32(src), _p32(dst))
    return src, dst


def rmat_thresholds(a: float = RMAT_A, b: float = RMAT_B, c: float = RMAT_C):
    """Cumulative quadrant probabilities scaled to 32-bit integer thresholds."""
    return (min(round(a * 2**32), 2**32 - 1), min(round((a + b) * 2**32), 2**32 - 1),
            min(round((a + b + c) * 2**32), 2**32 - 1))


def rmat_edges(scale: int, edge_factor: int, seed: int, permute: bool = True,
               a: float = RMAT_A, b: float = RMAT_B, c: float = RMAT_C):
    """edge_factor * 2^scale R-MAT draws on 2^scale vertices."""
    m = edge_factor << scale
    src = np.empty(m, dtype=np.uint32)
    dst = np.empty(m, dtype=np.uint32)
    ta, tab, tabc = rmat_thresholds(a, b, c)
    if m:
        _load().gg_rmat(scale, m, seed, ta, tab, tabc, int(permute), _p32(src), _p32(dst))
    return src, dst


def permutation(n: int, seed: int) -> np.ndarray:
    p = np.empty(n, dtype=np.uint32)
    _load().gg_permutation(n, seed, _p32(p))
    return p


def mesh_diagonals(rows: int, cols: int, p: float, seed: int) -> np.ndarray:
    """uint8 flags[(rows-1)*(cols-1)]: 1 where cell (i, j) holds its anti-diagonal."""
    cells = max(rows - 1, 0) * max(cols - 1, 0)
    flags = np.zeros(cells, dtype=np.uint8)
    thresh = min(int(p * 2**32), 2**32) if p < 1.0 else 2**32
    if cells:
        _load().gg_mesh_diagonals(rows, cols, thresh, seed,
                                  flags.ctypes.data_as(ctypes.POINTER(ctypes.c_uint8)))
    return flags


def mesh_edges(rows: int, cols: int, p: float, seed: int):
    """rows x cols 4-neighbour mesh plus random anti-diagonals; ids i*cols + j."""
    flags = mesh_diagonals(rows, cols, p, seed)
    cap = rows * max(cols - 1, 0) + max(rows - 1, 0) * cols + int(flags.sum())
    src = np.empty(cap, dtype=np.uint32)
    dst = np.empty(cap, dtype=np.uint32)
    fl = flags if flags.size else np.zeros(1, dtype=np.uint8)
    e = _load().gg_mesh_edges(rows, cols, fl.ctypes.data_as(ctypes.POINTER(ctypes.c_uint8)),
                              _p32(src), _p32(dst))
    assert e == cap
    return src, dst


# --------------------------------------------------------------------------
# Named workloads
# --------------------------------------------------------------------------

@dataclass(frozen=True)
class GraphSpec:
    """One synthetic graph: family, size parameters, seed and BFS root rule."""
    family: str           # "er" | "rmat" | "mesh"
    n: int                # number of vertices
    draws: int            # edge pairs drawn (before canonicalising)
    seed: int
    scale: int = 0        # rmat: log2 n
    edge_factor: int = 0  # rmat
    rows: int = 0         # mesh
    cols: int = 0         # mesh
    p: float = 0.0        # mesh diagonal probability
    root: str = "zero"    # "zero" (vertex 0 / mesh corner) | "maxdeg" (smallest id of max degree)

    def edges(self):
        if self.family == "er":
            return er_edges(self.n, self.draws, self.seed)
        if self.family == "rmat":
            return rmat_edges(self.scale, self.edge_factor, self.seed)
        if self.family == "mesh":
            return mesh_edges(self.rows, self.cols, self.p, self.seed)
        raise ValueError(self.family)


def er_spec(n: int, m: int, seed: int) -> GraphSpec:
    return GraphSpec("er", n, m, seed, root="zero")


def rmat_spec(scale: int, edge_factor: int, seed: int) -> GraphSpec:
    return GraphSpec("rmat", 1 << scale, edge_factor << scale, seed, scale=scale,
                     edge_factor=edge_factor, root="maxdeg")


def mesh_spec(rows: int, cols: int, p: float, seed: int) -> GraphSpec:
    return GraphSpec("mesh", rows * cols, 0, seed, rows=rows, cols=cols, p=p, root="zero")


# The single-graph workloads: ER G(1024, 8192) seed 1; R-MAT scale 24 edge
# factor 16 seed 2; 4096 x 4096 mesh with diagonals at p = 0.5, seed 7.
ER_1024 = er_spec(1024, 8192, 1)
RMAT_24 = rmat_spec(24, 16, 2)
MESH_4096 = mesh_spec(4096, 4096, 0.5, 7)


def _u01(seed: int, stream: int, i: int) -> float:
    return (hash64(seed, stream, i) >> 11) * (1.0 / 2**53)


def batched_specs(count: int = 4096, master_seed: int = 4, log2_min: int = 6,
                  log2_max: int = 16) -> list:
    """The batched workload: `count` graphs, n log-uniform on [2^log2_min, 2^log2_max].

    Even indices are Erdos-Renyi with mean degree uniform in [4, 64]
    (draws = n * d / 2); odd indices are R-MAT with scale = round(log2 n) and an
    edge factor uniform in {8, ..., 16}.  Per-graph seeds derive from the
    master seed (stream 10 sizes, 11 degrees, 12 seeds).
    """
    specs = []
    for g in range(count):
        x = log2_min + (log2_max - log2_min) * _u01(master_seed, 10, g)
        seed = hash64(master_seed, 12, g) & 0x7FFFFFFF
        if g % 2 == 0:
            n = max(2, int(math.floor(2.0 ** x)))
            d = 4.0 + 60.0 * _u01(master_seed, 11, g)
            specs.append(er_spec(n, int(n * d / 2), seed))
        else:
            scale = int(round(x))
            ef = 8 + int(hash64(master_seed, 11, g) % 9)
            specs.append(rmat_spec(scale, ef, seed))
    return specs

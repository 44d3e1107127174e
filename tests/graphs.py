"""Small hand-built graphs with closed-form triangle counts (test helpers).

Each builder returns (n, src, dst) as uint32 numpy arrays.
"""
import itertools

import numpy as np


def _arr(n, pairs):
    if not pairs:
        return n, np.zeros(0, np.uint32), np.zeros(0, np.uint32)
    s, d = zip(*pairs)
    return n, np.array(s, np.uint32), np.array(d, np.uint32)


def complete(n):
    """K_n: C(n, 3) triangles."""
    return _arr(n, list(itertools.combinations(range(n), 2)))


def complete_bipartite(a, b):
    """K_{a,b}: bipartite, no triangles."""
    return _arr(a + b, [(i, a + j) for i in range(a) for j in range(b)])


def wheel(n):
    """W_n: hub 0 joined to a rim cycle 1..n-1; n - 1 triangles for n >= 5."""
    rim = list(range(1, n))
    pairs = [(0, r) for r in rim] + [(rim[i], rim[(i + 1) % len(rim)]) for i in range(len(rim))]
    return _arr(n, pairs)


def path(n):
    return _arr(n, [(i, i + 1) for i in range(n - 1)])


def cycle(n):
    return _arr(n, [(i, (i + 1) % n) for i in range(n)])


def star(n):
    return _arr(n, [(0, i) for i in range(1, n)])


def diag_grid(r, c):
    """r x c grid, 4-neighbour edges plus every cell's anti-diagonal: 2(r-1)(c-1) triangles."""
    vid = lambda i, j: i * c + j
    pairs = []
    for i in range(r):
        for j in range(c):
            if j + 1 < c:
                pairs.append((vid(i, j), vid(i, j + 1)))
            if i + 1 < r:
                pairs.append((vid(i, j), vid(i + 1, j)))
            if i + 1 < r and j + 1 < c:
                pairs.append((vid(i + 1, j), vid(i, j + 1)))
    return _arr(r * c, pairs)


def random_gnp(n, p, seed):
    rng = np.random.default_rng(seed)
    pairs = [(i, j) for i in range(n) for j in range(i + 1, n) if rng.random() < p]
    return _arr(n, pairs)


def disjoint_union(*graphs):
    off = 0
    ss, dd = [], []
    for n, s, d in graphs:
        ss.append(s.astype(np.int64) + off)
        dd.append(d.astype(np.int64) + off)
        off += n
    return off, np.concatenate(ss).astype(np.uint32), np.concatenate(dd).astype(np.uint32)


def relabel(graph, seed):
    """Apply a random permutation of vertex ids."""
    n, s, d = graph
    perm = np.random.default_rng(seed).permutation(n).astype(np.uint32)
    return n, perm[s], perm[d]

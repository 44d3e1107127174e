"""Pins of the CPU oracle against facts fixed outside it (no GPU).

Closed forms, brute force (Algorithm Triples, tr(A^3)/6), an independent
algorithm (degree-ordered Forward), the cover-edge lemmas (H-E, HE2), and a
library BFS.  Each is chosen so that a plausible slip in the oracle (a dropped
term of the counting rule, u and v swapped, a wrong level index, a missed
restart) fails at least one of them.
"""
import itertools
from math import comb

import numpy as np
import pytest

import oracle
from paper_2403_02997_gb300 import gen
from tests import graphs


def run(g, root=0, want_cover=False):
    n, s, d = g
    r = oracle.count(n, s, d, root, want_cover=want_cover)
    assert r["T"] == r["c1"] + r["c2"] // 3, "Algorithm CETC-SM identity"
    assert r["c2"] % 3 == 0
    return r


# --------------------------------------------------------------------------
# Graph construction (undirected simple graph, Section Notations)
# --------------------------------------------------------------------------

def test_csr_matches_set_definition():
    rng = np.random.default_rng(5)
    for trial in range(20):
        n = int(rng.integers(1, 60))
        E = int(rng.integers(0, 300))
        s = rng.integers(0, n, E).astype(np.uint32)
        d = rng.integers(0, n, E).astype(np.uint32)
        rp, col = oracle.build_csr(n, s, d)
        nbrs = [set() for _ in range(n)]
        for a, b in zip(s.tolist(), d.tolist()):
            if a != b:
                nbrs[a].add(b)
                nbrs[b].add(a)
        assert rp[0] == 0 and rp.size == n + 1
        for v in range(n):
            assert col[rp[v]:rp[v + 1]].tolist() == sorted(nbrs[v])
        assert col.size == sum(len(x) for x in nbrs)


def test_csr_rejects_out_of_range():
    with pytest.raises(oracle.VertexRangeError):
        oracle.build_csr(4, np.array([0, 4], np.uint32), np.array([1, 2], np.uint32))


def test_empty_graphs():
    r = oracle.count(0, np.zeros(0, np.uint32), np.zeros(0, np.uint32), 0)
    assert r["T"] == 0 and r["m"] == 0
    r = oracle.count(5, np.zeros(0, np.uint32), np.zeros(0, np.uint32), 2)
    assert r["T"] == 0 and r["num_cover"] == 0
    assert r["level"].tolist() == [0, 0, 0, 0, 0]
    # only self-loops and repeats
    r = oracle.count(3, np.array([1, 1, 2], np.uint32), np.array([1, 1, 2], np.uint32), 0)
    assert r["m"] == 0 and r["T"] == 0


# --------------------------------------------------------------------------
# Closed forms
# --------------------------------------------------------------------------

@pytest.mark.parametrize("n", range(1, 13))
def test_complete_graph(n):
    g = graphs.complete(n)
    for root in range(n):
        r = run(g, root)
        assert r["T"] == comb(n, 3)
        # all vertices but the root share level 1: K_{n-1} is horizontal
        assert r["num_cover"] == comb(n - 1, 2)


@pytest.mark.parametrize("a,b", [(1, 1), (2, 3), (4, 4), (5, 9)])
def test_complete_bipartite_has_no_cover_edges(a, b):
    g = graphs.complete_bipartite(a, b)
    for root in range(a + b):
        r = run(g, root)
        assert r["T"] == 0 and r["num_cover"] == 0 and r["matches"] == 0


@pytest.mark.parametrize("n", [5, 6, 7, 12, 31])
def test_wheel(n):
    g = graphs.wheel(n)
    for root in [0, 1, n - 1]:
        r = run(g, root)
        assert r["T"] == n - 1
    # hub as root: every rim edge is horizontal, every apex is the hub (c1 only)
    r = run(g, 0)
    assert r["num_cover"] == n - 1 and r["c1"] == n - 1 and r["c2"] == 0


@pytest.mark.parametrize("rc", [(2, 2), (2, 5), (3, 3), (7, 4), (10, 13)])
def test_diagonal_grid(rc):
    r_, c_ = rc
    g = graphs.diag_grid(r_, c_)
    for root in [0, r_ * c_ - 1, (r_ // 2) * c_ + c_ // 2]:
        assert run(g, root)["T"] == 2 * (r_ - 1) * (c_ - 1)


@pytest.mark.parametrize("rows,cols,p,seed", [(5, 5, 0.5, 7), (17, 9, 0.5, 3), (32, 32, 1.0, 7),
                                              (40, 31, 0.25, 11), (12, 12, 0.0, 1)])
def test_mesh_closed_form(rows, cols, p, seed):
    """Anti-diagonal mesh from the corner: L(i,j) = i + j, S = the diagonals, T = 2 D."""
    s, d = gen.mesh_edges(rows, cols, p, seed)
    flags = gen.mesh_diagonals(rows, cols, p, seed)
    n = rows * cols
    r = oracle.count(n, s, d, 0, want_cover=True)
    i, j = np.divmod(np.arange(n), cols)
    assert np.array_equal(r["level"], (i + j).astype(np.int32))
    D = int(flags.sum())
    assert r["T"] == 2 * D and r["c1"] == 2 * D and r["c2"] == 0
    cells = np.nonzero(flags)[0]
    ci, cj = np.divmod(cells, cols - 1)
    a = (ci + 1) * cols + cj
    b = ci * cols + cj + 1
    expect = sorted(zip(np.minimum(a, b).tolist(), np.maximum(a, b).tolist()))
    got = list(zip(r["cover_u"].tolist(), r["cover_v"].tolist()))
    assert got == expect


@pytest.mark.parametrize("n", [1, 2, 3, 10, 50])
def test_path_levels(n):
    g = graphs.path(n)
    r = run(g, 0)
    assert r["level"].tolist() == list(range(n))
    assert r["num_cover"] == 0 and r["T"] == 0


@pytest.mark.parametrize("k", [1, 2, 3, 10])
def test_odd_cycle(k):
    n = 2 * k + 1
    for root in range(0, n, max(1, n // 4)):
        r = run(graphs.cycle(n), root, want_cover=True)
        assert r["num_cover"] == 1
        assert r["T"] == (1 if n == 3 else 0)
        u, v = int(r["cover_u"][0]), int(r["cover_v"][0])
        assert r["level"][u] == r["level"][v] == k


@pytest.mark.parametrize("n", [4, 6, 20])
def test_even_cycle_and_star(n):
    assert run(graphs.cycle(n))["num_cover"] == 0
    r = run(graphs.star(n), 3 % n)
    assert r["T"] == 0 and r["num_cover"] == 0


# --------------------------------------------------------------------------
# Brute force and library identities
# --------------------------------------------------------------------------

@pytest.mark.parametrize("seed", range(12))
def test_brute_force_triples(seed):
    rng = np.random.default_rng(seed)
    n = int(rng.integers(3, 40))
    p = float(rng.uniform(0.05, 0.9))
    g = graphs.random_gnp(n, p, seed)
    expect = oracle.triples(*g)
    for root in rng.choice(n, size=min(n, 5), replace=False):
        assert run(g, int(root))["T"] == expect


def test_triples_closed_forms():
    assert oracle.triples(*graphs.complete(9)) == comb(9, 3)
    assert oracle.triples(*graphs.wheel(8)) == 7
    assert oracle.triples(*graphs.complete_bipartite(4, 5)) == 0


@pytest.mark.parametrize("seed", range(6))
def test_trace_a_cubed(seed):
    rng = np.random.default_rng(100 + seed)
    n = int(rng.integers(50, 300))
    s, d = gen.er_edges(n, int(n * rng.uniform(2, 20)), seed)
    expect = oracle.trace_a3(n, s, d)
    assert oracle.count(n, s, d, int(rng.integers(0, n)))["T"] == expect


def test_forward_against_brute_force():
    for seed in range(8):
        g = graphs.random_gnp(30, 0.3, 200 + seed)
        rp, col = oracle.build_csr(*g)
        assert oracle.forward(rp, col) == oracle.triples(*g)


@pytest.mark.parametrize("family,seed", [("er", 1), ("er", 2), ("rmat", 3), ("rmat", 4)])
def test_forward_independent_count(family, seed):
    if family == "er":
        n = 3000
        s, d = gen.er_edges(n, 40000, seed)
    else:
        n = 1 << 12
        s, d = gen.rmat_edges(12, 16, seed)
    rp, col = oracle.build_csr(n, s, d)
    f = oracle.forward(rp, col)
    for root in [0, oracle.max_degree_root(rp), n // 2]:
        lv = oracle.bfs_levels(rp, col, root)
        r = oracle.cetc(rp, col, lv)
        assert r["T"] == f
        assert r["T"] == r["c1"] + r["c2"] // 3


def test_disconnected_union_counts_add():
    parts = [graphs.complete(6), graphs.wheel(7), graphs.cycle(3), graphs.path(4),
             graphs.diag_grid(3, 4), graphs.complete(1)]
    g = graphs.relabel(graphs.disjoint_union(*parts), 9)
    expect = comb(6, 3) + 6 + 1 + 0 + 2 * 2 * 3 + 0
    n = g[0]
    for root in range(0, n, 5):
        assert run(g, root)["T"] == expect


# --------------------------------------------------------------------------
# Lemmas on horizontal edges and the counting rule
# --------------------------------------------------------------------------

def _triangles(adj):
    n = adj.shape[0]
    return [(a, b, c) for a, b, c in itertools.combinations(range(n), 3)
            if adj[a, b] and adj[b, c] and adj[a, c]]


@pytest.mark.parametrize("seed", range(10))
def test_lemma_he2_and_rule(seed):
    """Every triangle has 1 or 3 horizontal edges; the rule counts it once."""
    rng = np.random.default_rng(seed)
    g = graphs.random_gnp(int(rng.integers(8, 36)), float(rng.uniform(0.1, 0.7)), 300 + seed)
    n = g[0]
    adj = oracle.adjacency_matrix(*g)
    root = int(rng.integers(0, n))
    r = run(g, root, want_cover=True)
    L = r["level"]
    S = set(zip(r["cover_u"].tolist(), r["cover_v"].tolist()))
    tris = _triangles(adj)
    hits = {t: 0 for t in tris}
    for (a, b, c) in tris:
        h = sum(L[x] == L[y] for x, y in [(a, b), (b, c), (a, c)])
        assert h in (1, 3)
        assert sum(((min(x, y), max(x, y)) in S) for x, y in [(a, b), (b, c), (a, c)]) == h
    # enumerate the rule by brute force over (cover edge, apex)
    for (u, v) in S:
        assert u < v and L[u] == L[v] and adj[u, v]
        per_edge = 0
        for w in range(n):
            if adj[u, w] and adj[v, w] and (L[w] != L[u] or v < w):
                hits[tuple(sorted((u, v, w)))] += 1
                per_edge += 1
        assert oracle.edge_count(r["row_ptr"], r["col"], L, u, v) == per_edge
    assert all(x == 1 for x in hits.values())
    assert r["T"] == len(tris)
    # every edge spans at most one level
    rp, col = r["row_ptr"], r["col"]
    src = np.repeat(np.arange(n), np.diff(rp))
    assert np.all(np.abs(L[src] - L[col]) <= 1)


def test_levels_match_networkx_with_restarts():
    nx = pytest.importorskip("networkx")
    for seed in range(4):
        n = 1 << 11
        s, d = gen.rmat_edges(11, 2, 50 + seed)
        rp, col = oracle.build_csr(n, s, d)
        root = oracle.max_degree_root(rp)
        L = oracle.bfs_levels(rp, col, root)
        G = nx.Graph()
        G.add_nodes_from(range(n))
        G.add_edges_from((int(a), int(b)) for a, b in zip(s, d) if a != b)
        expect = np.full(n, -1, np.int64)
        for v, dist in nx.single_source_shortest_path_length(G, root).items():
            expect[v] = dist
        for comp in sorted(nx.connected_components(G), key=min):
            start = min(comp)
            if expect[start] != -1:
                continue
            for v, dist in nx.single_source_shortest_path_length(G, start).items():
                expect[v] = dist
        assert np.array_equal(L.astype(np.int64), expect)


def test_edge_list_count_equals_full_loop():
    n = 1 << 11
    s, d = gen.rmat_edges(11, 8, 5)
    rp, col = oracle.build_csr(n, s, d)
    lv = oracle.bfs_levels(rp, col, 3)
    full = oracle.cetc(rp, col, lv, want_cover=True)
    part = oracle.cetc_edges(rp, col, lv, full["cover_u"], full["cover_v"])
    assert (part["T"], part["c1"], part["c2"]) == (full["T"], full["c1"], full["c2"])
    half = oracle.cetc_edges(rp, col, lv, full["cover_u"][::2], full["cover_v"][::2])
    other = oracle.cetc_edges(rp, col, lv, full["cover_u"][1::2], full["cover_v"][1::2])
    assert half["T"] + other["T"] == full["T"]


def test_parallel_edge_list_count():
    """The OpenMP edge loop (CETC-SM's form) sums the same per-edge counts: over all of S it
    gives C(n, 3) on K_n and the full loop's T, c1, c2 on an R-MAT graph; on a random subset it
    equals the single-thread loop."""
    k = 23
    s, d = zip(*[(a, b) for a in range(k) for b in range(a + 1, k)])
    rp, col = oracle.build_csr(k, np.array(s, np.uint32), np.array(d, np.uint32))
    lv = oracle.bfs_levels(rp, col, 0)
    full = oracle.cetc(rp, col, lv, want_cover=True)
    par = oracle.cetc_sm_edges(rp, col, lv, full["cover_u"], full["cover_v"])
    assert par["T"] == comb(k, 3)
    n = 1 << 11
    s, d = gen.rmat_edges(11, 8, 6)
    rp, col = oracle.build_csr(n, s, d)
    lv = oracle.bfs_levels(rp, col, 0)
    full = oracle.cetc(rp, col, lv, want_cover=True)
    par = oracle.cetc_sm_edges(rp, col, lv, full["cover_u"], full["cover_v"])
    assert (par["T"], par["c1"], par["c2"]) == (full["T"], full["c1"], full["c2"])
    idx = np.random.default_rng(3).integers(0, full["num_cover"], size=500)
    u, v = full["cover_u"][idx], full["cover_v"][idx]
    assert oracle.cetc_sm_edges(rp, col, lv, u, v) == oracle.cetc_edges(rp, col, lv, u, v)


def test_root_invariance_and_sampling():
    n = 1 << 10
    s, d = gen.rmat_edges(10, 8, 77)
    rp, col = oracle.build_csr(n, s, d)
    counts = set()
    for root in range(0, n, 97):
        lv = oracle.bfs_levels(rp, col, root)
        r = oracle.cetc(rp, col, lv)
        counts.add(r["T"])
        assert r["done"] == r["num_cover"]
        sm = oracle.cetc_sm(rp, col, lv)
        assert sm["T"] == r["T"] and sm["c1"] == r["c1"] and sm["c2"] == r["c2"]
        half = oracle.cetc(rp, col, lv, stride=2)
        assert half["done"] == (r["num_cover"] + 1) // 2
    assert len(counts) == 1


# --------------------------------------------------------------------------
# Generators (inputs shared by both sides)
# --------------------------------------------------------------------------

def test_splitmix64_vector():
    # SplitMix64 from state 0 gives 0xE220A8397B1DCDAF first (Vigna's reference
    # implementation); h(seed, stream, i) nests that function three times.
    assert _sm64_py(0) == 0xE220A8397B1DCDAF
    for args in [(0, 0, 0), (3, 4, 5), (2, 2, 123456789)]:
        seed, stream, i = args
        expect = _sm64_py((_sm64_py((_sm64_py(seed) + stream) & M64) + i) & M64)
        assert gen.hash64(*args) == expect


M64 = (1 << 64) - 1


def _sm64_py(x):
    x = (x + 0x9E3779B97F4A7C15) & M64
    x = ((x ^ (x >> 30)) * 0xBF58476D1CE4E5B9) & M64
    x = ((x ^ (x >> 27)) * 0x94D049BB133111EB) & M64
    return x ^ (x >> 31)


def test_generators_deterministic_and_shaped():
    a = gen.rmat_edges(10, 16, 5)
    b = gen.rmat_edges(10, 16, 5)
    assert np.array_equal(a[0], b[0]) and np.array_equal(a[1], b[1])
    assert a[0].size == 16 << 10 and a[0].max() < 1024
    # without the permutation, vertex 0 (all quadrant-a bits) is the heaviest
    s, d = gen.rmat_edges(12, 16, 5, permute=False)
    deg = np.bincount(np.concatenate([s, d]), minlength=4096)
    assert int(np.argmax(deg)) == 0
    # the permutation is a bijection
    p = gen.permutation(1000, 3)
    assert sorted(p.tolist()) == list(range(1000))
    e = gen.er_edges(1024, 8192, 1)
    assert e[0].size == 8192 and e[0].max() < 1024 and e[1].max() < 1024
    ms, md = gen.mesh_edges(4, 5, 1.0, 7)
    assert ms.size == 4 * 4 + 3 * 5 + 3 * 4


# --------------------------------------------------------------------------
# Algorithm CETC-Seq-S (split into G0 and G1)
# --------------------------------------------------------------------------

def _split(g, root):
    n, s, d = g
    rp, col = oracle.build_csr(n, s, d)
    lv = oracle.bfs_levels(rp, col, root) if n else np.zeros(0, np.int32)
    return oracle.cetc_split(rp, col, lv)


@pytest.mark.parametrize("n", range(1, 13))
def test_split_complete_graph(n):
    """K_n from vertex 0: the other n - 1 vertices share level 1, so G0 = K_{n-1}
    holds C(n-1, 3) triangles and the C(n-1, 2) triangles through the root have
    their apex on level 0."""
    r = _split(graphs.complete(n), 0)
    assert r["T0"] == comb(n - 1, 3) and r["T1"] == comb(n - 1, 2) and r["T"] == comb(n, 3)


@pytest.mark.parametrize("n", [5, 6, 9, 31])
def test_split_wheel(n):
    """W_n from the hub: G0 is the rim cycle (no triangle for n - 1 >= 4)."""
    r = _split(graphs.wheel(n), 0)
    assert (r["T0"], r["T1"]) == (0, n - 1)


@pytest.mark.parametrize("rows,cols,p,seed", [(5, 5, 0.5, 7), (17, 9, 1.0, 3)])
def test_split_mesh(rows, cols, p, seed):
    """Anti-diagonal mesh from the corner: every apex is off its diagonal's level."""
    s, d = gen.mesh_edges(rows, cols, p, seed)
    D = int(gen.mesh_diagonals(rows, cols, p, seed).sum())
    r = _split((rows * cols, s, d), 0)
    assert (r["T0"], r["T1"]) == (0, 2 * D)


@pytest.mark.parametrize("family,seed", [("er", 1), ("er", 5), ("rmat", 3), ("rmat", 6)])
def test_split_against_cetc_and_forward(family, seed):
    """T0 + T1 = T (Forward, an independent count); T1 = c1 and 3 T0 = c2 of
    the CETC-SM split, for several roots (restarts included)."""
    if family == "er":
        n = 2000
        s, d = gen.er_edges(n, 30000, seed)
    else:
        n = 1 << 11
        s, d = gen.rmat_edges(11, 16, seed)
    rp, col = oracle.build_csr(n, s, d)
    f = oracle.forward(rp, col)
    for root in [0, oracle.max_degree_root(rp), n - 1]:
        lv = oracle.bfs_levels(rp, col, root)
        sp = oracle.cetc_split(rp, col, lv)
        c = oracle.cetc(rp, col, lv)
        assert sp["T"] == f == c["T"]
        assert sp["T1"] == c["c1"] and 3 * sp["T0"] == c["c2"]


def test_split_disconnected():
    parts = [graphs.complete(6), graphs.wheel(7), graphs.cycle(3), graphs.path(4),
             graphs.diag_grid(3, 4), graphs.complete(1)]
    g = graphs.relabel(graphs.disjoint_union(*parts), 9)
    for root in range(0, g[0], 7):
        assert _split(g, root)["T"] == comb(6, 3) + 6 + 1 + 0 + 2 * 2 * 3 + 0


# --------------------------------------------------------------------------
# Degree ordering (Algorithms CETC-Seq-D / CETC-Seq-SD)
# --------------------------------------------------------------------------

def test_degree_order_worked_example():
    """A 4-cycle 0-1-2-3 with the chord 0-2: degrees 3, 2, 3, 2, so by decreasing degree
    and then increasing id the order is 0, 2, 1, 3 (worked by hand)."""
    s = np.array([0, 1, 2, 3, 0], np.uint32)
    d = np.array([1, 2, 3, 0, 2], np.uint32)
    rp, _ = oracle.build_csr(4, s, d)
    assert oracle.degree_order(rp).tolist() == [0, 2, 1, 3]


@pytest.mark.parametrize("family,seed", [("er", 3), ("rmat", 7), ("wheel", 0), ("union", 1)])
def test_degree_order(family, seed):
    if family == "er":
        n = 800
        s, d = gen.er_edges(n, 6000, seed)
    elif family == "rmat":
        n = 1 << 10
        s, d = gen.rmat_edges(10, 16, seed)
    elif family == "wheel":
        n, s, d = graphs.wheel(11)
    else:
        n, s, d = graphs.relabel(graphs.disjoint_union(graphs.complete(6), graphs.wheel(9),
                                                       graphs.path(5)), seed)
    rp, col = oracle.build_csr(n, s, d)
    deg = np.diff(rp)
    order = oracle.degree_order(rp)
    # the definition, restated with Python's sort
    assert order.tolist() == sorted(range(n), key=lambda v: (-int(deg[v]), v))
    assert np.all(np.diff(deg[order]) <= 0)
    # ties: among vertices of one degree the ids ascend
    tie = deg[order][:-1] == deg[order][1:]
    assert np.all(order[:-1][tie] < order[1:][tie])
    s2, d2 = oracle.relabel_edges(order, s, d)
    rp2, col2 = oracle.build_csr(n, s2, d2)
    assert np.array_equal(np.diff(rp2), deg[order])
    # relabelling keeps the count; the CETC count on the new graph (CETC-Seq-D)
    # and the split count on it (CETC-Seq-SD) agree with Forward
    f = oracle.forward(rp, col)
    assert oracle.forward(rp2, col2) == f
    lv2 = oracle.bfs_levels(rp2, col2, 0)
    assert oracle.cetc(rp2, col2, lv2)["T"] == f == oracle.cetc_split(rp2, col2, lv2)["T"]
    if family == "wheel":
        assert order[0] == 0  # the hub


# --------------------------------------------------------------------------
# Triangle listing and per-vertex counts
# --------------------------------------------------------------------------

@pytest.mark.parametrize("seed", range(8))
def test_listing_against_matrix_and_brute_force(seed):
    """Per-vertex counts = diag(A^3) / 2 (an exact int64 matrix product); the
    list = the brute-force set of pairwise adjacent triples; |list| = Forward."""
    rng = np.random.default_rng(seed)
    n = int(rng.integers(5, 60))
    m = int(rng.integers(0, n * 4))
    s = rng.integers(0, n, m).astype(np.uint32)
    d = rng.integers(0, n, m).astype(np.uint32)
    rp, col = oracle.build_csr(n, s, d)
    tri, vc = oracle.list_triangles(rp, col)
    a = oracle.adjacency_matrix(n, s, d).astype(np.int64)
    assert np.array_equal(vc.astype(np.int64), np.diag(a @ a @ a) // 2)
    brute = [t for t in itertools.combinations(range(n), 3)
             if a[t[0], t[1]] and a[t[1], t[2]] and a[t[0], t[2]]]
    assert [tuple(r) for r in tri.tolist()] == brute
    assert len(brute) == oracle.forward(rp, col)


@pytest.mark.parametrize("n", [3, 4, 7, 10])
def test_listing_closed_forms(n):
    rp, col = oracle.build_csr(*graphs.complete(n))
    tri, vc = oracle.list_triangles(rp, col)
    assert len(tri) == comb(n, 3) and np.all(vc == comb(n - 1, 2))
    rp, col = oracle.build_csr(*graphs.wheel(n + 2))
    tri, vc = oracle.list_triangles(rp, col)
    assert vc[0] == n + 1 and np.all(vc[1:] == 2)

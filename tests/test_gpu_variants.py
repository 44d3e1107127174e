"""The paper's CETC variants on the GPU against the oracle (needs a GB300).

- Algorithm CETC-Seq-S (tc_count_split): T = T0 + T1 bit-exact; c1 = T1 and
  c2 = 3 T0 against the oracle's literal CETC-Seq-S (which its own tests pin to
  closed forms and to CETC-SM's c1 / c2); levels and cover set as tc_count's.
- Algorithm Forward with degree ranking (tc_count_forward): T against the
  oracle's Forward.
- Algorithm CETC-Seq-FE (tc_count_fe): both branches give the same T.
Parameter sets send every pair through the inline merge, or through the
owner-hash pass with one or many chunks.
"""
from math import comb

import numpy as np
import pytest

import oracle
import paper_2403_02997_gb300 as tc
from paper_2403_02997_gb300 import gen
from tests import graphs

pytestmark = pytest.mark.gpu

PARAMS = {
    "default": {},
    "all_hash": dict(small_max_degree=0),
    "all_merge": dict(small_max_degree=1 << 30),
    "tiny_chunks": dict(small_max_degree=0, hash_chunk=32, edges_per_item=3),
    "long_items": dict(small_max_degree=0, hash_block=1024, hash_chunk=128, edges_per_item=4096),
}


@pytest.fixture(scope="module", autouse=True)
def built():
    from paper_2403_02997_gb300 import build
    build.build_all()
    oracle.build()


def _graphs():
    out = [("K12", graphs.complete(12), 0), ("wheel9", graphs.wheel(9), 0),
           ("diag_grid", graphs.diag_grid(7, 9), 5),
           ("union", graphs.relabel(graphs.disjoint_union(graphs.complete(6), graphs.wheel(7),
                                                            graphs.cycle(3), graphs.path(4)), 3), 4)]
    for seed in (1, 2):
        s, d = gen.er_edges(1500, 20000, seed)
        out.append((f"er{seed}", (1500, s, d), 0))
    for scale, ef, seed in ((10, 16, 3), (13, 16, 4), (12, 8, 5)):
        s, d = gen.rmat_edges(scale, ef, seed)
        out.append((f"rmat{scale}_{seed}", (1 << scale, s, d), "maxdeg"))
    s, d = gen.mesh_edges(40, 33, 0.5, 7)
    out.append(("mesh", (40 * 33, s, d), 0))
    return out


GRAPHS = _graphs()


@pytest.mark.parametrize("pname", list(PARAMS))
@pytest.mark.parametrize("gi", range(len(GRAPHS)))
def test_split_and_forward_match_oracle(gi, pname):
    name, (n, s, d), root = GRAPHS[gi]
    rp, col = oracle.build_csr(n, s, d)
    if root == "maxdeg":
        root = oracle.max_degree_root(rp)
    lv = oracle.bfs_levels(rp, col, root)
    sp = oracle.cetc_split(rp, col, lv)
    ref = oracle.cetc(rp, col, lv, want_cover=True)
    f = oracle.forward(rp, col)
    g = tc.Graph(s, d, n)
    try:
        g.set_params(**PARAMS[pname])
        T = g.count_split(root)
        st = g.stats()
        assert T == sp["T"] == ref["T"]
        assert (st["c1"], st["c2"]) == (sp["T1"], 3 * sp["T0"])
        assert st["num_cover"] == ref["num_cover"]
        assert np.array_equal(g.levels(), lv)
        u, v = g.cover_edges()
        o = np.lexsort((v, u))
        assert np.array_equal(u[o], ref["cover_u"]) and np.array_equal(v[o], ref["cover_v"])
        assert g.count_forward() == f
        with pytest.raises(tc.TCError):
            g.levels()  # no levels behind a forward count
        # the handle goes back to the cover-edge count unchanged
        assert g.count(root) == ref["T"]
        assert (g.stats()["c1"], g.stats()["c2"]) == (ref["c1"], ref["c2"])
    finally:
        g.close()


@pytest.mark.parametrize("gi", [0, 4, 6, 9])
def test_fe_both_branches(gi):
    name, (n, s, d), root = GRAPHS[gi]
    rp, col = oracle.build_csr(n, s, d)
    if root == "maxdeg":
        root = oracle.max_degree_root(rp)
    want = oracle.forward(rp, col)
    lv = oracle.bfs_levels(rp, col, root)
    c = oracle.cetc(rp, col, lv)["num_cover"] / max(1, col.size // 2)
    g = tc.Graph(s, d, n)
    try:
        T, used = g.count_fe(root, 2.0)       # c < 2 always: the cover-edge count
        assert T == want and not used
        assert np.array_equal(g.levels(), lv)
        T, used = g.count_fe(root, 0.0)       # c >= 0 always: the forward count
        assert T == want and used
        assert g.stats()["num_cover"] == round(c * (col.size // 2))
        T, used = g.count_fe(root, 0.7)       # the paper's threshold
        assert T == want and used == (c >= 0.7)
        with pytest.raises(tc.TCError):
            g.count_fe(root, -1.0)
    finally:
        g.close()


def test_variants_on_empty_and_tiny():
    for n, s, d in [(0, np.zeros(0, np.uint32), np.zeros(0, np.uint32)),
                    (5, np.zeros(0, np.uint32), np.zeros(0, np.uint32)),
                    graphs.complete(3), graphs.path(2)]:
        g = tc.Graph(s, d, n)
        try:
            want = 1 if n == 3 and s.size == 3 else 0
            assert g.count_split(0) == want
            assert g.count_forward() == want
            assert g.count_fe(0, 0.0)[0] == want
        finally:
            g.close()


def test_split_closed_form_complete():
    n, s, d = graphs.complete(20)
    g = tc.Graph(s, d, n)
    try:
        assert g.count_split(0) == comb(20, 3)
        st = g.stats()
        assert (st["c1"], st["c2"]) == (comb(19, 2), 3 * comb(19, 3))
    finally:
        g.close()


@pytest.mark.parametrize("gi", [0, 1, 3, 4, 6, 7, 9])
def test_degree_relabel_cetc_d_and_sd(gi):
    """tc_graph_relabel_degree against the oracle's degree ordering: the same
    permutation and CSR; on the new graph tc_count (CETC-Seq-D) and
    tc_count_split (CETC-Seq-SD) match the oracle's CETC on the relabelled
    edges (count, c1 / c2, levels, cover set) and the original count."""
    name, (n, s, d), _ = GRAPHS[gi]
    rp, col = oracle.build_csr(n, s, d)
    order = oracle.degree_order(rp)
    s2, d2 = oracle.relabel_edges(order, s, d)
    ref = oracle.count(n, s2, d2, 0, want_cover=True)
    g = tc.Graph(s, d, n)
    try:
        g2, perm = g.relabel_degree()
        try:
            assert np.array_equal(perm, order)
            rp2, col2 = g2.csr()
            assert np.array_equal(rp2.astype(np.int64), ref["row_ptr"])
            assert np.array_equal(col2, ref["col"])
            assert g2.max_degree_vertex() == 0 or g2.m == 0
            assert g2.count(0) == ref["T"] == oracle.forward(rp, col)
            st = g2.stats()
            assert (st["c1"], st["c2"], st["num_cover"]) == (ref["c1"], ref["c2"], ref["num_cover"])
            assert np.array_equal(g2.levels(), ref["level"])
            u, v = g2.cover_edges()
            o = np.lexsort((v, u))
            assert np.array_equal(u[o], ref["cover_u"]) and np.array_equal(v[o], ref["cover_v"])
            assert g2.count_split(0) == ref["T"]
        finally:
            g2.close()
    finally:
        g.close()


def test_relabel_empty():
    g = tc.Graph(np.zeros(0, np.uint32), np.zeros(0, np.uint32), 4)
    try:
        g2, perm = g.relabel_degree()
        assert perm.tolist() == [0, 1, 2, 3] and g2.m == 0 and g2.count(0) == 0
        g2.close()
    finally:
        g.close()


@pytest.mark.parametrize("pname", list(PARAMS))
@pytest.mark.parametrize("gi", [0, 1, 3, 4, 6, 9])
def test_triangle_listing(gi, pname):
    """tc_list_triangles against the oracle's enumeration: the same set of
    triangles (each once), per-vertex counts, each triple led by its cover edge
    (u < v on one level); a capacity below the count keeps the count and
    writes a subset."""
    name, (n, s, d), root = GRAPHS[gi]
    rp, col = oracle.build_csr(n, s, d)
    if root == "maxdeg":
        root = oracle.max_degree_root(rp)
    tri_ref, vc_ref = oracle.list_triangles(rp, col)
    lv = oracle.bfs_levels(rp, col, root)
    g = tc.Graph(s, d, n)
    try:
        g.set_params(**PARAMS[pname])
        T, tri, vc = g.list_triangles(root)
        assert T == len(tri_ref) and len(tri) == T
        assert np.all(tri[:, 0] < tri[:, 1]) and np.all(lv[tri[:, 0]] == lv[tri[:, 1]])
        srt = np.sort(tri, axis=1)
        srt = srt[np.lexsort((srt[:, 2], srt[:, 1], srt[:, 0]))]
        assert np.array_equal(srt, tri_ref.astype(np.int64))
        assert np.array_equal(vc, vc_ref)
        if T > 3:
            T2, part, none = g.list_triangles(root, capacity=T // 2, vertex_counts=False)
            assert T2 == T and len(part) == T // 2 and none is None
            ref_set = set(map(tuple, tri_ref.tolist()))
            got = [tuple(sorted(t)) for t in part.tolist()]
            assert len(set(got)) == len(got) and set(got) <= ref_set
        assert g.count(root) == T  # the handle counts as before
    finally:
        g.close()


def test_fe_with_learned_threshold():
    """The autotuner's CETC-Seq-FE threshold sends the graph down the branch that was faster on
    it, and that branch's count is the oracle's."""
    from paper_2403_02997_gb300 import autotune
    n = 1 << 14
    s, d = gen.rmat_edges(14, 16, 21)
    rp, col = oracle.build_csr(n, s, d)
    root = oracle.max_degree_root(rp)
    want = oracle.forward(rp, col)
    g = tc.Graph(s, d, n)
    try:
        fe = autotune.learn_fe_threshold(g, root, trials=2)
        T, used = g.count_fe(root, fe["threshold"])
        assert T == want and bool(used) == fe["forward_faster"]
    finally:
        g.close()

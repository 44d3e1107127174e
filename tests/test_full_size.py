"""Full-size workloads on the GPU, in the launch configuration the benchmark times.

* R-MAT scale 24 (edge factor 16, seed 2, root = max-degree vertex): the input
  is first confirmed identical to the one the oracle saw (edge-list checksum);
  then the count, c1, c2, m, |S|, d_max and root must equal the stored oracle
  values, and the CSR, the level array and the sorted cover-edge set must hash
  to the oracle's SHA-256 digests (an element-by-element comparison).
  Stored values: tests/golden/rmat24.json, written by make_golden.py.
* 4096 x 4096 mesh with anti-diagonals at p = 0.5 (seed 7, root = corner): the
  closed forms pinned in test_oracle: L(i, j) = i + j, S = the diagonals,
  T = 2 D.
* ER G(1024, 8192) (seed 1, root 0): everything against the oracle directly.
"""
import json
import os

import numpy as np
import pytest

import oracle
import paper_2403_02997_gb300 as tc
from paper_2403_02997_gb300 import gen
from tests.golden.make_golden import digest, edge_checksum

pytestmark = pytest.mark.gpu
HERE = os.path.dirname(os.path.abspath(__file__))


@pytest.fixture(scope="module", autouse=True)
def built():
    from paper_2403_02997_gb300 import build
    build.build_all()
    oracle.build()


def device_graph(src, dst, n):
    import torch
    s = torch.from_numpy(src.view(np.int32)).cuda()
    d = torch.from_numpy(dst.view(np.int32)).cuda()
    g = tc.Graph(s, d, n)
    del s, d
    return g


def sorted_cover_keys(u, v):
    return np.sort((u.astype(np.uint64) << np.uint64(32)) | v.astype(np.uint64))


def test_er1024_full():
    spec = gen.ER_1024
    src, dst = spec.edges()
    gold = json.load(open(os.path.join(HERE, "golden", "er1024.json")))
    assert edge_checksum(src, dst) == gold["edge_checksum"]
    ref = oracle.count(spec.n, src, dst, 0, want_cover=True)
    g = device_graph(src, dst, spec.n)
    try:
        assert g.count(0) == ref["T"] == gold["T"]
        st = g.stats()
        assert (st["c1"], st["c2"], st["num_cover"]) == (ref["c1"], ref["c2"], ref["num_cover"])
        assert np.array_equal(g.levels(), ref["level"])
        rp, col = g.csr()
        assert digest(rp.astype(np.int64), col) == gold["csr_sha256"]
        assert digest(g.levels()) == gold["level_sha256"]
        assert digest(sorted_cover_keys(*g.cover_edges())) == gold["cover_sha256"]
    finally:
        g.close()


def test_rmat24_full():
    gold = json.load(open(os.path.join(HERE, "golden", "rmat24.json")))
    spec = gen.RMAT_24
    src, dst = spec.edges()
    assert edge_checksum(src, dst) == gold["edge_checksum"], "generator differs on this machine"
    g = device_graph(src, dst, spec.n)
    del src, dst
    try:
        assert g.m == gold["m"] and g.d_max == gold["d_max"]
        root = g.max_degree_vertex()
        assert root == gold["root"]
        T = g.count(root)
        st = g.stats()
        assert T == gold["T"]
        assert (st["c1"], st["c2"], st["num_cover"]) == (gold["c1"], gold["c2"], gold["num_cover"])
        assert st["c2"] % 3 == 0 and st["c1"] + st["c2"] // 3 == T
        if "level_sha256" in gold:
            lv = g.levels()
            assert int(lv.max()) == gold["max_level"]
            assert digest(lv) == gold["level_sha256"]
            del lv
            assert digest(sorted_cover_keys(*g.cover_edges())) == gold["cover_sha256"]
            rp, col = g.csr()
            assert digest(rp.astype(np.int64), col) == gold["csr_sha256"]
        # a second root must give the same count (Lemma H-E: any BFS works)
        assert g.count(12345) == T
    finally:
        g.close()


def test_mesh4096_full():
    spec = gen.MESH_4096
    rows, cols = spec.rows, spec.cols
    src, dst = spec.edges()
    flags = gen.mesh_diagonals(rows, cols, spec.p, spec.seed)
    D = int(flags.sum())
    g = device_graph(src, dst, spec.n)
    del src, dst
    try:
        assert g.m == rows * (cols - 1) + (rows - 1) * cols + D
        T = g.count(0)
        assert T == 2 * D
        st = g.stats()
        assert st["num_levels"] == rows + cols - 1 and st["c2"] == 0
        lv = g.levels()
        i, j = np.divmod(np.arange(spec.n, dtype=np.int64), cols)
        assert np.array_equal(lv, (i + j).astype(np.int32))
        del lv, i, j
        cells = np.nonzero(flags)[0].astype(np.int64)
        ci, cj = np.divmod(cells, cols - 1)
        a, b = (ci + 1) * cols + cj, ci * cols + cj + 1
        want = np.sort((np.minimum(a, b).astype(np.uint64) << np.uint64(32)) |
                       np.maximum(a, b).astype(np.uint64))
        assert np.array_equal(sorted_cover_keys(*g.cover_edges()), want)
    finally:
        g.close()

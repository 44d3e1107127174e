"""tc_bfs_levels_noalloc (no device allocation) against the allocating path.

For callers that cannot call cudaMalloc, tc_bfs_levels_noalloc computes BFS
levels of a device CSR they own, using only a fixed scratch array compiled
into the library.  Its levels must equal those of tc_count + tc_get_levels on
the same graph and root, and those of the CPU oracle's BFS, on consecutive calls
(the scratch array keeps what the previous call left in it).  Integer output:
compared exactly.
"""
import numpy as np
import pytest

import oracle
import paper_2403_02997_gb300 as tc
from paper_2403_02997_gb300 import gen
from tests import graphs

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def built():
    from paper_2403_02997_gb300 import build
    build.build_all()


def _levels_both_ways(src, dst, n, root):
    import torch
    g = tc.Graph(src, dst, n)
    try:
        g.count(root)
        want = g.levels()
        rp, col = g.csr()
    finally:
        g.close()
    d_rp = torch.from_numpy(rp.view(np.int64)).cuda()
    d_col = torch.from_numpy(col.view(np.int32)).cuda()
    out = torch.full((n,), 7, dtype=torch.int32, device="cuda")  # stale values must vanish
    tc.tc_bfs_levels_noalloc(d_rp, d_col, n, root, out)
    torch.cuda.synchronize()
    return out.cpu().numpy(), want


def test_noalloc_levels_match_tc_count_on_consecutive_calls():
    s1, d1 = gen.rmat_edges(16, 16, 2)  # many components and isolated vertices
    n1 = 1 << 16
    g = tc.Graph(s1, d1, n1)
    root1 = g.max_degree_vertex()
    g.close()
    parts = [graphs.complete(9), graphs.wheel(12), graphs.path(30), graphs.cycle(7),
             graphs.star(40), graphs.complete(1), graphs.diag_grid(6, 9)]
    n2, s2, d2 = graphs.relabel(graphs.disjoint_union(*parts), 4)
    cases = [(s1, d1, n1, root1), (s2, d2, n2, 5), (s1, d1, n1, 777)]
    for src, dst, n, root in cases:
        got, want = _levels_both_ways(src, dst, n, root)
        assert np.array_equal(got, want)
        rp, col = oracle.build_csr(n, src, dst)
        assert np.array_equal(got, oracle.bfs_levels(rp, col, root))


def test_noalloc_rejects_oversized_graph():
    import torch
    dummy = torch.zeros(4, dtype=torch.int64, device="cuda")
    lv = torch.zeros(4, dtype=torch.int32, device="cuda")
    with pytest.raises(tc.TCError) as ei:
        tc.tc_bfs_levels_noalloc(dummy, dummy, (1 << 20) + 1, 0, lv)
    assert ei.value.status == 6  # TC_ERR_OVERFLOW, checked before any device work
    with pytest.raises(tc.TCError) as ei:
        tc.tc_bfs_levels_noalloc(dummy, dummy, 4, 4, lv)
    assert ei.value.status == 1  # root >= n

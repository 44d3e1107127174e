"""Serving loop: every answer equals the graph's count alone (GPU), and the
host-side admission respects the HBM budget (no GPU needed for the latter)."""
import numpy as np
import pytest

from paper_2403_02997_gb300 import gen


def test_footprint_grows_with_size():
    from paper_2403_02997_gb300.serve import footprint_bytes
    a = footprint_bytes(1000, 10_000)
    b = footprint_bytes(2000, 20_000)
    assert 0 < a < b < 3 * a


@pytest.mark.gpu
def test_results_alone_and_in_the_mix():
    import paper_2403_02997_gb300 as tc
    from paper_2403_02997_gb300 import build, serve
    build.build_all()
    specs = gen.batched_specs(48, master_seed=9, log2_min=6, log2_max=13)
    pool = [(*sp.edges(), sp.n, None if sp.root == "maxdeg" else 0) for sp in specs]
    alone = []
    for src, dst, n, root in pool:
        g = tc.Graph(src, dst, n)
        alone.append(g.count(g.max_degree_vertex() if root is None else root))
        g.close()
    budget = 3 * max(serve.footprint_bytes(n, s.size) for s, _, n, _ in pool)
    srv = serve.Server(hbm_budget_bytes=budget, max_batch=16)
    res = serve.run_arrivals(srv, pool, rate=2000.0, count=300, seed=3)
    srv.close()
    assert res["errors"] == 0
    for r in res["requests_list"]:
        idx = [i for i, p in enumerate(pool) if p[0] is r.src][0]
        assert r.count == alone[idx]
    assert srv.peak_used <= budget
    assert max(srv.batches) > 1          # requests were built and counted together
    assert res["p99_ms"] >= res["p50_ms"] > 0

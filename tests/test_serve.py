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


@pytest.mark.gpu
def test_device_memory_of_a_batch_within_footprint():
    """The device memory a request really takes (free-memory delta around one build and count
    of a group, with the pool keeping the build's peak reserved) stays within footprint_bytes,
    the bound admission charges against the HBM budget."""
    import torch

    import paper_2403_02997_gb300 as tc
    from paper_2403_02997_gb300 import build, serve
    build.build_all()
    specs = gen.batched_specs(32, master_seed=12, log2_min=8, log2_max=14)
    graphs = [(*sp.edges(), sp.n, None if sp.root == "maxdeg" else 0) for sp in specs]
    graphs += [(*gen.rmat_edges(17, 16, 30 + i), 1 << 17, None) for i in range(3)]
    reqs = [serve.Request(rid=i, src=s, dst=d, n=n, root=r) for i, (s, d, n, r) in enumerate(graphs)]
    backend = serve.GpuBackend()
    b, roots = backend.build(reqs[:4])       # warm-up: kernels loaded, pool and streams made
    backend.count(b, roots)
    backend.release(b)
    torch.cuda.synchronize()
    tc.pool_trim(0)
    torch.cuda.empty_cache()
    free0 = torch.cuda.mem_get_info()[0]
    b, roots = backend.build(reqs)
    counts = backend.count(b, roots)
    torch.cuda.synchronize()
    used = free0 - torch.cuda.mem_get_info()[0]
    reserved = tc.pool_reserved()
    backend.release(b)
    torch.cuda.synchronize()
    tc.pool_trim(0)
    assert len(counts) == len(reqs) and all(c >= 0 for c in counts)
    bound = sum(serve.footprint_bytes(r.n, int(r.src.size)) for r in reqs)
    assert 0 < used <= bound, (used, bound)
    assert reserved <= bound, (reserved, bound)


def test_overlap_of_intervals():
    from paper_2403_02997_gb300.serve import overlap_of
    r = overlap_of([(0.0, 2.0), (5.0, 6.0)], [(1.0, 3.0), (3.5, 5.5)])
    assert r["build_s"] == 3.0 and r["count_s"] == 4.0
    assert abs(r["overlap_s"] - 1.5) < 1e-12 and abs(r["build_overlap_frac"] - 0.5) < 1e-12
    assert overlap_of([], [(0.0, 1.0)])["overlap_s"] == 0.0


class OracleBackend:
    """A host stand-in for the device (the oracle counts each graph), so the
    serving loop's admission, grouping and answering run without a GPU."""

    def __init__(self, delay=0.002, fail_build=False):
        self.delay = delay
        self.fail_build = fail_build
        self.released = 0

    def build(self, group):
        import time
        time.sleep(self.delay)
        if self.fail_build:
            raise RuntimeError("build failed")
        return [(r.src, r.dst, r.n) for r in group], [r.root for r in group]

    def count(self, batch, roots):
        import time

        import oracle
        time.sleep(self.delay)
        out = []
        for s, d, n in batch:
            rp, col = oracle.build_csr(n, s, d)
            out.append(oracle.forward(rp, col))  # T does not depend on the root
        return out

    def release(self, batch):
        self.released += 1


def _pool(k=24):
    specs = gen.batched_specs(k, master_seed=7, log2_min=6, log2_max=10)
    return [(*sp.edges(), sp.n, None if sp.root == "maxdeg" else 0) for sp in specs]


def test_admission_respects_budget_and_answers_everything():
    import oracle
    from paper_2403_02997_gb300 import serve
    pool = _pool()
    want = []
    for s, d, n, _ in pool:
        rp, col = oracle.build_csr(n, s, d)
        want.append(oracle.forward(rp, col))
    budget = 3 * max(serve.footprint_bytes(n, s.size) for s, _, n, _ in pool)
    be = OracleBackend()
    srv = serve.Server(hbm_budget_bytes=budget, max_batch=6, backend=be)
    res = serve.run_arrivals(srv, pool, rate=20000.0, count=150, seed=2)
    srv.close()
    assert res["errors"] == 0 and len(srv.completed) == 150
    for r in res["requests_list"]:
        idx = [i for i, p in enumerate(pool) if p[0] is r.src][0]
        assert r.count == want[idx]
    assert 0 < srv.peak_used <= budget and srv.used == 0
    assert max(srv.batches) > 1 and max(srv.batches) <= 6      # grouped, never above max_batch
    assert be.released == len(srv.batches)
    assert res["p99_ms"] >= res["p50_ms"] > 0
    ov = srv.overlap_stats()          # every build and count interval was recorded
    assert ov["builds"] == ov["counts"] == len(srv.batches)
    assert 0.0 <= ov["overlap_s"] <= min(ov["build_s"], ov["count_s"])


def test_oversized_request_and_failed_build():
    from paper_2403_02997_gb300 import serve
    s, d, n, root = _pool(2)[1]
    small = serve.footprint_bytes(n, s.size)
    srv = serve.Server(hbm_budget_bytes=small - 1, backend=OracleBackend())
    r = srv.submit(serve.Request(rid=0, src=s, dst=d, n=n))
    assert r.event.is_set() and r.error and r.count is None
    srv.close()
    srv = serve.Server(hbm_budget_bytes=4 * small, backend=OracleBackend(fail_build=True))
    r = srv.submit(serve.Request(rid=1, src=s, dst=d, n=n))
    assert r.event.wait(10) and r.error == "build failed"
    srv.close()
    assert srv.used == 0

"""Host logic of bench.py on CPU: the CPU-baseline sampler and the reference arm."""
import json
import os
import subprocess
import sys

import numpy as np

import bench
import oracle
from paper_2403_02997_gb300 import gen

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_sampler_baselines():
    """One sample times both oracle forms; each full-graph estimate is the BFS and scan time
    plus the sampled seconds per cover edge times |S|, and the OpenMP form reports the host's
    thread count."""
    spec = gen.rmat_spec(12, 16, 5)
    src, dst = spec.edges()
    sam = bench.OracleSampler(spec, src, dst, 0, target_s=0.5)
    r = sam.step()
    lv = oracle.bfs_levels(sam.rp, sam.col, 0)
    assert r["num_cover"] == oracle.cetc(sam.rp, sam.col, lv)["num_cover"]
    for name, cores in (("seq", 1), ("omp", oracle.num_threads())):
        b = r[name]
        assert b["cores"] == cores and b["sampled_edges"] > 0 and b["sample_s"] > 0
        est = r["bfs_s"] + r["scan_s"] + b["sample_s"] / b["sampled_edges"] * r["num_cover"]
        assert abs(b["est_full_seconds"] - est) <= 1e-9 * est
        assert abs(b["value"] - sam.m / est) <= 1e-9 * b["value"]
    base = sam.baseline(r)
    assert base["kind"] == "oracle" and base["value"] == r["omp"]["value"]
    assert base["seq"]["cores"] == 1 and base["sample_wall_s"] >= r["omp"]["sample_s"]


def test_estimate_validation_runs():
    spec = gen.rmat_spec(12, 16, 5)
    src, dst = spec.edges()
    v = bench.validate_cpu_estimate(spec, src, dst, 0, 0.3)
    rp, col = oracle.build_csr(spec.n, src, dst)
    assert v["triangles"] == oracle.forward(rp, col)     # the full run counts every triangle
    assert v["full_seconds"] > 0 and v["estimated_seconds"] > 0
    assert v["relative_error"] == (v["estimated_seconds"] - v["full_seconds"]) / v["full_seconds"]


def test_reference_arm_line():
    r = subprocess.run([sys.executable, "bench.py", "--impl", "reference", "--workload", "rmat16",
                        "--steps", "1", "--warmup", "1"], capture_output=True, text=True,
                       timeout=600, cwd=ROOT)
    assert r.returncode == 0, r.stderr[-2000:]
    line = json.loads([x for x in r.stdout.splitlines() if x.startswith("{")][-1])
    assert line["impl"] == "reference" and line["unit"] == "edges/s" and line["value"] > 0
    assert line["cpu_baseline"]["kind"] == "oracle" and line["cpu_baseline"]["cores"] >= 1
    assert line["e2e"]["h2d_bytes_per_step"] == 0 and line["metric"] == bench.METRIC
    # the step time is the sample's measured wall time, the extrapolation is reported apart
    assert line["est_full_seconds"] > 0 and line["ms_per_step"] > 0
    assert abs(line["value"] - line["cpu_baseline"]["value"]) <= 1e-9 * line["value"]
    assert {"seq", "omp"} <= set(line["cpu_baseline"])


def test_hash_kernel_bytes_against_brute_force():
    """The roofline's algorithmic-byte model of the owner-hash kernel, recounted edge by edge:
    each owner-path cover edge streams the streamer's other-level neighbours and its same-level
    neighbours above v, and each owner's row is read once per work item."""
    import math
    spec = gen.rmat_spec(10, 16, 3)
    s, d = spec.edges()
    rp, col = oracle.build_csr(spec.n, s, d)
    root = oracle.max_degree_root(rp)
    lv = oracle.bfs_levels(rp, col, root)
    ref = oracle.count(spec.n, s, d, root, want_cover=True)
    assert np.array_equal(ref["level"], lv)
    cu, cv = ref["cover_u"].astype(np.int64), ref["cover_v"].astype(np.int64)
    deg = np.diff(rp.astype(np.int64))
    nbrs = [col[rp[x]:rp[x + 1]].astype(np.int64) for x in range(spec.n)]
    for smax, per_item in ((0, 3), (8, 512), (32, 7)):
        hb = bench.hash_kernel_bytes(rp, col, lv, ref["cover_u"], ref["cover_v"],
                                     {"small_max_degree": smax, "edges_per_item": per_item})
        streamed = edges = 0
        per_edge_bytes = 0
        owner_edges = {}
        for u, v in zip(cu.tolist(), cv.tolist()):
            if deg[u] <= smax and deg[v] <= smax:
                continue
            h, x = (v, u) if (deg[v] > deg[u] or (deg[v] == deg[u] and v > u)) else (u, v)
            vm = max(u, v)
            nx = nbrs[x]
            k = int(np.sum(lv[nx] != lv[x]) + np.sum((lv[nx] == lv[x]) & (nx > vm)))
            streamed += k
            edges += 1
            per_edge_bytes += 4 * k + 32 + 4 * math.ceil(math.log2(max(int(deg[x]), 2)))
            owner_edges[h] = owner_edges.get(h, 0) + 1
        items = sum(-(-c // per_item) for c in owner_edges.values())
        per_owner = sum(-(-c // per_item) * (4 * int(deg[h]) + 32) for h, c in owner_edges.items())
        assert hb["streamed_elements"] == streamed and hb["edges"] == edges
        assert hb["items"] == items and hb["bytes"] == per_edge_bytes + per_owner

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


def test_threaded_sample_equals_one_call():
    """The sampler's threads each run the oracle's edge loop on a slice of the
    sample; their sum is the single-call count (and, over all of S, T)."""
    spec = gen.rmat_spec(12, 16, 5)
    src, dst = spec.edges()
    one = bench.OracleSampler(spec, src, dst, 0, target_s=1.0, cores=1)
    many = bench.OracleSampler(spec, src, dst, 0, target_s=1.0, cores=4)
    lv = oracle.bfs_levels(one.rp, one.col, 0)
    cov = oracle.cetc(one.rp, one.col, lv, want_cover=True)
    us, vs = cov["cover_u"], cov["cover_v"]
    assert one._edges(lv, us, vs) == many._edges(lv, us, vs) == cov["T"]
    idx = np.random.default_rng(3).integers(0, us.size, 999)
    assert one._edges(lv, us[idx], vs[idx]) == many._edges(lv, us[idx], vs[idx])
    r = many.step()
    assert r["edges"] == one.m and r["est_seconds"] > 0 and r["done"] > 0


def test_reference_arm_line():
    r = subprocess.run([sys.executable, "bench.py", "--impl", "reference", "--workload", "rmat16",
                        "--steps", "1", "--warmup", "1"], capture_output=True, text=True,
                       timeout=600, cwd=ROOT)
    assert r.returncode == 0, r.stderr[-2000:]
    line = json.loads([x for x in r.stdout.splitlines() if x.startswith("{")][-1])
    assert line["impl"] == "reference" and line["unit"] == "edges/s" and line["value"] > 0
    assert line["cpu_baseline"]["kind"] == "oracle" and line["cpu_baseline"]["cores"] >= 1
    assert line["e2e"]["h2d_bytes_per_step"] == 0 and line["metric"] == bench.METRIC

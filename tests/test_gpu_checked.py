"""The checked build (-DTC_CHECKED) on the GPU (needs a GB300).

In the checked build the kernels test the preconditions of their
data-dependent accesses (vertex ids below n, row ranges inside the CSR, bucket
positions inside their bucket) and report a failure as TC_ERR_CUDA instead of
touching bad memory; it stands in for a memory checker.  On valid graphs no
check may fire and every count must still equal the oracle's.  The library is
loaded in a child process, so this process keeps the normal build.
"""
import os
import subprocess
import sys

import pytest

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

CHILD = r"""
import sys
sys.path.insert(0, ROOT)
import numpy as np
import oracle
import paper_2403_02997_gb300 as tc
from paper_2403_02997_gb300 import gen
from tests import graphs
tc.load_library(LIB)
cases = [graphs.complete(9), graphs.wheel(12), graphs.diag_grid(6, 7)]
for seed in (1, 2):
    s, d = gen.er_edges(1200, 15000, seed)
    cases.append((1200, s, d))
s, d = gen.rmat_edges(13, 16, 3)
cases.append((1 << 13, s, d))
params = [{}, dict(small_max_degree=0, hash_chunk=32, edges_per_item=3),
          dict(small_max_degree=0, hash_block=1024, hash_chunk=64, edges_per_item=700)]
for n, s, d in cases:
    rp, col = oracle.build_csr(n, s, d)
    root = oracle.max_degree_root(rp)
    lv = oracle.bfs_levels(rp, col, root)
    ref = oracle.cetc(rp, col, lv)
    for p in params:
        g = tc.Graph(s, d, n)
        g.set_params(**p)
        assert g.count(root) == ref["T"]
        st = g.stats()
        assert (st["c1"], st["c2"]) == (ref["c1"], ref["c2"])
        assert g.count_split(root) == ref["T"]
        assert g.count_forward() == ref["T"]
        assert g.list_triangles(root)[0] == ref["T"]
        g.close()
print("checked build ok", len(cases))
"""


def test_checked_build_counts_match_oracle():
    from paper_2403_02997_gb300 import build
    lib = build.build(checked=True)
    code = CHILD.replace("ROOT", repr(ROOT)).replace("LIB", repr(lib))
    r = subprocess.run([sys.executable, "-c", code], capture_output=True, text=True, timeout=900,
                       cwd=ROOT)
    assert r.returncode == 0, r.stdout[-2000:] + r.stderr[-4000:]
    assert "checked build ok" in r.stdout

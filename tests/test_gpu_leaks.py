"""Device memory is returned (needs a GB300).

Handles own all their device memory (counts allocate only the work-item table
and, for the forward and split counts, the oriented adjacency, inside the
handle); destroying a handle frees it.  After a warm-up round, repeated rounds
of create / every count / relabel / batch / destroy leave the device's free
memory where it was.
"""
import numpy as np
import pytest

import paper_2403_02997_gb300 as tc
from paper_2403_02997_gb300 import gen

pytestmark = pytest.mark.gpu


def _round(s, d, n):
    g = tc.Graph(s, d, n)
    r = g.max_degree_vertex()
    T = g.count(r)
    assert g.count_split(r) == T and g.count_forward() == T
    assert g.count_fe(r, 0.0)[0] == T
    assert g.list_triangles(r)[0] == T
    g2, _ = g.relabel_degree()
    assert g2.count(0) == T
    g2.close()
    b = tc.Batch([g])
    assert b.count([r]) == [T]
    b.close()
    g.close()


def test_no_device_memory_leak():
    import torch
    s, d = gen.rmat_edges(15, 16, 9)
    n = 1 << 15
    _round(s, d, n)  # warm-up: module loading, pinned staging
    torch.cuda.synchronize()
    torch.cuda.empty_cache()
    free0 = torch.cuda.mem_get_info()[0]
    for _ in range(4):
        _round(s, d, n)
    torch.cuda.synchronize()
    torch.cuda.empty_cache()
    free1 = torch.cuda.mem_get_info()[0]
    assert abs(free0 - free1) <= 16 << 20, (free0, free1)

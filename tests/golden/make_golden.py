"""Write the stored expected values for the full-size single-graph workloads.

Calls only the oracle (and the shared input generators).  Output:
tests/golden/<name>.json with the edge-list checksum (so a run on another
machine can confirm it generated the same input), n, m, the max-degree root,
the root's level count, |S| and the triangle count from two oracle routines:
Algorithm Forward with degree ordering (independent of BFS) and Algorithm
CETC-SM (c1, c2, T = c1 + c2 / 3).  It also stores SHA-256 digests of the
oracle's CSR (row_ptr as int64, col as uint32), of its level array (int32) and
of its cover-edge set (keys u << 32 | v, ascending, uint64), all little-endian,
so a full-size run can be compared element by element without re-running the
oracle.

    python tests/golden/make_golden.py rmat24      # R-MAT scale 24, ef 16, seed 2
    python tests/golden/make_golden.py er1024      # ER G(1024, 8192), seed 1
"""
import hashlib
import json
import os
import sys
import time

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

import oracle  # noqa: E402
from paper_2403_02997_gb300 import gen  # noqa: E402

SPECS = {"rmat24": gen.RMAT_24, "er1024": gen.ER_1024, "rmat16": gen.rmat_spec(16, 16, 2)}


def edge_checksum(src, dst) -> str:
    key = (src.astype(np.uint64) << np.uint64(32)) | dst.astype(np.uint64)
    mix = key * np.uint64(0x9E3779B97F4A7C15)
    return "%016x:%016x" % (int(np.bitwise_xor.reduce(mix)), int(mix.sum(dtype=np.uint64)))


def digest(*arrays) -> str:
    h = hashlib.sha256()
    for a in arrays:
        h.update(np.ascontiguousarray(a).astype(a.dtype.newbyteorder("<"), copy=False).tobytes())
    return h.hexdigest()


def main(name):
    spec = SPECS[name]
    t0 = time.time()
    src, dst = spec.edges()
    rp, col = oracle.build_csr(spec.n, src, dst)
    root = oracle.max_degree_root(rp) if spec.root == "maxdeg" else 0
    lv = oracle.bfs_levels(rp, col, root)
    t1 = time.time()
    fwd = oracle.forward(rp, col)
    t2 = time.time()
    sm = oracle.cetc_sm(rp, col, lv)
    t3 = time.time()
    assert sm["T"] == fwd, (sm, fwd)
    cov = oracle.cetc(rp, col, lv, stride=1 << 62, want_cover=True)
    keys = (cov["cover_u"].astype(np.uint64) << np.uint64(32)) | cov["cover_v"].astype(np.uint64)
    comp = np.diff(rp) > 0
    out = dict(name=name, family=spec.family, n=spec.n, draws=int(src.size), seed=spec.seed,
               edge_checksum=edge_checksum(src, dst), m=int(col.size // 2),
               d_max=int(np.diff(rp).max()) if spec.n else 0, root=root,
               max_level=int(lv.max()) if spec.n else 0,
               num_cover=int(cov["num_cover"]), T=int(fwd), c1=sm["c1"], c2=sm["c2"],
               nonisolated=int(comp.sum()),
               csr_sha256=digest(rp.astype(np.int64), col.astype(np.uint32)),
               level_sha256=digest(lv.astype(np.int32)),
               cover_sha256=digest(keys),
               seconds=dict(build_bfs=round(t1 - t0, 1), forward=round(t2 - t1, 1),
                            cetc_sm=round(t3 - t2, 1), threads=oracle.num_threads()))
    with open(os.path.join(HERE, name + ".json"), "w") as f:
        json.dump(out, f, indent=1)
        f.write("\n")
    print(json.dumps(out))


if __name__ == "__main__":
    for nm in sys.argv[1:]:
        main(nm)

"""Autotuner for the count's tunables (tc_params).

The tunables change speed only, never the count:
- ``small_max_degree``: degree bound of the inline-merge bin;
- ``medium_max_degree``: degree bound of the warp-merge bin;
- ``hash_block``: threads per owner-hash block (512, or 1024 with one block per SM);
- ``hash_chunk``: owner-row entries per shared-memory table;
- ``edges_per_item``: cover edges per owner-hash work item (up to 2x a 512-thread block, 4x a
  1024-thread one);
- ``bfs_alpha`` / ``bfs_beta``: the direction switches of the BFS.

``tune`` runs a coordinate descent. It starts from the defaults and, one parameter at a time, tries
each candidate value. The block size, chunk and item length only pay off together (a 1024-thread
block wants longer chunks and items than a 512-thread one), so one coordinate, ``shape``, moves the
three at once through ``SHAPES`` before each is refined alone. A value is kept only if the measured total time drops by more than
``min_gain``. Every candidate's count must equal the default's. Times are the library's own
CUDA-event totals (``ms_total`` of tc_stats), and the best of ``trials`` runs is kept.

Results are cached in a JSON table keyed by a workload signature: family, log2 n, log2 m,
log2 d_max, and batch size. ``lookup`` returns the tuned parameters for a signature, or None.

``learn_fe_threshold`` learns Algorithm CETC-Seq-FE's switch point for a graph family: the
variant takes the forward count when the covering ratio c = |S| / m after the BFS is at least
the threshold (the paper fixes 0.7). It times the cover-edge count and the forward count on a
graph of the family and puts the threshold just below that graph's c when the forward count
was faster, just above it otherwise; ``lookup_fe`` returns it for a signature.
"""
from __future__ import annotations

import json
import math
import os
import time
from typing import Dict, Iterable, Optional, Sequence

HERE = os.path.dirname(os.path.abspath(__file__))
CACHE = os.path.join(HERE, "tuned_params.json")

GRID: Dict[str, Sequence[int]] = {
    "hash_block": (512, 1024),
    "hash_chunk": (2048, 4096, 8192, 12288, 16384),
    "edges_per_item": (64, 128, 256, 512, 1024, 2048, 4096),
    "small_max_degree": (0, 8, 16, 32, 64, 128, 256, 512, 1024),
    "medium_max_degree": (0, 128, 256, 512, 1024),
    "bfs_alpha": (4, 15, 40),
    "bfs_beta": (8, 18, 48),
}
SHAPES = (
    {"hash_block": 512, "hash_chunk": 8192, "edges_per_item": 1024},
    {"hash_block": 1024, "hash_chunk": 12288, "edges_per_item": 4096},
    {"hash_block": 1024, "hash_chunk": 16384, "edges_per_item": 1024},
)
ORDER = ("small_max_degree", "medium_max_degree", "shape", "hash_block", "hash_chunk",
         "edges_per_item", "small_max_degree", "bfs_alpha", "bfs_beta")


def signature(n: int, m: int, d_max: int, family: str = "", batch: int = 1) -> str:
    lg = lambda x: int(round(math.log2(max(int(x), 1))))
    return f"{family or 'graph'}:n{lg(n)}:m{lg(m)}:d{lg(d_max)}:k{lg(batch)}"


def _measure(target, roots, params: dict, trials: int):
    target.set_params(**params)
    best, count = float("inf"), None
    for _ in range(trials):
        c = target.count(roots)
        st = target.stats()
        best = min(best, float(st["ms_total"]))
        if count is None:
            count = c
        elif c != count:
            raise RuntimeError("count changed between runs of one parameter set")
    return best, count


def tune(target, roots, grid: Optional[Dict[str, Iterable[int]]] = None, trials: int = 2,
         min_gain: float = 0.02, time_budget_s: float = 120.0,
         shapes: Optional[Sequence[dict]] = None) -> dict:
    """Coordinate descent over `grid` (and the joint `shapes`) for a tc.Graph (roots: int) or
    tc.Batch (roots: list)."""
    from paper_2403_02997_gb300 import tc_params_default
    if grid is None:  # the default search includes the joint shapes
        grid, shapes = dict(GRID), SHAPES if shapes is None else shapes
    else:
        grid, shapes = dict(grid), shapes or ()
    base = {k: v for k, v in tc_params_default().items()
            if k in ("small_max_degree", "medium_max_degree", "hash_block", "hash_chunk",
                     "edges_per_item", "bfs_alpha", "bfs_beta")}
    t0 = time.time()
    best_ms, want = _measure(target, roots, base, trials)
    history = [{"params": dict(base), "ms": best_ms}]
    cur = dict(base)
    for name in ORDER:
        if name == "shape":
            moves = [dict(m) for m in shapes if set(m) <= set(cur)]
        elif name not in grid or name not in cur:  # not a tunable of this library
            continue
        else:
            moves = [{name: int(v)} for v in grid[name]]
        for mv in moves:
            if all(cur[k] == v for k, v in mv.items()) or time.time() - t0 > time_budget_s:
                continue
            cand = dict(cur)
            cand.update(mv)
            try:
                ms, got = _measure(target, roots, cand, trials)
            except Exception as e:  # a value the library rejects is skipped
                history.append({"params": cand, "error": str(e)})
                continue
            if got != want:
                raise RuntimeError(f"count differs under {cand}: {got} != {want}")
            history.append({"params": cand, "ms": ms})
            if ms < best_ms * (1.0 - min_gain):
                best_ms, cur = ms, cand
    target.set_params(**cur)
    return {"params": cur, "ms": best_ms, "default_ms": history[0]["ms"], "history": history,
            "seconds": time.time() - t0}


def learn_fe_threshold(graph, root, trials: int = 2, margin: float = 0.05) -> dict:
    """CETC-Seq-FE's threshold for the family of `graph` (a tc.Graph, or any object with
    count(root), count_forward(), stats() and m)."""
    def best(fn):
        ms, val = float("inf"), None
        for _ in range(trials):
            v = fn()
            if val is not None and v != val:
                raise RuntimeError("count changed between runs")
            val = v
            ms = min(ms, float(graph.stats()["ms_total"]))
        return ms, val
    ms_cetc, t_cetc = best(lambda: graph.count(root))
    c = graph.stats()["num_cover"] / max(int(graph.m), 1)
    ms_fwd, t_fwd = best(lambda: graph.count_forward())
    if t_fwd != t_cetc:
        raise RuntimeError(f"forward count {t_fwd} != cover-edge count {t_cetc}")
    forward_wins = ms_fwd < ms_cetc
    thr = c * (1.0 - margin) if forward_wins else c * (1.0 + margin)
    return {"threshold": thr, "covering_ratio": c, "ms_cetc": ms_cetc, "ms_forward": ms_fwd,
            "forward_faster": forward_wins}


def store_fe(sig: str, fe: dict, path: str = CACHE) -> None:
    table = load_cache(path)
    table.setdefault(sig, {})["fe"] = fe
    with open(path, "w") as f:
        json.dump(table, f, indent=1, sort_keys=True)
        f.write("\n")


def lookup_fe(sig: str, path: str = CACHE) -> Optional[float]:
    entry = load_cache(path).get(sig, {}).get("fe")
    return None if entry is None else float(entry["threshold"])


def load_cache(path: str = CACHE) -> dict:
    if os.path.exists(path):
        with open(path) as f:
            return json.load(f)
    return {}


def store(sig: str, result: dict, path: str = CACHE) -> None:
    table = load_cache(path)
    table.setdefault(sig, {}).update({"params": result["params"], "ms": result["ms"],
                                      "default_ms": result["default_ms"]})
    with open(path, "w") as f:
        json.dump(table, f, indent=1, sort_keys=True)
        f.write("\n")


def lookup(sig: str, path: str = CACHE) -> Optional[dict]:
    entry = load_cache(path).get(sig)
    return None if entry is None or "params" not in entry else dict(entry["params"])


if __name__ == "__main__":
    # Tune the named single-graph workloads and the batched one on this GPU.
    import argparse

    import numpy as np
    import torch

    import paper_2403_02997_gb300 as tc
    from paper_2403_02997_gb300 import build, gen

    ap = argparse.ArgumentParser()
    ap.add_argument("workloads", nargs="*", default=["rmat24", "batched"])
    ap.add_argument("--trials", type=int, default=2)
    ap.add_argument("--budget", type=float, default=150.0)
    ap.add_argument("--out", default=CACHE, help="table to update (default: the package's)")
    ap.add_argument("--fe", action="store_true",
                    help="learn CETC-Seq-FE's threshold for single-graph workloads (no descent)")
    args = ap.parse_args()
    build.build_all()
    specs = {"rmat24": gen.RMAT_24, "rmat22": gen.rmat_spec(22, 16, 2), "mesh4096": gen.MESH_4096,
             "er1024": gen.ER_1024}
    for w in args.workloads:
        if w == "batched":
            sp = gen.batched_specs()
            gs = [tc.Graph(*s.edges(), s.n) for s in sp]
            roots = [g.max_degree_vertex() if s.root == "maxdeg" else 0 for g, s in zip(gs, sp)]
            target = tc.Batch(gs)
            sig = signature(sum(s.n for s in sp), sum(g.m for g in gs), max(g.d_max for g in gs),
                            "batched", len(gs))
            for g in gs:
                g.close()
        else:
            s = specs[w]
            src, dst = s.edges()
            target = tc.Graph(torch.from_numpy(src.view(np.int32)).cuda(),
                              torch.from_numpy(dst.view(np.int32)).cuda(), s.n)
            roots = target.max_degree_vertex() if s.root == "maxdeg" else 0
            sig = signature(s.n, target.m, target.d_max, s.family)
        if args.fe and w != "batched":
            tuned = lookup(sig, args.out)  # CETC-Seq as it runs: with its tuned parameters
            if tuned:
                target.set_params(**tuned)
            fe = learn_fe_threshold(target, roots, trials=args.trials)
            store_fe(sig, fe, args.out)
            print(json.dumps({"workload": w, "signature": sig, "fe": fe}), flush=True)
            target.close()
            continue
        res = tune(target, roots, trials=args.trials, time_budget_s=args.budget)
        store(sig, res, args.out)
        print(json.dumps({"workload": w, "signature": sig, "params": res["params"],
                          "ms": res["ms"], "default_ms": res["default_ms"],
                          "seconds": round(res["seconds"], 1)}), flush=True)
        target.close()

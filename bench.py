#!/usr/bin/env python3
"""Benchmark: cover-edge triangle counting on one GB300 (per rank).

Default workload: R-MAT scale 24 (2^24 vertices, edge factor 16, a=0.57
b=0.19 c=0.19 d=0.05, ids permuted, seed 2), BFS root = the smallest id of
largest degree.  One step = one tc_count on the device-resident CSR: BFS levels,
restarts, cover-edge extraction, intersections and the reduction, ending with
the count read back to the host.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--workload rmat24|er1024|mesh4096]
  python bench.py --impl reference ...   # the CPU oracle on bounded samples

Prints one JSON line (rank 0).  value = input edges/s (undirected edges after
canonicalising, summed over ranks, / the slowest rank's time).  With N > 1 each
rank counts its own replica graph (seed + rank): weak scaling, no collective on
the data path; only the timing uses a barrier and a max-reduction.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import math
import os
import statistics
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

from paper_2403_02997_gb300 import gen  # noqa: E402

WORKLOADS = {"rmat24": gen.RMAT_24, "er1024": gen.ER_1024, "mesh4096": gen.MESH_4096,
             # smaller cases of the same family, for profiling captures
             "rmat21": gen.rmat_spec(21, 16, 2), "rmat22": gen.rmat_spec(22, 16, 2),
             "rmat23": gen.rmat_spec(23, 16, 2),
             "rmat16": gen.rmat_spec(16, 16, 2)}
METRIC = "input edges/s (exact triangle count, tc_count on device-resident CSR)"
L2_BYTES = 129 * 2**20


def parse_args():
    p = argparse.ArgumentParser()
    p.add_argument("--gpus", type=int, default=1)
    p.add_argument("--steps", type=int, default=10)
    p.add_argument("--warmup", type=int, default=3)
    p.add_argument("--impl", choices=["ours", "reference"], default="ours")
    p.add_argument("--workload", choices=sorted(WORKLOADS) + ["batched", "serve"], default="rmat24")
    p.add_argument("--serve-requests", type=int, default=2000,
                   help="requests per arrival-rate point of the serving sweep")
    p.add_argument("--serve-budget-gb", type=float, default=96.0)
    p.add_argument("--batch-graphs", type=int, default=4096)
    p.add_argument("--no-tuned", action="store_true",
                   help="ignore the autotuner's table (paper_2403_02997_gb300/tuned_params.json)")
    p.add_argument("--params", default="",
                   help="JSON object of tc_params fields set after the tuned ones (single-graph "
                        "workloads), e.g. to profile a small graph with the headline's settings")
    p.add_argument("--cpu-seconds", type=float, default=15.0,
                   help="target seconds of oracle intersection work in the CPU baseline sample")
    p.add_argument("--no-cpu-baseline", action="store_true")
    p.add_argument("--e2e-steps", type=int, default=3)
    p.add_argument("--create-steps", type=int, default=3,
                   help="timed tc_graph_create calls from device-resident edges")
    p.add_argument("--no-extra", action="store_true",
                   help="R-MAT 24 headline only: skip the mesh, batched and serving keys")
    p.add_argument("--serve-requests-extra", type=int, default=1000,
                   help="requests per arrival-rate point of the serving key in the default line")
    p.add_argument("--cpu-validate", action="store_true",
                   help="time the full OpenMP oracle count and compare it with the sampled "
                        "estimate (CPU only)")
    return p.parse_args()


# ----------------------------------------------------------------------------
# distributed plumbing (replicas only)
# ----------------------------------------------------------------------------

def dist_setup(args=None):
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        import torch
        import torch.distributed as dist
        backend = "nccl" if torch.cuda.is_available() else "gloo"
        if torch.cuda.is_available():
            torch.cuda.set_device(local)
        dist.init_process_group(backend=backend)
    return world, rank, local


def barrier(world):
    if world > 1:
        import torch.distributed as dist
        dist.barrier()


def max_over_ranks(x: float, world: int) -> float:
    if world == 1:
        return x
    import torch
    import torch.distributed as dist
    dev = torch.device("cuda") if torch.cuda.is_available() else torch.device("cpu")
    t = torch.tensor([x], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def sum_over_ranks(x: float, world: int) -> float:
    if world == 1:
        return x
    import torch
    import torch.distributed as dist
    dev = torch.device("cuda") if torch.cuda.is_available() else torch.device("cpu")
    t = torch.tensor([x], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.SUM)
    return float(t.item())


def replica_spec(spec, rank):
    if rank == 0:
        return spec
    from dataclasses import replace
    return replace(spec, seed=spec.seed + 1000 * rank)


# ----------------------------------------------------------------------------
# clocks during the timed region
# ----------------------------------------------------------------------------

class ClockSampler:
    QUERY = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.proc = None
        self.path = None

    def start(self):
        fd, self.path = tempfile.mkstemp(suffix=".csv")
        os.close(fd)
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.QUERY}",
                 "--format=csv,noheader,nounits", "-lms", "100"],
                stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except OSError:
            self.proc = None
        time.sleep(0.3)

    def stop(self) -> dict:
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        time.sleep(0.15)
        self.proc.terminate()
        self.proc.wait()
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in open(self.path):
            f = [x.strip() for x in line.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                smax.append(float(f[2]))
            except ValueError:
                continue
            for nm, val in zip(names, f[5:9]):
                if val.lower().startswith("active"):
                    reasons.add(nm)
        os.unlink(self.path)
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(smax) if smax else None,
                "reasons": sorted(reasons), "samples": len(sm)}


def measured_peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(path):
        d = json.load(open(path))
        return float(d["hbm_gbs"]), "measured"
    return 6800.0, "fallback"


# ----------------------------------------------------------------------------
# algorithmic bytes of the owner-hash kernel
# ----------------------------------------------------------------------------

SPLIT_MAX = 1 << 62  # every row is streamed level-split


def hash_kernel_bytes(rp, col, level, cu, cv, params) -> dict:
    """Bytes the owner-hash kernel must move, from the graph, levels and cover set.

    Per owner-path cover edge {h, x} (h the owner: larger degree, ties larger id;
    x the streamer), with v = max(h, x): the elements of N(x) that can count --
    its neighbours on another level plus its same-level neighbours above v (the
    whole row if d(x) > SPLIT_MAX) -- 4 bytes each, plus its bucket entry (4),
    x's row offsets and split point (24) and the binary search for v (4 log2 d).
    Per work item (owner h, slice of its cover edges): the row N(h) (4 per entry)
    and the owner's offsets (32).
    """
    n = rp.size - 1
    deg = np.diff(rp.astype(np.int64))
    du = deg[cu].astype(np.int64)
    dv = deg[cv].astype(np.int64)
    smax = params["small_max_degree"]
    large = ~((du <= smax) & (dv <= smax))
    u = cu[large].astype(np.int64)
    v = cv[large].astype(np.int64)
    du, dv = du[large], dv[large]
    v_owns = (dv > du) | ((dv == du) & (v > u))
    owner = np.where(v_owns, v, u)
    x = np.where(v_owns, u, v)
    vmax = np.maximum(u, v)
    # same-level neighbours of every vertex as a sorted key list (row << 32 | id)
    rows = np.repeat(np.arange(n, dtype=np.int64), deg)
    same = level[rows] == level[col]
    keys = (rows[same] << 32) | col[same].astype(np.int64)
    same_deg = np.bincount(rows[same], minlength=n).astype(np.int64)
    del rows, same
    start = np.searchsorted(keys, x << 32)
    upto_v = np.searchsorted(keys, (x << 32) | (vmax + 1))
    above = same_deg[x] - (upto_v - start)
    dx = deg[x]
    streamed = np.where(dx > SPLIT_MAX, dx, (dx - same_deg[x]) + above)
    log_d = np.ceil(np.log2(np.maximum(dx, 2)))
    per_edge = 4 * streamed + 32 + 4 * log_d.astype(np.int64)
    owners, oc = np.unique(owner, return_counts=True)
    dh = deg[owners]
    per_item = params["edges_per_item"]
    slices = (oc + per_item - 1) // per_item
    per_owner = slices * (4 * dh + 32)
    return {"bytes": int(per_edge.sum() + per_owner.sum()), "edges": int(large.sum()),
            "items": int(slices.sum()), "streamed_elements": int(streamed.sum()),
            "row_elements": int(dx.sum())}


def kernel_source_sha() -> str:
    h = hashlib.sha256()
    for f in ["count.cu"]:
        h.update(open(os.path.join(ROOT, "paper_2403_02997_gb300", "csrc", f), "rb").read())
    return h.hexdigest()[:16]


def profiled_traffic(workload: str):
    """DRAM bytes per launch of the owner-hash kernel from the committed ncu summary.

    Returns (bytes or None, stale): stale is True when a summary exists but was taken on
    another revision of the kernel source, so its bytes no longer describe this kernel.
    """
    path = os.path.join(ROOT, "profiles", f"owner_hash_{workload}.json")
    if not os.path.exists(path):
        return None, False
    d = json.load(open(path))
    if d.get("source_sha") != kernel_source_sha():
        return None, True
    return d.get("dram_bytes_per_launch"), False


# ----------------------------------------------------------------------------
# CPU oracle timing (bounded sample)
# ----------------------------------------------------------------------------

class OracleSampler:
    """Times the oracle, as it stands, on a bounded sample of the workload.

    The graph is built by the oracle (not timed, as tc_graph_create is not in
    the GPU step).  One sample (`step`) times, on this host:

    * the oracle BFS over the whole graph with its restarts (one thread);
    * its cover-edge scan: the CETC-Seq edge loop with the intersections
      sampled out (orc_cetc with a stride beyond |S|; one thread);
    * the per-edge intersections of a seeded sample of S (random runs of 512
      consecutive cover edges, so the sample keeps the full loop's row locality),
      twice: ``seq``, the literal CETC-Seq edge loop on one thread (orc_cetc_edges),
      and ``omp``, Algorithm CETC-SM's parallel edge loop on all host threads
      (orc_cetc_sm_edges).  Each sample grows geometrically until it has used
      about its time budget.

    The full-graph time of each baseline is estimated as
    bfs + scan + (sample seconds / sampled edges) x |S|; `wall` is what the
    sample itself took.  Counts of the sampled edges are not used (the GPU arm
    checks its count against the oracle elsewhere).
    """

    def __init__(self, spec, src, dst, root, target_s, seed=11):
        import oracle
        self.o = oracle
        self.rp, self.col = oracle.build_csr(spec.n, src, dst)
        self.m = int(self.col.size // 2)
        self.root = root
        self.target_s = max(float(target_s), 0.2)
        self.rng = np.random.default_rng(seed)
        self.cores = int(oracle.num_threads())
        self.num_cover = None

    def _sample(self, fn, lv, cov, budget, cores):
        """Grows a uniform sample of S until about `budget` seconds.

        Returns (edges, seconds) of the batches that kept every thread busy (at least 1024 edges
        per thread), or of all batches when none did: the first, small batches mostly time the
        threads' start-up, which would bias the per-edge time upwards.
        """
        S = self.num_cover
        done, spent, k = 0, 0.0, 64
        batches = []
        run = 512  # consecutive cover edges per pick: the full loop's row locality is kept
        while S and spent < budget and done < 4 * S:
            k = min(k, S)
            starts = self.rng.integers(0, max(S - run, 0) + 1, size=max(1, k // run))
            idx = (starts[:, None] + np.arange(min(run, S))[None, :]).ravel()[:max(k, 1)]
            k = idx.size
            us, vs = cov["cover_u"][idx], cov["cover_v"][idx]
            t = time.perf_counter()
            fn(self.rp, self.col, lv, us, vs)
            dt = time.perf_counter() - t
            batches.append((k, dt))
            spent += dt
            done += k
            k = int(k * min(4.0, max(1.5, (budget - spent) / max(dt, 1e-6))))
        full = [(k_, t_) for k_, t_ in batches if k_ >= 1024 * cores] or batches
        return sum(k_ for k_, _ in full), sum(t_ for _, t_ in full)

    def step(self) -> dict:
        t0 = time.perf_counter()
        lv = self.o.bfs_levels(self.rp, self.col, self.root)
        t_bfs = time.perf_counter() - t0
        t = time.perf_counter()
        cov = self.o.cetc(self.rp, self.col, lv, stride=1 << 62, want_cover=True)
        t_scan = time.perf_counter() - t
        self.num_cover = S = cov["num_cover"]
        out = {"edges": self.m, "num_cover": S, "bfs_s": t_bfs, "scan_s": t_scan}
        for name, fn, share in (("seq", self.o.cetc_edges, 0.4), ("omp", self.o.cetc_sm_edges, 0.6)):
            done, spent = self._sample(fn, lv, cov, share * self.target_s,
                                       1 if name == "seq" else self.cores)
            est = t_bfs + t_scan + (spent / done) * S if done else t_bfs + t_scan
            out[name] = {"sampled_edges": done, "sample_s": spent, "est_full_seconds": est,
                         "cores": 1 if name == "seq" else self.cores,
                         "value": self.m / est if est > 0 else None}
        out["wall"] = time.perf_counter() - t0
        return out

    def describe(self, r) -> str:
        return (f"oracle BFS over the whole graph + full cover-edge scan (1 thread each), then the "
                f"per-edge intersections of seeded samples of S (random runs of 512 consecutive "
                f"cover edges; |S| = {r['num_cover']}): "
                f"{r['seq']['sampled_edges']} edges by the literal CETC-Seq loop on 1 thread, "
                f"{r['omp']['sampled_edges']} by the CETC-SM parallel loop on {self.cores} "
                f"threads; full-graph time = bfs + scan + sample seconds per edge x |S|")

    def baseline(self, r) -> dict:
        """The cpu_baseline object: the OpenMP form (all cores) with the one-thread form beside."""
        return {"value": r["omp"]["value"], "unit": "edges/s", "cores": self.cores,
                "kind": "oracle", "sample": self.describe(r),
                "est_full_seconds": r["omp"]["est_full_seconds"], "sample_wall_s": r["wall"],
                "seq": r["seq"], "omp": r["omp"]}


def validate_cpu_estimate(spec, src, dst, root, target_s):
    """The sampled full-graph estimate against a full timed run of the same loop.

    Times the OpenMP edge loop (orc_cetc_sm_edges) over all of S once and compares it with the
    sampler's estimate of the same (both after the same BFS and scan).
    """
    import oracle
    sam = OracleSampler(spec, src, dst, root, target_s)
    r = sam.step()
    lv = oracle.bfs_levels(sam.rp, sam.col, root)
    cov = oracle.cetc(sam.rp, sam.col, lv, stride=1 << 62, want_cover=True)
    t = time.perf_counter()
    full = oracle.cetc_sm_edges(sam.rp, sam.col, lv, cov["cover_u"], cov["cover_v"])
    t_full = time.perf_counter() - t + r["bfs_s"] + r["scan_s"]
    est = r["omp"]["est_full_seconds"]
    return {"workload": spec.family, "n": spec.n, "m": sam.m, "num_cover": r["num_cover"],
            "cores": sam.cores, "triangles": full["T"], "full_seconds": t_full,
            "estimated_seconds": est, "relative_error": (est - t_full) / t_full,
            "sampled_edges": r["omp"]["sampled_edges"], "sample_seconds": r["omp"]["sample_s"]}


# ----------------------------------------------------------------------------
# arms
# ----------------------------------------------------------------------------

def run_reference(args, world, rank):
    """The oracle as it stands on this host's cores (the reference arm).

    Each step is one bounded sample (OracleSampler.step); ms_per_step is its
    measured wall time.  value = input edges / the estimated full-graph time of
    Algorithm CETC-SM's parallel loop on all host threads (median over steps),
    the same figure as the GPU arm's cpu_baseline.
    """
    if rank != 0:
        return 0
    spec = WORKLOADS[args.workload]
    src, dst = spec.edges()
    import oracle
    rp, _ = oracle.build_csr(spec.n, src, dst)
    root = oracle.max_degree_root(rp) if spec.root == "maxdeg" else 0
    del rp
    budget = max(2.0, 90.0 / max(1, args.steps + args.warmup))
    sam = OracleSampler(spec, src, dst, root, target_s=budget)
    for _ in range(args.warmup):
        sam.step()
    walls, ests, last = [], [], None
    for _ in range(args.steps):
        last = sam.step()
        walls.append(last["wall"])
        ests.append(last["omp"]["est_full_seconds"])
    est = statistics.median(ests)
    value = sam.m / est
    base = dict(sam.baseline(last), value=value, est_full_seconds=est)
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": "edges/s",
            "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": 1000.0 * statistics.mean(walls), "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "int64", "data": "synthetic",
            "config": config_dict(spec, args),
            "timing": ("ms_per_step: measured wall time of one bounded sample; value: input edges "
                       "/ the estimated full-graph time of the CETC-SM oracle on all host threads"),
            "est_full_seconds": est,
            "cpu_baseline": base,
            "e2e": {"value": value, "unit": "edges/s", "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


def config_dict(spec, args):
    c = {"workload": args.workload, "family": spec.family, "n": spec.n, "seed": spec.seed,
         "root": "max-degree (smallest id)" if spec.root == "maxdeg" else "vertex 0",
         "l2": "inputs larger than L2 (CSR > 129 MB)" if args.workload != "er1024"
               else "input fits in L2 (small config)"}
    if spec.family == "rmat":
        c.update(scale=spec.scale, edge_factor=spec.edge_factor, abcd=[0.57, 0.19, 0.19, 0.05],
                 draws=spec.draws)
    elif spec.family == "mesh":
        c.update(rows=spec.rows, cols=spec.cols, p=spec.p)
    else:
        c.update(draws=spec.draws)
    c["parallelism"] = f"replicas x{args.gpus}"
    return c


def run_ours(args, world, rank, local):
    import torch
    import paper_2403_02997_gb300 as tc
    from paper_2403_02997_gb300 import build as tcbuild
    tcbuild.build_all()
    torch.cuda.set_device(local)
    spec = replica_spec(WORKLOADS[args.workload], rank)
    src, dst = spec.edges()
    E = int(src.size)
    stream = torch.cuda.Stream()
    h_src = torch.from_numpy(src.view(np.int32)).pin_memory()
    h_dst = torch.from_numpy(dst.view(np.int32)).pin_memory()
    with torch.cuda.stream(stream):
        d_src = h_src.to("cuda", non_blocking=True)
        d_dst = h_dst.to("cuda", non_blocking=True)
    stream.synchronize()
    # tc_graph_create from device-resident edges (radix-sort CSR build, allocation included),
    # host wall time with the device idle on both sides
    create_s = []
    for _ in range(args.create_steps):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        gc = tc.Graph(d_src, d_dst, spec.n, stream=stream)
        stream.synchronize()
        create_s.append(time.perf_counter() - t0)
        gc.close()
    g = tc.Graph(d_src, d_dst, spec.n, stream=stream)
    del d_src, d_dst
    root = g.max_degree_vertex() if spec.root == "maxdeg" else 0
    from paper_2403_02997_gb300 import autotune
    tuned = None if args.no_tuned else autotune.lookup(
        autotune.signature(spec.n, g.m, g.d_max, spec.family))
    if args.params:
        tuned = dict(tuned or {}, **json.loads(args.params))
    if tuned:
        g.set_params(**tuned)
    params = tc.tc_params_default()
    params.update(tuned or {})

    counts = []
    for _ in range(args.warmup):
        counts.append(g.count(root, stream=stream))
    barrier(world)
    torch.cuda.synchronize()
    clocks = ClockSampler(local)
    clocks.start()
    ev0 = torch.cuda.Event(enable_timing=True)
    ev1 = torch.cuda.Event(enable_timing=True)
    ms_hash, ms_bfs, ms_cover, ms_inter, launches = [], [], [], [], 0
    ev0.record(stream)
    for _ in range(args.steps):
        counts.append(g.count(root, stream=stream))
        st = g.stats()
        ms_hash.append(st["ms_hash"])
        ms_bfs.append(st["ms_bfs"])
        ms_cover.append(st["ms_cover"])
        ms_inter.append(st["ms_intersect"])
        launches += st["launches"]
    ev1.record(stream)
    stream.synchronize()
    barrier(world)
    torch.cuda.synchronize()
    clk = clocks.stop()
    elapsed_ms = ev0.elapsed_time(ev1)
    assert len(set(counts)) == 1, f"counts differ between steps: {set(counts)}"
    st = g.stats()
    T, m, n_cover = counts[0], g.m, st["num_cover"]

    max_ms = max_over_ranks(elapsed_ms, world)
    total_edges = sum_over_ranks(float(m) * args.steps, world)
    value = total_edges / (max_ms / 1000.0)

    # the paper's variants on the same graph and root (same count; not the headline)
    variants = {}
    for name, fn in (("cetc_seq_s", lambda: g.count_split(root, stream=stream)),
                     ("forward_degree_ranked", lambda: g.count_forward(stream=stream))):
        fn()
        ms = []
        for _ in range(3):
            assert fn() == T, name
            ms.append(g.stats()["ms_total"])
        variants[name] = {"ms": statistics.median(ms), "edges_per_s": m / (statistics.median(ms) / 1e3)}
    fe_count, fe_forward = g.count_fe(root, 0.7, stream=stream)
    assert fe_count == T
    variants["cetc_seq_fe_0.7"] = {"covering_ratio": n_cover / max(m, 1),
                                   "ran": "forward" if fe_forward else "cetc_seq"}
    # CETC-Seq-FE with the threshold the autotuner learned for this graph family
    fe_thr = None if args.no_tuned else autotune.lookup_fe(
        autotune.signature(spec.n, g.m, g.d_max, spec.family))
    if fe_thr is not None:
        ms = []
        for _ in range(3):
            fe_count, fe_forward = g.count_fe(root, fe_thr, stream=stream)
            assert fe_count == T
            ms.append(g.stats()["ms_total"])
        variants["cetc_seq_fe_learned"] = {
            "threshold": fe_thr, "covering_ratio": n_cover / max(m, 1),
            "ran": "forward" if fe_forward else "cetc_seq", "ms": statistics.median(ms),
            "edges_per_s": m / (statistics.median(ms) / 1e3)}
    # end to end through the C ABI from pinned host buffers
    e2e_steps = args.e2e_steps
    e2e_parts = {"create": [], "count": [], "close": []}
    for it in range(e2e_steps + 1 if e2e_steps else 0):
        if it == 1:  # one untimed warm-up step: the pool's first growth, first host staging
            for v in e2e_parts.values():
                v.clear()
            torch.cuda.synchronize()
            t0 = time.perf_counter()
        ta = time.perf_counter()
        gh = tc.Graph(h_src.numpy().view(np.uint32), h_dst.numpy().view(np.uint32), spec.n,
                      stream=stream)
        if tuned:  # the parameters the device-resident count ran with
            gh.set_params(**tuned)
        r = gh.max_degree_vertex() if spec.root == "maxdeg" else 0
        tb = time.perf_counter()
        c = gh.count(r, stream=stream)
        tc_ = time.perf_counter()
        gh.close()
        td = time.perf_counter()
        assert c == T
        for k, v in (("create", tb - ta), ("count", tc_ - tb), ("close", td - tc_)):
            e2e_parts[k].append(v)
    if e2e_steps:
        t_e2e = (time.perf_counter() - t0) / e2e_steps
        e2e_max = max_over_ranks(t_e2e, world)
        e2e_value = sum_over_ranks(float(m), world) / e2e_max
    else:  # profiling runs skip the end-to-end leg
        e2e_max, e2e_value = None, None

    # roofline of the dominant kernel (owner-hash intersection), algorithmic bytes.  The host-side
    # byte model allocates and frees many GB of host memory, which slows the driver's calls for a
    # while afterwards, so it runs after the end-to-end leg; the levels and cover set are those of
    # a CETC-Seq count (the variants above may have run the forward count last).
    assert g.count(root, stream=stream) == T
    rp, col = g.csr()
    cu, cv = g.cover_edges()
    hb = hash_kernel_bytes(rp, col, g.levels(), cu, cv, params)
    deg = np.diff(rp.astype(np.int64))
    survey_bytes = int(24 * m + 12 * spec.n + 16 * n_cover +
                       4 * (deg[cu].sum() + deg[cv].sum()) + 4 * (st["c1"] + st["c2"]))
    del rp, col, cu, cv, deg
    peak, peak_kind = measured_peaks()
    hash_ms = statistics.mean(ms_hash) if ms_hash else 0.0
    achieved = hb["bytes"] / (hash_ms / 1e3) / 1e9 if hash_ms > 0 else 0.0
    traffic, traffic_stale = profiled_traffic(args.workload)
    dram_rate = traffic / (hash_ms / 1e3) / 1e9 if traffic and hash_ms > 0 else None

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        try:
            sam = OracleSampler(spec, src, dst, root, target_s=args.cpu_seconds)
            cpu = sam.baseline(sam.step())
        except Exception as e:  # keep the GPU line even if the host runs short
            cpu = {"value": None, "unit": "edges/s", "cores": 1, "kind": "oracle",
                   "sample": f"failed: {e}"}

    line = {
        "metric": METRIC, "value": value, "unit": "edges/s", "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": max_ms / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "int64",
        "data": "synthetic (seeded counter-based generator)",
        "config": dict(config_dict(spec, args), params=params,
                       params_source=("--params" if args.params else "autotuned" if tuned else "defaults")),
        "triangles": T, "m": m, "num_cover": n_cover, "covering_ratio": n_cover / max(m, 1),
        "cover_intersections_per_s": n_cover / (statistics.mean(ms_inter) / 1e3)
        if statistics.mean(ms_inter) > 0 else None,
        "phase_ms": {"bfs": statistics.mean(ms_bfs), "cover": statistics.mean(ms_cover),
                     "intersect": statistics.mean(ms_inter), "owner_hash": hash_ms},
        "bfs": {"levels": st["num_levels"], "steps": st["bfs_steps"],
                "bottom_up_steps": st["bottom_up_steps"], "restarted": st["restarted"]},
        "roofline": {"bound": "hbm", "kernel": "k_owner_hash", "achieved": achieved,
                     "peak": peak, "unit": "GB/s", "frac": achieved / peak if peak else None,
                     "peak_kind": peak_kind, "traffic": traffic, "traffic_stale": traffic_stale,
                     "frac_alg": achieved / peak if peak else None,
                     "frac_dram": dram_rate / peak if dram_rate and peak else None,
                     "achieved_dram": dram_rate,
                     "alg_bytes_per_launch": hb["bytes"], "hash_edges": hb["edges"],
                     "hash_items": hb["items"], "streamed_elements": hb["streamed_elements"],
                     "streamer_row_elements": hb["row_elements"],
                     "survey_alg_bytes_per_count": survey_bytes},
        "create": {"seconds": statistics.median(create_s) if create_s else None,
                   "input_edges_per_s": E / statistics.median(create_s) if create_s else None,
                   "input_bytes_per_s": 8 * E / statistics.median(create_s) if create_s else None,
                   "what": "tc_graph_create from device-resident edge lists: key build, radix "
                           "sort, dedup, CSR (allocation included)"},
        "e2e": {"value": e2e_value, "unit": "edges/s", "h2d_bytes_per_step": 8 * E,
                "d2h_bytes_per_step": 8, "seconds_per_step": e2e_max,
                "parts_ms": {k: [round(x * 1e3, 1) for x in v] for k, v in e2e_parts.items()},
                "what": "host edge lists (pinned) -> tc_graph_create (H2D + CSR build) -> "
                        "tc_count -> tc_graph_destroy"},
        "gpu_launches": launches,
        "clocks": clk,
        "cpu_baseline": cpu,
        "variants": variants,
    }
    g.close()
    del g
    torch.cuda.synchronize()
    if args.workload == "rmat24" and not args.no_extra:
        # the other workloads of the same campaign, each with its own clock record
        line["mesh4096"] = measure_mesh(args, world, rank, local)
        line["batched"] = measure_batched(args, world, rank, local)
        line["serve"] = measure_serve(args, world, rank, local, requests=args.serve_requests_extra,
                                      loads=(0.1, 0.6, 0.9))
    if rank == 0:
        print(json.dumps(line), flush=True)
    return 0


def measure_mesh(args, world, rank, local) -> dict:
    """tc_count on the 4096 x 4096 random-diagonal mesh (about 8191 BFS levels).

    Its count must equal the closed form 2 D (D = diagonals present): each
    anti-diagonal lies in exactly two triangles and the 4-neighbour grid has none.
    """
    import torch
    import paper_2403_02997_gb300 as tc
    from paper_2403_02997_gb300 import autotune
    spec = replica_spec(gen.MESH_4096, rank)
    src, dst = spec.edges()
    diagonals = int(gen.mesh_diagonals(spec.rows, spec.cols, spec.p, spec.seed).sum())
    stream = torch.cuda.Stream()
    d_src = torch.from_numpy(src.view(np.int32)).cuda()
    d_dst = torch.from_numpy(dst.view(np.int32)).cuda()
    g = tc.Graph(d_src, d_dst, spec.n, stream=stream)
    del d_src, d_dst
    tuned = None if args.no_tuned else autotune.lookup(
        autotune.signature(spec.n, g.m, g.d_max, spec.family))
    if tuned:
        g.set_params(**tuned)
    for _ in range(max(args.warmup, 3)):
        T = g.count(0, stream=stream)
    steps = max(args.steps, 5)
    barrier(world)
    torch.cuda.synchronize()
    clocks = ClockSampler(local)
    clocks.start()
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    ev0.record(stream)
    for _ in range(steps):
        assert g.count(0, stream=stream) == T
    ev1.record(stream)
    stream.synchronize()
    clk = clocks.stop()
    st = g.stats()
    ms = max_over_ranks(ev0.elapsed_time(ev1) / steps, world)
    m = g.m
    g.close()
    return {"workload": "mesh 4096 x 4096, 4-neighbour + anti-diagonals p=0.5 (seed 7), root 0",
            "ms_per_count": ms, "edges_per_s": sum_over_ranks(float(m), world) / (ms / 1e3),
            "m": m, "triangles": T, "closed_form_2D": 2 * diagonals,
            "closed_form_ok": T == 2 * diagonals, "levels": st["num_levels"],
            "phase_ms": {"bfs": st["ms_bfs"], "cover": st["ms_cover"],
                         "intersect": st["ms_intersect"]},
            "steps": steps, "params": tuned or "defaults", "clocks": clk}


def measure_batched(args, world, rank, local) -> dict:
    """The batched workload: graphs of uneven size counted together.

    value = graphs counted per second by tc_batch_count on device-resident
    graphs (whole job over ranks); beside it, the same graphs counted one
    tc_count at a time on the same GPU, and tc_count_many end to end from host
    edge lists (graph builds included).
    """
    import torch
    import paper_2403_02997_gb300 as tc
    from paper_2403_02997_gb300 import build as tcbuild
    tcbuild.build_all()
    torch.cuda.set_device(local)
    specs = gen.batched_specs(args.batch_graphs, master_seed=4 + 1000 * rank)
    edges = [sp.edges() for sp in specs]
    stream = torch.cuda.Stream()
    t0 = time.perf_counter()
    gs = [tc.Graph(s, d, sp.n, stream=stream) for sp, (s, d) in zip(specs, edges)]
    t_create = time.perf_counter() - t0
    roots = [g.max_degree_vertex() if sp.root == "maxdeg" else 0 for g, sp in zip(gs, specs)]
    m_total = sum(g.m for g in gs)
    b = tc.Batch(gs, stream=stream)
    from paper_2403_02997_gb300 import autotune
    tuned = None if args.no_tuned else autotune.lookup(autotune.signature(
        sum(sp.n for sp in specs), m_total, max(g.d_max for g in gs), "batched", len(gs)))
    if tuned:
        b.set_params(**tuned)
    counts = None
    for _ in range(args.warmup):
        counts = b.count(roots, stream=stream)
    barrier(world)
    torch.cuda.synchronize()
    clocks = ClockSampler(local)
    clocks.start()
    ev0 = torch.cuda.Event(enable_timing=True)
    ev1 = torch.cuda.Event(enable_timing=True)
    ev0.record(stream)
    for _ in range(args.steps):
        c = b.count(roots, stream=stream)
        assert counts is None or c == counts
        counts = c
    ev1.record(stream)
    stream.synchronize()
    barrier(world)
    clk = clocks.stop()
    st = b.stats()
    ms = max_over_ranks(ev0.elapsed_time(ev1), world)
    graphs_total = sum_over_ranks(float(len(gs)) * args.steps, world)
    value = graphs_total / (ms / 1e3)
    # the fixed cost of a batch: the 64 smallest graphs counted as one batch
    small_ix = sorted(range(len(gs)), key=lambda i: gs[i].m)[:64]
    sb = tc.Batch([gs[i] for i in small_ix], stream=stream)
    if tuned:
        sb.set_params(**tuned)
    small_roots = [roots[i] for i in small_ix]
    for _ in range(3):
        sb.count(small_roots, stream=stream)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for _ in range(20):
        sb.count(small_roots, stream=stream)
    small_ms = (time.perf_counter() - t0) / 20 * 1e3
    small_launches = sb.stats()["launches"]
    small_edges = int(sum(gs[i].m for i in small_ix))
    # the same small batch and the whole batch in one persistent launch (one graph per block)
    assert sb.count_persistent(small_roots, stream=stream) == sb.count(small_roots, stream=stream)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for _ in range(20):
        sb.count_persistent(small_roots, stream=stream)
    small_persist_ms = (time.perf_counter() - t0) / 20 * 1e3
    sb.close()
    assert b.count_persistent(roots, stream=stream) == counts
    persist_ms = []
    for _ in range(3):
        b.count_persistent(roots, stream=stream)
        persist_ms.append(b.stats()["ms_total"])
    persist_ms = statistics.median(persist_ms)
    # one tc_count per graph, same GPU, same graphs
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    single = [g.count(r, stream=stream) for g, r in zip(gs, roots)]
    t_single = time.perf_counter() - t0
    assert single == counts
    b.close()
    # end to end: host edge lists -> one batch built from them -> count -> host counts
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    eb = tc.Batch.from_edges([(s, d, sp.n) for sp, (s, d) in zip(specs, edges)], stream=stream)
    if tuned:
        eb.set_params(**tuned)
    e2e_counts = eb.count(roots, stream=stream)
    eb.close()
    t_e2e = time.perf_counter() - t0
    assert e2e_counts == counts
    # the same through per-graph handles and tc_count_many
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    hs = [tc.Graph(s, d, sp.n, stream=stream) for sp, (s, d) in zip(specs, edges)]
    many_counts = tc.count_many(hs, roots, stream=stream)
    for h in hs:
        h.close()
    t_many = time.perf_counter() - t0
    assert many_counts == counts
    for g in gs:
        g.close()
    h2d = sum(8 * int(s.size) for s, _ in edges)
    return {
        "metric": f"graphs/s (batched count of {len(gs)} graphs, device-resident)",
        "graphs_per_s": value, "ms_per_batch": ms / args.steps, "steps": args.steps,
        "config": {"workload": "batched", "graphs": len(gs), "n_log_uniform": [64, 65536],
                   "families": "even: ER mean degree U[4,64]; odd: R-MAT ef U{8..16}",
                   "master_seed": 4, "vertices": int(sum(sp.n for sp in specs)),
                   "edges_undirected": int(m_total), "parallelism": f"replicas x{world}",
                   "l2": "inputs larger than L2", "params": tuned or "defaults"},
        "edges_per_s": sum_over_ranks(float(m_total) * args.steps, world) / (ms / 1e3),
        "one_count_per_graph": {"graphs_per_s": len(gs) / t_single, "seconds": t_single},
        "speedup_vs_one_count_per_graph": (len(gs) / (ms / 1e3 / args.steps)) / (len(gs) / t_single),
        "triangles_total": int(sum(counts)),
        "phase_ms": {"bfs": st["ms_bfs"], "cover": st["ms_cover"],
                     "intersect": st["ms_intersect"], "owner_hash": st["ms_hash"]},
        "graph_build_seconds": t_create,
        "e2e": {"value": len(gs) / t_e2e, "unit": "graphs/s", "h2d_bytes_per_step": h2d,
                "d2h_bytes_per_step": 8 * len(gs), "seconds_per_step": t_e2e,
                "what": "host edge lists -> tc_batch_create_from_edges -> tc_batch_count"},
        "e2e_per_graph_handles": {"graphs_per_s": len(gs) / t_many, "seconds": t_many,
                                  "what": "tc_graph_create per graph + tc_count_many"},
        "gpu_launches": st["launches"] * args.steps,
        "launches_per_batch": st["launches"],
        "small_batch": {"graphs": len(small_ix), "edges": small_edges, "ms_per_batch": small_ms,
                        "launches": small_launches, "persistent_ms_per_batch": small_persist_ms,
                        "what": "the 64 smallest graphs as one batch: the fixed cost of a batch; "
                                "persistent = tc_batch_count_persistent (one launch)"},
        "persistent": {"ms_per_batch": persist_ms, "graphs_per_s": len(gs) / (persist_ms / 1e3),
                       "launches": 1,
                       "what": "tc_batch_count_persistent: the whole batch in one launch, one "
                               "graph per block (the same counts)"},
        "clocks": clk,
    }


def run_batched(args, world, rank, local):
    """The batched workload as its own JSON line (graphs/s)."""
    r = measure_batched(args, world, rank, local)
    if rank != 0:
        return 0
    line = {"metric": r["metric"], "value": r["graphs_per_s"], "unit": "graphs/s",
            "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": r["ms_per_batch"], "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "int64",
            "data": "synthetic (seeded counter-based generator)"}
    line.update({k: v for k, v in r.items() if k not in ("metric", "graphs_per_s")})
    print(json.dumps(line), flush=True)
    return 0


def measure_serve(args, world, rank, local, requests=None, loads=(0.1, 0.3, 0.6, 0.9, 1.2)) -> dict:
    """The serving workload: Poisson arrivals of count requests.

    Requests are drawn from the batched distribution, a pool of 512 graphs with n log-uniform on
    [2^6, 2^16], seed 5. Every 100th request is an R-MAT scale-22, edge-factor-16 graph, which is
    the 1 %. The capacity is first measured with every request arriving at once. The sweep then
    runs at the given fractions of that capacity and reports graphs/s and p50/p99 latency from
    arrival to count, and how much of the device time the batch builds overlapped with counts.
    """
    import torch
    from paper_2403_02997_gb300 import autotune, serve
    torch.cuda.set_device(local)
    requests = requests or args.serve_requests
    specs = gen.batched_specs(512, master_seed=5 + 1000 * rank)
    pool = [(*sp.edges(), sp.n, None if sp.root == "maxdeg" else 0) for sp in specs]
    big = [(*gen.rmat_spec(22, 16, 22 + i + 1000 * rank).edges(), 1 << 22, None) for i in range(2)]
    tuned = None if args.no_tuned else autotune.lookup("batched:n25:m29:d13:k12")
    budget = int(args.serve_budget_gb * (1 << 30))
    srv = serve.Server(hbm_budget_bytes=budget, params=tuned)
    serve.run_arrivals(srv, pool, rate=1e6, count=200, seed=1)          # warm-up
    clocks = ClockSampler(local)
    clocks.start()
    sat = serve.run_arrivals(srv, pool, rate=1e9, count=requests, seed=2,
                             big_every=100, big_pool=big)
    sat.pop("requests_list")
    capacity = sat["graphs_per_s"]
    points = []
    for f in loads:
        r = serve.run_arrivals(srv, pool, rate=f * capacity, count=requests,
                               seed=int(100 * f), big_every=100, big_pool=big)
        r.pop("requests_list")
        r["load"] = f
        points.append(r)
    clk = clocks.stop()
    batches = list(srv.batches)
    overlap = srv.overlap_stats()
    srv.close()
    knee = next((p["load"] for p in points if p["p99_ms"] and points[0]["p99_ms"] and
                 p["p99_ms"] > 5 * points[0]["p99_ms"]), None)
    return {
        "metric": "served graphs/s and p50/p99 latency (continuous batching, Poisson arrivals)",
        "graphs_per_s": max(p["graphs_per_s"] for p in points),
        "config": {"workload": "serve", "pool": "512 graphs, n log-uniform [2^6, 2^16] (seed 5)",
                   "big": "1 % R-MAT scale 22 ef 16", "requests_per_point": requests,
                   "hbm_budget_gb": args.serve_budget_gb, "params": tuned or "defaults"},
        "capacity_graphs_per_s": capacity, "saturated": sat, "sweep": points,
        "p99_knee_load": knee,
        "mean_batch": float(np.mean(batches)) if batches else None,
        "max_batch": int(max(batches)) if batches else None,
        "overlap": overlap, "clocks": clk,
    }


def run_serve(args, world, rank, local):
    """The serving workload as its own JSON line (peak served graphs/s over the sweep)."""
    from paper_2403_02997_gb300 import build as tcbuild
    tcbuild.build_all()
    r = measure_serve(args, world, rank, local)
    if rank != 0:
        return 0
    line = {"metric": r["metric"], "value": r["graphs_per_s"], "unit": "graphs/s",
            "n_gpus": world, "steps": len(r["sweep"]), "warmup": 1, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "int64",
            "data": "synthetic (seeded counter-based generator)"}
    line.update({k: v for k, v in r.items() if k not in ("metric", "graphs_per_s")})
    print(json.dumps(line), flush=True)
    return 0


def main():
    args = parse_args()
    world, rank, local = dist_setup(args)
    try:
        if args.cpu_validate:
            spec = WORKLOADS[args.workload]
            src, dst = spec.edges()
            import oracle
            rp, _ = oracle.build_csr(spec.n, src, dst)
            root = oracle.max_degree_root(rp) if spec.root == "maxdeg" else 0
            del rp
            print(json.dumps(validate_cpu_estimate(spec, src, dst, root, args.cpu_seconds)))
            return 0
        if args.impl == "reference":
            if args.workload in ("batched", "serve"):
                print(json.dumps({"impl": "reference", "unavailable":
                                  f"the {args.workload} workload is timed for the GPU arm only"}))
                return 0
            return run_reference(args, world, rank)
        if args.workload == "batched":
            return run_batched(args, world, rank, local)
        if args.workload == "serve":
            return run_serve(args, world, rank, local)
        return run_ours(args, world, rank, local)
    finally:
        if world > 1:
            import torch.distributed as dist
            dist.destroy_process_group()


if __name__ == "__main__":
    sys.exit(main())

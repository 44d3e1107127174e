// Cover edges and their intersections: the counting step of Algorithm CETC-Seq
// (Section "Cover-Edge Triangle Counting"), computed in the parallel shape of
// Algorithm CETC-SM.
//
// Counting rule (Algorithm CETC-Seq): for a cover edge {u, v}, u < v, a common
// neighbour w counts when L(w) != L(u) (c1 of Algorithm CETC-SM), or when
// L(w) == L(u) and v < w.  Every path below tallies c1 and c2' = the number of
// same-level common neighbours with v < w, so T = c1 + c2'.  The CETC-SM
// statistic c2 (all same-level common neighbours) equals 3 c2': a same-level
// apex exists only in a triangle with three horizontal edges (Lemma "HE2"),
// which each of its three cover edges sees, and exactly one of them, the edge
// of its two smallest vertices, sees with the apex above v.
//
// k_cover        one thread per adjacency entry (u, v): a horizontal edge with
//                u < v (L(u) == L(v), Definition "BFS-Edge") is a cover edge
//                (Theorem "Cover-Edge Set Generation") and joins the cover
//                list.  If both degrees are <= small_max_degree the thread merges
//                the two rows itself (two pointers, Algorithm EMP); otherwise the
//                edge goes to its endpoint of larger degree, the "owner".
// k_level_split  per row x: a copy of N(x) reordered as [neighbours on L(x) |
//                neighbours on another level], each part ascending (a stable
//                partition; rows up to kSplitMax by one warp, longer rows in
//                tiles of kSplitTile by k_split_tile_*).  A streamer then skips
//                its same-level neighbours w <= v, which can never count, and
//                what it streams -- its same-level neighbours above v, then
//                all its other-level ones -- is one contiguous range.
// k_bucket       groups the owner-path edges by owner (counting sort).
// k_owner_hash   one CTA per work item (owner h, slice of h's cover edges):
//                N(h) is taken in chunks; each chunk goes into a shared-memory
//                hash table (the scatter / probe scheme of Algorithm EHP; two-
//                table cuckoo hashing, one slot per bucket: every lookup is two
//                4-byte loads, hit or miss), and every edge {h, x} of the slice
//                streams its segments of N(x), 128 ids per warp step, up to the
//                chunk's largest id through it.
// Per-thread counts are reduced by warp shuffles and one atomic per CTA.
//
// The same machinery serves the paper's variants and the listing:
// k_g1_pairs       Algorithm CETC-Seq-S's T1: the cover edges with the
//                  intersections of their G1 rows (the other-level parts of the
//                  level-split rows);
// k_orient, k_forward_pairs
//                  Algorithm Forward's orientation by (degree, id) and its
//                  pairs |A+(x) ∩ A+(w)| (CETC-Seq-S's T0 on G0, and the whole
//                  graph for CETC-Seq-FE's forward branch); k_owner_hash's plain
//                  instances intersect the pairs of both that are too long for
//                  a thread's merge;
// k_horizontal     |S|, for CETC-Seq-FE's covering ratio;
// kEmit instances  of k_cover and k_owner_hash emit every triangle they count
//                  (triangle listing and per-vertex counts).
#include "tc_internal.cuh"

namespace tc {

namespace {

constexpr int kCoverBlock = 256;
constexpr int kCoverEntriesPerBlock = 2048;
constexpr uint32_t kEmpty = 0xFFFFFFFFu;
constexpr int kHashBlock = 512;         // threads of an owner-hash block (or 2x, see hash_block)
constexpr uint32_t kSplitMax = 4096;    // rows longer than this are split in tiles
constexpr uint32_t kSplitTile = 4096;   // entries per tile of a long row
constexpr int kTileBlock = 512;         // threads per tile block (8 entries each)
constexpr uint32_t kHashA = 2654435761u;  // multiplicative hashing constants (odd)
constexpr uint32_t kHashB = 0x85EBCA77u;
constexpr int kCuckooRounds = 96;

__device__ __forceinline__ void warp_append_pair(bool take, uint2 value, uint2* list,
                                                 unsigned long long* len) {
  const unsigned mask = __ballot_sync(0xffffffffu, take);
  if (!mask) return;
  const unsigned lane = lane_id();
  const unsigned leader = __ffs(mask) - 1;
  unsigned long long base = 0;
  if (lane == leader) base = atomicAdd(len, (unsigned long long)__popc(mask));
  base = __shfl_sync(0xffffffffu, base, leader);
  if (take) list[base + __popc(mask & ((1u << lane) - 1u))] = value;
}

// Largest u in [lo, hi] with row_ptr[u] <= j.
__device__ __forceinline__ uint32_t row_of(const unsigned long long* row_ptr, uint32_t lo,
                                          uint32_t hi, unsigned long long j) {
  while (lo < hi) {
    uint32_t mid = lo + (hi - lo + 1) / 2;
    if (row_ptr[mid] <= j) lo = mid; else hi = mid - 1;
  }
  return lo;
}

// Four ids of a sorted row from position p on, kEmpty past its end e (four
// independent loads).
__device__ __forceinline__ void load4(const uint32_t* __restrict__ col, unsigned long long p,
                                      unsigned long long e, uint32_t& w0, uint32_t& w1,
                                      uint32_t& w2, uint32_t& w3) {
  w0 = p < e ? col[p] : kEmpty;
  w1 = p + 1 < e ? col[p + 1] : kEmpty;
  w2 = p + 2 < e ? col[p + 2] : kEmpty;
  w3 = p + 3 < e ? col[p + 3] : kEmpty;
}

// The two-pointer merge of Algorithm EMP over the sorted rows arr[ba, ea) and
// arr[bb, eb), taken four ids at a time on each side: all 16 pairs of the two
// current blocks are compared, then the block whose last id is smaller moves
// on (both on a tie) with its next four ids loaded together.  A plain merge
// waits for one dependent load per step; this one for one per four ids.
// Every common id w is reported once, by hit(w): a block moves past w only
// after the other row's block that holds w has been current (its last id
// would otherwise be below w, and the smaller-last rule would have moved it
// instead).  Ids are below 2^31, so kEmpty past a row's end matches nothing.
template <typename Hit>
__device__ __forceinline__ void block_merge(const uint32_t* __restrict__ arr, unsigned long long ba,
                                            unsigned long long ea, unsigned long long bb,
                                            unsigned long long eb, Hit&& hit) {
  uint32_t a0, a1, a2, a3, b0, b1, b2, b3;
  load4(arr, ba, ea, a0, a1, a2, a3);
  load4(arr, bb, eb, b0, b1, b2, b3);
  while (ba < ea && bb < eb) {
    if (a0 == b0 || a0 == b1 || a0 == b2 || a0 == b3) hit(a0);
    if (a1 != kEmpty && (a1 == b0 || a1 == b1 || a1 == b2 || a1 == b3)) hit(a1);
    if (a2 != kEmpty && (a2 == b0 || a2 == b1 || a2 == b2 || a2 == b3)) hit(a2);
    if (a3 != kEmpty && (a3 == b0 || a3 == b1 || a3 == b2 || a3 == b3)) hit(a3);
    const bool step_a = a3 <= b3, step_b = b3 <= a3;
    if (step_a) {
      ba += 4;
      load4(arr, ba, ea, a0, a1, a2, a3);
    }
    if (step_b) {
      bb += 4;
      load4(arr, bb, eb, b0, b1, b2, b3);
    }
  }
}

// c1 and c2' of one thread (see the file comment).
struct Tally {
  unsigned long long c1 = 0, c2c = 0;
};

__device__ __forceinline__ void flush_tally(Tally tl, DevCounters* ctr) {
  __shared__ unsigned long long red[2][32];
  tl.c1 = warp_sum(tl.c1);
  tl.c2c = warp_sum(tl.c2c);
  const unsigned lane = lane_id(), warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
  if (lane == 0) {
    red[0][warp] = tl.c1;
    red[1][warp] = tl.c2c;
  }
  __syncthreads();
  if (warp == 0) {
    unsigned long long a = lane < nw ? red[0][lane] : 0, b = lane < nw ? red[1][lane] : 0;
    a = warp_sum(a);
    b = warp_sum(b);
    if (lane == 0) {
      if (a + b) atomicAdd(&ctr->tri, a + b);
      if (a) atomicAdd(&ctr->c1, a);
      if (b) atomicAdd(&ctr->c2, 3ull * b);
    }
  }
}

// Triangle emission of a listing count.  Every triangle is found once, at its
// cover edge {a, b} (a < b) with apex w.
struct Emit {
  uint32_t* tri;               // triples (a, b, w); NULL: no list
  unsigned long long cap;      // triples that fit
  unsigned long long* cursor;  // triangles found so far (device)
  unsigned long long* vcount;  // per-vertex counts; NULL: none
  uint32_t a, b;               // the cover edge of the hits passed to put()
  // Warp-collective (all 32 lanes, converged): lane hits `hit` (0 or 1) with
  // apex w.  One cursor atomic per call; a and b's counts are added per edge
  // by the caller.
  __device__ __forceinline__ void put(uint32_t hit, uint32_t w) const {
    const unsigned m = __ballot_sync(0xffffffffu, hit);
    if (!m) return;
    if (vcount && hit) atomicAdd(&vcount[w], 1ull);
    if (!tri) return;
    const unsigned lane = lane_id(), leader = __ffs(m) - 1;
    unsigned long long base = 0;
    if (lane == leader) base = atomicAdd(cursor, (unsigned long long)__popc(m));
    base = __shfl_sync(0xffffffffu, base, leader);
    const unsigned long long pos = base + __popc(m & ((1u << lane) - 1u));
    if (hit && pos < cap) {
      tri[3 * pos] = a;
      tri[3 * pos + 1] = b;
      tri[3 * pos + 2] = w;
    }
  }
};

// Cover edges, compacted: k_cover queues the cover edges its lanes find (ballot
// ranks into a per-warp shared-memory queue) and, once 32 are queued, appends
// them to the cover list with one atomic and every lane bins one of them (bin_cover: its rows' offsets, then the small-bin
// merge or an append).  Without the queue only the lanes whose entry happened
// to be a cover edge -- about a quarter of them -- would do that work while
// the rest of the warp waited.  In batch mode the hits go to u's graph.
constexpr int kSmallQueue = 64;  // per warp: up to 31 left over + 32 queued in one step

struct BatchRun {  // a thread's run of hits for one graph of a batch
  uint32_t g = 0xFFFFFFFFu;
  unsigned long long hits = 0, lo = 0, hi = 0;  // graph g holds the vertices [lo, hi)
  __device__ __forceinline__ void add(uint32_t u, unsigned long long here,
                                      const unsigned long long* __restrict__ voff, uint32_t nb,
                                      unsigned long long* __restrict__ gcount) {
    if (u < lo || u >= hi) {  // another graph than the run's
      if (hits) atomicAdd(&gcount[g], hits);
      g = batch_graph_of(voff, 0, nb - 1, u);
      lo = voff[g];
      hi = voff[g + 1];
      hits = 0;
    }
    hits += here;
  }
  __device__ __forceinline__ void flush(unsigned long long* __restrict__ gcount) {
    if (hits) atomicAdd(&gcount[g], hits);
  }
};

// Bins one queued cover edge {u, v} and counts it if it is in the small bin;
// called by every lane of the warp (the appends are warp-collective), with
// `valid` false on lanes that hold no edge.  Small bin (both degrees <=
// small_max): the blocked merge of N(u) and N(v); a common neighbour w counts
// as in Algorithm CETC-Seq, c1 when L(w) != L(u), c2' when L(w) == L(u) and
// v < w.  Medium bin: appended for k_warp_merge.  Otherwise: appended for the
// owner-hash pass as (owner, streamer), the owner the endpoint of larger
// degree (ties: larger id), and counted in ocount[owner].
__device__ __forceinline__ void bin_cover(bool valid, uint2 e,
                                          const unsigned long long* __restrict__ row_ptr,
                                          const uint32_t* __restrict__ col,
                                          const int32_t* __restrict__ level, uint32_t small_max,
                                          uint32_t medium_max, uint32_t* __restrict__ ocount,
                                          uint2* __restrict__ medium, uint2* __restrict__ large,
                                          DevCounters* ctr,
                                          const unsigned long long* __restrict__ voff,
                                          uint32_t nb, unsigned long long* __restrict__ gcount,
                                          Tally& tl, BatchRun& run) {
  bool is_medium = false, is_large = false;
  uint2 le = make_uint2(0, 0);
  if (valid) {
    const uint32_t u = e.x, v = e.y;
    const unsigned long long bu = row_ptr[u], eu = row_ptr[u + 1];
    const unsigned long long bv = row_ptr[v], ev = row_ptr[v + 1];
    const int32_t lu = level[u];
    const unsigned long long du = eu - bu, dv = ev - bv;
    if (du <= small_max && dv <= small_max) {
      uint32_t here = 0;
      block_merge(col, bu, eu, bv, ev, [&](uint32_t w) {
        if (level[w] != lu) {
          ++tl.c1;
          ++here;
        } else if (v < w) {
          ++tl.c2c;
          ++here;
        }
      });
      if (nb && here) run.add(u, here, voff, nb, gcount);
    } else if (du <= medium_max && dv <= medium_max) {
      is_medium = true;
    } else {
      is_large = true;
      const bool v_owns = dv > du || (dv == du && v > u);
      le = v_owns ? make_uint2(v, u) : make_uint2(u, v);
    }
  }
  // the lanes with one owner (queued edges often share a hub) add to its
  // count with one atomic
  const uint32_t key = is_large ? le.x : kEmpty;
  const unsigned peers = __match_any_sync(0xffffffffu, key);
  if (is_large && lane_id() == (unsigned)__ffs(peers) - 1)
    atomicAdd(&ocount[le.x], (uint32_t)__popc(peers));
  warp_append_pair(is_medium, e, medium, &ctr->num_medium);
  warp_append_pair(is_large, le, large, &ctr->num_large);
}

template <bool kEmit>
__global__ void __launch_bounds__(kCoverBlock) k_cover(const unsigned long long* __restrict__ row_ptr,
                                                       const uint32_t* __restrict__ col,
                                                       const uint32_t* __restrict__ erow,
                                                       const int32_t* __restrict__ level, uint32_t n,
                                                       unsigned long long nnz, uint32_t small_max,
                                                       uint2* __restrict__ cover,
                                                       uint2* __restrict__ large,
                                                       uint32_t* __restrict__ ocount,
                                                       uint32_t medium_max,
                                                       uint2* __restrict__ medium,
                                                       const unsigned long long* __restrict__ voff,
                                                       uint32_t nb,
                                                       unsigned long long* __restrict__ gcount,
                                                       DevCounters* ctr, Emit em) {
  __shared__ uint2 s_q[kEmit ? 1 : kCoverBlock / kWarp][kEmit ? 1 : kSmallQueue];
  Tally tl;
  // batch mode: the merges' hits go to their graph, one atomic per run of
  // edges of the same graph seen by this thread
  BatchRun run;
  uint32_t qn = 0;  // cover edges queued by this warp (warp-uniform)
  uint2* const q = s_q[kEmit ? 0 : threadIdx.x / kWarp];
  // each block takes tiles of consecutive entries; a thread's entries in a
  // tile are kCoverBlock apart (coalesced), and their rows come from erow
  for (unsigned long long e0 = (unsigned long long)blockIdx.x * kCoverEntriesPerBlock; e0 < nnz;
       e0 += (unsigned long long)gridDim.x * kCoverEntriesPerBlock) {
    const unsigned long long e1 = min(nnz, e0 + kCoverEntriesPerBlock);
    for (unsigned long long b = e0; b < e1; b += kCoverBlock) {
      const unsigned long long j = b + threadIdx.x;
      bool is_cover = false, is_large = false, is_medium = false;
      uint2 ce = make_uint2(0, 0), le = make_uint2(0, 0);
      if (j < e1) {
        const uint32_t u = erow[j];
        const uint32_t v = col[j];
        if (check_failed(v >= n, ctr)) {
        } else if (v > u) {
          const int32_t lu = level[u];
          if (level[v] == lu) {
            is_cover = true;
            ce = make_uint2(u, v);
            if (kEmit) {  // listing: binned and merged by this thread
              const unsigned long long bu = row_ptr[u], eu = row_ptr[u + 1];
              const unsigned long long bv = row_ptr[v], ev = row_ptr[v + 1];
              const unsigned long long du = eu - bu, dv = ev - bv;
              if (du <= small_max && dv <= small_max) {
                // merge of N(u) and N(v), then again to write its triangles to
                // the slots reserved for them
                uint32_t here = 0;
                block_merge(col, bu, eu, bv, ev, [&](uint32_t w) {
                  if (level[w] != lu) {
                    ++tl.c1;
                    ++here;
                  } else if (v < w) {
                    ++tl.c2c;
                    ++here;
                  }
                });
                if (here) {
                  unsigned long long pos =
                      em.tri ? atomicAdd(em.cursor, (unsigned long long)here) : 0;
                  if (em.vcount) {
                    atomicAdd(&em.vcount[u], (unsigned long long)here);
                    atomicAdd(&em.vcount[v], (unsigned long long)here);
                  }
                  block_merge(col, bu, eu, bv, ev, [&](uint32_t w) {
                    if (level[w] != lu || v < w) {
                      if (em.tri && pos < em.cap) {
                        em.tri[3 * pos] = u;
                        em.tri[3 * pos + 1] = v;
                        em.tri[3 * pos + 2] = w;
                      }
                      ++pos;
                      if (em.vcount) atomicAdd(&em.vcount[w], 1ull);
                    }
                  });
                }
              } else if (du <= medium_max && dv <= medium_max) {
                is_medium = true;
              } else {
                is_large = true;
                const bool v_owns = dv > du || (dv == du && v > u);
                le = v_owns ? make_uint2(v, u) : make_uint2(u, v);
                atomicAdd(&ocount[le.x], 1u);
              }
            }
          }
        }
      }
      if (kEmit) {
        warp_append_pair(is_cover, ce, cover, &ctr->num_cover);
        warp_append_pair(is_medium, ce, medium, &ctr->num_medium);
        warp_append_pair(is_large, le, large, &ctr->num_large);
      } else {
        const unsigned lane = lane_id();
        const unsigned m = __ballot_sync(0xffffffffu, is_cover);
        if (is_cover) q[qn + __popc(m & ((1u << lane) - 1u))] = ce;
        qn += __popc(m);
        if (qn >= kWarp) {  // every lane bins one queued cover edge (and lists it)
          __syncwarp();
          const uint2 qe = q[lane];
          warp_append_pair(true, qe, cover, &ctr->num_cover);
          bin_cover(true, qe, row_ptr, col, level, small_max, medium_max, ocount, medium,
                    large, ctr, voff, nb, gcount, tl, run);
          __syncwarp();
          if (lane < qn - kWarp) q[lane] = q[kWarp + lane];
          qn -= kWarp;
          __syncwarp();
        }
      }
    }
  }
  if (!kEmit) {
    __syncwarp();
    const unsigned lane = lane_id();
    const uint2 qe = lane < qn ? q[lane] : make_uint2(0, 0);
    warp_append_pair(lane < qn, qe, cover, &ctr->num_cover);
    bin_cover(lane < qn, qe, row_ptr, col, level, small_max, medium_max, ocount, medium, large,
              ctr, voff, nb, gcount, tl, run);
  }
  if (nb) run.flush(gcount);
  flush_tally(tl, ctr);
}

// Warp merge of the medium bin: one warp per cover edge {u, v} (u < v), both
// degrees <= kMediumCap.  The longer row is staged in the warp's shared-memory
// slice; each lane takes every 32nd id of the shorter row and binary-searches
// it there (ids of a row ascend, so a lane's searches start where its previous
// one ended).  A hit w counts as in Algorithm CETC-Seq: c1 when L(w) != L(u),
// c2' when L(w) == L(u) and v < w.
constexpr int kWarpMergeBlock = 256;
constexpr uint32_t kMediumCap = 1024;

__global__ void __launch_bounds__(kWarpMergeBlock) k_warp_merge(
    const unsigned long long* __restrict__ row_ptr, const uint32_t* __restrict__ col,
    const int32_t* __restrict__ level, const uint2* __restrict__ medium, unsigned long long count,
    const unsigned long long* __restrict__ voff, uint32_t nb,
    unsigned long long* __restrict__ gcount, DevCounters* ctr) {
  __shared__ uint32_t s_row[kWarpMergeBlock / 32][kMediumCap];
  const unsigned lane = lane_id(), warp = threadIdx.x >> 5;
  uint32_t* row = s_row[warp];
  const unsigned long long warps = (unsigned long long)gridDim.x * blockDim.x / 32;
  Tally tl;
  uint32_t run_g = 0xFFFFFFFFu;
  unsigned long long run = 0;
  for (unsigned long long e = ((unsigned long long)blockIdx.x * blockDim.x + threadIdx.x) / 32;
       e < count; e += warps) {
    const uint2 ed = medium[e];
    const uint32_t u = ed.x, v = ed.y;
    const unsigned long long bu = row_ptr[u], eu = row_ptr[u + 1];
    const unsigned long long bv = row_ptr[v], ev = row_ptr[v + 1];
    const bool u_long = eu - bu >= ev - bv;
    const unsigned long long lb = u_long ? bu : bv, le = u_long ? eu : ev;
    const unsigned long long sb = u_long ? bv : bu, se = u_long ? ev : eu;
    const uint32_t nl = (uint32_t)(le - lb);
    for (uint32_t j = lane; j < nl; j += 32) row[j] = col[lb + j];
    __syncwarp();
    const int32_t lu = level[u];
    uint32_t lo = 0, c1 = 0, c2c = 0;
    for (unsigned long long j = sb + lane; j < se; j += 32) {
      const uint32_t w = col[j];
      uint32_t a = lo, b = nl;
      while (a < b) {
        const uint32_t mid = (a + b) >> 1;
        if (row[mid] < w) a = mid + 1; else b = mid;
      }
      lo = a;
      if (a < nl && row[a] == w) {
        if (level[w] != lu) ++c1;
        else if (v < w) ++c2c;
      }
    }
    tl.c1 += c1;
    tl.c2c += c2c;
    if (nb) {
      const unsigned long long here = warp_sum((unsigned long long)(c1 + c2c));
      if (lane == 0 && here) {
        const uint32_t gid = batch_graph_of(voff, 0, nb - 1, u);
        if (gid != run_g) {
          if (run) atomicAdd(&gcount[run_g], run);
          run_g = gid;
          run = 0;
        }
        run += here;
      }
    }
    __syncwarp();
  }
  if (run) atomicAdd(&gcount[run_g], run);
  flush_tally(tl, ctr);
}

// The level split of one row x = [b, e) (kSplitMax >= e - b > 0) by the whole
// warp: pass 1 counts the neighbours on another level, pass 2 writes both
// parts in order with ballot ranks, the same-level part first (rows of up to
// 128 entries in one pass, their ids and level tests held in registers).
__device__ __forceinline__ void split_row_warp(const uint32_t* __restrict__ col,
                                               const int32_t* __restrict__ level,
                                               unsigned long long b, unsigned long long e,
                                               int32_t lx, uint32_t* __restrict__ lcol,
                                               unsigned long long* lsplit_x) {
  const unsigned lane = lane_id();
  const unsigned lt = (1u << lane) - 1u;
  if (e - b <= 128) {
    uint32_t w[4];
    unsigned mo[4], ms[4];
    unsigned long long other = 0;
#pragma unroll
    for (int t = 0; t < 4; ++t) {
      const unsigned long long j = b + 32 * t + lane;
      const bool valid = j < e;
      w[t] = valid ? col[j] : 0u;
      const bool o = valid && level[w[t]] != lx;
      mo[t] = __ballot_sync(0xffffffffu, o);
      ms[t] = __ballot_sync(0xffffffffu, valid && !o);
      other += __popc(mo[t]);
    }
    unsigned long long ps = b, po = e - other;
#pragma unroll
    for (int t = 0; t < 4; ++t) {
      if (mo[t] & (1u << lane)) lcol[po + __popc(mo[t] & lt)] = w[t];
      else if (ms[t] & (1u << lane)) lcol[ps + __popc(ms[t] & lt)] = w[t];
      po += __popc(mo[t]);
      ps += __popc(ms[t]);
    }
    if (lane == 0) *lsplit_x = e - other;
    return;
  }
  unsigned long long other = 0;
  for (unsigned long long j0 = b; j0 < e; j0 += 32) {
    const unsigned long long j = j0 + lane;
    const bool o = j < e && level[col[j]] != lx;
    other += __popc(__ballot_sync(0xffffffffu, o));
  }
  unsigned long long ps = b, po = e - other;
  for (unsigned long long j0 = b; j0 < e; j0 += 32) {
    const unsigned long long j = j0 + lane;
    uint32_t w = 0;
    const bool valid = j < e;
    bool o = false;
    if (valid) {
      w = col[j];
      o = level[w] != lx;
    }
    const unsigned mo = __ballot_sync(0xffffffffu, valid && o);
    const unsigned ms = __ballot_sync(0xffffffffu, valid && !o);
    if (valid) {
      if (o) lcol[po + __popc(mo & lt)] = w;
      else lcol[ps + __popc(ms & lt)] = w;
    }
    po += __popc(mo);
    ps += __popc(ms);
  }
  if (lane == 0) *lsplit_x = e - other;
}

// Level split of the rows of degree <= kSplitMax: per row x a copy of N(x) as
// [same-level part | other-level part], each ascending; lsplit[x] is where the
// other-level part starts.  A warp takes 32 consecutive rows (grid-stride):
// a row of at most kLaneRow entries goes to its own lane (ids and level tests
// in registers, so many short rows have their loads in flight together), the
// longer ones to the whole warp, one after another.  Rows longer than
// kSplitMax are left to the tile kernels below.
constexpr uint32_t kLaneRow = 16;

__global__ void k_level_split(const unsigned long long* __restrict__ row_ptr,
                              const uint32_t* __restrict__ col, const int32_t* __restrict__ level,
                              uint32_t n, uint32_t* __restrict__ lcol,
                              unsigned long long* __restrict__ lsplit) {
  const unsigned lane = lane_id();
  const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;  // rows per sweep (32 per warp)
  for (uint64_t x0 = (uint64_t)blockIdx.x * blockDim.x + (threadIdx.x & ~31u); x0 < n;
       x0 += stride) {
    const uint64_t x = x0 + lane;
    const bool valid = x < n;
    const unsigned long long b = valid ? row_ptr[x] : 0, e = valid ? row_ptr[x + 1] : 0;
    const unsigned long long d = e - b;
    const int32_t lx = valid && d ? level[x] : 0;
    if (valid && d <= kLaneRow) {  // this lane's row
      uint32_t w[kLaneRow];
      uint32_t obits = 0;
#pragma unroll
      for (uint32_t i = 0; i < kLaneRow; ++i) w[i] = i < d ? col[b + i] : 0u;
#pragma unroll
      for (uint32_t i = 0; i < kLaneRow; ++i)
        if (i < d && level[w[i]] != lx) obits |= 1u << i;
      const uint32_t other = __popc(obits);
      unsigned long long ps = b, po = e - other;
#pragma unroll
      for (uint32_t i = 0; i < kLaneRow; ++i) {
        if (i >= d) break;
        if (obits & (1u << i)) lcol[po++] = w[i];
        else lcol[ps++] = w[i];
      }
      lsplit[x] = e - other;
    }
    unsigned long_rows = __ballot_sync(0xffffffffu, valid && d > kLaneRow && d <= kSplitMax);
    while (long_rows) {  // warp-uniform
      const unsigned l = __ffs(long_rows) - 1;
      long_rows &= long_rows - 1;
      const unsigned long long rb = __shfl_sync(0xffffffffu, b, l);
      const unsigned long long re = __shfl_sync(0xffffffffu, e, l);
      const int32_t rl = __shfl_sync(0xffffffffu, lx, l);
      split_row_warp(col, level, rb, re, rl, lcol, &lsplit[x0 + l]);
    }
  }
}

// Tiles of the rows longer than kSplitMax: tiles[x] = ceil(d(x) / kSplitTile).
__global__ void k_split_tiles(const unsigned long long* __restrict__ row_ptr, uint32_t n,
                              uint32_t* __restrict__ tiles) {
  for (uint64_t x = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; x < n;
       x += (uint64_t)gridDim.x * blockDim.x) {
    const unsigned long long d = row_ptr[x + 1] - row_ptr[x];
    tiles[x] = d > kSplitMax ? (uint32_t)((d + kSplitTile - 1) / kSplitTile) : 0u;
  }
}

__global__ void k_tile_rows(const unsigned long long* __restrict__ toff, uint32_t n,
                            uint32_t* __restrict__ tile_row) {
  for (uint64_t x = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; x < n;
       x += (uint64_t)gridDim.x * blockDim.x)
    for (unsigned long long t = toff[x]; t < toff[x + 1]; ++t) tile_row[t] = (uint32_t)x;
}

// Block per tile: number of entries on another level than the row's vertex.
__global__ void __launch_bounds__(kTileBlock) k_split_tile_count(
    const unsigned long long* __restrict__ row_ptr, const uint32_t* __restrict__ col,
    const int32_t* __restrict__ level, const uint32_t* __restrict__ tile_row,
    const unsigned long long* __restrict__ toff, uint32_t* __restrict__ tcnt) {
  __shared__ uint32_t tmp[kTileBlock / 32 + 1];
  const uint32_t t = blockIdx.x;
  const uint32_t x = tile_row[t];
  const unsigned long long b = row_ptr[x], e = row_ptr[x + 1];
  const unsigned long long tb = b + (unsigned long long)(t - toff[x]) * kSplitTile;
  const unsigned long long te = min(e, tb + kSplitTile);
  const int32_t lx = level[x];
  uint32_t c = 0;
  for (unsigned long long j = tb + threadIdx.x; j < te; j += kTileBlock) c += level[col[j]] != lx;
  c = block_sum(c, tmp);
  if (threadIdx.x == 0) tcnt[t] = c;
}

// Block per tile: writes the tile's entries to their places in both parts.
// Thread i holds the tile's entries 8i..8i+7 (input order), so block-wide
// exclusive scans of the per-thread counts give stable ranks.
__global__ void __launch_bounds__(kTileBlock) k_split_tile_write(
    const unsigned long long* __restrict__ row_ptr, const uint32_t* __restrict__ col,
    const int32_t* __restrict__ level, const uint32_t* __restrict__ tile_row,
    const unsigned long long* __restrict__ toff, const uint32_t* __restrict__ tcnt,
    uint32_t* __restrict__ lcol, unsigned long long* __restrict__ lsplit) {
  constexpr int kPer = kSplitTile / kTileBlock;
  __shared__ unsigned long long tmp[kTileBlock / 32 + 1];
  const uint32_t t = blockIdx.x;
  const uint32_t x = tile_row[t];
  const unsigned long long b = row_ptr[x], e = row_ptr[x + 1];
  const unsigned long long t0 = toff[x], nt = toff[x + 1] - t0, k = t - t0;
  const unsigned long long tb = b + k * kSplitTile;
  const int32_t lx = level[x];
  // other-level entries of the earlier tiles, and of the whole row
  unsigned long long before = 0, all = 0;
  for (unsigned long long q = threadIdx.x; q < nt; q += kTileBlock) {
    const unsigned long long c = tcnt[t0 + q];
    all += c;
    if (q < k) before += c;
  }
  before = block_sum(before, tmp);
  all = block_sum(all, tmp);
  uint32_t w[kPer];
  unsigned flags = 0, mine = 0, valid = 0;
#pragma unroll
  for (int i = 0; i < kPer; ++i) {
    const unsigned long long j = tb + (unsigned long long)threadIdx.x * kPer + i;
    w[i] = 0;
    if (j < e) {
      w[i] = col[j];
      valid |= 1u << i;
      if (level[w[i]] != lx) {
        flags |= 1u << i;
        ++mine;
      }
    }
  }
  unsigned long long tot;
  unsigned long long po = block_exclusive_scan((unsigned long long)mine, tmp, &tot);
  unsigned long long ps = block_exclusive_scan((unsigned long long)(__popc(valid) - mine), tmp, &tot);
  po += e - all + before;
  ps += b + (k * kSplitTile - before);
#pragma unroll
  for (int i = 0; i < kPer; ++i) {
    if (!(valid & (1u << i))) continue;
    if (flags & (1u << i)) lcol[po++] = w[i];
    else lcol[ps++] = w[i];
  }
  if (k == 0 && threadIdx.x == 0) lsplit[x] = e - all;
}

__global__ void k_bucket(const uint2* __restrict__ large, unsigned long long count,
                         const unsigned long long* __restrict__ ooff, uint32_t* __restrict__ ofill,
                         uint32_t* __restrict__ ostream, uint32_t n, DevCounters* ctr) {
  // the lanes of a warp holding pairs of one owner (consecutive pairs often
  // share it: the cover scan emits a row's entries together) take their slots
  // with one atomic
  const unsigned lane = lane_id(), lt = (1u << lane) - 1u;
  const unsigned long long stride = (unsigned long long)gridDim.x * blockDim.x;  // multiple of 32
  for (unsigned long long i0 = (unsigned long long)blockIdx.x * blockDim.x + (threadIdx.x & ~31u);
       i0 < count; i0 += stride) {
    const unsigned long long i = i0 + lane;
    uint2 e = make_uint2(kEmpty, 0u);
    if (i < count) e = large[i];
    const bool ok = i < count && !check_failed(e.x >= n, ctr);
    const uint32_t key = ok ? e.x : kEmpty;
    const unsigned peers = __match_any_sync(0xffffffffu, key);
    const unsigned leader = __ffs(peers) - 1;
    uint32_t start = 0;
    if (ok && lane == leader) start = atomicAdd(&ofill[e.x], (uint32_t)__popc(peers));
    start = __shfl_sync(0xffffffffu, start, leader);
    if (!ok) continue;
    const unsigned long long pos = ooff[e.x] + start + __popc(peers & lt);
    if (check_failed(pos >= count || pos >= ooff[e.x + 1], ctr)) continue;
    ostream[pos] = e.y;
  }
}

// Work items per owner h: ceil(ocount[h] / edges_per_item) slices of its cover edges.
__global__ void k_item_counts(const uint32_t* __restrict__ ocount, uint32_t n, uint32_t per_item,
                              uint32_t* __restrict__ icount) {
  for (uint64_t h = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; h < n;
       h += (uint64_t)gridDim.x * blockDim.x)
    icount[h] = (ocount[h] + per_item - 1) / per_item;
}

__global__ void k_item_owner(const unsigned long long* __restrict__ ioff, uint32_t n,
                             uint32_t* __restrict__ item_owner) {
  for (uint64_t h = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; h < n;
       h += (uint64_t)gridDim.x * blockDim.x)
    for (unsigned long long i = ioff[h]; i < ioff[h + 1]; ++i) item_owner[i] = (uint32_t)h;
}

// ---- the owner-hash kernel ----------------------------------------------

// Row ranges of an owner-hash pass (see k_owner_hash).
struct HashRows {
  const unsigned long long* tb;  // owner h's table: tcol[tb[h], te[h])
  const unsigned long long* te;
  const uint32_t* tcol;
  const unsigned long long* sb;  // streamer x's (first) segment: scol[sb[x], se[x])
  const unsigned long long* se;
  const uint32_t* scol;
};

// Shared memory of k_owner_hash: the chunk's hash tables (or its sorted copy).
extern __shared__ uint32_t s_table[];

// Dynamic shared memory of k_owner_hash for chunks of up to `chunk` entries:
// two cuckoo tables of chunk + chunk / 4 + 1 slots.
__host__ __device__ constexpr size_t owner_hash_smem(uint32_t chunk) {
  return sizeof(uint32_t) * 2 * ((size_t)chunk + chunk / 4 + 1);
}

// Cuckoo hashing with two tables of one slot per bucket: an id w sits either
// at T1[h1(w)] or at T2[h2(w)] (T1 = s_table[0, size), T2 = s_table[size,
// 2 size)), so a lookup is two 4-byte shared loads and two compares, the same
// instructions for a hit and a miss (no divergence inside the warp).  Each
// table has `size` >= 5/4 x entries slots (load <= 0.4, below the 1/2
// threshold of two-table cuckoo hashing); indices are multiplicative hashes
// reduced to [0, size) by a high multiply.
struct Cuckoo {
  uint32_t size;
  __device__ __forceinline__ uint32_t h1(uint32_t w) const { return __umulhi(w * kHashA, size); }
  __device__ __forceinline__ uint32_t h2(uint32_t w) const {
    return size + __umulhi(w * kHashB, size);
  }
  // Insert w; false if it could not be placed (the caller falls back).
  __device__ __forceinline__ bool insert(uint32_t w) const {
    uint32_t cur = w;
    for (int it = 0; it < kCuckooRounds; ++it) {
      uint32_t* s1 = &s_table[h1(cur)];
      if (*s1 == kEmpty && atomicCAS(s1, kEmpty, cur) == kEmpty) return true;
      uint32_t* s2 = &s_table[h2(cur)];
      if (*s2 == kEmpty && atomicCAS(s2, kEmpty, cur) == kEmpty) return true;
      cur = atomicExch((it & 1) ? s2 : s1, cur);  // evict; the evicted id moves on
      if (cur == kEmpty) return true;
    }
    return false;
  }
  __device__ __forceinline__ uint32_t contains(uint32_t w) const {
    return (uint32_t)((s_table[h1(w)] == w) | (s_table[h2(w)] == w));
  }
};

// Sorted-array lookup in s_table[0, len), used for a chunk whose cuckoo build
// failed.
__device__ __forceinline__ uint32_t sorted_contains(uint32_t len, uint32_t w) {
  uint32_t lo = 0, hi = len;
  while (lo < hi) {
    const uint32_t mid = (lo + hi) >> 1;
    if (s_table[mid] < w) lo = mid + 1; else hi = mid;
  }
  return lo < len && s_table[lo] == w;
}

// Lookup of one streamed id in the chunk: the cuckoo table, or for a chunk
// whose table could not be built, the sorted copy.
template <bool kSorted>
__device__ __forceinline__ uint32_t chunk_hit(const Cuckoo ck, uint32_t sorted_len, uint32_t w) {
  if (kSorted) return sorted_contains(sorted_len, w);
  return ck.contains(w);
}

// The warp streams arr[cur, end) up to the first id above hi (kBounded; the
// last chunk of a row is unbounded), looking every element up in the chunk;
// returns the new cursor and adds the hits.  One step is 128 ids: lane l holds
// ids l, l + 32, l + 64 and l + 96 of the step (coalesced loads).  The next
// step is loaded before the current one is looked up -- in a bounded pass only
// while the current step ends at or below hi, so a pass reads at most one step
// past its part (read again by the next chunk).  In the last step, whole rows
// of 32 ids past end or above hi are skipped and the rest is masked per id.  A
// segment is one row's part: shorter than n < 2^31.
// One step's ids at p (lane l: p[0], p[32], p[64], p[96], p = the step's
// start + l), kEmpty from len on (len = ids from p to the end, as int); a
// step wholly before the end (full, warp-uniform) loads without per-id tests.
__device__ __forceinline__ void load_step(const uint32_t* p, uint32_t len, bool full,
                                          uint32_t (&w)[4]) {
  if (full) {
#pragma unroll
    for (int t = 0; t < 4; ++t) w[t] = __ldg(p + 32 * t);
  } else {
#pragma unroll
    for (int t = 0; t < 4; ++t) w[t] = (int)len > 32 * t ? __ldg(p + 32 * t) : kEmpty;
  }
}

// One step of stream_segment on the ids in w, the next step's loaded into wn
// first (p, len: this step's; advanced to the next).  Returns true after the
// last step, with the new cursor in out.
template <bool kBounded, bool kSorted, bool kEmit>
__device__ __forceinline__ bool segment_step(const uint32_t* __restrict__ arr, const uint32_t*& p,
                                             uint32_t& len, const uint32_t (&w)[4],
                                             uint32_t (&wn)[4], const uint32_t hi,
                                             const Cuckoo ck, const uint32_t sorted_len,
                                             const Emit& em, uint32_t& hits,
                                             unsigned long long& out) {
  const uint32_t lane = lane_id();
  const int rem = (int)(len + lane);  // ids from the step's first to the end
  bool more = rem > 128;
  if (kBounded) more = more && __shfl_sync(0xffffffffu, w[3], 31) <= hi;
  if (more) {
    load_step(p + 128, len - 128, rem >= 256, wn);
#pragma unroll
    for (int t = 0; t < 4; ++t) {
      const uint32_t hit = chunk_hit<kSorted>(ck, sorted_len, w[t]);
      hits += hit;
      if (kEmit) em.put(hit, w[t]);
    }
    p += 128;
    len -= 128;
    return false;
  }
  // ids ascend with 32 t + lane, so the ids taken (before end, at most hi)
  // form a prefix of the step: stop at the first row of 32 with none
  uint32_t taken = 0;
#pragma unroll
  for (int t = 0; t < 4; ++t) {
    const bool in = (int)len > 32 * t && (!kBounded || w[t] <= hi);
    const unsigned m = __ballot_sync(0xffffffffu, in);
    if (!m) break;
    taken += __popc(m);
    const uint32_t hit = (uint32_t)in & chunk_hit<kSorted>(ck, sorted_len, w[t]);
    hits += hit;
    if (kEmit) em.put(hit, w[t]);
  }
  // the new cursor follows the ids taken
  out = (unsigned long long)(p - lane - arr) + taken;
  return true;
}

template <bool kBounded, bool kSorted, bool kEmit>
__device__ __forceinline__ unsigned long long stream_segment(
    const uint32_t* __restrict__ arr, const unsigned long long cur, const unsigned long long end,
    const uint32_t hi, const Cuckoo ck, const uint32_t sorted_len, const Emit& em,
    uint32_t& hits) {
  if (cur >= end) return end;
  const uint32_t lane = lane_id();
  const uint32_t* p = arr + cur + lane;
  uint32_t len = (uint32_t)(end - cur) - lane;  // ids from p to end (as int: may be <= 0)
  uint32_t w[4], wn[4];
  load_step(p, len, (int)(len + lane) >= 128, w);
  unsigned long long out = end;
  // two steps per iteration, w and wn trading roles (no register copies)
  for (;;) {
    if (segment_step<kBounded, kSorted, kEmit>(arr, p, len, w, wn, hi, ck, sorted_len, em, hits, out))
      return out;
    if (segment_step<kBounded, kSorted, kEmit>(arr, p, len, wn, w, hi, ck, sorted_len, em, hits, out))
      return out;
  }
}

// Cursors and hits of one cover edge after a chunk.
struct EdgePass {
  unsigned long long a, b;  // cursors of the other-level and same-level segments
  uint32_t c1, c2c;         // hits in each
};

// Both segments of one cover edge for one chunk.  A segment is part of one row,
// so it holds fewer than n < 2^31 ids (stream_segment's length is an int).
template <bool kBounded, bool kSorted, bool kEmit>
__device__ __forceinline__ EdgePass stream_edge(const uint32_t* __restrict__ lcol,
                                                unsigned long long a, unsigned long long ae,
                                                unsigned long long b, unsigned long long be,
                                                uint32_t hi, const Cuckoo ck,
                                                uint32_t sorted_len, const Emit& em) {
  EdgePass r{a, b, 0, 0};
#pragma unroll 1
  for (int part = 0; part < 2; ++part) {  // one copy of the loop for both segments
    uint32_t hits = 0;
    const unsigned long long cur = stream_segment<kBounded, kSorted, kEmit>(
        lcol, part ? b : a, part ? be : ae, hi, ck, sorted_len, em, hits);
    if (part) {
      r.b = cur;
      r.c2c = hits;
    } else {
      r.a = cur;
      r.c1 = hits;
    }
  }
  return r;
}

// Lookups of one 128-id step (lane l holds ids l, l + 32, l + 64, l + 96),
// tallied as c2' for the ids of position < q2 in the step and as c1 from q2
// on; kMasked: only the step's first rem ids (rem <= 128; len = rem - lane)
// count, and rows of 32 past them are skipped.
template <bool kMasked, bool kEmit>
__device__ __forceinline__ void fused_step(const uint32_t (&w)[4], int len, int rem, int q2,
                                           const Cuckoo ck, const Emit& em, uint32_t& c1,
                                           uint32_t& c2c) {
  const int lane = (int)lane_id();
  if (kMasked || (q2 > 0 && q2 < 128)) {  // per id (the last step, or the boundary's)
#pragma unroll
    for (int t = 0; t < 4; ++t) {
      if (kMasked && 32 * t >= rem) break;  // warp-uniform
      uint32_t hit = ck.contains(w[t]);
      if (kMasked) hit &= (uint32_t)(len > 32 * t);
      if (32 * t + lane < q2) c2c += hit; else c1 += hit;
      if (kEmit) em.put(hit, w[t]);
    }
  } else {  // the whole step on one side of the boundary
    uint32_t h = 0;
#pragma unroll
    for (int t = 0; t < 4; ++t) {
      const uint32_t hit = ck.contains(w[t]);
      h += hit;
      if (kEmit) em.put(hit, w[t]);
    }
    if (q2 > 0) c2c += h; else c1 += h;
  }
}

// Against an owner of one chunk (unbounded), the two segments of a cover edge
// as one range arr[cur, end): its same-level ids above v, [cur, bnd), tallied
// as c2', then its other-level ids, [bnd, end), tallied as c1 -- one pass, and
// the same-level part fills the first step of the other-level part instead of
// taking a partial step of its own.  Same step structure as stream_segment.
// A row holds fewer than n < 2^31 ids.
template <bool kEmit>
__device__ __forceinline__ bool fused_seg_step(const uint32_t*& p, uint32_t& len, const int rb,
                                               const uint32_t (&w)[4], uint32_t (&wn)[4],
                                               const Cuckoo ck, const Emit& em, uint32_t& c1,
                                               uint32_t& c2c) {
  const int rem = (int)(len + lane_id());  // ids from the step's first to end
  const int q2 = rem - rb;                 // same-level ids from the step's first on
  if (rem > 128) {
    load_step(p + 128, len - 128, rem >= 256, wn);
    fused_step<false, kEmit>(w, (int)len, rem, q2, ck, em, c1, c2c);
    p += 128;
    len -= 128;
    return false;
  }
  fused_step<true, kEmit>(w, (int)len, rem, q2, ck, em, c1, c2c);
  return true;
}

template <bool kEmit>
__device__ __forceinline__ void stream_fused(const uint32_t* __restrict__ arr,
                                             unsigned long long cur, unsigned long long bnd,
                                             unsigned long long end, const Cuckoo ck,
                                             const Emit& em, uint32_t& c1, uint32_t& c2c) {
  if (cur >= end) return;
  const uint32_t lane = lane_id();
  const uint32_t* p = arr + cur + lane;
  uint32_t len = (uint32_t)(end - cur) - lane;  // ids from p to end (as int: may be <= 0)
  const int rb = (int)(end - bnd);              // ids of the other-level part
  uint32_t w[4], wn[4];
  load_step(p, len, (int)(len + lane) >= 128, w);
  for (;;) {
    if (fused_seg_step<kEmit>(p, len, rb, w, wn, ck, em, c1, c2c)) return;
    if (fused_seg_step<kEmit>(p, len, rb, wn, w, ck, em, c1, c2c)) return;
  }
}

// The rare path (a chunk kept as a sorted array), out of line so it does not
// weigh on the registers of the hot loop.  Arguments and result go by value:
// nothing of the caller's has its address taken (which would put it in local
// memory).
template <bool kEmit>
__device__ __noinline__ EdgePass stream_edge_sorted(const uint32_t* __restrict__ lcol,
                                                    unsigned long long a, unsigned long long ae,
                                                    unsigned long long b, unsigned long long be,
                                                    bool bounded, uint32_t hi,
                                                    uint32_t sorted_len, const Emit em) {
  const Cuckoo none{0};
  if (bounded) return stream_edge<true, true, kEmit>(lcol, a, ae, b, be, hi, none, sorted_len, em);
  return stream_edge<false, true, kEmit>(lcol, a, ae, b, be, hi, none, sorted_len, em);
}

// First index in arr[a, b) (sorted) with arr[i] >= t.
__device__ __forceinline__ unsigned long long lower_bound_u32(const uint32_t* __restrict__ arr,
                                                              unsigned long long a,
                                                              unsigned long long b, uint32_t t) {
  while (a < b) {
    const unsigned long long mid = a + (b - a) / 2;
    if (arr[mid] < t) a = mid + 1; else b = mid;
  }
  return a;
}

// Work item = (owner h, slice of h's cover edges).  N(h) is taken in chunks of
// `chunk` entries; per chunk the table is rebuilt and every edge of the slice
// streams both parts of its level-split row -- all neighbours on another level,
// and the same-level neighbours above v -- from the part's cursor up to the
// chunk's largest id (rows are sorted: cursors only move forward, and each
// streamed element is looked up in exactly one chunk; the last chunk takes the
// rest).  Warps take edges one at a time from a shared counter.
//
// The rows are given as HashRows.  Cover edges of Algorithm CETC-Seq
// (kPlain = false): the owner's table is its whole row, col[tb[h], te[h]) with
// tb = row_ptr, te = row_ptr + 1, and the streamer x streams two segments of
// its level-split row scol = lcol = [same-level | other-level]: its other-level
// part [sb[x], se[x]) (sb = lsplit, se = row_ptr + 1; tallied as c1) and its
// same-level part above v, [first id > v in [tb[x], sb[x]), sb[x]) (tallied as
// c2').  The two are adjacent: against an owner of one chunk they go as one
// range (stream_fused).  Plain pairs (kPlain = true): the table is
// tcol[tb[h], te[h]) and the streamer streams the one segment scol[sb[x],
// se[x]); hits are tallied as c1, or as c2' when plain_as_c2 is set.
// Edges per work item that the cursor arrays of k_owner_hash hold.  With
// 32-bit positions (graphs of fewer than 2^32 adjacency entries) a cursor
// takes half the shared memory of a 64-bit one, and the slices are longer:
// fewer items, so fewer builds of each owner's tables.
template <int kThreads, typename Pos>
__host__ __device__ constexpr uint32_t owner_hash_cap() {
  return sizeof(Pos) == 4 ? (kThreads == 2 * kHashBlock ? 4u : 2u) * (uint32_t)kThreads
                          : (uint32_t)kThreads;
}

template <int kThreads, bool kPlain, bool kEmit, typename Pos = unsigned long long>
__global__ void __launch_bounds__(kThreads, 1024 / kThreads) k_owner_hash(
    const HashRows rows, const unsigned long long* __restrict__ ooff,
    const uint32_t* __restrict__ ostream, const unsigned long long* __restrict__ ioff,
    const uint32_t* __restrict__ item_owner, unsigned long long nitems, uint32_t chunk,
    uint32_t per_item, uint32_t force_sorted, uint32_t plain_as_c2,
    const unsigned long long* __restrict__ voff, uint32_t nb,
    unsigned long long* __restrict__ gcount, DevCounters* ctr, Emit em, uint32_t n,
    unsigned long long nnz_cap) {
  const unsigned long long* __restrict__ tb = rows.tb;
  const unsigned long long* __restrict__ te = rows.te;
  const uint32_t* __restrict__ col = rows.tcol;
  const uint32_t* __restrict__ lcol = rows.scol;
  __shared__ unsigned long long s_item;
  __shared__ uint32_t s_next, s_fail;
  // cursors of the slice's edges (positions in the rows: Pos holds nnz_cap)
  constexpr uint32_t kCap = owner_hash_cap<kThreads, Pos>();
  __shared__ Pos s_a[kCap], s_ae[kCap];
  __shared__ Pos s_b[kCap], s_be[kCap];
  __shared__ uint32_t s_x[kEmit ? kCap : 1];  // streamers (listing only)
  const unsigned lane = lane_id();
  Tally tl;
  if (check_failed(per_item > kCap || (sizeof(Pos) == 4 && nnz_cap >= (1ull << 32)), ctr)) return;
  for (;;) {
    if (threadIdx.x == 0) s_item = atomicAdd(&ctr->item_cursor, 1ull);
    __syncthreads();
    const unsigned long long item = s_item;
    if (item >= nitems) break;
    const uint32_t h = item_owner[item];
    if (check_failed(h >= n, ctr)) continue;  // block-uniform
    const unsigned long long hb = tb[h], he = te[h];
    if (check_failed(hb > he || he > nnz_cap, ctr)) continue;
    const uint32_t chunks = (uint32_t)((he - hb + chunk - 1) / chunk);
    const unsigned long long eb = ooff[h] + (item - ioff[h]) * per_item;
    unsigned long long item_hits = 0;  // this thread's hits in this item (batch mode)
    const uint32_t ne = (uint32_t)min((unsigned long long)per_item, ooff[h + 1] - eb);
    for (uint32_t i = threadIdx.x; i < ne; i += blockDim.x) {
      const uint32_t x = ostream[eb + i];
      if (kEmit) s_x[i] = x;
      if (check_failed(x >= n, ctr)) {  // an empty edge instead
        s_a[i] = s_ae[i] = s_b[i] = s_be[i] = 0;
        continue;
      }
      const unsigned long long os = rows.sb[x];  // the other-level part: [os, se[x])
      s_a[i] = os;
      s_ae[i] = rows.se[x];
      if (kPlain) {
        s_b[i] = s_be[i] = 0;
      } else {  // the same-level part [tb[x], os): its ids above v
        const uint32_t v = x > h ? x : h;
        s_b[i] = lower_bound_u32(lcol, tb[x], os, v + 1);
        s_be[i] = os;
      }
      if (check_failed(s_a[i] > s_ae[i] || s_ae[i] > nnz_cap || s_b[i] > s_be[i] ||
                       s_be[i] > nnz_cap, ctr))
        s_a[i] = s_ae[i] = s_b[i] = s_be[i] = 0;
    }
    // An owner whose row spans several chunks is taken in its two level parts
    // (the other-level and the same-level neighbours of the level-split row,
    // each sorted): a streamer's other-level ids can only meet the owner's
    // other-level neighbours, and its same-level ids above v only the owner's
    // same-level ones, so each segment passes over its own part's chunks only.
    // A single-chunk owner keeps one table of its whole row.
    const bool split = !kPlain && chunks > 1;
    // start of the other-level part (end of the same-level part) of h's row
    const unsigned long long hs = split ? rows.sb[h] : hb;
    const uint32_t* __restrict__ tsrc = split ? lcol : col;
    for (uint32_t part = 0; part < (split ? 2u : 1u); ++part) {
      // part 0: [hs, he) (the other-level part, or the whole row); part 1: [hb, hs)
      const unsigned long long pb = part ? hb : hs, pe = part ? hs : he;
      const uint32_t pchunks = (uint32_t)((pe - pb + chunk - 1) / chunk);
    for (uint32_t c = 0; c < pchunks; ++c) {
      const unsigned long long cb = pb + (unsigned long long)c * chunk;
      const unsigned long long ce = min(pe, cb + chunk);
      const uint32_t entries = (uint32_t)(ce - cb);
      const bool bounded = c + 1 < pchunks;
      const uint32_t hi_id = bounded ? tsrc[ce - 1] : kEmpty;
      // two tables of >= 5/4 x entries slots each (load <= 0.4)
      const uint32_t size = entries + entries / 4 + 1;
      const Cuckoo ck{size};
      for (uint32_t i = threadIdx.x; i < 2 * size; i += blockDim.x) s_table[i] = kEmpty;
      if (threadIdx.x == 0) {
        s_next = 0;
        s_fail = force_sorted;
      }
      __syncthreads();
      if (!force_sorted) {
        // four loads in flight per thread before its inserts, instead of one
        // dependent load latency per entry
        unsigned long long j = cb + threadIdx.x;
        for (; j + 3 * blockDim.x < ce; j += 4 * blockDim.x) {
          const uint32_t w0 = tsrc[j], w1 = tsrc[j + blockDim.x], w2 = tsrc[j + 2 * blockDim.x],
                         w3 = tsrc[j + 3 * blockDim.x];
          bool ok = ck.insert(w0);
          ok = ck.insert(w1) && ok;
          ok = ck.insert(w2) && ok;
          ok = ck.insert(w3) && ok;
          if (!ok) s_fail = 1;
        }
        for (; j < ce; j += blockDim.x)
          if (!ck.insert(tsrc[j])) s_fail = 1;
      }
      __syncthreads();
      const bool sorted = s_fail != 0;
      if (sorted) {  // rare: keep the chunk as a sorted array instead
        for (uint32_t i = threadIdx.x; i < entries; i += blockDim.x) s_table[i] = tsrc[cb + i];
        __syncthreads();
      }
      for (;;) {
        uint32_t i = 0;
        if (lane == 0) i = atomicAdd(&s_next, 1u);
        i = __shfl_sync(0xffffffffu, i, 0);
        if (i >= ne) break;
        // with the row split, part 0 streams only the other-level segment and
        // part 1 only the same-level one (the other passed in empty)
        const unsigned long long ae = s_ae[i], be = s_be[i];
        const unsigned long long a = split && part ? ae : s_a[i];
        const unsigned long long b = split && !part ? be : s_b[i];
        Emit ed = em;
        if (kEmit) {
          const uint32_t x = s_x[i];
          ed.a = min(h, x);
          ed.b = max(h, x);
        }
        EdgePass r;
        if (!sorted) {
          if (kPlain || split) {  // one segment: the part's own (plain pairs: [a, ae))
            const bool seg1 = !kPlain && part;
            const unsigned long long cur = seg1 ? b : a, end = seg1 ? be : ae;
            uint32_t hits = 0;
            const unsigned long long nc =
                bounded ? stream_segment<true, false, kEmit>(lcol, cur, end, hi_id, ck, 0, ed, hits)
                        : stream_segment<false, false, kEmit>(lcol, cur, end, hi_id, ck, 0, ed, hits);
            r = seg1 ? EdgePass{a, nc, 0, hits} : EdgePass{nc, b, hits, 0};
          } else {  // one chunk: [b, be) and [a, ae) are adjacent (be == a)
            r = EdgePass{ae, be, 0, 0};
            stream_fused<kEmit>(lcol, b, be, ae, ck, ed, r.c1, r.c2c);
          }
        } else {
          r = stream_edge_sorted<kEmit>(lcol, a, ae, b, be, bounded, hi_id, entries, ed);
        }
        if (kEmit && em.vcount) {  // the cover edge's endpoints, once per edge and chunk
          const unsigned long long eh = warp_sum((unsigned long long)(r.c1 + r.c2c));
          if (lane == 0 && eh) {
            atomicAdd(&em.vcount[h], eh);
            atomicAdd(&em.vcount[s_x[i]], eh);
          }
        }
        if (lane == 0) {
          if (!(split && part)) s_a[i] = r.a;
          if (!(split && !part)) s_b[i] = r.b;
        }
        const uint32_t c1 = r.c1, c2c = r.c2c;
        if (kPlain && plain_as_c2) {
          tl.c2c += c1;
        } else {
          tl.c1 += c1;
          tl.c2c += c2c;
        }
        item_hits += c1 + c2c;
      }
      __syncthreads();
    }
    }
    if (nb) {  // one atomic per warp per item into the owner's graph
      item_hits = warp_sum(item_hits);
      if (lane == 0 && item_hits) atomicAdd(&gcount[batch_graph_of(voff, 0, nb - 1, h)], item_hits);
    }
  }
  flush_tally(tl, ctr);
}

// ---- a batch counted in one persistent launch, one graph per block ---------
//
// k_batch_graphs takes the graphs of a batch from a device work queue (largest
// first) and runs the whole path for a graph inside one block of kFuseThreads
// threads: BFS levels from its root (top-down, the frontier's edges spread
// over the block by a scan of its degrees), the restart rule (union-find over
// the still-unvisited vertices, each root the smallest id of its component,
// then one multi-source BFS from those roots), the cover-edge scan, and the
// intersections under the counting rule of Algorithm CETC-Seq.  A graph's CSR
// (a few MB at most in the batches it serves) stays in L2 while its block
// works on it.  Everything a graph needs lives in its own slices of the
// union's arrays: level / queues / parents over its vertices, the pairs of
// high-degree cover edges over its half of the entries.
//  - both degrees <= small_max: the cover edge is queued per warp and merged
//    by one lane (block_merge);
//  - otherwise: a warp takes the pair and each lane binary-searches every
//    32nd id of the shorter row in the longer one.
constexpr int kFuseThreads = 1024;
constexpr int kFuseWarps = kFuseThreads / kWarp;

// Block-level BFS: levels lvl0 + 1, ... from the qlen vertices in q (all at
// level lvl0), queues q / nq ping-ponging; all threads call it.  Each level
// takes the frontier in tiles of kFuseThreads vertices; a block scan of their
// degrees hands every thread whole edges, so a hub's row is spread over the
// block.  A vertex is claimed with atomicCAS(level, -1, l + 1).
__device__ void block_bfs(const unsigned long long* __restrict__ row_ptr,
                          const uint32_t* __restrict__ col, int32_t* level, uint32_t* q,
                          uint32_t* nq, uint32_t qlen, int32_t lvl0, uint32_t* s_v,
                          unsigned long long* s_b, unsigned long long* s_off,
                          unsigned long long* s_tmp, uint32_t* s_len) {
  const unsigned lane = lane_id();
  int32_t lvl = lvl0;
  while (qlen > 0) {
    if (threadIdx.x == 0) *s_len = 0;
    __syncthreads();
    for (uint32_t t0 = 0; t0 < qlen; t0 += kFuseThreads) {
      const uint32_t i = t0 + threadIdx.x;
      const uint32_t u = i < qlen ? __ldcg(q + i) : kNoLevel;
      unsigned long long b = 0, d = 0;
      if (u != kNoLevel) {
        b = row_ptr[u];
        d = row_ptr[u + 1] - b;
      }
      unsigned long long total;
      const unsigned long long off = block_exclusive_scan(d, s_tmp, &total);
      s_v[threadIdx.x] = u;
      s_b[threadIdx.x] = b;
      s_off[threadIdx.x] = off;
      __syncthreads();
      const uint32_t tv = min((uint32_t)kFuseThreads, qlen - t0);
      for (unsigned long long j0 = 0; j0 < total; j0 += kFuseThreads) {
        const unsigned long long j = j0 + threadIdx.x;
        bool take = false;
        uint32_t w = 0;
        if (j < total) {
          uint32_t lo = 0, hi = tv - 1;  // last vertex of the tile whose edges start at or before j
          while (lo < hi) {
            const uint32_t mid = (lo + hi + 1) >> 1;
            if (s_off[mid] <= j) lo = mid; else hi = mid - 1;
          }
          w = col[s_b[lo] + (j - s_off[lo])];
          take = atomicCAS(&level[w], -1, lvl + 1) == -1;
        }
        const unsigned m = __ballot_sync(0xffffffffu, take);
        if (m) {
          const unsigned leader = __ffs(m) - 1;
          uint32_t base = 0;
          if (lane == leader) base = atomicAdd(s_len, (uint32_t)__popc(m));
          base = __shfl_sync(0xffffffffu, base, leader);
          if (take) nq[base + __popc(m & ((1u << lane) - 1u))] = w;
        }
      }
      __syncthreads();  // s_v / s_b / s_off are rewritten by the next tile
    }
    qlen = *s_len;
    uint32_t* t = q;
    q = nq;
    nq = t;
    ++lvl;
    __syncthreads();  // every thread has read *s_len before it is reset
  }
}

// Union-find over the graph's unvisited vertices: the larger root is hooked
// under the smaller with a CAS, so a root is always the smallest id of its
// tree (find with path halving; any ancestor is a valid parent).
__device__ __forceinline__ uint32_t fuse_find(uint32_t* parent, uint32_t x) {
  uint32_t p = parent[x];
  while (p != x) {
    const uint32_t gp = parent[p];
    if (gp != p) parent[x] = gp;
    x = p;
    p = gp;
  }
  return x;
}

__global__ void __launch_bounds__(kFuseThreads, 1) k_batch_graphs(
    const unsigned long long* __restrict__ row_ptr, const uint32_t* __restrict__ col,
    const uint32_t* __restrict__ erow, int32_t* level, uint32_t* qa, uint32_t* qb,
    uint32_t* parent, uint2* pairs, const unsigned long long* __restrict__ voff,
    const uint32_t* __restrict__ roots, const uint32_t* __restrict__ order, uint32_t k,
    uint32_t small_max, unsigned long long* __restrict__ gcount, DevCounters* ctr) {
  __shared__ uint32_t s_v[kFuseThreads];
  __shared__ unsigned long long s_b[kFuseThreads], s_off[kFuseThreads];
  __shared__ unsigned long long s_tmp[kFuseWarps + 1];
  __shared__ uint2 s_q[kFuseWarps][kSmallQueue];
  __shared__ uint32_t s_g, s_len, s_npairs;
  const unsigned lane = lane_id(), warp = threadIdx.x / kWarp;
  uint2* const q = s_q[warp];
  Tally tl;
  for (;;) {
    if (threadIdx.x == 0) s_g = (uint32_t)atomicAdd(&ctr->item_cursor, 1ull);
    __syncthreads();
    if (s_g >= k) break;
    const uint32_t g = order[s_g];
    const unsigned long long v0 = voff[g], v1 = voff[g + 1];
    const unsigned long long E0 = row_ptr[v0], E1 = row_ptr[v1];
    unsigned long long hits = 0, covers = 0;  // this thread's, in graph g
    if (v1 > v0) {
      // ---- levels: BFS from the root, then the restart rule
      for (unsigned long long v = v0 + threadIdx.x; v < v1; v += kFuseThreads) level[v] = -1;
      __syncthreads();
      if (threadIdx.x == 0) {
        const uint32_t r = roots[g];
        level[r] = 0;
        qa[v0] = r;
      }
      __syncthreads();
      block_bfs(row_ptr, col, level, qa + v0, qb + v0, 1, 0, s_v, s_b, s_off, s_tmp, &s_len);
      unsigned long long left = 0;
      for (unsigned long long v = v0 + threadIdx.x; v < v1; v += kFuseThreads) {
        const bool un = level[v] == -1;
        left += un;
        if (un) parent[v] = (uint32_t)v;
      }
      left = block_sum(left, s_tmp);
      if (left) {
        // union-find over the unvisited vertices (every edge of one joins two)
        for (unsigned long long j = E0 + threadIdx.x; j < E1; j += kFuseThreads) {
          const uint32_t u = erow[j], w = col[j];
          if (w >= u || level[u] != -1) continue;
          uint32_t a = u, c = w;
          for (;;) {
            a = fuse_find(parent, a);
            c = fuse_find(parent, c);
            if (a == c) break;
            const uint32_t hi = a > c ? a : c, lo = a > c ? c : a;
            if (atomicCAS(&parent[hi], hi, lo) == hi) break;
          }
        }
        if (threadIdx.x == 0) s_len = 0;
        __syncthreads();
        // the roots (each its component's smallest id) seed one multi-source BFS
        for (unsigned long long v0b = v0; v0b < v1; v0b += kFuseThreads) {
          const unsigned long long v = v0b + threadIdx.x;
          const bool seed = v < v1 && level[v] == -1 && parent[v] == (uint32_t)v;
          if (seed) level[v] = 0;
          const unsigned m = __ballot_sync(0xffffffffu, seed);
          if (m) {
            const unsigned leader = __ffs(m) - 1;
            uint32_t base = 0;
            if (lane == leader) base = atomicAdd(&s_len, (uint32_t)__popc(m));
            base = __shfl_sync(0xffffffffu, base, leader);
            if (seed) qa[v0 + base + __popc(m & ((1u << lane) - 1u))] = (uint32_t)v;
          }
        }
        __syncthreads();
        const uint32_t seeds = s_len;
        __syncthreads();
        block_bfs(row_ptr, col, level, qa + v0, qb + v0, seeds, 0, s_v, s_b, s_off, s_tmp,
                  &s_len);
      }
      // ---- cover edges: small pairs merged by a lane, the others listed
      if (threadIdx.x == 0) s_npairs = 0;
      __syncthreads();
      uint2* gp = pairs + E0 / 2;  // the graph's half of the entries: room for all its edges
      uint32_t qn = 0;
      for (unsigned long long j0 = E0; j0 < E1; j0 += kFuseThreads) {
        const unsigned long long j = j0 + threadIdx.x;
        bool is_cover = false;
        uint2 ce = make_uint2(0, 0);
        if (j < E1) {
          const uint32_t u = erow[j], v = col[j];
          if (v > u && level[v] == level[u]) {
            is_cover = true;
            ce = make_uint2(u, v);
          }
        }
        const unsigned m = __ballot_sync(0xffffffffu, is_cover);
        if (is_cover) q[qn + __popc(m & ((1u << lane) - 1u))] = ce;
        qn += __popc(m);
        const bool last = j0 + kFuseThreads >= E1;
        while (qn >= kWarp || (last && qn)) {
          // every lane bins one queued cover edge (the last step drains the rest)
          __syncwarp();
          const uint32_t take = min(qn, (uint32_t)kWarp);
          bool big = false;
          uint2 e = make_uint2(0, 0);
          if (lane < take) {
            e = q[lane];
            ++covers;
            const unsigned long long bu = row_ptr[e.x], eu = row_ptr[e.x + 1];
            const unsigned long long bv = row_ptr[e.y], ev = row_ptr[e.y + 1];
            if (eu - bu <= small_max && ev - bv <= small_max) {
              const int32_t lu = level[e.x];
              const uint32_t vv = e.y;
              block_merge(col, bu, eu, bv, ev, [&](uint32_t w) {
                if (level[w] != lu) {
                  ++tl.c1;
                  ++hits;
                } else if (vv < w) {
                  ++tl.c2c;
                  ++hits;
                }
              });
            } else {
              big = true;
            }
          }
          const unsigned mb = __ballot_sync(0xffffffffu, big);
          if (mb) {
            const unsigned leader = __ffs(mb) - 1;
            uint32_t base = 0;
            if (lane == leader) base = atomicAdd(&s_npairs, (uint32_t)__popc(mb));
            base = __shfl_sync(0xffffffffu, base, leader);
            if (big) gp[base + __popc(mb & ((1u << lane) - 1u))] = e;
          }
          __syncwarp();
          if (lane + take < qn) q[lane] = q[take + lane];
          qn -= take;
          __syncwarp();
        }
      }
      __syncthreads();
      // ---- pairs with a high-degree endpoint: a warp per pair, each lane
      // binary-searching every 32nd id of the shorter row in the longer one
      const uint32_t np = s_npairs;
      for (uint32_t p = warp; p < np; p += kFuseWarps) {
        const uint2 e = gp[p];
        const uint32_t u = e.x, v = e.y;
        const int32_t lu = level[u];
        const unsigned long long bu = row_ptr[u], eu = row_ptr[u + 1];
        const unsigned long long bv = row_ptr[v], ev = row_ptr[v + 1];
        const bool u_short = eu - bu <= ev - bv;
        const unsigned long long sb = u_short ? bu : bv, se = u_short ? eu : ev;
        const unsigned long long lb = u_short ? bv : bu, le = u_short ? ev : eu;
        unsigned long long lo = lb;
        for (unsigned long long t = sb + lane; t < se; t += kWarp) {
          const uint32_t w = col[t];
          unsigned long long a = lo, b = le;
          while (a < b) {
            const unsigned long long mid = a + (b - a) / 2;
            if (col[mid] < w) a = mid + 1; else b = mid;
          }
          lo = a;
          if (a < le && col[a] == w) {
            if (level[w] != lu) {
              ++tl.c1;
              ++hits;
            } else if (v < w) {
              ++tl.c2c;
              ++hits;
            }
          }
        }
      }
    }
    // ---- the graph's count
    hits = block_sum(hits, s_tmp);
    covers = block_sum(covers, s_tmp);
    if (threadIdx.x == 0) {
      gcount[g] = hits;
      if (covers) atomicAdd(&ctr->num_cover, covers);
    }
    __syncthreads();
  }
  flush_tally(tl, ctr);
}

}  // namespace

namespace {

// ---- Algorithm Forward and Algorithm CETC-Seq-S --------------------------

// deg[x] = end[x] - beg[x]: the lengths of the rows an orientation ranks by.
__global__ void k_row_degrees(const unsigned long long* __restrict__ beg,
                              const unsigned long long* __restrict__ end, uint32_t n,
                              uint32_t* __restrict__ deg) {
  for (uint64_t x = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; x < n;
       x += (uint64_t)gridDim.x * blockDim.x)
    deg[x] = (uint32_t)(end[x] - beg[x]);
}

// The orientation of Algorithm Forward (Section "Related Work"), ranking the
// vertices by degree as the paper's reordering does: A+(x) = the w in
// arr[beg[x], end[x]) with (deg[w], w) > (deg[x], x), kept in ascending id
// order.  Every edge of the row set lies in exactly one A+(), and
// |A+(x)| <= sqrt(2 m).  One warp per row; with out == nullptr it writes
// |A+(x)| to cnt[x], else A+(x) to out[obeg[x] ...] (ballot ranks keep order).
__global__ void k_orient(const unsigned long long* __restrict__ beg,
                         const unsigned long long* __restrict__ end,
                         const uint32_t* __restrict__ arr, const uint32_t* __restrict__ deg,
                         uint32_t n, uint32_t* __restrict__ cnt,
                         const unsigned long long* __restrict__ obeg,
                         uint32_t* __restrict__ out) {
  const unsigned lane = lane_id();
  const unsigned lt = (1u << lane) - 1u;
  const uint64_t warps = (uint64_t)gridDim.x * blockDim.x / 32;
  for (uint64_t xx = ((uint64_t)blockIdx.x * blockDim.x + threadIdx.x) / 32; xx < n; xx += warps) {
    const uint32_t x = (uint32_t)xx;
    const unsigned long long b = beg[x], e = end[x];
    const uint32_t dx = deg[x];
    unsigned long long pos = out ? obeg[x] : 0;
    uint32_t c = 0;
    for (unsigned long long j0 = b; j0 < e; j0 += 32) {
      const unsigned long long j = j0 + lane;
      bool keep = false;
      uint32_t w = 0;
      if (j < e) {
        w = arr[j];
        const uint32_t dw = deg[w];
        keep = dw > dx || (dw == dx && w > x);
      }
      const unsigned m = __ballot_sync(0xffffffffu, keep);
      if (out && keep) out[pos + __popc(m & lt)] = w;
      pos += __popc(m);
      c += __popc(m);
    }
    if (!out && lane == 0) cnt[x] = c;
  }
}

// Pairs of an oriented adjacency (obeg, ocol), one thread per entry (x, w):
// |A+(x) ∩ A+(w)| counts each triangle of the row set once (at its two
// lowest-ranked vertices).  Both lists of at most small_max ids: merged by the
// thread (two pointers); otherwise the pair goes to the owner-hash pass as
// (owner, streamer), the owner holding the longer list (ties: larger id).
// Hits are tallied as c1, or as c2' when as_c2 is set.
__global__ void __launch_bounds__(kCoverBlock) k_forward_pairs(
    const unsigned long long* __restrict__ obeg, const uint32_t* __restrict__ ocol, uint32_t n,
    unsigned long long total, uint32_t small_max, uint32_t as_c2, uint2* __restrict__ large,
    uint32_t* __restrict__ ocount, DevCounters* ctr) {
  __shared__ uint32_t s_lo, s_hi;
  Tally tl;
  for (unsigned long long e0 = (unsigned long long)blockIdx.x * kCoverEntriesPerBlock; e0 < total;
       e0 += (unsigned long long)gridDim.x * kCoverEntriesPerBlock) {
    const unsigned long long e1 = min(total, e0 + kCoverEntriesPerBlock);
    __syncthreads();
    if (threadIdx.x == 0) {
      s_lo = row_of(obeg, 0, n - 1, e0);
      s_hi = row_of(obeg, s_lo, n - 1, e1 - 1);
    }
    __syncthreads();
    const uint32_t lo = s_lo, hi = s_hi;
    for (unsigned long long b = e0; b < e1; b += kCoverBlock) {
      const unsigned long long j = b + threadIdx.x;
      bool is_large = false;
      uint2 le = make_uint2(0, 0);
      if (j < e1) {
        const uint32_t x = row_of(obeg, lo, hi, j);
        const uint32_t w = check_failed(ocol[j] >= n, ctr) ? x : ocol[j];
        const unsigned long long bx = obeg[x], ex = obeg[x + 1];
        const unsigned long long bw = obeg[w], ew = obeg[w + 1];
        const unsigned long long dx = ex - bx, dw = ew - bw;
        if (dw > 0) {
          if (dx <= small_max && dw <= small_max) {
            uint32_t here = 0;
            block_merge(ocol, bx, ex, bw, ew, [&](uint32_t) { ++here; });
            if (as_c2) tl.c2c += here; else tl.c1 += here;
          } else {
            is_large = true;
            const bool w_owns = dw > dx || (dw == dx && w > x);
            le = w_owns ? make_uint2(w, x) : make_uint2(x, w);
            atomicAdd(&ocount[le.x], 1u);
          }
        }
      }
      warp_append_pair(is_large, le, large, &ctr->num_large);
    }
  }
  flush_tally(tl, ctr);
}

// The cover edges of Algorithm CETC-Seq-S: one thread per adjacency entry
// (u, v); a horizontal edge with u < v joins the cover list, and the
// intersection of its endpoints' G1 rows (the other-level parts of the
// level-split rows, lcol[lsplit[x], row_ptr[x + 1])) is merged by the thread when
// both have at most small_max ids, else sent to the owner-hash pass (owner:
// the longer G1 row, ties larger id).  Hits are tallied as c1.
__global__ void __launch_bounds__(kCoverBlock) k_g1_pairs(
    const unsigned long long* __restrict__ row_ptr, const uint32_t* __restrict__ col,
    const uint32_t* __restrict__ erow, const int32_t* __restrict__ level,
    const uint32_t* __restrict__ lcol,
    const unsigned long long* __restrict__ lsplit, uint32_t n, unsigned long long nnz,
    uint32_t small_max, uint2* __restrict__ cover, uint2* __restrict__ large,
    uint32_t* __restrict__ ocount, DevCounters* ctr) {
  Tally tl;
  for (unsigned long long e0 = (unsigned long long)blockIdx.x * kCoverEntriesPerBlock; e0 < nnz;
       e0 += (unsigned long long)gridDim.x * kCoverEntriesPerBlock) {
    const unsigned long long e1 = min(nnz, e0 + kCoverEntriesPerBlock);
    for (unsigned long long b = e0; b < e1; b += kCoverBlock) {
      const unsigned long long j = b + threadIdx.x;
      bool is_cover = false, is_large = false;
      uint2 ce = make_uint2(0, 0), le = make_uint2(0, 0);
      if (j < e1) {
        const uint32_t u = erow[j];
        const uint32_t v = col[j];
        if (v > u && level[v] == level[u]) {
          is_cover = true;
          ce = make_uint2(u, v);
          const unsigned long long bu = lsplit[u], eu = row_ptr[u + 1];
          const unsigned long long bv = lsplit[v], ev = row_ptr[v + 1];
          const unsigned long long du = eu - bu, dv = ev - bv;
          if (du > 0 && dv > 0) {
            if (du <= small_max && dv <= small_max) {
              uint32_t here = 0;
              block_merge(lcol, bu, eu, bv, ev, [&](uint32_t) { ++here; });
              tl.c1 += here;
            } else {
              is_large = true;
              const bool v_owns = dv > du || (dv == du && v > u);
              le = v_owns ? make_uint2(v, u) : make_uint2(u, v);
              atomicAdd(&ocount[le.x], 1u);
            }
          }
        }
      }
      warp_append_pair(is_cover, ce, cover, &ctr->num_cover);
      warp_append_pair(is_large, le, large, &ctr->num_large);
    }
  }
  flush_tally(tl, ctr);
}

// |S|: the horizontal edges {u, v}, u < v (one thread per adjacency entry).
__global__ void __launch_bounds__(kCoverBlock) k_horizontal(
    const uint32_t* __restrict__ erow, const uint32_t* __restrict__ col,
    const int32_t* __restrict__ level, unsigned long long nnz, DevCounters* ctr) {
  unsigned long long mine = 0;
  for (unsigned long long j = (unsigned long long)blockIdx.x * blockDim.x + threadIdx.x; j < nnz;
       j += (unsigned long long)gridDim.x * blockDim.x) {
    const uint32_t u = erow[j], v = col[j];
    mine += v > u && level[v] == level[u];
  }
  mine = warp_sum(mine);
  if (lane_id() == 0 && mine) atomicAdd(&ctr->num_cover, mine);
}

// erow[j] = the row of entry j, one thread per entry: each block takes a tile
// of kCoverEntriesPerBlock consecutive entries, finds the rows the tile spans
// (two searches of row_ptr by one thread) and every thread its entry's row
// within them.  Runs once per graph, at creation.
__global__ void __launch_bounds__(kCoverBlock) k_fill_rows(
    const unsigned long long* __restrict__ row_ptr, uint32_t n, unsigned long long nnz,
    uint32_t* __restrict__ erow) {
  __shared__ uint32_t s_lo, s_hi;
  for (unsigned long long e0 = (unsigned long long)blockIdx.x * kCoverEntriesPerBlock; e0 < nnz;
       e0 += (unsigned long long)gridDim.x * kCoverEntriesPerBlock) {
    const unsigned long long e1 = min(nnz, e0 + kCoverEntriesPerBlock);
    __syncthreads();
    if (threadIdx.x == 0) {
      s_lo = row_of(row_ptr, 0, n - 1, e0);
      s_hi = row_of(row_ptr, s_lo, n - 1, e1 - 1);
    }
    __syncthreads();
    const uint32_t lo = s_lo, hi = s_hi;
    for (unsigned long long j = e0 + threadIdx.x; j < e1; j += kCoverBlock)
      erow[j] = row_of(row_ptr, lo, hi, j);
  }
}

// Level-split rows of the whole graph: short rows by warps, long rows in tiles.
tc_status run_level_split(tc_graph* g, cudaStream_t st) {
  const uint32_t n = g->n;
  const int sms = num_sms();
  k_level_split<<<sms * 16, 256, 0, st>>>(g->row_ptr, g->col, g->level, n, g->lcol, g->lsplit); TC_LAUNCHED();
  if (g->d_max > kSplitMax) {
    k_split_tiles<<<grid_for(n, 256, sms * 16), 256, 0, st>>>(g->row_ptr, n, g->fdeg); TC_LAUNCHED();
    TC_TRY(exclusive_scan_u32(g->fdeg, g->ioff, n, g->scan, st));
    TC_CUDA_TRY(cudaMemcpyAsync(&g->ctr_host->scan_total, g->ioff + n, sizeof(unsigned long long),
                                cudaMemcpyDeviceToHost, st));
    TC_CUDA_TRY(cudaStreamSynchronize(st));
    const unsigned long long ntiles = g->ctr_host->scan_total;
    if (ntiles > g->tile_cap) return TC_ERR_OVERFLOW;
    if (ntiles > 0) {
      k_tile_rows<<<grid_for(n, 256, sms * 16), 256, 0, st>>>(g->ioff, n, g->tile_row); TC_LAUNCHED();
      k_split_tile_count<<<(unsigned)ntiles, kTileBlock, 0, st>>>(g->row_ptr, g->col, g->level,
                                                                 g->tile_row, g->ioff, g->tile_cnt); TC_LAUNCHED();
      k_split_tile_write<<<(unsigned)ntiles, kTileBlock, 0, st>>>(g->row_ptr, g->col, g->level,
                                                                 g->tile_row, g->ioff, g->tile_cnt,
                                                                 g->lcol, g->lsplit); TC_LAUNCHED();
    }
  }
  TC_CUDA_TRY(cudaGetLastError());
  return TC_OK;
}

// One owner-hash pass over the nlarge (owner, streamer) pairs in g->large,
// whose per-owner counts are in g->ocount and their exclusive scan in g->ooff:
// bucket the streamers by owner, slice each owner's bucket into work items of
// edges_per_item, and launch k_owner_hash over the items.
template <bool kPlain, bool kEmit = false>
tc_status run_owner_pass(tc_graph* g, unsigned long long nlarge, const HashRows& rows,
                         uint32_t plain_as_c2, const unsigned long long* voff, uint32_t nb,
                         unsigned long long* gcount, cudaStream_t st, const Emit& em = Emit{}) {
  const uint32_t n = g->n;
  const int sms = num_sms();
  TC_CUDA_TRY(cudaMemsetAsync(g->ofill, 0, sizeof(uint32_t) * n, st));
  k_bucket<<<grid_for(nlarge, 256, sms * 16), 256, 0, st>>>(g->large, nlarge, g->ooff, g->ofill,
                                                           g->ostream, n, g->ctr); TC_LAUNCHED();
  const uint32_t chunk = g->params.hash_chunk;
  const bool wide = g->params.hash_block == 2 * kHashBlock;
  const int threads = wide ? 2 * kHashBlock : kHashBlock;
  // 32-bit cursor positions when every position of the rows fits
  const bool pos32 = g->nnz < (1ull << 32);
  const uint32_t cap = wide ? (pos32 ? owner_hash_cap<2 * kHashBlock, uint32_t>()
                                     : owner_hash_cap<2 * kHashBlock, unsigned long long>())
                            : (pos32 ? owner_hash_cap<kHashBlock, uint32_t>()
                                     : owner_hash_cap<kHashBlock, unsigned long long>());
  const uint32_t per_item = g->params.edges_per_item < cap ? g->params.edges_per_item : cap;
  k_item_counts<<<grid_for(n, 256, sms * 16), 256, 0, st>>>(g->ocount, n, per_item, g->fdeg); TC_LAUNCHED();
  TC_CUDA_TRY(cudaGetLastError());
  TC_TRY(exclusive_scan_u32(g->fdeg, g->ioff, n, g->scan, st));
  TC_CUDA_TRY(cudaMemcpyAsync(&g->ctr->items, g->ioff + n, sizeof(unsigned long long),
                              cudaMemcpyDeviceToDevice, st));
  TC_CUDA_TRY(cudaMemcpyAsync(&g->ctr_host->items, g->ioff + n, sizeof(unsigned long long),
                              cudaMemcpyDeviceToHost, st));
  TC_CUDA_TRY(cudaMemsetAsync(&g->ctr->item_cursor, 0, sizeof(unsigned long long), st));
  TC_CUDA_TRY(cudaStreamSynchronize(st));
  const unsigned long long nitems = g->ctr_host->items;
  if (nitems > g->item_cap) {
    dev_free(g, g->item_owner, st);
    g->item_owner = nullptr;
    g->item_cap = 0;
    const unsigned long long want = nitems + nitems / 4 + 1024;
    TC_CUDA_TRY(dev_alloc(g, &g->item_owner, want, st));
    g->item_cap = want;
  }
  k_item_owner<<<grid_for(n, 256, sms * 16), 256, 0, st>>>(g->ioff, n, g->item_owner); TC_LAUNCHED();
  const size_t smem = owner_hash_smem(chunk);
  using u64 = unsigned long long;
  const void* kern =
      wide ? (pos32 ? (const void*)k_owner_hash<2 * kHashBlock, kPlain, kEmit, uint32_t>
                    : (const void*)k_owner_hash<2 * kHashBlock, kPlain, kEmit, u64>)
           : (pos32 ? (const void*)k_owner_hash<kHashBlock, kPlain, kEmit, uint32_t>
                    : (const void*)k_owner_hash<kHashBlock, kPlain, kEmit, u64>);
  TC_CUDA_TRY(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  int per_sm = 0;
  TC_CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, threads, smem));
  if (per_sm < 1) per_sm = 1;
  unsigned grid = (unsigned)(sms * per_sm);
  if (nitems < grid) grid = (unsigned)nitems;
  TC_CUDA_TRY(cudaEventRecord(g->ev[4], st));
  const uint32_t force_sorted = g->params.sorted_lookup ? 1u : 0u;
#define TC_OWNER_HASH_ARGS                                                                     \
  rows, g->ooff, g->ostream, g->ioff, g->item_owner, nitems, chunk, per_item, force_sorted,   \
      plain_as_c2, voff, nb, gcount, g->ctr, em, n, g->nnz
  if (wide && pos32)
    k_owner_hash<2 * kHashBlock, kPlain, kEmit, uint32_t><<<grid, threads, smem, st>>>(TC_OWNER_HASH_ARGS);
  else if (wide)
    k_owner_hash<2 * kHashBlock, kPlain, kEmit, u64><<<grid, threads, smem, st>>>(TC_OWNER_HASH_ARGS);
  else if (pos32)
    k_owner_hash<kHashBlock, kPlain, kEmit, uint32_t><<<grid, threads, smem, st>>>(TC_OWNER_HASH_ARGS);
  else
    k_owner_hash<kHashBlock, kPlain, kEmit, u64><<<grid, threads, smem, st>>>(TC_OWNER_HASH_ARGS);
#undef TC_OWNER_HASH_ARGS
  TC_LAUNCHED();
  TC_CUDA_TRY(cudaGetLastError());
  return TC_OK;
}

// Scan of the per-owner counts and the number of owner-path pairs.
tc_status scan_owners(tc_graph* g, cudaStream_t st, unsigned long long* nlarge) {
  TC_TRY(exclusive_scan_u32(g->ocount, g->ooff, g->n, g->scan, st));
  TC_CUDA_TRY(cudaMemcpyAsync(g->ctr_host, g->ctr, sizeof(DevCounters), cudaMemcpyDeviceToHost, st));
  TC_CUDA_TRY(cudaStreamSynchronize(st));
  *nlarge = g->ctr_host->num_large;
  return TC_OK;
}

}  // namespace

tc_status owner_hash_fits(uint32_t chunk, uint32_t hash_block) {
  const bool wide = hash_block == 2 * kHashBlock;
  // the 32-bit-position instances hold the longer cursor arrays
  const void* kern = wide ? (const void*)k_owner_hash<2 * kHashBlock, false, false, uint32_t>
                          : (const void*)k_owner_hash<kHashBlock, false, false, uint32_t>;
  cudaFuncAttributes fa;
  TC_CUDA_TRY(cudaFuncGetAttributes(&fa, kern));
  int dev = 0, optin = 0;
  TC_CUDA_TRY(cudaGetDevice(&dev));
  TC_CUDA_TRY(cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev));
  const size_t need = owner_hash_smem(chunk) + fa.sharedSizeBytes;
  return need <= (size_t)optin ? TC_OK : TC_ERR_INVALID_ARG;
}

tc_status run_batch_graphs(tc_graph* u, const unsigned long long* voff, const uint32_t* roots,
                           const uint32_t* order, uint32_t k, unsigned long long* gcount,
                           cudaStream_t st) {
  TC_CUDA_TRY(cudaMemsetAsync(u->ctr, 0, sizeof(DevCounters), st));
  TC_CUDA_TRY(cudaEventRecord(u->ev[4], st));
  if (k == 0) return TC_OK;
  const uint32_t small_max = u->params.small_max_degree;
  k_batch_graphs<<<num_sms(), kFuseThreads, 0, st>>>(
      u->row_ptr, u->col, u->erow, u->level, u->queue_a, u->queue_b, u->parent, u->large, voff,
      roots, order, k, small_max, gcount, u->ctr); TC_LAUNCHED();
  TC_CUDA_TRY(cudaGetLastError());
  return TC_OK;
}

tc_status fill_entry_rows(tc_graph* g, cudaStream_t st) {
  if (g->nnz == 0 || g->n == 0) return TC_OK;
  k_fill_rows<<<grid_for(g->nnz, kCoverEntriesPerBlock, num_sms() * 16), kCoverBlock, 0, st>>>(
      g->row_ptr, g->n, g->nnz, g->erow); TC_LAUNCHED();
  TC_CUDA_TRY(cudaGetLastError());
  return TC_OK;
}

tc_status run_cover_and_count(tc_graph* g, cudaStream_t st) {
  const uint32_t n = g->n;
  const int sms = num_sms();
  TC_CUDA_TRY(cudaMemsetAsync(g->ctr, 0, sizeof(DevCounters), st));
  if (g->nnz == 0) {
    TC_CUDA_TRY(cudaEventRecord(g->ev[2], st));
    return TC_OK;
  }
  TC_CUDA_TRY(cudaMemsetAsync(g->ocount, 0, sizeof(uint32_t) * n, st));
  const uint32_t small_max = g->params.small_max_degree;
  k_cover<false><<<grid_for(g->nnz, kCoverEntriesPerBlock, sms * 16), kCoverBlock, 0, st>>>(
      g->row_ptr, g->col, g->erow, g->level, n, g->nnz, small_max, g->cover, g->large, g->ocount,
      g->params.medium_max_degree > kMediumCap ? kMediumCap : g->params.medium_max_degree,
      g->medium, g->voff, g->batch_k, g->gcount, g->ctr, Emit{}); TC_LAUNCHED();
  TC_CUDA_TRY(cudaGetLastError());
  TC_CUDA_TRY(cudaEventRecord(g->ev[2], st));
  unsigned long long nlarge = 0;
  TC_TRY(scan_owners(g, st, &nlarge));
  const unsigned long long nmedium = g->ctr_host->num_medium;
  if (nmedium > 0) {
    k_warp_merge<<<grid_for(nmedium * 32, kWarpMergeBlock, sms * 16), kWarpMergeBlock, 0, st>>>(
        g->row_ptr, g->col, g->level, g->medium, nmedium, g->voff, g->batch_k, g->gcount,
        g->ctr); TC_LAUNCHED();
    TC_CUDA_TRY(cudaGetLastError());
  }
  if (nlarge == 0) return TC_OK;
  TC_TRY(run_level_split(g, st));
  const HashRows rows{g->row_ptr, g->row_ptr + 1, g->col, g->lsplit, g->row_ptr + 1, g->lcol};
  return run_owner_pass<false>(g, nlarge, rows, 0, g->voff, g->batch_k, g->gcount, st);
}

namespace {

// Oriented adjacency storage (obeg[n+1], ocol[m]), allocated on first use.
tc_status ensure_oriented(tc_graph* g, cudaStream_t st) {
  if (!g->obeg) TC_CUDA_TRY(dev_alloc(g, &g->obeg, (size_t)g->n + 1, st));
  if (!g->ocol) TC_CUDA_TRY(dev_alloc(g, &g->ocol, (size_t)g->m + 1, st));
  return TC_OK;
}

// A+() of the rows arr[beg[x], end[x]) into (g->obeg, g->ocol); *total = its size.
tc_status orient(tc_graph* g, const unsigned long long* beg, const unsigned long long* end,
                 const uint32_t* arr, cudaStream_t st, unsigned long long* total) {
  const uint32_t n = g->n;
  const int sms = num_sms();
  TC_TRY(ensure_oriented(g, st));
  k_row_degrees<<<grid_for(n, 256, sms * 16), 256, 0, st>>>(beg, end, n, g->fdeg); TC_LAUNCHED();
  k_orient<<<sms * 16, 256, 0, st>>>(beg, end, arr, g->fdeg, n, g->ocount, nullptr, nullptr); TC_LAUNCHED();
  TC_TRY(exclusive_scan_u32(g->ocount, g->obeg, n, g->scan, st));
  TC_CUDA_TRY(cudaMemcpyAsync(&g->ctr_host->scan_total, g->obeg + n, sizeof(unsigned long long),
                              cudaMemcpyDeviceToHost, st));
  TC_CUDA_TRY(cudaStreamSynchronize(st));
  *total = g->ctr_host->scan_total;
  if (*total > g->m) return TC_ERR_OVERFLOW;  // every edge lies in one A+() at most
  k_orient<<<sms * 16, 256, 0, st>>>(beg, end, arr, g->fdeg, n, nullptr, g->obeg, g->ocol); TC_LAUNCHED();
  TC_CUDA_TRY(cudaGetLastError());
  return TC_OK;
}

// The pairs of the oriented adjacency in (g->obeg, g->ocol): inline merges and
// one owner-hash pass.
tc_status forward_pairs(tc_graph* g, unsigned long long total, uint32_t as_c2, cudaStream_t st) {
  if (total == 0) return TC_OK;
  const uint32_t n = g->n;
  const int sms = num_sms();
  TC_CUDA_TRY(cudaMemsetAsync(g->ocount, 0, sizeof(uint32_t) * n, st));
  TC_CUDA_TRY(cudaMemsetAsync(&g->ctr->num_large, 0, sizeof(unsigned long long), st));
  k_forward_pairs<<<grid_for(total, kCoverEntriesPerBlock, sms * 16), kCoverBlock, 0, st>>>(
      g->obeg, g->ocol, n, total, g->params.small_max_degree, as_c2, g->large, g->ocount, g->ctr); TC_LAUNCHED();
  TC_CUDA_TRY(cudaGetLastError());
  unsigned long long nlarge = 0;
  TC_TRY(scan_owners(g, st, &nlarge));
  if (nlarge == 0) return TC_OK;
  const HashRows rows{g->obeg, g->obeg + 1, g->ocol, g->obeg, g->obeg + 1, g->ocol};
  return run_owner_pass<true>(g, nlarge, rows, as_c2, nullptr, 0, nullptr, st);
}

}  // namespace

tc_status run_forward_count(tc_graph* g, cudaStream_t st) {
  TC_CUDA_TRY(cudaMemsetAsync(g->ctr, 0, sizeof(DevCounters), st));
  if (g->nnz == 0) {
    TC_CUDA_TRY(cudaEventRecord(g->ev[2], st));
    return TC_OK;
  }
  unsigned long long total = 0;
  TC_TRY(orient(g, g->row_ptr, g->row_ptr + 1, g->col, st, &total));
  TC_CUDA_TRY(cudaEventRecord(g->ev[2], st));
  return forward_pairs(g, total, 0, st);
}

tc_status run_split_count(tc_graph* g, cudaStream_t st) {
  const uint32_t n = g->n;
  const int sms = num_sms();
  TC_CUDA_TRY(cudaMemsetAsync(g->ctr, 0, sizeof(DevCounters), st));
  if (g->nnz == 0) {
    TC_CUDA_TRY(cudaEventRecord(g->ev[2], st));
    return TC_OK;
  }
  // G1 rows are the other-level parts, G0 rows the same-level parts, of the
  // level-split rows
  TC_TRY(run_level_split(g, st));
  // T1: intersections of G1 rows over the edges of G0 (the cover edges)
  TC_CUDA_TRY(cudaMemsetAsync(g->ocount, 0, sizeof(uint32_t) * n, st));
  k_g1_pairs<<<grid_for(g->nnz, kCoverEntriesPerBlock, sms * 16), kCoverBlock, 0, st>>>(
      g->row_ptr, g->col, g->erow, g->level, g->lcol, g->lsplit, n, g->nnz, g->params.small_max_degree,
      g->cover, g->large, g->ocount, g->ctr); TC_LAUNCHED();
  TC_CUDA_TRY(cudaGetLastError());
  TC_CUDA_TRY(cudaEventRecord(g->ev[2], st));
  unsigned long long nlarge = 0;
  TC_TRY(scan_owners(g, st, &nlarge));
  if (nlarge > 0) {
    const HashRows rows{g->lsplit, g->row_ptr + 1, g->lcol, g->lsplit, g->row_ptr + 1, g->lcol};
    TC_TRY(run_owner_pass<true>(g, nlarge, rows, 0, nullptr, 0, nullptr, st));
  }
  // T0: Algorithm forward-hashed on G0, tallied as c2' (c2 = 3 T0)
  unsigned long long total = 0;
  TC_TRY(orient(g, g->row_ptr, g->lsplit, g->lcol, st, &total));
  return forward_pairs(g, total, 1, st);
}

tc_status run_count_horizontal(tc_graph* g, cudaStream_t st, unsigned long long* num_cover) {
  const int sms = num_sms();
  TC_CUDA_TRY(cudaMemsetAsync(g->ctr, 0, sizeof(DevCounters), st));
  if (g->nnz > 0) {
    k_horizontal<<<grid_for(g->nnz, kCoverBlock, sms * 16), kCoverBlock, 0, st>>>(
        g->erow, g->col, g->level, g->nnz, g->ctr); TC_LAUNCHED();
    TC_CUDA_TRY(cudaGetLastError());
  }
  TC_CUDA_TRY(cudaMemcpyAsync(g->ctr_host, g->ctr, sizeof(DevCounters), cudaMemcpyDeviceToHost, st));
  TC_CUDA_TRY(cudaStreamSynchronize(st));
  *num_cover = g->ctr_host->num_cover;
  return TC_OK;
}

tc_status run_cover_and_list(tc_graph* g, const EmitSink& sink, cudaStream_t st) {
  const uint32_t n = g->n;
  const int sms = num_sms();
  TC_CUDA_TRY(cudaMemsetAsync(g->ctr, 0, sizeof(DevCounters), st));
  TC_CUDA_TRY(cudaEventRecord(g->ev[2], st));
  if (g->nnz == 0) return TC_OK;
  const Emit em{sink.tri, sink.cap, &g->ctr->listed, sink.vcount, 0, 0};
  TC_CUDA_TRY(cudaMemsetAsync(g->ocount, 0, sizeof(uint32_t) * n, st));
  k_cover<true><<<grid_for(g->nnz, kCoverEntriesPerBlock, sms * 16), kCoverBlock, 0, st>>>(
      g->row_ptr, g->col, g->erow, g->level, n, g->nnz, g->params.small_max_degree, g->cover,
      g->large, g->ocount, 0, g->medium, nullptr, 0, nullptr, g->ctr, em); TC_LAUNCHED();
  TC_CUDA_TRY(cudaGetLastError());
  unsigned long long nlarge = 0;
  TC_TRY(scan_owners(g, st, &nlarge));
  if (nlarge == 0) return TC_OK;
  TC_TRY(run_level_split(g, st));
  const HashRows rows{g->row_ptr, g->row_ptr + 1, g->col, g->lsplit, g->row_ptr + 1, g->lcol};
  return run_owner_pass<false, true>(g, nlarge, rows, 0, nullptr, 0, nullptr, st, em);
}

}  // namespace tc

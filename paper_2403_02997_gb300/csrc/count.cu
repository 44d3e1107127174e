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
// k_level_split  per row x: a copy of N(x) reordered as [neighbours on another
//                level | neighbours on L(x)], each part ascending (a stable
//                partition; rows up to kSplitMax by one warp, longer rows in
//                tiles of kSplitTile by k_split_tile_*).  A streamer then skips
//                its same-level neighbours w <= v, which can never count.
// k_bucket       groups the owner-path edges by owner (counting sort).
// k_owner_hash   one CTA per work item (owner h, slice of h's cover edges):
//                N(h) is taken in chunks; each chunk goes into a shared-memory
//                hash table (the scatter / probe scheme of Algorithm EHP; two-
//                table cuckoo hashing, one slot per bucket: every lookup is two
//                4-byte loads, hit or miss), and every edge {h, x} of the slice
//                streams its segments of N(x), 128 ids per warp step, up to the
//                chunk's largest id through it.
// Per-thread counts are reduced by warp shuffles and one atomic per CTA.
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

__global__ void __launch_bounds__(kCoverBlock) k_cover(const unsigned long long* __restrict__ row_ptr,
                                                       const uint32_t* __restrict__ col,
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
                                                       DevCounters* ctr) {
  __shared__ uint32_t s_lo, s_hi, s_g0, s_g1;
  Tally tl;
  // batch mode: counts of the inline merges go to their graph, one atomic per
  // run of edges of the same graph seen by this thread
  uint32_t run_g = 0xFFFFFFFFu;
  unsigned long long run = 0;
  for (unsigned long long e0 = (unsigned long long)blockIdx.x * kCoverEntriesPerBlock; e0 < nnz;
       e0 += (unsigned long long)gridDim.x * kCoverEntriesPerBlock) {
    const unsigned long long e1 = min(nnz, e0 + kCoverEntriesPerBlock);
    __syncthreads();
    if (threadIdx.x == 0) {
      s_lo = row_of(row_ptr, 0, n - 1, e0);
      s_hi = row_of(row_ptr, s_lo, n - 1, e1 - 1);
      if (nb) {
        s_g0 = batch_graph_of(voff, 0, nb - 1, s_lo);
        s_g1 = batch_graph_of(voff, s_g0, nb - 1, s_hi);
      }
    }
    __syncthreads();
    const uint32_t lo = s_lo, hi = s_hi;
    for (unsigned long long b = e0; b < e1; b += kCoverBlock) {
      const unsigned long long j = b + threadIdx.x;
      bool is_cover = false, is_large = false, is_medium = false;
      uint2 ce = make_uint2(0, 0), le = make_uint2(0, 0);
      if (j < e1) {
        const uint32_t u = row_of(row_ptr, lo, hi, j);
        const uint32_t v = col[j];
        if (v > u) {
          const int32_t lu = level[u];
          if (level[v] == lu) {
            is_cover = true;
            ce = make_uint2(u, v);
            const unsigned long long bu = row_ptr[u], eu = row_ptr[u + 1];
            const unsigned long long bv = row_ptr[v], ev = row_ptr[v + 1];
            const unsigned long long du = eu - bu, dv = ev - bv;
            if (du <= small_max && dv <= small_max) {
              // two-pointer merge of N(u) and N(v)
              unsigned long long x = bu, y = bv;
              uint32_t here = 0;
              while (x < eu && y < ev) {
                const uint32_t a = col[x], c = col[y];
                if (a == c) {
                  if (level[a] != lu) {
                    ++tl.c1;
                    ++here;
                  } else if (v < a) {
                    ++tl.c2c;
                    ++here;
                  }
                  ++x;
                  ++y;
                } else if (a < c) {
                  ++x;
                } else {
                  ++y;
                }
              }
              if (nb && here) {
                const uint32_t gid = s_g0 == s_g1 ? s_g0 : batch_graph_of(voff, s_g0, s_g1, u);
                if (gid != run_g) {
                  if (run) atomicAdd(&gcount[run_g], run);
                  run_g = gid;
                  run = 0;
                }
                run += here;
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
      warp_append_pair(is_cover, ce, cover, &ctr->num_cover);
      warp_append_pair(is_medium, ce, medium, &ctr->num_medium);
      warp_append_pair(is_large, le, large, &ctr->num_large);
    }
  }
  if (run) atomicAdd(&gcount[run_g], run);
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

// One warp per row of degree <= kSplitMax (grid-stride).  Pass 1 counts the
// neighbours on another level; pass 2 writes both parts in order with ballot
// ranks.  Longer rows are left to the tile kernels below.
__global__ void k_level_split(const unsigned long long* __restrict__ row_ptr,
                              const uint32_t* __restrict__ col, const int32_t* __restrict__ level,
                              uint32_t n, uint32_t* __restrict__ lcol,
                              unsigned long long* __restrict__ lsplit) {
  const unsigned lane = lane_id();
  const unsigned lt = (1u << lane) - 1u;
  const uint64_t warps = (uint64_t)gridDim.x * blockDim.x / 32;
  for (uint64_t x = ((uint64_t)blockIdx.x * blockDim.x + threadIdx.x) / 32; x < n; x += warps) {
    const unsigned long long b = row_ptr[x], e = row_ptr[x + 1];
    if (e - b > kSplitMax) continue;
    if (e == b) {
      if (lane == 0) lsplit[x] = b;
      continue;
    }
    const int32_t lx = level[x];
    unsigned long long other = 0;
    for (unsigned long long j0 = b; j0 < e; j0 += 32) {
      const unsigned long long j = j0 + lane;
      const bool o = j < e && level[col[j]] != lx;
      other += __popc(__ballot_sync(0xffffffffu, o));
    }
    unsigned long long po = b, ps = b + other;
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
    if (lane == 0) lsplit[x] = b + other;
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
  po += b + before;
  ps += b + all + (k * kSplitTile - before);
#pragma unroll
  for (int i = 0; i < kPer; ++i) {
    if (!(valid & (1u << i))) continue;
    if (flags & (1u << i)) lcol[po++] = w[i];
    else lcol[ps++] = w[i];
  }
  if (k == 0 && threadIdx.x == 0) lsplit[x] = b + all;
}

__global__ void k_bucket(const uint2* __restrict__ large, unsigned long long count,
                         const unsigned long long* __restrict__ ooff, uint32_t* __restrict__ ofill,
                         uint32_t* __restrict__ ostream) {
  for (unsigned long long i = (unsigned long long)blockIdx.x * blockDim.x + threadIdx.x; i < count;
       i += (unsigned long long)gridDim.x * blockDim.x) {
    const uint2 e = large[i];
    const unsigned long long pos = ooff[e.x] + atomicAdd(&ofill[e.x], 1u);
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
template <bool kBounded, bool kSorted>
__device__ __forceinline__ unsigned long long stream_segment(
    const uint32_t* __restrict__ arr, const unsigned long long cur, const unsigned long long end,
    const uint32_t hi, const Cuckoo ck, const uint32_t sorted_len, uint32_t& hits) {
  if (cur >= end) return end;
  const uint32_t lane = lane_id();
  const uint32_t* p = arr + cur + lane;
  uint32_t len = (uint32_t)(end - cur) - lane;  // ids from p to end (as int: may be <= 0)
  uint32_t w[4];
#pragma unroll
  for (int t = 0; t < 4; ++t) w[t] = (int)len > 32 * t ? __ldg(p + 32 * t) : kEmpty;
  for (;;) {
    bool more = (int)(len + lane) > 128;
    if (kBounded) more = more && __shfl_sync(0xffffffffu, w[3], 31) <= hi;
    uint32_t wn[4];
    if (more) {
#pragma unroll
      for (int t = 0; t < 4; ++t) wn[t] = (int)len > 128 + 32 * t ? __ldg(p + 128 + 32 * t) : kEmpty;
#pragma unroll
      for (int t = 0; t < 4; ++t) hits += chunk_hit<kSorted>(ck, sorted_len, w[t]);
    } else {
      // ids ascend with 32 t + lane, so the ids taken (before end, at most hi)
      // form a prefix of the step: stop at the first row of 32 with none
      uint32_t taken = 0;
#pragma unroll
      for (int t = 0; t < 4; ++t) {
        const bool in = (int)len > 32 * t && (!kBounded || w[t] <= hi);
        const unsigned m = __ballot_sync(0xffffffffu, in);
        if (!m) break;
        taken += __popc(m);
        hits += (uint32_t)in & chunk_hit<kSorted>(ck, sorted_len, w[t]);
      }
      // the new cursor follows the ids taken
      return (unsigned long long)(p - lane - arr) + taken;
    }
    p += 128;
    len -= 128;
#pragma unroll
    for (int t = 0; t < 4; ++t) w[t] = wn[t];
  }
}

// Cursors and hits of one cover edge after a chunk.
struct EdgePass {
  unsigned long long a, b;  // cursors of the other-level and same-level segments
  uint32_t c1, c2c;         // hits in each
};

// Both segments of one cover edge for one chunk.  A segment is part of one row,
// so it holds fewer than n < 2^31 ids (stream_segment's length is an int).
template <bool kBounded, bool kSorted>
__device__ __forceinline__ EdgePass stream_edge(const uint32_t* __restrict__ lcol,
                                                unsigned long long a, unsigned long long ae,
                                                unsigned long long b, unsigned long long be,
                                                uint32_t hi, const Cuckoo ck,
                                                uint32_t sorted_len) {
  EdgePass r{a, b, 0, 0};
#pragma unroll 1
  for (int part = 0; part < 2; ++part) {  // one copy of the loop for both segments
    uint32_t hits = 0;
    const unsigned long long cur = stream_segment<kBounded, kSorted>(
        lcol, part ? b : a, part ? be : ae, hi, ck, sorted_len, hits);
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

// The rare path (a chunk kept as a sorted array), out of line so it does not
// weigh on the registers of the hot loop.  Arguments and result go by value:
// nothing of the caller's has its address taken (which would put it in local
// memory).
__device__ __noinline__ EdgePass stream_edge_sorted(const uint32_t* __restrict__ lcol,
                                                    unsigned long long a, unsigned long long ae,
                                                    unsigned long long b, unsigned long long be,
                                                    bool bounded, uint32_t hi,
                                                    uint32_t sorted_len) {
  const Cuckoo none{0};
  if (bounded) return stream_edge<true, true>(lcol, a, ae, b, be, hi, none, sorted_len);
  return stream_edge<false, true>(lcol, a, ae, b, be, hi, none, sorted_len);
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
template <int kThreads>
__global__ void __launch_bounds__(kThreads, 1024 / kThreads) k_owner_hash(
    const unsigned long long* __restrict__ row_ptr, const uint32_t* __restrict__ col,
    const uint32_t* __restrict__ lcol, const unsigned long long* __restrict__ lsplit,
    const unsigned long long* __restrict__ ooff, const uint32_t* __restrict__ ostream,
    const unsigned long long* __restrict__ ioff, const uint32_t* __restrict__ item_owner,
    unsigned long long nitems, uint32_t chunk, uint32_t per_item, uint32_t force_sorted,
    const unsigned long long* __restrict__ voff, uint32_t nb,
    unsigned long long* __restrict__ gcount, DevCounters* ctr) {
  __shared__ unsigned long long s_item;
  __shared__ uint32_t s_next, s_fail;
  // cursors of the slice's edges (edges_per_item <= kThreads)
  __shared__ unsigned long long s_a[kThreads], s_ae[kThreads];
  __shared__ unsigned long long s_b[kThreads], s_be[kThreads];
  const unsigned lane = lane_id();
  Tally tl;
  for (;;) {
    if (threadIdx.x == 0) s_item = atomicAdd(&ctr->item_cursor, 1ull);
    __syncthreads();
    const unsigned long long item = s_item;
    if (item >= nitems) break;
    const uint32_t h = item_owner[item];
    const unsigned long long hb = row_ptr[h], he = row_ptr[h + 1];
    const uint32_t chunks = (uint32_t)((he - hb + chunk - 1) / chunk);
    const unsigned long long eb = ooff[h] + (item - ioff[h]) * per_item;
    unsigned long long item_hits = 0;  // this thread's hits in this item (batch mode)
    const uint32_t ne = (uint32_t)min((unsigned long long)per_item, ooff[h + 1] - eb);
    for (uint32_t i = threadIdx.x; i < ne; i += blockDim.x) {
      const uint32_t x = ostream[eb + i];
      const uint32_t v = x > h ? x : h;
      const unsigned long long sp = lsplit[x], xe = row_ptr[x + 1];
      s_a[i] = row_ptr[x];
      s_ae[i] = sp;
      s_b[i] = lower_bound_u32(lcol, sp, xe, v + 1);
      s_be[i] = xe;
    }
    for (uint32_t c = 0; c < chunks; ++c) {
      const unsigned long long cb = hb + (unsigned long long)c * chunk;
      const unsigned long long ce = min(he, cb + chunk);
      const uint32_t entries = (uint32_t)(ce - cb);
      const bool bounded = c + 1 < chunks;
      const uint32_t hi_id = bounded ? col[ce - 1] : kEmpty;
      // two tables of >= 5/4 x entries slots each (load <= 0.4)
      const uint32_t size = entries + entries / 4 + 1;
      const Cuckoo ck{size};
      for (uint32_t i = threadIdx.x; i < 2 * size; i += blockDim.x) s_table[i] = kEmpty;
      if (threadIdx.x == 0) {
        s_next = 0;
        s_fail = force_sorted;
      }
      __syncthreads();
      if (!force_sorted)
        for (unsigned long long j = cb + threadIdx.x; j < ce; j += blockDim.x)
          if (!ck.insert(col[j])) s_fail = 1;
      __syncthreads();
      const bool sorted = s_fail != 0;
      if (sorted) {  // rare: keep the chunk as a sorted array instead
        for (uint32_t i = threadIdx.x; i < entries; i += blockDim.x) s_table[i] = col[cb + i];
        __syncthreads();
      }
      for (;;) {
        uint32_t i = 0;
        if (lane == 0) i = atomicAdd(&s_next, 1u);
        i = __shfl_sync(0xffffffffu, i, 0);
        if (i >= ne) break;
        const unsigned long long a = s_a[i], b = s_b[i];
        const unsigned long long ae = s_ae[i], be = s_be[i];
        EdgePass r;
        if (!sorted) {
          if (bounded) r = stream_edge<true, false>(lcol, a, ae, b, be, hi_id, ck, entries);
          else r = stream_edge<false, false>(lcol, a, ae, b, be, hi_id, ck, entries);
        } else {
          r = stream_edge_sorted(lcol, a, ae, b, be, bounded, hi_id, entries);
        }
        if (lane == 0) {
          s_a[i] = r.a;
          s_b[i] = r.b;
        }
        const uint32_t c1 = r.c1, c2c = r.c2c;
        tl.c1 += c1;
        tl.c2c += c2c;
        item_hits += c1 + c2c;
      }
      __syncthreads();
    }
    if (nb) {  // one atomic per warp per item into the owner's graph
      item_hits = warp_sum(item_hits);
      if (lane == 0 && item_hits) atomicAdd(&gcount[batch_graph_of(voff, 0, nb - 1, h)], item_hits);
    }
  }
  flush_tally(tl, ctr);
}

}  // namespace

tc_status owner_hash_fits(uint32_t chunk, uint32_t hash_block) {
  const bool wide = hash_block == 2 * kHashBlock;
  const void* kern = wide ? (const void*)k_owner_hash<2 * kHashBlock>
                          : (const void*)k_owner_hash<kHashBlock>;
  cudaFuncAttributes fa;
  TC_CUDA_TRY(cudaFuncGetAttributes(&fa, kern));
  int dev = 0, optin = 0;
  TC_CUDA_TRY(cudaGetDevice(&dev));
  TC_CUDA_TRY(cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev));
  const size_t need = owner_hash_smem(chunk) + fa.sharedSizeBytes;
  return need <= (size_t)optin ? TC_OK : TC_ERR_INVALID_ARG;
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
  k_cover<<<grid_for(g->nnz, kCoverEntriesPerBlock, sms * 16), kCoverBlock, 0, st>>>(
      g->row_ptr, g->col, g->level, n, g->nnz, small_max, g->cover, g->large, g->ocount,
      g->params.medium_max_degree > kMediumCap ? kMediumCap : g->params.medium_max_degree,
      g->medium, g->voff, g->batch_k, g->gcount, g->ctr); TC_LAUNCHED();
  TC_CUDA_TRY(cudaGetLastError());
  TC_CUDA_TRY(cudaEventRecord(g->ev[2], st));
  TC_TRY(exclusive_scan_u32(g->ocount, g->ooff, n, g->scan, st));
  TC_CUDA_TRY(cudaMemcpyAsync(g->ctr_host, g->ctr, sizeof(DevCounters), cudaMemcpyDeviceToHost, st));
  TC_CUDA_TRY(cudaStreamSynchronize(st));
  const unsigned long long nmedium = g->ctr_host->num_medium;
  if (nmedium > 0) {
    k_warp_merge<<<grid_for(nmedium * 32, kWarpMergeBlock, sms * 16), kWarpMergeBlock, 0, st>>>(
        g->row_ptr, g->col, g->level, g->medium, nmedium, g->voff, g->batch_k, g->gcount,
        g->ctr); TC_LAUNCHED();
    TC_CUDA_TRY(cudaGetLastError());
  }
  const unsigned long long nlarge = g->ctr_host->num_large;
  if (nlarge == 0) return TC_OK;
  // level-split rows: short rows by warps, long rows in tiles
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
  TC_CUDA_TRY(cudaMemsetAsync(g->ofill, 0, sizeof(uint32_t) * n, st));
  k_bucket<<<grid_for(nlarge, 256, sms * 16), 256, 0, st>>>(g->large, nlarge, g->ooff, g->ofill,
                                                           g->ostream); TC_LAUNCHED();
  const uint32_t chunk = g->params.hash_chunk;
  const uint32_t per_item = g->params.edges_per_item;
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
    cudaFree(g->item_owner);
    g->item_owner = nullptr;
    g->item_cap = 0;
    const unsigned long long want = nitems + nitems / 4 + 1024;
    TC_CUDA_TRY(cudaMalloc(&g->item_owner, sizeof(uint32_t) * want));
    g->item_cap = want;
  }
  k_item_owner<<<grid_for(n, 256, sms * 16), 256, 0, st>>>(g->ioff, n, g->item_owner); TC_LAUNCHED();
  const size_t smem = owner_hash_smem(chunk);
  const bool wide = g->params.hash_block == 2 * kHashBlock;
  const int threads = wide ? 2 * kHashBlock : kHashBlock;
  const void* kern = wide ? (const void*)k_owner_hash<2 * kHashBlock>
                          : (const void*)k_owner_hash<kHashBlock>;
  TC_CUDA_TRY(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  int per_sm = 0;
  TC_CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, threads, smem));
  if (per_sm < 1) per_sm = 1;
  unsigned grid = (unsigned)(sms * per_sm);
  if (nitems < grid) grid = (unsigned)nitems;
  TC_CUDA_TRY(cudaEventRecord(g->ev[4], st));
  const uint32_t force_sorted = g->params.sorted_lookup ? 1u : 0u;
  if (wide)
    k_owner_hash<2 * kHashBlock><<<grid, threads, smem, st>>>(
        g->row_ptr, g->col, g->lcol, g->lsplit, g->ooff, g->ostream, g->ioff, g->item_owner,
        nitems, chunk, per_item, force_sorted, g->voff, g->batch_k, g->gcount, g->ctr);
  else
    k_owner_hash<kHashBlock><<<grid, threads, smem, st>>>(
        g->row_ptr, g->col, g->lcol, g->lsplit, g->ooff, g->ostream, g->ioff, g->item_owner,
        nitems, chunk, per_item, force_sorted, g->voff, g->batch_k, g->gcount, g->ctr);
  TC_LAUNCHED();
  TC_CUDA_TRY(cudaGetLastError());
  return TC_OK;
}

}  // namespace tc

// Cover edges and their intersections: the counting step of Algorithm CETC-Seq
// (Section "Cover-Edge Triangle Counting"), computed in the parallel shape of
// Algorithm CETC-SM.
//
// k_cover        one thread per adjacency entry (u, v): a horizontal edge with
//                u < v (L(u) == L(v), Definition "BFS-Edge") is a cover edge
//                (Theorem "Cover-Edge Set Generation").  It is appended to the
//                cover list.  If both degrees are <= small_max_degree the thread
//                intersects the two rows itself (the two-pointer merge of
//                Algorithm EMP); otherwise the edge goes to the endpoint of
//                larger degree, its "owner", for the hash path.
// k_bucket       groups the hash-path edges by owner (counting sort).
// k_owner_hash   one CTA per work item (owner h, chunk c of N(h), slice of h's
//                cover edges): chunk c is loaded into a shared-memory hash table
//                (the scatter / probe / clear scheme of Algorithm EHP), tagged
//                per entry with L(w) == L(h); each cover edge {h, x} then
//                streams the part of N(x) inside the chunk's id range through
//                the table.  Each common neighbour w is counted by the rule of
//                Algorithm CETC-Seq: when L(w) != L(u), or L(w) == L(u) and
//                v < w, with u < v the edge's endpoints; c1 / c2 of Algorithm
//                CETC-SM are kept beside T.
// Per-thread counts are reduced by warp shuffles and one atomic per CTA.
#include "tc_internal.cuh"

namespace tc {

namespace {

constexpr int kCoverBlock = 256;
constexpr int kCoverEntriesPerBlock = 2048;
constexpr uint32_t kEmpty = 0xFFFFFFFFu;
constexpr uint32_t kSameLevel = 0x80000000u;
constexpr int kHashBlock = 512;

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

struct Tally {
  unsigned long long t = 0, c1 = 0, c2 = 0;
  __device__ __forceinline__ void add(bool same, uint32_t v, uint32_t w) {
    if (!same) {
      ++t;
      ++c1;
    } else {
      ++c2;
      if (v < w) ++t;
    }
  }
};

__device__ __forceinline__ void flush_tally(Tally tl, DevCounters* ctr) {
  __shared__ unsigned long long red[3][32];
  tl.t = warp_sum(tl.t);
  tl.c1 = warp_sum(tl.c1);
  tl.c2 = warp_sum(tl.c2);
  const unsigned lane = lane_id(), warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
  if (lane == 0) {
    red[0][warp] = tl.t;
    red[1][warp] = tl.c1;
    red[2][warp] = tl.c2;
  }
  __syncthreads();
  if (warp == 0) {
    unsigned long long a = lane < nw ? red[0][lane] : 0, b = lane < nw ? red[1][lane] : 0,
                       c = lane < nw ? red[2][lane] : 0;
    a = warp_sum(a);
    b = warp_sum(b);
    c = warp_sum(c);
    if (lane == 0) {
      if (a) atomicAdd(&ctr->tri, a);
      if (b) atomicAdd(&ctr->c1, b);
      if (c) atomicAdd(&ctr->c2, c);
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
                                                       DevCounters* ctr) {
  __shared__ uint32_t s_lo, s_hi;
  Tally tl;
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
    for (unsigned long long b = e0; b < e1; b += kCoverBlock) {
      const unsigned long long j = b + threadIdx.x;
      bool is_cover = false, is_large = false;
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
              while (x < eu && y < ev) {
                const uint32_t a = col[x], c = col[y];
                if (a == c) {
                  tl.add(level[a] == lu, v, a);
                  ++x;
                  ++y;
                } else if (a < c) {
                  ++x;
                } else {
                  ++y;
                }
              }
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

// Work items per owner: ceil(d(h) / chunk) chunks x ceil(ocount / edges_per_item) slices.
__global__ void k_item_counts(const unsigned long long* __restrict__ row_ptr,
                              const uint32_t* __restrict__ ocount, uint32_t n, uint32_t chunk,
                              uint32_t per_item, uint32_t* __restrict__ icount,
                              DevCounters* ctr) {
  for (uint64_t h = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; h < n;
       h += (uint64_t)gridDim.x * blockDim.x) {
    const uint32_t oc = ocount[h];
    unsigned long long items = 0;
    if (oc) {
      const unsigned long long d = row_ptr[h + 1] - row_ptr[h];
      const unsigned long long chunks = (d + chunk - 1) / chunk;
      const unsigned long long slices = (oc + per_item - 1) / per_item;
      items = chunks * slices;
      if (items > 0xFFFFFFFFull) {  // tunables too fine for this owner: report, skip
        atomicOr(&ctr->err, kErrOverflow);
        items = 0;
      }
    }
    icount[h] = (uint32_t)items;
  }
}

__global__ void k_item_owner(const unsigned long long* __restrict__ ioff, uint32_t n,
                             uint32_t* __restrict__ item_owner) {
  for (uint64_t h = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; h < n;
       h += (uint64_t)gridDim.x * blockDim.x)
    for (unsigned long long i = ioff[h]; i < ioff[h + 1]; ++i) item_owner[i] = (uint32_t)h;
}

// First index in the sorted range col[a, b) whose value is >= t (warp-wide
// 32-ary search; all lanes get the answer).
__device__ __forceinline__ unsigned long long warp_lower_bound(const uint32_t* __restrict__ col,
                                                               unsigned long long a,
                                                               unsigned long long b, uint32_t t) {
  const unsigned lane = lane_id();
  while (b - a > 32) {
    const unsigned long long step = (b - a + 31) / 32;
    const unsigned long long idx = a + lane * step;
    const uint32_t val = idx < b ? col[idx] : 0xFFFFFFFFu;
    const unsigned k = __popc(__ballot_sync(0xffffffffu, val < t));
    if (k == 0) return a;
    const unsigned long long na = a + (k - 1) * step + 1;
    const unsigned long long nb = a + (unsigned long long)k * step;
    a = na;
    if (nb < b) b = nb;
  }
  const unsigned long long idx = a + lane;
  const uint32_t val = idx < b ? col[idx] : 0xFFFFFFFFu;
  return a + __popc(__ballot_sync(0xffffffffu, val < t));
}

__device__ __forceinline__ uint32_t hash_slot(uint32_t w, uint32_t mask) {
  return (w * 2654435761u) & mask;
}

__global__ void __launch_bounds__(kHashBlock) k_owner_hash(
    const unsigned long long* __restrict__ row_ptr, const uint32_t* __restrict__ col,
    const int32_t* __restrict__ level, uint32_t n, const unsigned long long* __restrict__ ooff,
    const uint32_t* __restrict__ ostream, const unsigned long long* __restrict__ ioff,
    const uint32_t* __restrict__ item_owner, unsigned long long nitems, uint32_t chunk,
    uint32_t per_item, DevCounters* ctr) {
  extern __shared__ uint32_t table[];
  __shared__ unsigned long long s_item;
  const unsigned lane = lane_id(), warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
  Tally tl;
  for (;;) {
    if (threadIdx.x == 0) s_item = atomicAdd(&ctr->item_cursor, 1ull);
    __syncthreads();
    const unsigned long long item = s_item;
    if (item >= nitems) break;
    const uint32_t h = item_owner[item];
    const unsigned long long hb = row_ptr[h], he = row_ptr[h + 1];
    const unsigned long long dh = he - hb;
    const uint32_t chunks = (uint32_t)((dh + chunk - 1) / chunk);
    const unsigned long long local = item - ioff[h];
    const uint32_t c = (uint32_t)(local % chunks);
    const unsigned long long s = local / chunks;
    const unsigned long long cb = hb + (unsigned long long)c * chunk;
    const unsigned long long ce = min(he, cb + chunk);
    const uint32_t lo_id = col[cb], hi_id = col[ce - 1];
    const int32_t lh = level[h];
    const unsigned long long eb = ooff[h] + s * per_item;
    const unsigned long long ee = min(ooff[h + 1], eb + per_item);

    // table size for this chunk: a power of two >= 2 * entries (load <= 1/2)
    uint32_t cap = 64;
    while (cap < 2 * (uint32_t)(ce - cb)) cap <<= 1;
    const uint32_t mask = cap - 1;
    for (uint32_t i = threadIdx.x; i < cap; i += blockDim.x) table[i] = kEmpty;
    __syncthreads();
    for (unsigned long long j = cb + threadIdx.x; j < ce; j += blockDim.x) {
      const uint32_t w = col[j];
      const uint32_t key = w | (level[w] == lh ? kSameLevel : 0u);
      uint32_t slot = hash_slot(w, mask);
      while (atomicCAS(&table[slot], kEmpty, key) != kEmpty) slot = (slot + 1) & mask;
    }
    __syncthreads();
    for (unsigned long long e = eb + warp; e < ee; e += nw) {
      const uint32_t x = ostream[e];
      const uint32_t v = x > h ? x : h;
      unsigned long long xb = row_ptr[x], xe = row_ptr[x + 1];
      if (chunks > 1) {
        xb = warp_lower_bound(col, xb, xe, lo_id);
        xe = warp_lower_bound(col, xb, xe, hi_id + 1);
      }
      for (unsigned long long j = xb + lane; j < xe; j += 32) {
        const uint32_t w = col[j];
        uint32_t slot = hash_slot(w, mask);
        for (;;) {
          const uint32_t k = table[slot];
          if (k == kEmpty) break;
          if ((k & ~kSameLevel) == w) {
            tl.add((k & kSameLevel) != 0, v, w);
            break;
          }
          slot = (slot + 1) & mask;
        }
      }
    }
    __syncthreads();
  }
  flush_tally(tl, ctr);
}

}  // namespace

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
      g->row_ptr, g->col, g->level, n, g->nnz, small_max, g->cover, g->large, g->ocount, g->ctr); TC_LAUNCHED();
  TC_CUDA_TRY(cudaGetLastError());
  TC_CUDA_TRY(cudaEventRecord(g->ev[2], st));
  TC_TRY(exclusive_scan_u32(g->ocount, g->ooff, n, g->scan, st));
  TC_CUDA_TRY(cudaMemcpyAsync(g->ctr_host, g->ctr, sizeof(DevCounters), cudaMemcpyDeviceToHost, st));
  TC_CUDA_TRY(cudaStreamSynchronize(st));
  const unsigned long long nlarge = g->ctr_host->num_large;
  if (nlarge == 0) return TC_OK;
  TC_CUDA_TRY(cudaMemsetAsync(g->ofill, 0, sizeof(uint32_t) * n, st));
  k_bucket<<<grid_for(nlarge, 256, sms * 16), 256, 0, st>>>(g->large, nlarge, g->ooff, g->ofill,
                                                           g->ostream); TC_LAUNCHED();
  const uint32_t chunk = g->params.hash_chunk;
  const uint32_t per_item = g->params.edges_per_item;
  k_item_counts<<<grid_for(n, 256, sms * 16), 256, 0, st>>>(g->row_ptr, g->ocount, n, chunk,
                                                           per_item, g->fdeg, g->ctr); TC_LAUNCHED();
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
  const uint32_t cap = 2 * chunk;
  const size_t smem = sizeof(uint32_t) * cap;
  TC_CUDA_TRY(cudaFuncSetAttribute(k_owner_hash, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                   (int)smem));
  int per_sm = 0;
  TC_CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_owner_hash, kHashBlock, smem));
  if (per_sm < 1) per_sm = 1;
  unsigned grid = (unsigned)(sms * per_sm);
  if (nitems < grid) grid = (unsigned)nitems;
  TC_CUDA_TRY(cudaEventRecord(g->ev[4], st));
  k_owner_hash<<<grid, kHashBlock, smem, st>>>(g->row_ptr, g->col, g->level, n, g->ooff,
                                              g->ostream, g->ioff, g->item_owner, nitems, chunk,
                                              per_item, g->ctr); TC_LAUNCHED();
  TC_CUDA_TRY(cudaGetLastError());
  return TC_OK;
}

}  // namespace tc

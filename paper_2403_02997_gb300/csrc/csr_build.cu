// Graph construction on the device: canonical undirected simple graph -> CSR
// with rows sorted ascending (the input form of every routine in the paper's
// evaluation framework, Section "Open Source Evaluation Framework"; the graph is
// undirected and simple per Section "Notations and Definitions").
//
//   1. k_make_keys     each pair (u, v), u != v, becomes the two keys
//                      (u << kb) | v and (v << kb) | u; self-loops become the
//                      all-ones sentinel, which sorts last;
//   2. LSD radix sort  8-bit digits over the 2*kb key bits: per pass a tile
//                      histogram, a scan of the digit-major histogram table and
//                      a stable scatter (warp match + per-warp digit counts);
//   3. k_dedup_*       drop repeats (a key equal to its predecessor) with a
//                      reduce-then-scan, write col[] and fill row_ptr[] at row
//                      starts, so empty rows get the offset of the next row.
#include "tc_internal.cuh"

namespace tc {

namespace {

constexpr unsigned long long kSentinel = ~0ull;

__global__ void k_make_keys(const uint32_t* __restrict__ src, const uint32_t* __restrict__ dst,
                            uint64_t E, uint32_t n, int kb, ulonglong2* __restrict__ keys,
                            DevCounters* ctr) {
  const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
  for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < E; i += stride) {
    uint32_t u = src[i], v = dst[i];
    ulonglong2 k;
    if (u >= n || v >= n) {
      atomicOr(&ctr->err, kErrVertexRange);
      k.x = k.y = kSentinel;
    } else if (u == v) {
      k.x = k.y = kSentinel;
    } else {
      k.x = ((unsigned long long)u << kb) | v;
      k.y = ((unsigned long long)v << kb) | u;
    }
    keys[i] = k;
  }
}

// The same for several graphs' edges in one array (EdgeGroups): a block takes a
// tile of edges and finds the graphs at its two ends once; each endpoint is
// checked against its own graph's vertex count and offset into the union.
constexpr unsigned long long kKeyTile = 2048;
__global__ void k_make_keys_multi(const uint32_t* __restrict__ src, const uint32_t* __restrict__ dst,
                                  uint64_t E, EdgeGroups grp, int kb,
                                  ulonglong2* __restrict__ keys, DevCounters* ctr) {
  __shared__ uint32_t s_g0, s_g1;
  for (unsigned long long t0 = (unsigned long long)blockIdx.x * kKeyTile; t0 < E;
       t0 += (unsigned long long)gridDim.x * kKeyTile) {
    const unsigned long long t1 = min((unsigned long long)E, t0 + kKeyTile);
    __syncthreads();
    if (threadIdx.x == 0) {
      s_g0 = batch_graph_of(grp.ein, 0, grp.k - 1, t0);
      s_g1 = batch_graph_of(grp.ein, s_g0, grp.k - 1, t1 - 1);
    }
    __syncthreads();
    const uint32_t g0 = s_g0, g1 = s_g1;
    for (unsigned long long i = t0 + threadIdx.x; i < t1; i += blockDim.x) {
      const uint32_t g = g0 == g1 ? g0 : batch_graph_of(grp.ein, g0, g1, i);
      const uint32_t u = src[i], v = dst[i], ng = grp.nvert[g];
      const unsigned long long off = grp.voff[g];
      ulonglong2 k;
      if (u >= ng || v >= ng) {
        atomicOr(&ctr->err, kErrVertexRange);
        k.x = k.y = kSentinel;
      } else if (u == v) {
        k.x = k.y = kSentinel;
      } else {
        k.x = ((off + u) << kb) | (off + v);
        k.y = ((off + v) << kb) | (off + u);
      }
      keys[i] = k;
    }
  }
}

constexpr int kRadixBits = 8;
constexpr int kRadix = 1 << kRadixBits;
constexpr int kSortBlock = 256;  // == kRadix: one digit owner per thread
constexpr int kSortItems = 16;  // 4096 keys (32 KB) per tile: 16 keys per digit on average
constexpr uint64_t kSortTile = (uint64_t)kSortBlock * kSortItems;
constexpr int kSortWarps = kSortBlock / 32;
static_assert(kSortBlock == kRadix, "digit ownership assumes one thread per digit");

__global__ void __launch_bounds__(kSortBlock) k_radix_hist(const unsigned long long* __restrict__ keys,
                                                           uint64_t N, int shift, uint32_t nb,
                                                           uint32_t* __restrict__ hist) {
  __shared__ uint32_t cnt[kRadix];
  cnt[threadIdx.x] = 0;
  __syncthreads();
  const uint64_t base = (uint64_t)blockIdx.x * kSortTile;
#pragma unroll 8
  for (int k = 0; k < kSortItems; ++k) {
    uint64_t i = base + (uint64_t)k * kSortBlock + threadIdx.x;
    if (i < N) atomicAdd(&cnt[(unsigned)(keys[i] >> shift) & (kRadix - 1)], 1u);
  }
  __syncthreads();
  hist[(uint64_t)threadIdx.x * nb + blockIdx.x] = cnt[threadIdx.x];
}

// Stable scatter, staged through shared memory so that the writes to each
// digit's output range go out as contiguous runs (about kSortTile / kRadix
// keys per digit and tile) instead of one scattered 8-byte write per key.
// The tile's keys are first ranked by digit in index order: they are taken in
// rounds of kSortBlock (round r, thread t holds key r*kSortBlock + t) and
// ranked within a round by (warp, lane), so equal digits keep their input
// order; thread d owns digit d and turns the per-warp counts of the round
// into positions in the tile's digit-sorted copy in shared memory.  Then the
// copy is written out in order, key p of the copy (digit d) to the digit's
// global offset for this tile plus p minus the digit's start in the copy.
__global__ void __launch_bounds__(kSortBlock) k_radix_scatter(const unsigned long long* __restrict__ in,
                                                              unsigned long long* __restrict__ out,
                                                              uint64_t N, int shift, uint32_t nb,
                                                              const unsigned long long* __restrict__ offs) {
  extern __shared__ unsigned long long s_keys[];  // kSortTile keys, digit-sorted
  __shared__ uint32_t wcnt[kSortWarps][kRadix];
  __shared__ uint32_t pos[kSortWarps][kRadix];
  __shared__ uint32_t s_start[kRadix];             // digit d's first position in s_keys
  __shared__ unsigned long long s_goff[kRadix];    // digit d's first output position
  const unsigned lane = lane_id(), warp = threadIdx.x >> 5, dd = threadIdx.x;
  const uint64_t base = (uint64_t)blockIdx.x * kSortTile;
  const uint32_t tile_n = (uint32_t)(N - base < kSortTile ? N - base : kSortTile);
  // the tile's digit counts are the steps of the histogram's scan (digit-
  // major, tile-minor: the entry after (d, tile) is the next one in the
  // scan's order, the total at the end), and their scan gives s_start
  __shared__ uint32_t s_tmp[kSortWarps + 1];
  const uint64_t hi = (uint64_t)dd * nb + blockIdx.x;
  const unsigned long long g0 = offs[hi];
  s_goff[dd] = g0;
  const uint32_t cnt = (uint32_t)(offs[hi + 1] - g0);
  uint32_t total = 0;
  s_start[dd] = block_exclusive_scan(cnt, s_tmp, &total);
#pragma unroll
  for (int w = 0; w < kSortWarps; ++w) wcnt[w][dd] = 0;
  __syncthreads();
  uint32_t run_off = s_start[dd];
  const unsigned lt_mask = (1u << lane) - 1u;
  for (int r = 0; r < kSortItems; ++r) {
    const uint32_t i = (uint32_t)r * kSortBlock + threadIdx.x;
    const bool valid = i < tile_n;
    const unsigned long long key = valid ? in[base + i] : 0ull;
    const unsigned d = valid ? ((unsigned)(key >> shift) & (kRadix - 1)) : (unsigned)kRadix;
    const unsigned peers = __match_any_sync(0xffffffffu, d);
    const unsigned lower = __popc(peers & lt_mask);
    if (valid && lower == 0) wcnt[warp][d] = __popc(peers);
    __syncthreads();
#pragma unroll
    for (int w = 0; w < kSortWarps; ++w) {
      const uint32_t c = wcnt[w][dd];
      wcnt[w][dd] = 0;
      pos[w][dd] = run_off;
      run_off += c;
    }
    __syncthreads();
    if (valid) s_keys[pos[warp][d] + lower] = key;
  }
  __syncthreads();
  for (uint32_t p = threadIdx.x; p < tile_n; p += kSortBlock) {
    const unsigned long long key = s_keys[p];
    const unsigned d = (unsigned)(key >> shift) & (kRadix - 1);
    out[s_goff[d] + (p - s_start[d])] = key;
  }
}

// The scatter's static plus dynamic shared memory is above the 48 KB a launch
// gets without opting in.
cudaError_t radix_scatter_smem() {
  return cudaFuncSetAttribute(k_radix_scatter, cudaFuncAttributeMaxDynamicSharedMemorySize,
                              (int)(kSortTile * sizeof(unsigned long long)));
}

constexpr int kDedupBlock = 512;
constexpr int kDedupItems = 8;
constexpr uint64_t kDedupTile = (uint64_t)kDedupBlock * kDedupItems;

__device__ __forceinline__ bool is_kept(const unsigned long long* keys, uint64_t i,
                                        unsigned long long k) {
  return k != kSentinel && (i == 0 || keys[i - 1] != k);
}

__global__ void __launch_bounds__(kDedupBlock) k_dedup_reduce(const unsigned long long* __restrict__ keys,
                                                              uint64_t N,
                                                              unsigned long long* __restrict__ sums) {
  __shared__ unsigned long long tmp[kDedupBlock / 32 + 1];
  const uint64_t base = (uint64_t)blockIdx.x * kDedupTile;
  unsigned long long c = 0;
#pragma unroll
  for (int k = 0; k < kDedupItems; ++k) {
    uint64_t i = base + (uint64_t)k * kDedupBlock + threadIdx.x;
    if (i < N && is_kept(keys, i, keys[i])) ++c;
  }
  c = block_sum(c, tmp);
  if (threadIdx.x == 0) sums[blockIdx.x] = c;
}

// Writes col[] and row_ptr[].  A kept key that starts row u sets row_ptr[x] for
// every x in (previous key's row, u]; the last non-sentinel key (kept or a
// repeat) sets row_ptr[x] = nnz for x in (its row, n].
__global__ void __launch_bounds__(kDedupBlock) k_dedup_write(const unsigned long long* __restrict__ keys,
                                                             uint64_t N, int kb, uint32_t n,
                                                             const unsigned long long* __restrict__ offs,
                                                             const unsigned long long* __restrict__ nnz_ptr,
                                                             uint32_t* __restrict__ col,
                                                             unsigned long long* __restrict__ row_ptr) {
  __shared__ unsigned long long tmp[kDedupBlock / 32 + 1];
  const uint64_t base = (uint64_t)blockIdx.x * kDedupTile + (uint64_t)threadIdx.x * kDedupItems;
  const unsigned long long vmask = (1ull << kb) - 1ull;
  unsigned long long kv[kDedupItems];
  unsigned flags = 0;
  unsigned long long c = 0;
#pragma unroll
  for (int k = 0; k < kDedupItems; ++k) {
    uint64_t i = base + k;
    kv[k] = i < N ? keys[i] : kSentinel;
    if (i < N && is_kept(keys, i, kv[k])) {
      flags |= 1u << k;
      ++c;
    }
  }
  unsigned long long total;
  unsigned long long p = block_exclusive_scan(c, tmp, &total) + offs[blockIdx.x];
#pragma unroll
  for (int k = 0; k < kDedupItems; ++k) {
    const uint64_t i = base + k;
    const unsigned long long key = kv[k];
    if (key == kSentinel) continue;
    const long long u = (long long)(key >> kb);
    if (flags & (1u << k)) {
      col[p] = (uint32_t)(key & vmask);
      const long long prev_u = (i == 0) ? -1ll : (long long)(keys[i - 1] >> kb);
      if (prev_u < u)
        for (long long x = prev_u + 1; x <= u; ++x) row_ptr[x] = p;
      ++p;
    }
    if (i + 1 == N || keys[i + 1] == kSentinel) {
      const unsigned long long nnz = *nnz_ptr;
      for (long long x = u + 1; x <= (long long)n; ++x) row_ptr[x] = nnz;
    }
  }
}

__global__ void k_degree_stats(const unsigned long long* __restrict__ row_ptr, uint32_t n,
                               unsigned int* dmax) {
  unsigned best = 0;
  for (uint64_t v = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; v < n;
       v += (uint64_t)gridDim.x * blockDim.x)
    best = max(best, (unsigned)(row_ptr[v + 1] - row_ptr[v]));
  best = __reduce_max_sync(0xffffffffu, best);
  if (lane_id() == 0) atomicMax(dmax, best);
}

__global__ void k_maxdeg_vertex(const unsigned long long* __restrict__ row_ptr, uint32_t n,
                                const unsigned int* dmax, unsigned int* vmin) {
  const unsigned target = *dmax;
  unsigned best = 0xFFFFFFFFu;
  for (uint64_t v = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; v < n;
       v += (uint64_t)gridDim.x * blockDim.x)
    if ((unsigned)(row_ptr[v + 1] - row_ptr[v]) == target) best = min(best, (unsigned)v);
  best = __reduce_min_sync(0xffffffffu, best);
  if (lane_id() == 0 && best != 0xFFFFFFFFu) atomicMin(vmin, best);
}

}  // namespace

// Bits of a vertex id below n (at least 1).
int key_bits(uint32_t n) {
  if (n <= 2) return 1;
  uint32_t x = n - 1;
  int b = 0;
  while (x) {
    ++b;
    x >>= 1;
  }
  return b;
}


tc_status sort_keys(unsigned long long** keys, unsigned long long** tmp, uint64_t N, int bits,
                    cudaStream_t st) {
  if (N == 0) return TC_OK;
  const uint64_t nb = (N + kSortTile - 1) / kSortTile;
  if (nb > 0x7FFFFFFFull) return TC_ERR_OVERFLOW;
  const uint64_t hcount = (uint64_t)kRadix * nb;
  uint32_t* hist = nullptr;
  unsigned long long* hoff = nullptr;
  ScanScratch ss;
  ss.capacity = scan_scratch_entries(hcount + 1);
  tc_status status = TC_OK;
  if (cudaMalloc(&hist, sizeof(uint32_t) * hcount) != cudaSuccess ||
      cudaMalloc(&hoff, sizeof(unsigned long long) * (hcount + 1)) != cudaSuccess ||
      cudaMalloc(&ss.sums, sizeof(unsigned long long) * ss.capacity) != cudaSuccess)
    status = TC_ERR_OOM;
  if (status == TC_OK && radix_scatter_smem() != cudaSuccess) status = TC_ERR_CUDA;
  for (int shift = 0; shift < bits && status == TC_OK; shift += kRadixBits) {
    k_radix_hist<<<(unsigned)nb, kSortBlock, 0, st>>>(*keys, N, shift, (uint32_t)nb, hist); TC_LAUNCHED();
    status = exclusive_scan_u32(hist, hoff, hcount, ss, st);
    if (status != TC_OK) break;
    k_radix_scatter<<<(unsigned)nb, kSortBlock, kSortTile * sizeof(unsigned long long), st>>>(*keys, *tmp, N, shift, (uint32_t)nb, hoff); TC_LAUNCHED();
    unsigned long long* t = *keys;
    *keys = *tmp;
    *tmp = t;
  }
  if (status == TC_OK && cudaStreamSynchronize(st) != cudaSuccess) status = TC_ERR_CUDA;
  cudaFree(hist);
  cudaFree(hoff);
  cudaFree(ss.sums);
  return status;
}

tc_status build_csr(tc_graph* g, const uint32_t* d_src, const uint32_t* d_dst, uint64_t E,
                    cudaStream_t st, const EdgeGroups* groups) {
  const uint32_t n = g->n;
  const int kb = key_bits(n);
  const uint64_t N = 2 * E;
  unsigned long long* keys_a = nullptr;
  unsigned long long* keys_b = nullptr;
  uint32_t* hist = nullptr;
  unsigned long long* hoff = nullptr;
  tc_status status = TC_OK;
  auto fail = [&](tc_status s) {
    status = s;
    return s;
  };

  TC_CUDA_TRY(cudaMemsetAsync(g->ctr, 0, sizeof(DevCounters), st));
  g->row_ptr = nullptr;
  TC_CUDA_TRY(dev_alloc(g, &g->row_ptr, (size_t)n + 1, st));
  if (N == 0) {
    TC_CUDA_TRY(cudaMemsetAsync(g->row_ptr, 0, sizeof(unsigned long long) * ((size_t)n + 1), st));
    g->nnz = 0;
    g->m = 0;
  } else {
    const uint64_t nb = (N + kSortTile - 1) / kSortTile;
    const uint64_t ndb = (N + kDedupTile - 1) / kDedupTile;
    if (nb > 0x7FFFFFFFull) return TC_ERR_OVERFLOW;
    do {
      if (dev_alloc(g, &keys_a, N, st) != cudaSuccess) { fail(TC_ERR_OOM); break; }
      if (dev_alloc(g, &keys_b, N, st) != cudaSuccess) { fail(TC_ERR_OOM); break; }
      if (dev_alloc(g, &hist, (size_t)kRadix * nb, st) != cudaSuccess) { fail(TC_ERR_OOM); break; }
      const uint64_t hcount = (uint64_t)kRadix * nb;
      const uint64_t off_entries = (hcount > ndb ? hcount : ndb) + 1;
      if (dev_alloc(g, &hoff, off_entries, st) != cudaSuccess) { fail(TC_ERR_OOM); break; }
      ScanScratch ss;
      ss.capacity = scan_scratch_entries(off_entries);
      if (dev_alloc(g, &ss.sums, ss.capacity, st) != cudaSuccess) { fail(TC_ERR_OOM); break; }

      if (groups)
        k_make_keys_multi<<<grid_for(E, kKeyTile, 152 * 64), 256, 0, st>>>(
            d_src, d_dst, E, *groups, kb, reinterpret_cast<ulonglong2*>(keys_a), g->ctr);
      else
        k_make_keys<<<grid_for(E, 256, 152 * 64), 256, 0, st>>>(d_src, d_dst, E, n, kb,
                                                               reinterpret_cast<ulonglong2*>(keys_a),
                                                               g->ctr);
      TC_LAUNCHED();
      if (radix_scatter_smem() != cudaSuccess) fail(TC_ERR_CUDA);
      for (int shift = 0; shift < 2 * kb && status == TC_OK; shift += kRadixBits) {
        k_radix_hist<<<(unsigned)nb, kSortBlock, 0, st>>>(keys_a, N, shift, (uint32_t)nb, hist); TC_LAUNCHED();
        if (exclusive_scan_u32(hist, hoff, hcount, ss, st) != TC_OK) { fail(TC_ERR_CUDA); break; }
        k_radix_scatter<<<(unsigned)nb, kSortBlock, kSortTile * sizeof(unsigned long long), st>>>(keys_a, keys_b, N, shift, (uint32_t)nb, hoff); TC_LAUNCHED();
        unsigned long long* t = keys_a;
        keys_a = keys_b;
        keys_b = t;
      }
      if (status != TC_OK) { dev_free(g, ss.sums, st); break; }
      k_dedup_reduce<<<(unsigned)ndb, kDedupBlock, 0, st>>>(keys_a, N, hoff); TC_LAUNCHED();
      if (exclusive_scan_u64(hoff, hoff, ndb, ss, st) != TC_OK) { dev_free(g, ss.sums, st); fail(TC_ERR_CUDA); break; }
      unsigned long long nnz = 0;
      unsigned int err = 0;
      cudaMemcpyAsync(&nnz, hoff + ndb, sizeof(nnz), cudaMemcpyDeviceToHost, st);
      cudaMemcpyAsync(&err, &g->ctr->err, sizeof(err), cudaMemcpyDeviceToHost, st);
      if (cudaStreamSynchronize(st) != cudaSuccess) { dev_free(g, ss.sums, st); fail(TC_ERR_CUDA); break; }
      dev_free(g, ss.sums, st);
      if (err & kErrVertexRange) { fail(TC_ERR_VERTEX_RANGE); break; }
      g->nnz = nnz;
      g->m = nnz / 2;
      if (nnz == 0) {
        cudaMemsetAsync(g->row_ptr, 0, sizeof(unsigned long long) * ((size_t)n + 1), st);
        break;
      }
      // padded to a multiple of 4 entries plus 4, so 16-byte loads of any
      // aligned quad that starts inside the array stay inside the allocation
      const size_t col_alloc = ((size_t)nnz + 7) & ~(size_t)3;
      if (dev_alloc(g, &g->col, col_alloc, st) != cudaSuccess) { fail(TC_ERR_OOM); break; }
      cudaMemsetAsync(g->col + nnz, 0, sizeof(uint32_t) * (col_alloc - nnz), st);
      k_dedup_write<<<(unsigned)ndb, kDedupBlock, 0, st>>>(keys_a, N, kb, n, hoff, hoff + ndb, g->col,
                                                           g->row_ptr); TC_LAUNCHED();
    } while (0);
    cudaError_t e = cudaGetLastError();
    if (status == TC_OK && e != cudaSuccess) {
      set_last_cuda_error(e);
      status = TC_ERR_CUDA;
    }
    cudaStreamSynchronize(st);
    dev_free(g, keys_a, st);
    dev_free(g, keys_b, st);
    dev_free(g, hist, st);
    dev_free(g, hoff, st);
    if (status != TC_OK) return status;
  }
  // degree statistics: largest degree and the smallest vertex id that has it
  TC_CUDA_TRY(cudaMemsetAsync(g->ctr, 0, sizeof(DevCounters), st));
  TC_CUDA_TRY(cudaMemsetAsync(&g->ctr->dmax_vertex, 0xFF, sizeof(unsigned int), st));
  if (n > 0) {
    k_degree_stats<<<grid_for(n, 256, 152 * 16), 256, 0, st>>>(g->row_ptr, n, &g->ctr->dmax); TC_LAUNCHED();
    k_maxdeg_vertex<<<grid_for(n, 256, 152 * 16), 256, 0, st>>>(g->row_ptr, n, &g->ctr->dmax,
                                                               &g->ctr->dmax_vertex); TC_LAUNCHED();
    TC_CUDA_TRY(cudaGetLastError());
  }
  TC_CUDA_TRY(cudaMemcpyAsync(g->ctr_host, g->ctr, sizeof(DevCounters), cudaMemcpyDeviceToHost, st));
  TC_CUDA_TRY(cudaStreamSynchronize(st));
  g->d_max = g->ctr_host->dmax;
  g->maxdeg_vertex = (n == 0 || g->ctr_host->dmax_vertex == 0xFFFFFFFFu) ? 0 : g->ctr_host->dmax_vertex;
  TC_CUDA_TRY(cudaMemsetAsync(g->ctr, 0, sizeof(DevCounters), st));
  return TC_OK;
}

}  // namespace tc

// Batched counting: k graphs counted together as one disjoint union.
//
// The union's CSR is the concatenation of the graphs' CSRs, with per-graph
// vertex offsets voff and entry offsets eoff (vertex v of graph i becomes
// voff[i] + v).  Because the graphs share no vertex:
//  - one multi-source BFS from every graph's root gives each graph's levels
//    (a BFS never crosses into another graph);
//  - the restart rule is unchanged: every other component of graph i still
//    starts at its smallest id, which stays the smallest after the offset;
//  - every cover edge and every apex lies inside one graph, so the count
//    kernels add each hit to that graph's counter.
// All phases therefore run as single launches over the whole batch -- one
// sequence of launches for all k graphs instead of k sequences.
#include <algorithm>
#include <cstring>
#include <new>
#include <vector>

#include "tc_internal.cuh"

struct tc_batch {
  tc_graph* u = nullptr;                   // the union (owns its CSR and count state)
  uint32_t k = 0;
  std::vector<uint32_t> part_n;            // vertices of each graph (the handles are not kept)
  std::vector<unsigned long long> voff_h;  // k + 1
  unsigned long long* voff = nullptr;      // device copies
  unsigned long long* eoff = nullptr;
  unsigned long long* gcount = nullptr;
  uint32_t* roots = nullptr;               // device, k
  uint32_t* order = nullptr;               // device, k: graphs largest first (persistent count)
  std::vector<uint32_t> order_h;           // host copy, made on the first persistent count
};

namespace tc {
namespace {

struct PartDesc {
  const unsigned long long* row_ptr;
  const uint32_t* col;
};

constexpr int kGatherBlock = 256;
constexpr unsigned long long kGatherTile = 4096;

// Union row offsets: row_ptr[voff[g] + v] = eoff[g] + part_g.row_ptr[v].
__global__ void k_gather_rows(const PartDesc* __restrict__ parts,
                              const unsigned long long* __restrict__ voff,
                              const unsigned long long* __restrict__ eoff, uint32_t k,
                              unsigned long long N, unsigned long long* __restrict__ row_ptr) {
  for (unsigned long long v = (unsigned long long)blockIdx.x * blockDim.x + threadIdx.x; v < N;
       v += (unsigned long long)gridDim.x * blockDim.x) {
    const uint32_t g = batch_graph_of(voff, 0, k - 1, v);
    row_ptr[v] = eoff[g] + parts[g].row_ptr[v - voff[g]];
  }
  if (blockIdx.x == 0 && threadIdx.x == 0) row_ptr[N] = eoff[k];
}

// Union neighbour ids: col[eoff[g] + j] = part_g.col[j] + voff[g].  A block
// takes a tile of entries and finds the graphs at its two ends once.
__global__ void __launch_bounds__(kGatherBlock) k_gather_cols(
    const PartDesc* __restrict__ parts, const unsigned long long* __restrict__ voff,
    const unsigned long long* __restrict__ eoff, uint32_t k, unsigned long long NNZ,
    uint32_t* __restrict__ col) {
  __shared__ uint32_t s_g0, s_g1;
  for (unsigned long long t0 = (unsigned long long)blockIdx.x * kGatherTile; t0 < NNZ;
       t0 += (unsigned long long)gridDim.x * kGatherTile) {
    const unsigned long long t1 = min(NNZ, t0 + kGatherTile);
    __syncthreads();
    if (threadIdx.x == 0) {
      s_g0 = batch_graph_of(eoff, 0, k - 1, t0);
      s_g1 = batch_graph_of(eoff, s_g0, k - 1, t1 - 1);
    }
    __syncthreads();
    const uint32_t g0 = s_g0, g1 = s_g1;
    for (unsigned long long j = t0 + threadIdx.x; j < t1; j += kGatherBlock) {
      const uint32_t g = g0 == g1 ? g0 : batch_graph_of(eoff, g0, g1, j);
      col[j] = parts[g].col[j - eoff[g]] + (uint32_t)voff[g];
    }
  }
}

__global__ void k_seed_roots(const uint32_t* __restrict__ roots, uint32_t k, int32_t* level,
                             uint32_t* queue) {
  for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < k; i += gridDim.x * blockDim.x) {
    level[roots[i]] = 0;
    queue[i] = roots[i];
  }
}

// Largest (degree, -local id) per graph: after the pass, best[g] >> 32 is the
// largest degree of graph g and ~best[g] & 0xFFFFFFFF its smallest such id.
__global__ void __launch_bounds__(kGatherBlock) k_batch_maxdeg(
    const unsigned long long* __restrict__ row_ptr, const unsigned long long* __restrict__ voff,
    uint32_t k, unsigned long long N, unsigned long long* best) {
  __shared__ uint32_t s_g0, s_g1;
  for (unsigned long long t0 = (unsigned long long)blockIdx.x * kGatherTile; t0 < N;
       t0 += (unsigned long long)gridDim.x * kGatherTile) {
    const unsigned long long t1 = min(N, t0 + kGatherTile);
    __syncthreads();
    if (threadIdx.x == 0) {
      s_g0 = batch_graph_of(voff, 0, k - 1, t0);
      s_g1 = batch_graph_of(voff, s_g0, k - 1, t1 - 1);
    }
    __syncthreads();
    const uint32_t g0 = s_g0, g1 = s_g1;
    for (unsigned long long v = t0 + threadIdx.x; v < t1; v += kGatherBlock) {
      const uint32_t g = g0 == g1 ? g0 : batch_graph_of(voff, g0, g1, v);
      const unsigned long long deg = row_ptr[v + 1] - row_ptr[v];
      const unsigned long long key = (deg << 32) | (0xFFFFFFFFull - (v - voff[g]));
      atomicMax(&best[g], key);
    }
  }
}

// Entry offsets of the graphs: out[g] = row_ptr[voff[g]], g = 0..k.
__global__ void k_graph_entries(const unsigned long long* __restrict__ row_ptr,
                                const unsigned long long* __restrict__ voff, uint32_t k,
                                unsigned long long* __restrict__ out) {
  for (uint32_t g = blockIdx.x * blockDim.x + threadIdx.x; g <= k; g += gridDim.x * blockDim.x)
    out[g] = row_ptr[voff[g]];
}

// Counters, host mirror and events of a union handle (a pooled handle's
// mirror is pageable: freeing pinned memory would synchronise the device).
tc_status init_union(tc_graph* u, cudaStream_t st) {
  params_default(&u->params);
  std::memset(&u->stats, 0, sizeof(u->stats));
  if (dev_alloc(u, &u->ctr, 1, st) != cudaSuccess) {
    cudaGetLastError();
    return TC_ERR_OOM;
  }
  if (u->pooled) {
    u->ctr_host = new (std::nothrow) DevCounters();
    if (!u->ctr_host) return TC_ERR_OOM;
  } else if (cudaMallocHost(reinterpret_cast<void**>(&u->ctr_host), sizeof(DevCounters)) !=
             cudaSuccess) {
    cudaGetLastError();
    return TC_ERR_OOM;
  }
  std::memset(u->ctr_host, 0, sizeof(DevCounters));
  for (cudaEvent_t& e : u->ev)
    if (cudaEventCreate(&e) != cudaSuccess) return TC_ERR_CUDA;
  return TC_OK;
}

// Frees a batch.  Every call on it finished its work before returning, so a
// pooled batch's memory goes back on the library's stream, with no
// device-wide synchronisation.
void free_batch(tc_batch* b) {
  if (!b) return;
  tc_graph* u = b->u;
  cudaStream_t fs = u && u->pooled ? free_stream() : nullptr;
  dev_free(u, b->voff, fs);
  dev_free(u, b->eoff, fs);
  dev_free(u, b->gcount, fs);
  dev_free(u, b->roots, fs);
  dev_free(u, b->order, fs);
  if (u) {
    u->voff = nullptr;
    u->gcount = nullptr;
    free_graph(u);
  }
  delete b;
}

}  // namespace
}  // namespace tc

using namespace tc;

extern "C" {

tc_status tc_batch_create(tc_graph* const* gs, size_t k, void* stream, tc_batch** out) {
  if (!out) return TC_ERR_INVALID_ARG;
  *out = nullptr;
  if (k == 0 || !gs || k > 0xFFFFFFFFull) return TC_ERR_INVALID_ARG;
  for (size_t i = 0; i < k; ++i)
    if (!gs[i]) return TC_ERR_INVALID_ARG;
  {  // the handles must be distinct
    std::vector<const tc_graph*> sorted(gs, gs + k);
    std::sort(sorted.begin(), sorted.end());
    if (std::adjacent_find(sorted.begin(), sorted.end()) != sorted.end()) return TC_ERR_INVALID_ARG;
  }
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  tc_batch* b = new (std::nothrow) tc_batch();
  if (!b) return TC_ERR_OOM;
  b->k = (uint32_t)k;
  b->part_n.resize(k);
  for (size_t i = 0; i < k; ++i) b->part_n[i] = gs[i]->n;
  std::vector<unsigned long long> voff(k + 1, 0), eoff(k + 1, 0);
  uint32_t dmax = 0;
  for (size_t i = 0; i < k; ++i) {
    voff[i + 1] = voff[i] + gs[i]->n;
    eoff[i + 1] = eoff[i] + gs[i]->nnz;
    dmax = gs[i]->d_max > dmax ? gs[i]->d_max : dmax;
  }
  if (voff[k] >= 0x80000000ull) {
    delete b;
    return TC_ERR_OVERFLOW;
  }
  b->voff_h = voff;
  tc_status s = TC_OK;
  PartDesc* d_parts = nullptr;
  do {
    tc_graph* u = new (std::nothrow) tc_graph();
    if (!u) { s = TC_ERR_OOM; break; }
    b->u = u;
    if ((s = init_union(u, st)) != TC_OK) break;
    u->n = (uint32_t)voff[k];
    u->nnz = eoff[k];
    u->m = u->nnz / 2;
    u->d_max = dmax;
    const size_t col_alloc = ((size_t)u->nnz + 7) & ~(size_t)3;
    if (cudaMalloc(&u->row_ptr, sizeof(unsigned long long) * (voff[k] + 1)) != cudaSuccess ||
        cudaMalloc(&u->col, sizeof(uint32_t) * col_alloc) != cudaSuccess ||
        cudaMalloc(&b->voff, sizeof(unsigned long long) * (k + 1)) != cudaSuccess ||
        cudaMalloc(&b->eoff, sizeof(unsigned long long) * (k + 1)) != cudaSuccess ||
        cudaMalloc(&b->gcount, sizeof(unsigned long long) * k) != cudaSuccess ||
        cudaMalloc(&b->roots, sizeof(uint32_t) * k) != cudaSuccess ||
        cudaMalloc(&d_parts, sizeof(PartDesc) * k) != cudaSuccess) {
      cudaGetLastError();
      s = TC_ERR_OOM;
      break;
    }
    std::vector<PartDesc> pd(k);
    for (size_t i = 0; i < k; ++i) pd[i] = PartDesc{gs[i]->row_ptr, gs[i]->col};
    if (cudaMemcpyAsync(d_parts, pd.data(), sizeof(PartDesc) * k, cudaMemcpyHostToDevice, st) != cudaSuccess ||
        cudaMemcpyAsync(b->voff, voff.data(), sizeof(unsigned long long) * (k + 1), cudaMemcpyHostToDevice, st) != cudaSuccess ||
        cudaMemcpyAsync(b->eoff, eoff.data(), sizeof(unsigned long long) * (k + 1), cudaMemcpyHostToDevice, st) != cudaSuccess ||
        cudaMemsetAsync(u->col + u->nnz, 0, sizeof(uint32_t) * (col_alloc - u->nnz), st) != cudaSuccess) {
      s = TC_ERR_CUDA;
      break;
    }
    const int sms = num_sms();
    k_gather_rows<<<grid_for(voff[k] + 1, 256, sms * 16), 256, 0, st>>>(d_parts, b->voff, b->eoff,
                                                                        b->k, voff[k], u->row_ptr);
    if (u->nnz)
      k_gather_cols<<<grid_for(u->nnz, kGatherTile, sms * 16), kGatherBlock, 0, st>>>(
          d_parts, b->voff, b->eoff, b->k, u->nnz, u->col);
    if (cudaGetLastError() != cudaSuccess) { s = TC_ERR_CUDA; break; }
    if ((s = alloc_count_state(u, st)) != TC_OK) break;
    u->batch_k = b->k;
    u->voff = b->voff;
    u->gcount = b->gcount;
    if (cudaStreamSynchronize(st) != cudaSuccess) { s = TC_ERR_CUDA; break; }
  } while (0);
  if (d_parts) {
    cudaStreamSynchronize(st);
    cudaFree(d_parts);
  }
  if (s != TC_OK) {
    free_batch(b);
    return s;
  }
  *out = b;
  return TC_OK;
}

tc_status tc_batch_create_from_edges(const uint32_t* src, const uint32_t* dst,
                                     const uint64_t* edge_offsets, const uint32_t* num_vertices,
                                     size_t k, int edges_on_device, void* stream, tc_batch** out) {
  if (!out) return TC_ERR_INVALID_ARG;
  *out = nullptr;
  if (k == 0 || k > 0xFFFFFFFFull || !edge_offsets || !num_vertices || edge_offsets[0] != 0)
    return TC_ERR_INVALID_ARG;
  for (size_t i = 0; i < k; ++i)
    if (edge_offsets[i + 1] < edge_offsets[i]) return TC_ERR_INVALID_ARG;
  const uint64_t E = edge_offsets[k];
  if (E > 0 && (!src || !dst)) return TC_ERR_INVALID_ARG;
  if (E > (1ull << 34)) return TC_ERR_OVERFLOW;
  std::vector<unsigned long long> voff(k + 1, 0);
  for (size_t i = 0; i < k; ++i) voff[i + 1] = voff[i] + num_vertices[i];
  if (voff[k] >= 0x80000000ull) return TC_ERR_OVERFLOW;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  tc_batch* b = new (std::nothrow) tc_batch();
  if (!b) return TC_ERR_OOM;
  b->k = (uint32_t)k;
  b->part_n.assign(num_vertices, num_vertices + k);
  b->voff_h = voff;
  tc_status s = TC_OK;
  uint32_t *staged_src = nullptr, *staged_dst = nullptr, *d_nvert = nullptr;
  do {
    tc_graph* u = new (std::nothrow) tc_graph();
    if (!u) { s = TC_ERR_OOM; break; }
    b->u = u;
    u->pooled = true;  // built and freed while other batches count (serving)
    if ((s = init_union(u, st)) != TC_OK) break;
    u->n = (uint32_t)voff[k];
    if (dev_alloc(u, &b->voff, k + 1, st) != cudaSuccess ||
        dev_alloc(u, &b->eoff, k + 1, st) != cudaSuccess ||
        dev_alloc(u, &b->gcount, k, st) != cudaSuccess ||
        dev_alloc(u, &b->roots, k, st) != cudaSuccess ||
        dev_alloc(u, &d_nvert, k, st) != cudaSuccess) {
      cudaGetLastError();
      s = TC_ERR_OOM;
      break;
    }
    // b->eoff holds the input edge offsets during the build
    if (cudaMemcpyAsync(b->voff, voff.data(), sizeof(unsigned long long) * (k + 1), cudaMemcpyHostToDevice, st) != cudaSuccess ||
        cudaMemcpyAsync(b->eoff, edge_offsets, sizeof(unsigned long long) * (k + 1), cudaMemcpyHostToDevice, st) != cudaSuccess ||
        cudaMemcpyAsync(d_nvert, num_vertices, sizeof(uint32_t) * k, cudaMemcpyHostToDevice, st) != cudaSuccess) {
      s = TC_ERR_CUDA;
      break;
    }
    const uint32_t* d_src = src;
    const uint32_t* d_dst = dst;
    if (E > 0 && !edges_on_device) {
      if (dev_alloc(u, &staged_src, E, st) != cudaSuccess ||
          dev_alloc(u, &staged_dst, E, st) != cudaSuccess) {
        cudaGetLastError();
        s = TC_ERR_OOM;
        break;
      }
      if (cudaMemcpyAsync(staged_src, src, sizeof(uint32_t) * E, cudaMemcpyHostToDevice, st) != cudaSuccess ||
          cudaMemcpyAsync(staged_dst, dst, sizeof(uint32_t) * E, cudaMemcpyHostToDevice, st) != cudaSuccess) {
        s = TC_ERR_CUDA;
        break;
      }
      d_src = staged_src;
      d_dst = staged_dst;
    }
    const EdgeGroups grp{b->eoff, b->voff, d_nvert, b->k};
    if ((s = build_csr(u, d_src, d_dst, E, st, &grp)) != TC_OK) break;
    if ((s = alloc_count_state(u, st)) != TC_OK) break;
    u->batch_k = b->k;
    u->voff = b->voff;
    u->gcount = b->gcount;
    if (cudaStreamSynchronize(st) != cudaSuccess) { s = TC_ERR_CUDA; break; }
  } while (0);
  // the staging and group arrays go back in stream order after their last use
  dev_free(b->u, staged_src, st);
  dev_free(b->u, staged_dst, st);
  dev_free(b->u, d_nvert, st);
  cudaStreamSynchronize(st);
  if (s != TC_OK) {
    free_batch(b);
    return s;
  }
  *out = b;
  return TC_OK;
}

tc_status tc_batch_max_degree_vertices(tc_batch* b, void* stream, uint32_t* host_roots) {
  if (!b || !host_roots) return TC_ERR_INVALID_ARG;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  tc_graph* u = b->u;
  std::vector<unsigned long long> best(b->k, 0);
  if (u->n > 0) {
    TC_CUDA_TRY(cudaMemsetAsync(b->gcount, 0, sizeof(unsigned long long) * b->k, st));
    k_batch_maxdeg<<<grid_for(u->n, kGatherTile, num_sms() * 16), kGatherBlock, 0, st>>>(
        u->row_ptr, b->voff, b->k, u->n, b->gcount);
    TC_CUDA_TRY(cudaGetLastError());
    TC_CUDA_TRY(cudaMemcpyAsync(best.data(), b->gcount, sizeof(unsigned long long) * b->k,
                                cudaMemcpyDeviceToHost, st));
    TC_CUDA_TRY(cudaStreamSynchronize(st));
  }
  for (uint32_t i = 0; i < b->k; ++i)
    host_roots[i] = b->part_n[i] ? (uint32_t)(0xFFFFFFFFull - (best[i] & 0xFFFFFFFFull)) : 0u;
  return TC_OK;
}

tc_status tc_batch_destroy(tc_batch* b) {
  if (!b) return TC_OK;
  free_batch(b);
  return TC_OK;
}

tc_status tc_batch_set_params(tc_batch* b, const tc_params* p) {
  if (!b || !b->u) return TC_ERR_INVALID_ARG;
  return tc_set_params(b->u, p);
}

tc_status tc_batch_count(tc_batch* b, const uint32_t* roots, void* stream, uint64_t* counts) {
  if (!b || !roots || !counts) return TC_ERR_INVALID_ARG;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  tc_graph* u = b->u;
  const uint32_t k = b->k;
  std::vector<uint32_t> ur;
  ur.reserve(k);
  for (uint32_t i = 0; i < k; ++i) {
    const uint32_t n = b->part_n[i];
    if (n == 0) continue;
    if (roots[i] >= n) return TC_ERR_INVALID_ARG;
    ur.push_back((uint32_t)(b->voff_h[i] + roots[i]));
  }
  std::memset(&u->stats, 0, sizeof(u->stats));
  u->stats.m = u->m;
  u->counted = false;
  if (u->n == 0) {
    for (uint32_t i = 0; i < k; ++i) counts[i] = 0;
    return TC_OK;
  }
  const uint32_t launches0 = g_launches;
  TC_CUDA_TRY(cudaEventRecord(u->ev[0], st));
  TC_CUDA_TRY(cudaMemcpyAsync(b->roots, ur.data(), sizeof(uint32_t) * ur.size(),
                              cudaMemcpyHostToDevice, st));
  TC_CUDA_TRY(cudaMemsetAsync(b->gcount, 0, sizeof(unsigned long long) * k, st));
  TC_CUDA_TRY(cudaMemsetAsync(u->level, 0xFF, sizeof(int32_t) * u->n, st));
  k_seed_roots<<<grid_for(ur.size(), 256, 1024), 256, 0, st>>>(b->roots, (uint32_t)ur.size(),
                                                              u->level, u->queue_a); TC_LAUNCHED();
  TC_CUDA_TRY(cudaGetLastError());
  TC_TRY(run_bfs_from_queue(u, ur.size(), st));
  TC_CUDA_TRY(cudaEventRecord(u->ev[1], st));
  TC_TRY(run_cover_and_count(u, st));
  TC_CUDA_TRY(cudaEventRecord(u->ev[3], st));
  std::vector<unsigned long long> gc(k);
  TC_CUDA_TRY(cudaMemcpyAsync(gc.data(), b->gcount, sizeof(unsigned long long) * k,
                              cudaMemcpyDeviceToHost, st));
  TC_CUDA_TRY(cudaMemcpyAsync(u->ctr_host, u->ctr, sizeof(DevCounters), cudaMemcpyDeviceToHost, st));
  TC_CUDA_TRY(cudaStreamSynchronize(st));
  const DevCounters& c = *u->ctr_host;
  if (c.err & kErrTimeout) return TC_ERR_TIMEOUT;
  if (c.err & kErrOverflow) return TC_ERR_OVERFLOW;
  if (c.err) return TC_ERR_CUDA;
  for (uint32_t i = 0; i < k; ++i) counts[i] = gc[i];
  u->stats.triangles = c.tri;
  u->stats.c1 = c.c1;
  u->stats.c2 = c.c2;
  u->stats.num_cover = c.num_cover;
  cudaEventElapsedTime(&u->stats.ms_bfs, u->ev[0], u->ev[1]);
  cudaEventElapsedTime(&u->stats.ms_cover, u->ev[1], u->ev[2]);
  cudaEventElapsedTime(&u->stats.ms_intersect, u->ev[2], u->ev[3]);
  cudaEventElapsedTime(&u->stats.ms_total, u->ev[0], u->ev[3]);
  if (c.items) cudaEventElapsedTime(&u->stats.ms_hash, u->ev[4], u->ev[3]);
  u->stats.launches = g_launches - launches0;
  u->stats.hash_items = c.items;
  u->stats.hash_edges = c.num_large;
  u->counted = true;
  return TC_OK;
}

tc_status tc_batch_count_persistent(tc_batch* b, const uint32_t* roots, void* stream,
                                    uint64_t* counts) {
  if (!b || !roots || !counts) return TC_ERR_INVALID_ARG;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  tc_graph* u = b->u;
  const uint32_t k = b->k;
  std::vector<uint32_t> gr(k, 0);
  for (uint32_t i = 0; i < k; ++i) {
    const uint32_t n = b->part_n[i];
    if (n == 0) continue;
    if (roots[i] >= n) return TC_ERR_INVALID_ARG;
    gr[i] = (uint32_t)(b->voff_h[i] + roots[i]);
  }
  std::memset(&u->stats, 0, sizeof(u->stats));
  u->stats.m = u->m;
  u->counted = false;
  const uint32_t launches0 = g_launches;
  if (!b->order) {  // once per batch: the graphs by entries, largest first
    unsigned long long* ent = nullptr;
    TC_CUDA_TRY(dev_alloc(u, &ent, (size_t)k + 1, st));
    k_graph_entries<<<grid_for(k + 1, 256, 64), 256, 0, st>>>(u->row_ptr, b->voff, k, ent); TC_LAUNCHED();
    std::vector<unsigned long long> eh(k + 1);
    cudaError_t e = cudaMemcpyAsync(eh.data(), ent, sizeof(unsigned long long) * (k + 1),
                                    cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    dev_free(u, ent, st);
    if (e != cudaSuccess) {
      set_last_cuda_error(e);
      return TC_ERR_CUDA;
    }
    b->order_h.resize(k);
    for (uint32_t i = 0; i < k; ++i) b->order_h[i] = i;
    std::stable_sort(b->order_h.begin(), b->order_h.end(), [&](uint32_t x, uint32_t y) {
      return eh[x + 1] - eh[x] > eh[y + 1] - eh[y];
    });
    TC_CUDA_TRY(dev_alloc(u, &b->order, k, st));
    TC_CUDA_TRY(cudaMemcpyAsync(b->order, b->order_h.data(), sizeof(uint32_t) * k,
                                cudaMemcpyHostToDevice, st));
  }
  TC_CUDA_TRY(cudaEventRecord(u->ev[0], st));
  TC_CUDA_TRY(cudaMemcpyAsync(b->roots, gr.data(), sizeof(uint32_t) * k, cudaMemcpyHostToDevice,
                              st));
  TC_TRY(run_batch_graphs(u, b->voff, b->roots, b->order, k, b->gcount, st));
  TC_CUDA_TRY(cudaEventRecord(u->ev[3], st));
  std::vector<unsigned long long> gc(k);
  TC_CUDA_TRY(cudaMemcpyAsync(gc.data(), b->gcount, sizeof(unsigned long long) * k,
                              cudaMemcpyDeviceToHost, st));
  TC_CUDA_TRY(cudaMemcpyAsync(u->ctr_host, u->ctr, sizeof(DevCounters), cudaMemcpyDeviceToHost, st));
  TC_CUDA_TRY(cudaStreamSynchronize(st));
  const DevCounters& c = *u->ctr_host;
  if (c.err) return TC_ERR_CUDA;
  for (uint32_t i = 0; i < k; ++i) counts[i] = gc[i];
  u->stats.triangles = c.tri;
  u->stats.c1 = c.c1;
  u->stats.c2 = c.c2;
  u->stats.num_cover = c.num_cover;
  cudaEventElapsedTime(&u->stats.ms_total, u->ev[0], u->ev[3]);
  u->stats.ms_intersect = u->stats.ms_total;
  u->stats.launches = g_launches - launches0;
  u->counted = true;
  return TC_OK;
}

tc_status tc_batch_get_stats(const tc_batch* b, tc_stats* out) {
  if (!b || !out) return TC_ERR_INVALID_ARG;
  *out = b->u->stats;
  return TC_OK;
}

tc_status tc_batch_get_levels(const tc_batch* b, size_t i, int32_t* host_levels) {
  if (!b || i >= b->k || !b->u->counted) return TC_ERR_INVALID_ARG;
  const uint32_t n = b->part_n[i];
  if (n == 0) return TC_OK;
  if (!host_levels) return TC_ERR_INVALID_ARG;
  TC_CUDA_TRY(cudaDeviceSynchronize());
  std::vector<int32_t> tmp(n);
  TC_CUDA_TRY(cudaMemcpy(tmp.data(), b->u->level + b->voff_h[i], sizeof(int32_t) * n,
                         cudaMemcpyDeviceToHost));
  for (uint32_t v = 0; v < n; ++v) host_levels[v] = tmp[v];
  return TC_OK;
}

tc_status tc_count_many(tc_graph* const* gs, const uint32_t* roots, size_t k, void* stream,
                        uint64_t* counts) {
  if (k == 0) return TC_OK;
  if (!gs || !roots || !counts) return TC_ERR_INVALID_ARG;
  for (size_t i = 0; i < k; ++i) {
    if (!gs[i]) return TC_ERR_INVALID_ARG;
    if (gs[i]->n > 0 && roots[i] >= gs[i]->n) return TC_ERR_INVALID_ARG;
  }
  tc_batch* b = nullptr;
  TC_TRY(tc_batch_create(gs, k, stream, &b));
  b->u->params = gs[0]->params;
  b->u->params.test_barrier_skip = 0;
  const tc_status s = tc_batch_count(b, roots, stream, counts);
  tc_batch_destroy(b);
  return s;
}

}  // extern "C"

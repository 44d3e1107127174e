// C ABI of libtc (declared in include/tc.h).  Argument checks, ownership of
// device memory, and the order of the phases; the arithmetic is in the kernels
// of csr_build.cu, bfs.cu and count.cu.
#include <cstdlib>
#include <cstring>
#include <mutex>
#include <new>
#include <vector>

#include "tc_internal.cuh"

namespace tc {

static thread_local cudaError_t g_last_cuda_error = cudaSuccess;

void set_last_cuda_error(cudaError_t e) { g_last_cuda_error = e; }

thread_local uint32_t g_launches = 0;

namespace {
constexpr int kMaxDevices = 64;
std::mutex g_dev_mu;
int g_sms[kMaxDevices] = {};
cudaMemPool_t g_pool[kMaxDevices] = {};
cudaStream_t g_free_stream[kMaxDevices] = {};

int current_device() {
  int dev = 0;
  cudaGetDevice(&dev);
  return dev >= 0 && dev < kMaxDevices ? dev : 0;
}

// The library's pool on the current device, created on first use.  Its
// release threshold is the largest value, so memory freed into it stays
// reserved for the next stream-ordered allocation instead of going back to
// the driver at every synchronisation (tc_pool_trim returns it).
cudaError_t lib_pool(cudaMemPool_t* pool) {
  const int dev = current_device();
  std::lock_guard<std::mutex> lock(g_dev_mu);
  if (!g_pool[dev]) {
    cudaMemPoolProps props;
    std::memset(&props, 0, sizeof(props));
    props.allocType = cudaMemAllocationTypePinned;
    props.location.type = cudaMemLocationTypeDevice;
    props.location.id = dev;
    cudaMemPool_t p = nullptr;
    cudaError_t e = cudaMemPoolCreate(&p, &props);
    if (e != cudaSuccess) return e;
    unsigned long long keep = ~0ull;
    e = cudaMemPoolSetAttribute(p, cudaMemPoolAttrReleaseThreshold, &keep);
    if (e != cudaSuccess) {
      cudaMemPoolDestroy(p);
      return e;
    }
    g_pool[dev] = p;
  }
  *pool = g_pool[dev];
  return cudaSuccess;
}
}  // namespace

int num_sms() {
  const int dev = current_device();
  std::lock_guard<std::mutex> lock(g_dev_mu);
  if (g_sms[dev] == 0) {
    int v = 0;
    cudaDeviceGetAttribute(&v, cudaDevAttrMultiProcessorCount, dev);
    g_sms[dev] = v > 0 ? v : 1;
  }
  return g_sms[dev];
}

cudaStream_t free_stream() {
  const int dev = current_device();
  std::lock_guard<std::mutex> lock(g_dev_mu);
  if (!g_free_stream[dev]) cudaStreamCreateWithFlags(&g_free_stream[dev], cudaStreamNonBlocking);
  return g_free_stream[dev];
}

cudaError_t dev_malloc(const tc_graph* g, void** p, size_t bytes, cudaStream_t st) {
  *p = nullptr;
  if (g && g->pooled) {
    cudaMemPool_t pool = nullptr;
    cudaError_t e = lib_pool(&pool);
    if (e != cudaSuccess) return e;
    return cudaMallocFromPoolAsync(p, bytes, pool, st);
  }
  return cudaMalloc(p, bytes);
}

void dev_free(const tc_graph* g, void* p, cudaStream_t st) {
  if (!p) return;
  if (g && g->pooled) cudaFreeAsync(p, st);
  else cudaFree(p);
}

namespace {

template <typename T>
tc_status dalloc(const tc_graph* g, T** p, size_t count, cudaStream_t st) {
  cudaError_t e = dev_alloc(g, p, count, st);
  if (e != cudaSuccess) {
    set_last_cuda_error(e);
    cudaGetLastError();
    return TC_ERR_OOM;
  }
  return TC_OK;
}

}  // namespace

void free_graph(tc_graph* g) {
  if (!g) return;
  void* ptrs[] = {g->row_ptr, g->col,   g->erow,   g->level,  g->queue_a, g->queue_b, g->qoff,
                  g->ooff,    g->ioff,  g->parent, g->fdeg,    g->ocount,  g->ofill,
                  g->cover,   g->large, g->ostream, g->item_owner, g->ctr, g->scan.sums,
                  g->lcol,    g->lsplit, g->tile_row, g->tile_cnt, g->medium, g->obeg,
                  g->ocol};
  // every call on the handle finished its work before returning: nothing is
  // pending on this memory, so pooled memory goes back on the library's stream
  cudaStream_t fs = g->pooled ? free_stream() : nullptr;
  for (void* p : ptrs) dev_free(g, p, fs);
  if (g->ctr_host) {
    if (g->pooled) delete g->ctr_host;
    else cudaFreeHost(g->ctr_host);
  }
  for (cudaEvent_t e : g->ev)
    if (e) cudaEventDestroy(e);
  delete g;
}

tc_status alloc_count_state(tc_graph* g, cudaStream_t st) {
  const size_t n = g->n, m = g->m;
  TC_TRY(dalloc(g, &g->level, n, st));
  TC_TRY(dalloc(g, &g->queue_a, n, st));
  TC_TRY(dalloc(g, &g->queue_b, n, st));
  TC_TRY(dalloc(g, &g->qoff, n + 1, st));
  TC_TRY(dalloc(g, &g->ooff, n + 1, st));
  TC_TRY(dalloc(g, &g->ioff, n + 1, st));
  TC_TRY(dalloc(g, &g->parent, n, st));
  TC_TRY(dalloc(g, &g->fdeg, n, st));
  TC_TRY(dalloc(g, &g->ocount, n, st));
  TC_TRY(dalloc(g, &g->ofill, n, st));
  TC_TRY(dalloc(g, &g->cover, m, st));
  TC_TRY(dalloc(g, &g->large, m, st));
  TC_TRY(dalloc(g, &g->ostream, m, st));
  TC_TRY(dalloc(g, &g->medium, m, st));
  TC_TRY(dalloc(g, &g->lcol, g->nnz, st));
  TC_TRY(dalloc(g, &g->lsplit, n, st));
  // tiles of rows longer than 4096 entries, 4096 per tile: at most nnz / 2048
  g->tile_cap = g->nnz / 2048 + 1;
  TC_TRY(dalloc(g, &g->tile_row, g->tile_cap, st));
  TC_TRY(dalloc(g, &g->tile_cnt, g->tile_cap, st));
  g->scan.capacity = scan_scratch_entries(n + 1);
  TC_TRY(dalloc(g, &g->scan.sums, g->scan.capacity, st));
  TC_TRY(dalloc(g, &g->erow, g->nnz, st));
  return fill_entry_rows(g, st);
}

void params_default(tc_params* p) {
  std::memset(p, 0, sizeof(*p));
  p->small_max_degree = 32;
  p->hash_chunk = 8192;
  p->edges_per_item = 512;
  p->bfs_alpha = 15;
  p->bfs_beta = 18;
  p->persistent_bfs = 1;
  p->barrier_timeout_ms = 2000;
  p->hash_block = 512;
  p->cluster_bfs = 1;
}

namespace {

tc_status sync_status(tc_graph* g, cudaStream_t st) {
  cudaError_t e = cudaStreamSynchronize(st);
  if (e != cudaSuccess) {
    set_last_cuda_error(e);
    return TC_ERR_CUDA;
  }
  (void)g;
  return TC_OK;
}

}  // namespace
}  // namespace tc

using namespace tc;

extern "C" {

tc_status tc_params_default(tc_params* p) {
  if (!p) return TC_ERR_INVALID_ARG;
  params_default(p);
  return TC_OK;
}

tc_status tc_set_params(tc_graph* g, const tc_params* p) {
  if (!g || !p) return TC_ERR_INVALID_ARG;
  const uint32_t c = p->hash_chunk;
  if (c < 32 || c > 16384 || c % 32 != 0) return TC_ERR_INVALID_ARG;
  if (p->hash_block != 512 && p->hash_block != 1024) return TC_ERR_INVALID_ARG;
  // edges per item: up to 2x (512-thread blocks) or 4x (1024) the block size
  // (above the block size they are clamped to it on graphs of 2^32 or more
  // adjacency entries, whose cursors take 64 bits)
  if (p->edges_per_item == 0 || p->edges_per_item > (p->hash_block == 1024 ? 4096u : 1024u) ||
      p->bfs_alpha == 0 ||
      p->bfs_beta == 0)
    return TC_ERR_INVALID_ARG;
  if (p->barrier_timeout_ms == 0 || p->barrier_timeout_ms > 600000) return TC_ERR_INVALID_ARG;
  if (p->medium_max_degree > 1024) return TC_ERR_INVALID_ARG;
  if (p->cluster_bfs > 1) return TC_ERR_INVALID_ARG;
  TC_TRY(owner_hash_fits(c, p->hash_block));
  g->params = *p;
  return TC_OK;
}

tc_status tc_graph_create(const uint32_t* src, const uint32_t* dst, uint64_t num_edges,
                          uint32_t num_vertices, int edges_on_device, void* stream,
                          tc_graph** out) {
  if (!out) return TC_ERR_INVALID_ARG;
  *out = nullptr;
  if (num_edges > 0 && (!src || !dst)) return TC_ERR_INVALID_ARG;
  if (num_vertices >= 0x80000000u) return TC_ERR_INVALID_ARG;
  if (num_edges > (1ull << 34)) return TC_ERR_OVERFLOW;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  tc_graph* g = new (std::nothrow) tc_graph();
  if (!g) return TC_ERR_OOM;
  // device memory comes stream-ordered from the library's pool: a graph built
  // after another was destroyed reuses its memory without mapping new pages,
  // and destroying one does not wait for the whole device
  g->pooled = true;
  params_default(&g->params);
  std::memset(&g->stats, 0, sizeof(g->stats));
  g->n = num_vertices;
  tc_status s = TC_OK;
  uint32_t* staged_src = nullptr;
  uint32_t* staged_dst = nullptr;
  do {
    if ((s = dalloc(g, &g->ctr, 1, st)) != TC_OK) break;
    // pageable: freeing pinned memory would synchronise the device
    g->ctr_host = new (std::nothrow) DevCounters();
    if (!g->ctr_host) {
      s = TC_ERR_OOM;
      break;
    }
    std::memset(g->ctr_host, 0, sizeof(DevCounters));
    bool ev_ok = true;
    for (cudaEvent_t& e : g->ev) ev_ok = ev_ok && cudaEventCreate(&e) == cudaSuccess;
    if (!ev_ok) { s = TC_ERR_CUDA; break; }
    const uint32_t* d_src = src;
    const uint32_t* d_dst = dst;
    if (num_edges > 0 && !edges_on_device) {
      if ((s = dalloc(g, &staged_src, num_edges, st)) != TC_OK) break;
      if ((s = dalloc(g, &staged_dst, num_edges, st)) != TC_OK) break;
      if (cudaMemcpyAsync(staged_src, src, sizeof(uint32_t) * num_edges, cudaMemcpyHostToDevice, st) != cudaSuccess ||
          cudaMemcpyAsync(staged_dst, dst, sizeof(uint32_t) * num_edges, cudaMemcpyHostToDevice, st) != cudaSuccess) {
        s = TC_ERR_CUDA;
        break;
      }
      d_src = staged_src;
      d_dst = staged_dst;
    }
    if ((s = build_csr(g, d_src, d_dst, num_edges, st)) != TC_OK) break;
    if ((s = alloc_count_state(g, st)) != TC_OK) break;
    s = sync_status(g, st);
  } while (0);
  // the staging buffers go back to the pool after the build that read them
  dev_free(g, staged_src, st);
  dev_free(g, staged_dst, st);
  if (s != TC_OK) {
    cudaStreamSynchronize(st);  // nothing of the failed build may still use the memory
    free_graph(g);
    return s;
  }
  *out = g;
  return TC_OK;
}

tc_status tc_graph_destroy(tc_graph* g) {
  if (!g) return TC_OK;
  // every call on the handle synchronised its own stream before returning, so
  // no work on its memory is pending: no device-wide synchronisation here
  free_graph(g);
  return TC_OK;
}

tc_status tc_pool_trim(uint64_t keep_bytes) {
  cudaMemPool_t pool = nullptr;
  TC_CUDA_TRY(lib_pool(&pool));
  TC_CUDA_TRY(cudaStreamSynchronize(free_stream()));
  TC_CUDA_TRY(cudaMemPoolTrimTo(pool, (size_t)keep_bytes));
  return TC_OK;
}

tc_status tc_pool_reserved(uint64_t* bytes) {
  if (!bytes) return TC_ERR_INVALID_ARG;
  cudaMemPool_t pool = nullptr;
  TC_CUDA_TRY(lib_pool(&pool));
  unsigned long long v = 0;
  TC_CUDA_TRY(cudaMemPoolGetAttribute(pool, cudaMemPoolAttrReservedMemCurrent, &v));
  *bytes = v;
  return TC_OK;
}

tc_status tc_graph_info(const tc_graph* g, uint32_t* n, uint64_t* m, uint32_t* d_max) {
  if (!g) return TC_ERR_INVALID_ARG;
  if (n) *n = g->n;
  if (m) *m = g->m;
  if (d_max) *d_max = g->d_max;
  return TC_OK;
}

tc_status tc_max_degree_vertex(const tc_graph* g, uint32_t* v) {
  if (!g || !v) return TC_ERR_INVALID_ARG;
  *v = g->maxdeg_vertex;
  return TC_OK;
}

namespace {

// Reads the counters of a count run on `st` (which events 0..3 bracket) into
// *count and the handle's statistics.
tc_status finish_count(tc_graph* g, cudaStream_t st, uint64_t* count, uint32_t launches0) {
  TC_CUDA_TRY(cudaEventRecord(g->ev[3], st));
  TC_CUDA_TRY(cudaMemcpyAsync(g->ctr_host, g->ctr, sizeof(DevCounters), cudaMemcpyDeviceToHost, st));
  TC_TRY(sync_status(g, st));
  const DevCounters& c = *g->ctr_host;
  if (c.err & kErrTimeout) return TC_ERR_TIMEOUT;
  if (c.err & kErrOverflow) return TC_ERR_OVERFLOW;
  if (c.err) return TC_ERR_CUDA;
  *count = c.tri;
  g->stats.triangles = c.tri;
  g->stats.c1 = c.c1;
  g->stats.c2 = c.c2;
  g->stats.num_cover = c.num_cover;
  cudaEventElapsedTime(&g->stats.ms_bfs, g->ev[0], g->ev[1]);
  cudaEventElapsedTime(&g->stats.ms_cover, g->ev[1], g->ev[2]);
  cudaEventElapsedTime(&g->stats.ms_intersect, g->ev[2], g->ev[3]);
  cudaEventElapsedTime(&g->stats.ms_total, g->ev[0], g->ev[3]);
  g->stats.ms_hash = 0.f;
  if (c.items) cudaEventElapsedTime(&g->stats.ms_hash, g->ev[4], g->ev[3]);
  g->stats.launches = g_launches - launches0;
  g->stats.hash_items = c.items;
  g->stats.hash_edges = c.num_large;
  return TC_OK;
}

// Common start of a count: statistics reset, argument checks.  Returns false
// (with *status set) when the count is finished or refused here.
bool begin_count(tc_graph* g, uint32_t root, bool needs_root, uint64_t* count, tc_status* status) {
  *status = TC_OK;
  if (!g || !count) {
    *status = TC_ERR_INVALID_ARG;
    return false;
  }
  std::memset(&g->stats, 0, sizeof(g->stats));
  g->stats.m = g->m;
  g->counted = false;
  if (g->n == 0) {
    *count = 0;
    g->counted = true;
    return false;
  }
  if (needs_root && root >= g->n) {
    *status = TC_ERR_INVALID_ARG;
    return false;
  }
  return true;
}

}  // namespace

tc_status tc_count(tc_graph* g, uint32_t root, void* stream, uint64_t* count) {
  tc_status s;
  if (!begin_count(g, root, true, count, &s)) return s;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  const uint32_t launches0 = g_launches;
  TC_CUDA_TRY(cudaEventRecord(g->ev[0], st));
  TC_TRY(run_bfs(g, root, st));
  TC_CUDA_TRY(cudaEventRecord(g->ev[1], st));
  TC_TRY(run_cover_and_count(g, st));
  TC_TRY(finish_count(g, st, count, launches0));
  g->counted = true;
  g->last_root = root;
  return TC_OK;
}

tc_status tc_list_triangles(tc_graph* g, uint32_t root, void* stream, uint32_t* triangles,
                            uint64_t capacity, uint64_t* vertex_counts, uint64_t* count,
                            uint64_t* written) {
  if (written) *written = 0;
  if (g && vertex_counts && g->n)
    TC_CUDA_TRY(cudaMemsetAsync(vertex_counts, 0, sizeof(uint64_t) * g->n,
                                static_cast<cudaStream_t>(stream)));
  tc_status s;
  if (!begin_count(g, root, true, count, &s)) return s;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  const uint32_t launches0 = g_launches;
  TC_CUDA_TRY(cudaEventRecord(g->ev[0], st));
  TC_TRY(run_bfs(g, root, st));
  TC_CUDA_TRY(cudaEventRecord(g->ev[1], st));
  const EmitSink sink{triangles, triangles ? capacity : 0,
                      reinterpret_cast<unsigned long long*>(vertex_counts)};
  TC_TRY(run_cover_and_list(g, sink, st));
  TC_TRY(finish_count(g, st, count, launches0));
  // every counted triangle was emitted exactly once
  if (triangles && g->ctr_host->listed != g->ctr_host->tri) return TC_ERR_CUDA;
  if (written) *written = triangles ? (*count < capacity ? *count : capacity) : 0;
  g->counted = true;
  g->last_root = root;
  return TC_OK;
}

tc_status tc_count_split(tc_graph* g, uint32_t root, void* stream, uint64_t* count) {
  tc_status s;
  if (!begin_count(g, root, true, count, &s)) return s;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  const uint32_t launches0 = g_launches;
  TC_CUDA_TRY(cudaEventRecord(g->ev[0], st));
  TC_TRY(run_bfs(g, root, st));
  TC_CUDA_TRY(cudaEventRecord(g->ev[1], st));
  TC_TRY(run_split_count(g, st));
  TC_TRY(finish_count(g, st, count, launches0));
  g->counted = true;
  g->last_root = root;
  return TC_OK;
}

tc_status tc_count_forward(tc_graph* g, void* stream, uint64_t* count) {
  tc_status s;
  if (!begin_count(g, 0, false, count, &s)) return s;
  g->counted = false;  // no levels or cover set behind this count
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  const uint32_t launches0 = g_launches;
  TC_CUDA_TRY(cudaEventRecord(g->ev[0], st));
  TC_CUDA_TRY(cudaEventRecord(g->ev[1], st));
  TC_TRY(run_forward_count(g, st));
  return finish_count(g, st, count, launches0);
}

tc_status tc_count_fe(tc_graph* g, uint32_t root, float threshold, void* stream, uint64_t* count,
                      int* used_forward) {
  tc_status s;
  if (used_forward) *used_forward = 0;
  if (!begin_count(g, root, true, count, &s)) return s;
  if (!(threshold >= 0.f)) return TC_ERR_INVALID_ARG;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  const uint32_t launches0 = g_launches;
  TC_CUDA_TRY(cudaEventRecord(g->ev[0], st));
  TC_TRY(run_bfs(g, root, st));
  unsigned long long num_cover = 0;
  TC_TRY(run_count_horizontal(g, st, &num_cover));
  TC_CUDA_TRY(cudaEventRecord(g->ev[1], st));
  const double c = g->m ? (double)num_cover / (double)g->m : 0.0;
  if (c < threshold) {
    TC_TRY(run_cover_and_count(g, st));
    TC_TRY(finish_count(g, st, count, launches0));
    g->counted = true;
    g->last_root = root;
    return TC_OK;
  }
  if (used_forward) *used_forward = 1;
  TC_TRY(run_forward_count(g, st));
  TC_TRY(finish_count(g, st, count, launches0));
  g->stats.num_cover = num_cover;
  return TC_OK;
}

tc_status tc_get_levels(const tc_graph* g, int32_t* host_levels) {
  if (!g || !host_levels) return TC_ERR_INVALID_ARG;
  if (!g->counted) return TC_ERR_INVALID_ARG;
  if (g->n == 0) return TC_OK;
  TC_CUDA_TRY(cudaDeviceSynchronize());
  TC_CUDA_TRY(cudaMemcpy(host_levels, g->level, sizeof(int32_t) * g->n, cudaMemcpyDeviceToHost));
  return TC_OK;
}

tc_status tc_get_cover_edges(const tc_graph* g, uint64_t* num_cover, uint32_t* host_u,
                             uint32_t* host_v) {
  if (!g || !num_cover) return TC_ERR_INVALID_ARG;
  if (!g->counted) return TC_ERR_INVALID_ARG;
  *num_cover = g->stats.num_cover;
  if (!host_u || !host_v || g->stats.num_cover == 0) return TC_OK;
  TC_CUDA_TRY(cudaDeviceSynchronize());
  std::vector<uint2> tmp(g->stats.num_cover);
  TC_CUDA_TRY(cudaMemcpy(tmp.data(), g->cover, sizeof(uint2) * tmp.size(), cudaMemcpyDeviceToHost));
  for (size_t i = 0; i < tmp.size(); ++i) {
    host_u[i] = tmp[i].x;
    host_v[i] = tmp[i].y;
  }
  return TC_OK;
}

tc_status tc_get_csr(const tc_graph* g, uint64_t* host_row_ptr, uint32_t* host_col) {
  if (!g || !host_row_ptr || (!host_col && g->nnz)) return TC_ERR_INVALID_ARG;
  TC_CUDA_TRY(cudaDeviceSynchronize());
  TC_CUDA_TRY(cudaMemcpy(host_row_ptr, g->row_ptr, sizeof(uint64_t) * ((size_t)g->n + 1),
                         cudaMemcpyDeviceToHost));
  if (g->nnz)
    TC_CUDA_TRY(cudaMemcpy(host_col, g->col, sizeof(uint32_t) * g->nnz, cudaMemcpyDeviceToHost));
  return TC_OK;
}

tc_status tc_get_stats(const tc_graph* g, tc_stats* out) {
  if (!g || !out) return TC_ERR_INVALID_ARG;
  *out = g->stats;
  return TC_OK;
}

const char* tc_status_string(tc_status s) {
  switch (s) {
    case TC_OK: return "TC_OK";
    case TC_ERR_INVALID_ARG: return "TC_ERR_INVALID_ARG: invalid argument";
    case TC_ERR_VERTEX_RANGE: return "TC_ERR_VERTEX_RANGE: edge endpoint >= num_vertices";
    case TC_ERR_OOM: return "TC_ERR_OOM: device allocation failed";
    case TC_ERR_CUDA: return "TC_ERR_CUDA: CUDA runtime error";
    case TC_ERR_TIMEOUT: return "TC_ERR_TIMEOUT: bounded device wait expired";
    case TC_ERR_OVERFLOW: return "TC_ERR_OVERFLOW: size beyond supported limits";
  }
  return "unknown tc_status";
}

}  // extern "C"

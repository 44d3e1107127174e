// tc_bfs_levels_noalloc: BFS levels of a caller-owned device CSR with no
// device allocation at all.
//
// Who needs it: applications that own every byte of device memory through
// their own pool or a fixed budget, and services that must not allocate once
// they are running (cudaMalloc may synchronise the device, and may fail under
// memory pressure at the worst moment).  They bring the graph (row offsets and
// neighbour ids) and the output array; the scratch this computation needs (two
// frontier queues, union-find parents and two counters) is one file-scope
// __device__ array of fixed size, present on every device that loads the
// library until the process exits.
//
// The kernels are variants of the level-synchronous search in bfs.cu: a
// top-down step with one warp per frontier vertex (no frontier scan, so no
// offset array), then the same restart rule -- every vertex not reached from
// the root gets its level from a search started at the smallest id of its
// component, found by union-find that hooks the larger root under the smaller.
#include <mutex>

#include "tc_internal.cuh"

namespace tc {
namespace {

constexpr uint32_t kNoallocMaxVertices = 1u << 20;
constexpr size_t kNoallocHeader = 256;  // counters
constexpr size_t kNoallocBytes = kNoallocHeader + 3 * sizeof(uint32_t) * (size_t)kNoallocMaxVertices;
constexpr int kMaxDevices = 64;

// Shared by every call on a device.  Calls whose device work overlaps (two
// streams, or two host threads, at the same time) race on it.
static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoallocBytes];

struct Scratch {
  unsigned long long* next_n;  // vertices appended to the next queue
  unsigned long long* unvisited;
  uint32_t* queue_a;
  uint32_t* queue_b;
  uint32_t* parent;
};

std::mutex g_mu;
void* g_base[kMaxDevices] = {};

// Device address of the scratch array on the current device, looked up once
// per device (cudaGetSymbolAddress with that device current).
tc_status scratch_on_current_device(Scratch* s) {
  int dev = 0;
  TC_CUDA_TRY(cudaGetDevice(&dev));
  if (dev < 0 || dev >= kMaxDevices) return TC_ERR_OVERFLOW;
  void* base = nullptr;
  {
    std::lock_guard<std::mutex> lock(g_mu);
    if (!g_base[dev]) {
      void* p = nullptr;
      const cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
      if (e != cudaSuccess || !p) {
        set_last_cuda_error(e);
        return TC_ERR_CUDA;
      }
      g_base[dev] = p;
    }
    base = g_base[dev];
  }
  unsigned char* b = static_cast<unsigned char*>(base);
  s->next_n = reinterpret_cast<unsigned long long*>(b);
  s->unvisited = reinterpret_cast<unsigned long long*>(b + 8);
  uint32_t* q = reinterpret_cast<uint32_t*>(b + kNoallocHeader);
  s->queue_a = q;
  s->queue_b = q + kNoallocMaxVertices;
  s->parent = q + 2 * (size_t)kNoallocMaxVertices;
  return TC_OK;
}

__device__ __forceinline__ void na_append(bool take, uint32_t value, uint32_t* queue,
                                          unsigned long long* len) {
  const unsigned mask = __ballot_sync(0xffffffffu, take);
  if (!mask) return;
  const unsigned lane = lane_id();
  const unsigned leader = __ffs(mask) - 1;
  unsigned long long base = 0;
  if (lane == leader) base = atomicAdd(len, (unsigned long long)__popc(mask));
  base = __shfl_sync(0xffffffffu, base, leader);
  if (take) queue[base + __popc(mask & ((1u << lane) - 1u))] = value;
}

__global__ void k_na_root(int32_t* level, uint32_t* queue, uint32_t root) {
  level[root] = 0;
  queue[0] = root;
}

// Top-down step, one warp per frontier vertex.
__global__ void k_na_td(const unsigned long long* __restrict__ row_ptr,
                        const uint32_t* __restrict__ col, int32_t* __restrict__ level,
                        const uint32_t* __restrict__ queue, unsigned long long qlen,
                        int32_t next_level, uint32_t* __restrict__ next_queue,
                        unsigned long long* next_n) {
  const unsigned lane = lane_id();
  const unsigned long long warps = (unsigned long long)gridDim.x * blockDim.x / 32;
  for (unsigned long long i = ((unsigned long long)blockIdx.x * blockDim.x + threadIdx.x) / 32;
       i < qlen; i += warps) {
    const uint32_t u = queue[i];
    const unsigned long long b = row_ptr[u], e = row_ptr[u + 1];
    for (unsigned long long j0 = b; j0 < e; j0 += 32) {
      const unsigned long long j = j0 + lane;
      bool take = false;
      uint32_t w = 0;
      if (j < e) {
        w = col[j];
        if (level[w] == -1) take = atomicCAS(&level[w], -1, next_level) == -1;
      }
      na_append(take, w, next_queue, next_n);
    }
  }
}

__global__ void k_na_unvisited(const int32_t* __restrict__ level, uint32_t n,
                               unsigned long long* unvisited) {
  unsigned long long c = 0;
  for (uint64_t v = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; v < n;
       v += (uint64_t)gridDim.x * blockDim.x)
    c += level[v] == -1;
  c = warp_sum(c);
  if (lane_id() == 0 && c) atomicAdd(unvisited, c);
}

__global__ void k_na_cc_init(uint32_t* parent, uint32_t n) {
  for (uint64_t v = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; v < n;
       v += (uint64_t)gridDim.x * blockDim.x)
    parent[v] = (uint32_t)v;
}

__device__ __forceinline__ uint32_t na_find(uint32_t* parent, uint32_t x) {
  uint32_t p = parent[x];
  while (p != x) {
    const uint32_t gp = parent[p];
    if (gp != p) parent[x] = gp;
    x = p;
    p = gp;
  }
  return x;
}

// Union over every edge {v, w}, w < v, of an unvisited vertex v (rows need not
// be sorted).  The larger root is hooked under the smaller with a CAS.
__global__ void k_na_cc_hook(const unsigned long long* __restrict__ row_ptr,
                             const uint32_t* __restrict__ col, const int32_t* __restrict__ level,
                             uint32_t* parent, uint32_t n) {
  const uint64_t warps = (uint64_t)gridDim.x * blockDim.x / 32;
  for (uint64_t v = ((uint64_t)blockIdx.x * blockDim.x + threadIdx.x) / 32; v < n; v += warps) {
    if (level[v] != -1) continue;
    const unsigned long long b = row_ptr[v], e = row_ptr[v + 1];
    for (unsigned long long j = b + lane_id(); j < e; j += 32) {
      const uint32_t w = col[j];
      if (w >= v) continue;
      uint32_t a = (uint32_t)v, c = w;
      for (;;) {
        a = na_find(parent, a);
        c = na_find(parent, c);
        if (a == c) break;
        const uint32_t hi = a > c ? a : c, lo = a > c ? c : a;
        if (atomicCAS(&parent[hi], hi, lo) == hi) break;
      }
    }
  }
}

__global__ void k_na_cc_seed(const uint32_t* __restrict__ parent, int32_t* __restrict__ level,
                             uint32_t n, uint32_t* __restrict__ queue,
                             unsigned long long* next_n) {
  const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
  const uint64_t iters = ((uint64_t)n + stride - 1) / stride;
  for (uint64_t it = 0; it < iters; ++it) {
    const uint64_t v = it * stride + (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
    bool take = false;
    if (v < n && level[v] == -1 && parent[v] == (uint32_t)v) {
      level[v] = 0;
      take = true;
    }
    na_append(take, (uint32_t)v, queue, next_n);
  }
}

tc_status read_u64(const unsigned long long* dev, unsigned long long* host, cudaStream_t st) {
  TC_CUDA_TRY(cudaMemcpyAsync(host, dev, sizeof(*host), cudaMemcpyDeviceToHost, st));
  TC_CUDA_TRY(cudaStreamSynchronize(st));
  return TC_OK;
}

// Level-synchronous top-down search from the qlen vertices in s.queue_a.
tc_status na_levels(const unsigned long long* row_ptr, const uint32_t* col, int32_t* level,
                    unsigned long long qlen, const Scratch& s, cudaStream_t st) {
  const int sms = num_sms();
  uint32_t* q = s.queue_a;
  uint32_t* nq = s.queue_b;
  for (int32_t lvl = 0; qlen > 0; ++lvl) {
    TC_CUDA_TRY(cudaMemsetAsync(s.next_n, 0, sizeof(unsigned long long), st));
    k_na_td<<<grid_for(qlen * 32, 256, sms * 8), 256, 0, st>>>(row_ptr, col, level, q, qlen,
                                                             lvl + 1, nq, s.next_n); TC_LAUNCHED();
    TC_CUDA_TRY(cudaGetLastError());
    TC_TRY(read_u64(s.next_n, &qlen, st));
    uint32_t* t = q;
    q = nq;
    nq = t;
  }
  return TC_OK;
}

}  // namespace
}  // namespace tc

using namespace tc;

extern "C" tc_status tc_bfs_levels_noalloc(const uint64_t* row_ptr, const uint32_t* col,
                                           uint32_t n, uint32_t root, int32_t* levels,
                                           void* stream) {
  if (n == 0) return TC_OK;
  if (!row_ptr || !col || !levels || root >= n) return TC_ERR_INVALID_ARG;
  if (n > kNoallocMaxVertices) return TC_ERR_OVERFLOW;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  Scratch s;
  TC_TRY(scratch_on_current_device(&s));
  const unsigned long long* rp = reinterpret_cast<const unsigned long long*>(row_ptr);
  const int sms = num_sms();
  // the scratch keeps the previous call's contents: every part used below is
  // written before it is read (queues by appends, parents by k_na_cc_init,
  // counters by the memsets)
  TC_CUDA_TRY(cudaMemsetAsync(levels, 0xFF, sizeof(int32_t) * n, st));
  k_na_root<<<1, 1, 0, st>>>(levels, s.queue_a, root); TC_LAUNCHED();
  TC_CUDA_TRY(cudaGetLastError());
  TC_TRY(na_levels(rp, col, levels, 1, s, st));
  TC_CUDA_TRY(cudaMemsetAsync(s.unvisited, 0, sizeof(unsigned long long), st));
  k_na_unvisited<<<sms * 8, 256, 0, st>>>(levels, n, s.unvisited); TC_LAUNCHED();
  TC_CUDA_TRY(cudaGetLastError());
  unsigned long long left = 0;
  TC_TRY(read_u64(s.unvisited, &left, st));
  if (left == 0) return TC_OK;
  k_na_cc_init<<<sms * 8, 256, 0, st>>>(s.parent, n); TC_LAUNCHED();
  k_na_cc_hook<<<sms * 16, 256, 0, st>>>(rp, col, levels, s.parent, n); TC_LAUNCHED();
  TC_CUDA_TRY(cudaMemsetAsync(s.next_n, 0, sizeof(unsigned long long), st));
  k_na_cc_seed<<<sms * 8, 256, 0, st>>>(s.parent, levels, n, s.queue_a, s.next_n); TC_LAUNCHED();
  TC_CUDA_TRY(cudaGetLastError());
  unsigned long long seeds = 0;
  TC_TRY(read_u64(s.next_n, &seeds, st));
  TC_TRY(na_levels(rp, col, levels, seeds, s, st));
  return TC_OK;
}

// BFS levels (Definition "BFS-Edge": L(v) = shortest distance from the root)
// with the restart rule of Algorithm CETC-Seq (a new search from every vertex
// still unvisited, taken in ascending id order), computed level-synchronously.
//
// Root phase: level-synchronous, direction-optimising (Beamer et al.):
//   top-down  k_bfs_td    frontier queue; edges of the frontier are spread
//                         evenly over the grid through a scan of frontier
//                         degrees, so a hub row uses every SM; a vertex is
//                         claimed with atomicCAS(level, -1, l+1);
//   bottom-up k_bfs_bu    every unvisited vertex scans its row (8 lanes per
//                         vertex, early exit) for a neighbour at level l.
//   Switch to bottom-up when the frontier's edges exceed the unexplored edges
//   / alpha; back to top-down when the frontier falls below n / beta.
// Small frontiers (long, thin graphs such as meshes and road networks, and the
//   tails of every search) run in one persistent cooperative kernel,
//   k_bfs_persistent: one block per SM, one warp per frontier vertex, and a
//   device-side grid barrier between levels, until the frontier empties or
//   grows past kPersistMaxVerts / kPersistMaxEdges.  Every barrier wait is
//   bounded by barrier_timeout_ms (%globaltimer); past it the kernel records
//   kErrTimeout and every block leaves, so a count fails with TC_ERR_TIMEOUT
//   instead of hanging.
// Restart phase: the vertices left unvisited form whole components.  Their
//   components are found by union-find that always hooks the larger root under
//   the smaller, so each root is its component's smallest id — exactly the
//   vertex the ascending restart loop starts from.  One multi-source BFS from
//   all those roots (level 0) then gives every level at once; components do not
//   interact, so the levels equal those of the sequential restarts.
#include <cooperative_groups.h>

#include "tc_internal.cuh"

namespace tc {

namespace {

constexpr int kTdBlock = 256;
constexpr int kTdEdgesPerBlock = 2048;
constexpr int kBuBlock = 256;
constexpr int kBuGroup = 8;

constexpr int kPersistBlock = 512;
constexpr unsigned long long kPersistMaxVerts = 1ull << 16;
constexpr unsigned long long kPersistMaxEdges = 1ull << 19;
constexpr unsigned int kPersistMaxDeg = 4096;  // one warp expands a vertex in the persistent kernel

__global__ void k_set_root(int32_t* level, uint32_t* queue, uint32_t root) {
  level[root] = 0;
  queue[0] = root;
}

__global__ void k_frontier_degrees(const uint32_t* __restrict__ queue, uint64_t qlen,
                                   const unsigned long long* __restrict__ row_ptr,
                                   uint32_t* __restrict__ fdeg, unsigned int* fmaxdeg) {
  unsigned int mx = 0;
  for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < qlen;
       i += (uint64_t)gridDim.x * blockDim.x) {
    uint32_t u = queue[i];
    const uint32_t d = (uint32_t)(row_ptr[u + 1] - row_ptr[u]);
    fdeg[i] = d;
    mx = d > mx ? d : mx;
  }
  mx = __reduce_max_sync(0xffffffffu, mx);
  if (lane_id() == 0 && mx) atomicMax(fmaxdeg, mx);
}

// Largest i in [lo, hi] with qoff[i] <= e (qoff nondecreasing, qoff[lo] <= e).
__device__ __forceinline__ uint64_t frontier_index(const unsigned long long* qoff, uint64_t lo,
                                                   uint64_t hi, unsigned long long e) {
  while (lo < hi) {
    uint64_t mid = lo + (hi - lo + 1) / 2;
    if (qoff[mid] <= e) lo = mid; else hi = mid - 1;
  }
  return lo;
}

__device__ __forceinline__ void warp_append(bool take, uint32_t value, uint32_t* queue,
                                            unsigned long long* len) {
  const unsigned mask = __ballot_sync(0xffffffffu, take);
  if (!mask) return;
  const unsigned lane = lane_id();
  unsigned long long base = 0;
  const unsigned leader = __ffs(mask) - 1;
  if (lane == leader) base = atomicAdd(len, (unsigned long long)__popc(mask));
  base = __shfl_sync(0xffffffffu, base, leader);
  if (take) queue[base + __popc(mask & ((1u << lane) - 1u))] = value;
}

__global__ void __launch_bounds__(kTdBlock) k_bfs_td(const unsigned long long* __restrict__ row_ptr,
                                                     const uint32_t* __restrict__ col,
                                                     int32_t* __restrict__ level,
                                                     const uint32_t* __restrict__ queue,
                                                     uint64_t qlen,
                                                     const unsigned long long* __restrict__ qoff,
                                                     int32_t next_level,
                                                     uint32_t* __restrict__ next_queue,
                                                     DevCounters* ctr) {
  __shared__ uint64_t s_lo, s_hi;
  const unsigned long long total = qoff[qlen];
  for (unsigned long long e0 = (unsigned long long)blockIdx.x * kTdEdgesPerBlock; e0 < total;
       e0 += (unsigned long long)gridDim.x * kTdEdgesPerBlock) {
    const unsigned long long e1 = min(total, e0 + kTdEdgesPerBlock);
    __syncthreads();
    if (threadIdx.x == 0) {
      s_lo = frontier_index(qoff, 0, qlen - 1, e0);
      s_hi = frontier_index(qoff, s_lo, qlen - 1, e1 - 1);
    }
    __syncthreads();
    const uint64_t lo = s_lo, hi = s_hi;
    for (unsigned long long b = e0; b < e1; b += kTdBlock) {
      const unsigned long long e = b + threadIdx.x;
      bool take = false;
      uint32_t w = 0;
      if (e < e1) {
        const uint64_t i = frontier_index(qoff, lo, hi, e);
        const uint32_t u = queue[i];
        w = col[row_ptr[u] + (e - qoff[i])];
        if (level[w] == -1) take = atomicCAS(&level[w], -1, next_level) == -1;
      }
      warp_append(take, w, next_queue, &ctr->next_n);
    }
  }
}

__global__ void __launch_bounds__(kBuBlock) k_bfs_bu(const unsigned long long* __restrict__ row_ptr,
                                                     const uint32_t* __restrict__ col,
                                                     int32_t* __restrict__ level, uint32_t n,
                                                     int32_t cur_level, DevCounters* ctr) {
  const unsigned lane = lane_id();
  const unsigned sub = lane & (kBuGroup - 1);
  const unsigned gmask = 0xFFu << (lane & ~(kBuGroup - 1u));
  const uint64_t groups = (uint64_t)gridDim.x * blockDim.x / kBuGroup;
  unsigned long long found = 0;
  for (uint64_t v = ((uint64_t)blockIdx.x * blockDim.x + threadIdx.x) / kBuGroup; v < n;
       v += groups) {
    if (level[v] != -1) continue;
    const unsigned long long b = row_ptr[v], e = row_ptr[v + 1];
    bool hit_any = false;
    for (unsigned long long j0 = b; j0 < e; j0 += kBuGroup) {
      const unsigned long long j = j0 + sub;
      const bool hit = j < e && level[col[j]] == cur_level;
      if (__ballot_sync(gmask, hit) & gmask) {
        hit_any = true;
        break;
      }
    }
    if (hit_any && sub == 0) {
      level[v] = cur_level + 1;
      ++found;
    }
  }
  found = warp_sum(found);
  if (lane == 0 && found) atomicAdd(&ctr->next_n, found);
}

__global__ void k_collect_level(const int32_t* __restrict__ level, uint32_t n, int32_t want,
                                uint32_t* __restrict__ queue, DevCounters* ctr) {
  const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
  const uint64_t iters = ((uint64_t)n + stride - 1) / stride;
  for (uint64_t it = 0; it < iters; ++it) {
    const uint64_t v = it * stride + (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const bool take = v < n && level[v] == want;
    warp_append(take, (uint32_t)v, queue, &ctr->next_n);
  }
}

__global__ void k_count_unvisited(const int32_t* __restrict__ level, uint32_t n, DevCounters* ctr) {
  unsigned long long c = 0;
  for (uint64_t v = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; v < n;
       v += (uint64_t)gridDim.x * blockDim.x)
    c += level[v] == -1;
  c = warp_sum(c);
  if (lane_id() == 0 && c) atomicAdd(&ctr->unvisited, c);
}

// ---- persistent search for small frontiers --------------------------------

__device__ __forceinline__ unsigned long long global_ns() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

// Grid-wide barrier for a co-resident grid (cooperative launch).  The last
// block to arrive resets the count and advances the generation; the others
// wait for the generation to change, each for at most budget_ns, and give up
// (recording kErrTimeout) when the budget runs out or another block already
// gave up.  Returns false, to every thread of the block, when it gave up.
__device__ bool grid_barrier(DevCounters* c, unsigned nblocks, unsigned long long budget_ns) {
  __shared__ int s_ok;
  __syncthreads();
  if (threadIdx.x == 0) {
    int ok = 1;
    volatile unsigned int* genp = &c->bar_gen;
    volatile unsigned int* errp = &c->err;
    const unsigned int gen = *genp;
    __threadfence();
    if (atomicAdd(&c->bar_count, 1u) == nblocks - 1) {
      atomicExch(&c->bar_count, 0u);
      __threadfence();
      atomicAdd(&c->bar_gen, 1u);
    } else {
      const unsigned long long t0 = global_ns();
      while (*genp == gen) {
        if ((*errp & kErrTimeout) || global_ns() - t0 > budget_ns) {
          atomicOr(&c->err, kErrTimeout);
          ok = 0;
          break;
        }
        __nanosleep(100);
      }
    }
    __threadfence();
    s_ok = ok;
  }
  __syncthreads();
  return s_ok != 0;
}

__global__ void k_persist_init(DevCounters* c, unsigned long long qlen) {
  c->plen[0] = qlen;
  c->plen[1] = c->plen[2] = 0;
  c->pedges[0] = c->pedges[1] = c->pedges[2] = 0;
  c->pmaxdeg[0] = c->pmaxdeg[1] = c->pmaxdeg[2] = 0;
  c->bar_count = 0;
}

// Levels lvl0, lvl0+1, ... top-down from the frontier in q0 (its length in
// plen[0]).  Iteration it reads the frontier of slot it%3 from queue it&1 and
// appends the next one to slot (it+1)%3 / queue (it+1)&1; block 0 clears slot
// (it+2)%3, which every block finished reading before the previous barrier.
// Queues and slot counters written by other blocks are read with __ldcg (L2),
// never through a stale L1 line.
__global__ void __launch_bounds__(kPersistBlock) k_bfs_persistent(
    const unsigned long long* __restrict__ row_ptr, const uint32_t* __restrict__ col,
    int32_t* level, uint32_t* q0, uint32_t* q1, int32_t lvl0, unsigned long long budget_ns,
    int test_skip, DevCounters* c) {
  const unsigned lane = lane_id();
  const unsigned long long gwarp = ((unsigned long long)blockIdx.x * blockDim.x + threadIdx.x) / 32;
  const unsigned long long nwarps = (unsigned long long)gridDim.x * blockDim.x / 32;
  int32_t lvl = lvl0;
  for (unsigned it = 0;; ++it) {
    const unsigned cur = it % 3, nxt = (it + 1) % 3, old = (it + 2) % 3;
    const uint32_t* q = (it & 1) ? q1 : q0;
    uint32_t* nq = (it & 1) ? q0 : q1;
    const unsigned long long qlen = __ldcg(&c->plen[cur]);
    if (blockIdx.x == 0 && threadIdx.x == 0) {
      c->plen[old] = 0;
      c->pedges[old] = 0;
      c->pmaxdeg[old] = 0;
    }
    for (unsigned long long i = gwarp; i < qlen; i += nwarps) {
      const uint32_t u = __ldcg(q + i);
      const unsigned long long b = row_ptr[u], e = row_ptr[u + 1];
      for (unsigned long long j0 = b; j0 < e; j0 += 32) {
        const unsigned long long j = j0 + lane;
        bool take = false;
        uint32_t w = 0;
        unsigned long long deg = 0;
        if (j < e) {
          w = col[j];
          if (__ldcg(level + w) == -1) take = atomicCAS(&level[w], -1, lvl + 1) == -1;
          if (take) deg = row_ptr[w + 1] - row_ptr[w];
        }
        warp_append(take, w, nq, &c->plen[nxt]);
        const unsigned int dmax = __reduce_max_sync(0xffffffffu, (unsigned int)deg);
        deg = warp_sum(deg);
        if (lane == 0 && deg) {
          atomicAdd(&c->pedges[nxt], deg);
          atomicMax(&c->pmaxdeg[nxt], dmax);
        }
      }
    }
    if (test_skip && blockIdx.x == 0) return;  // testing: this block never arrives
    if (!grid_barrier(c, gridDim.x, budget_ns)) return;
    const unsigned long long nlen = __ldcg(&c->plen[nxt]);
    const unsigned long long nedges = __ldcg(&c->pedges[nxt]);
    const unsigned int nmax = __ldcg(&c->pmaxdeg[nxt]);
    ++lvl;
    if (nlen == 0 || nlen > kPersistMaxVerts || nedges > kPersistMaxEdges ||
        nmax > kPersistMaxDeg) {
      if (blockIdx.x == 0 && threadIdx.x == 0) {
        c->p_level = (unsigned)lvl;
        c->p_slot = nxt;
        c->p_buf = (it + 1) & 1;
      }
      return;
    }
  }
}

// ---- cluster search for small, low-degree frontiers -----------------------
//
// Long, thin graphs (meshes, road networks) run thousands of levels whose
// frontiers hold a few thousand low-degree vertices; a level's cost is then
// the latency of its chain of dependent memory operations (queue entry, row
// offsets, neighbour, the claiming CAS, the append).
// k_bfs_cluster keeps that chain short: a group of kClusterGroup lanes takes a
// frontier vertex and each lane one of its edges, and each group takes
// kClusterPer vertices with their loads issued together, so a level is about
// five dependent steps however its edges fall.  It runs in one thread-block
// cluster of kClusterCtas blocks (one per SM): a level ends at the hardware
// cluster barrier, and the next frontier's length is counted in block 0's
// shared memory through distributed-shared-memory atomics (one per warp and
// step, ballot ranks).  Every block reads the same counters after the
// barrier, so all take the same exit: the next frontier empty, above
// kClusterMaxVerts, or the level just expanded had a vertex of degree above
// kClusterGroup (expanded anyway, in further steps).  There is no spin-wait,
// hence no timeout path.  Queues written by other blocks are read with
// __ldcg (L2), never through a stale L1 line.
constexpr int kClusterCtas = 8;
constexpr int kClusterThreads = 1024;
constexpr uint32_t kClusterGroup = 8;
constexpr uint32_t kClusterPer = 4;
constexpr uint32_t kClusterGroups = (uint32_t)kClusterCtas * kClusterThreads / kClusterGroup;
constexpr unsigned long long kClusterMaxVerts =
    (unsigned long long)kClusterGroups * kClusterPer;  // 4096
constexpr unsigned int kClusterMaxDeg = kClusterGroup;

__global__ void __cluster_dims__(kClusterCtas, 1, 1) __launch_bounds__(kClusterThreads)
    k_bfs_cluster(const unsigned long long* __restrict__ row_ptr, const uint32_t* __restrict__ col,
                  int32_t* level, uint32_t* q0, uint32_t* q1, uint32_t qlen0, int32_t lvl0,
                  DevCounters* c) {
  namespace cg = cooperative_groups;
  cg::cluster_group cluster = cg::this_cluster();
  // next-frontier counters of block 0 in three slots: level `it` reads slot
  // it%3, appends to slot (it+1)%3, and block 0 clears slot (it+2)%3, which
  // every block read before the barrier that ended the previous level
  __shared__ uint32_t s_len[3];
  __shared__ int s_big[3];
  const unsigned rank = cluster.block_rank(), lane = lane_id();
  uint32_t* len0 = cluster.map_shared_rank(s_len, 0);
  int* big0 = cluster.map_shared_rank(s_big, 0);
  if (rank == 0 && threadIdx.x == 0) {
    s_len[0] = qlen0;
    s_len[1] = s_len[2] = 0;
    s_big[0] = s_big[1] = s_big[2] = 0;
  }
  cluster.sync();
  const uint32_t grp = (rank * kClusterThreads + threadIdx.x) / kClusterGroup;
  const uint32_t gl = lane % kClusterGroup;
  int32_t lvl = lvl0;
  for (unsigned it = 0;; ++it) {
    const unsigned cur = it % 3, nxt = (it + 1) % 3, old = (it + 2) % 3;
    const uint32_t* q = (it & 1) ? q1 : q0;
    uint32_t* nq = (it & 1) ? q0 : q1;
    const uint32_t qlen = len0[cur];
    if (rank == 0 && threadIdx.x == 0) {
      s_len[old] = 0;
      s_big[old] = 0;
    }
    uint32_t u[kClusterPer];
    unsigned long long b[kClusterPer], e[kClusterPer];
#pragma unroll
    for (uint32_t k = 0; k < kClusterPer; ++k) {
      const uint32_t i = grp + k * kClusterGroups;
      u[k] = i < qlen ? __ldcg(q + i) : kNoLevel;
    }
    unsigned long long dmax = 0;
#pragma unroll
    for (uint32_t k = 0; k < kClusterPer; ++k) {
      b[k] = e[k] = 0;
      if (u[k] != kNoLevel) {
        b[k] = row_ptr[u[k]];
        e[k] = row_ptr[u[k] + 1];
      }
      dmax = max(dmax, e[k] - b[k]);
    }
    if (dmax > kClusterMaxDeg && gl == 0) big0[nxt] = 1;
    // steps of kClusterGroup edges (one for every vertex of degree <= kClusterGroup)
    const unsigned steps = __reduce_max_sync(
        0xffffffffu, (unsigned)((dmax + kClusterGroup - 1) / kClusterGroup));
    for (unsigned t = 0; t < steps; ++t) {
      uint32_t w[kClusterPer];
      bool take[kClusterPer];
#pragma unroll
      for (uint32_t k = 0; k < kClusterPer; ++k) {
        const unsigned long long j = b[k] + (unsigned long long)t * kClusterGroup + gl;
        w[k] = j < e[k] ? col[j] : kNoLevel;
      }
      // the claiming CAS without a level read first: it returns the old level,
      // so a visited neighbour costs one atomic instead of a load on the chain
#pragma unroll
      for (uint32_t k = 0; k < kClusterPer; ++k)
        take[k] = w[k] != kNoLevel && atomicCAS(&level[w[k]], -1, lvl + 1) == -1;
#pragma unroll
      for (uint32_t k = 0; k < kClusterPer; ++k) {
        const unsigned m = __ballot_sync(0xffffffffu, take[k]);
        if (m) {
          const unsigned leader = __ffs(m) - 1;
          uint32_t base = 0;
          if (lane == leader) base = atomicAdd(&len0[nxt], (uint32_t)__popc(m));
          base = __shfl_sync(0xffffffffu, base, leader);
          if (take[k]) nq[base + __popc(m & ((1u << lane) - 1u))] = w[k];
        }
      }
    }
    cluster.sync();
    const uint32_t nlen = len0[nxt];
    const bool big = big0[nxt] != 0;
    ++lvl;
    if (nlen == 0 || nlen > kClusterMaxVerts || big) {
      if (rank == 0 && threadIdx.x == 0) {
        c->p_level = (unsigned)lvl;
        c->plen[0] = nlen;
        c->p_buf = (it + 1) & 1;
      }
      cluster.sync();  // block 0's counters stay alive until every block has read them
      return;
    }
  }
}

// ---- restart components -------------------------------------------------

__global__ void k_cc_init(uint32_t* parent, uint32_t n) {
  for (uint64_t v = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; v < n;
       v += (uint64_t)gridDim.x * blockDim.x)
    parent[v] = (uint32_t)v;
}

__device__ __forceinline__ uint32_t cc_find(uint32_t* parent, uint32_t x) {
  uint32_t p = parent[x];
  while (p != x) {
    uint32_t gp = parent[p];
    if (gp != p) parent[x] = gp;  // path halving; any ancestor is a valid parent
    x = p;
    p = gp;
  }
  return x;
}

// Union of the endpoints of every edge {v, w}, w < v, of an unvisited vertex v
// (all its neighbours are unvisited too).  The larger root is hooked under the
// smaller one with a CAS, so a root is always the minimum of its tree.
__global__ void k_cc_hook(const unsigned long long* __restrict__ row_ptr,
                          const uint32_t* __restrict__ col, const int32_t* __restrict__ level,
                          uint32_t* parent, uint32_t n) {
  const uint64_t warps = (uint64_t)gridDim.x * blockDim.x / 32;
  for (uint64_t v = ((uint64_t)blockIdx.x * blockDim.x + threadIdx.x) / 32; v < n; v += warps) {
    if (level[v] != -1) continue;
    const unsigned long long b = row_ptr[v], e = row_ptr[v + 1];
    for (unsigned long long j = b + lane_id(); j < e; j += 32) {
      uint32_t w = col[j];
      if (w >= v) break;  // rows are sorted
      uint32_t a = (uint32_t)v, c = w;
      for (;;) {
        a = cc_find(parent, a);
        c = cc_find(parent, c);
        if (a == c) break;
        uint32_t hi = a > c ? a : c, lo = a > c ? c : a;
        if (atomicCAS(&parent[hi], hi, lo) == hi) break;
      }
    }
  }
}

// Roots (parent[v] == v after hooking) of unvisited vertices start the
// restart search at level 0.
__global__ void k_cc_seed(const uint32_t* __restrict__ parent, int32_t* __restrict__ level,
                          uint32_t n, uint32_t* __restrict__ queue, DevCounters* ctr) {
  const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
  const uint64_t iters = ((uint64_t)n + stride - 1) / stride;
  for (uint64_t it = 0; it < iters; ++it) {
    const uint64_t v = it * stride + (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
    bool take = false;
    if (v < n && level[v] == -1 && parent[v] == (uint32_t)v) {
      level[v] = 0;
      take = true;
    }
    warp_append(take, (uint32_t)v, queue, &ctr->next_n);
  }
}

tc_status read_counters(tc_graph* g, cudaStream_t st) {
  TC_CUDA_TRY(cudaMemcpyAsync(g->ctr_host, g->ctr, sizeof(DevCounters), cudaMemcpyDeviceToHost, st));
  TC_CUDA_TRY(cudaStreamSynchronize(st));
  return TC_OK;
}

tc_status reset_next(tc_graph* g, cudaStream_t st) {
  TC_CUDA_TRY(cudaMemsetAsync(&g->ctr->next_n, 0, sizeof(unsigned long long), st));
  return TC_OK;
}

// One persistent run from the frontier q (qlen vertices at level lvl).  On
// return the search has advanced to *next_lvl, whose frontier (*next_len
// vertices, possibly none) is in nq when *next_in_b, else in q.
tc_status run_persistent(tc_graph* g, uint32_t* q, uint32_t* nq, uint64_t qlen, int32_t lvl,
                         cudaStream_t st, int32_t* next_lvl, uint64_t* next_len, bool* next_in_b) {
  static int coop = -1, per_sm = 0;
  if (coop < 0) {
    int dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&coop, cudaDevAttrCooperativeLaunch, dev);
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_bfs_persistent, kPersistBlock, 0);
  }
  if (!coop || per_sm < 1) return TC_ERR_CUDA;
  k_persist_init<<<1, 1, 0, st>>>(g->ctr, qlen); TC_LAUNCHED();
  TC_CUDA_TRY(cudaGetLastError());
  const unsigned long long budget_ns = 1000000ull * g->params.barrier_timeout_ms;
  int test_skip = g->params.test_barrier_skip ? 1 : 0;
  const unsigned long long* rp = g->row_ptr;
  const uint32_t* cl = g->col;
  int32_t* lv = g->level;
  DevCounters* c = g->ctr;
  void* args[] = {(void*)&rp, (void*)&cl, (void*)&lv, (void*)&q, (void*)&nq, (void*)&lvl,
                  (void*)&budget_ns, (void*)&test_skip, (void*)&c};
  TC_CUDA_TRY(cudaLaunchCooperativeKernel((const void*)k_bfs_persistent, dim3(num_sms()),
                                          dim3(kPersistBlock), args, 0, st)); TC_LAUNCHED();
  TC_TRY(read_counters(g, st));
  const DevCounters& h = *g->ctr_host;
  if (h.err & kErrTimeout) return TC_ERR_TIMEOUT;
  *next_lvl = (int32_t)h.p_level;
  *next_len = h.plen[h.p_slot];
  *next_in_b = h.p_buf == 1;
  return TC_OK;
}

// One k_bfs_cluster run from the frontier q (qlen <= kClusterMaxVerts vertices
// at level lvl); results as run_persistent.
tc_status run_cluster(tc_graph* g, uint32_t* q, uint32_t* nq, uint64_t qlen, int32_t lvl,
                      cudaStream_t st, int32_t* next_lvl, uint64_t* next_len, bool* next_in_b) {
  k_bfs_cluster<<<kClusterCtas, kClusterThreads, 0, st>>>(g->row_ptr, g->col, g->level, q, nq,
                                                          (uint32_t)qlen, lvl, g->ctr); TC_LAUNCHED();
  TC_CUDA_TRY(cudaGetLastError());
  TC_TRY(read_counters(g, st));
  const DevCounters& h = *g->ctr_host;
  *next_lvl = (int32_t)h.p_level;
  *next_len = h.plen[0];
  *next_in_b = h.p_buf == 1;
  return TC_OK;
}

// Level-synchronous search from the vertices already in queue_a (qlen of them,
// all at level 0).  Returns the number of levels (1 + deepest level).
tc_status level_loop(tc_graph* g, uint64_t qlen, cudaStream_t st, uint32_t* levels_out) {
  const uint32_t n = g->n;
  const int sms = num_sms();
  uint32_t* q = g->queue_a;
  uint32_t* nq = g->queue_b;
  bool bottom_up = false;
  long double unexplored = (long double)g->nnz;
  int32_t lvl = 0;
  const uint32_t alpha = g->params.bfs_alpha ? g->params.bfs_alpha : 15;
  const uint32_t beta = g->params.bfs_beta ? g->params.bfs_beta : 18;
  uint64_t prev_frontier = qlen;
  while (true) {
    unsigned long long fedges = 0;
    if (!bottom_up) {
      if (qlen == 0) break;
      TC_CUDA_TRY(cudaMemsetAsync(&g->ctr->fmaxdeg, 0, sizeof(unsigned int), st));
      k_frontier_degrees<<<grid_for(qlen, 256, sms * 16), 256, 0, st>>>(q, qlen, g->row_ptr, g->fdeg,
                                                                        &g->ctr->fmaxdeg); TC_LAUNCHED();
      TC_CUDA_TRY(cudaGetLastError());
      TC_TRY(exclusive_scan_u32(g->fdeg, g->qoff, qlen, g->scan, st));
      TC_CUDA_TRY(cudaMemcpyAsync(&g->ctr_host->scan_total, g->qoff + qlen, sizeof(unsigned long long),
                                  cudaMemcpyDeviceToHost, st));
      TC_CUDA_TRY(cudaMemcpyAsync(&g->ctr_host->fmaxdeg, &g->ctr->fmaxdeg, sizeof(unsigned int),
                                  cudaMemcpyDeviceToHost, st));
      TC_CUDA_TRY(cudaStreamSynchronize(st));
      fedges = g->ctr_host->scan_total;
      if ((long double)fedges * alpha > unexplored && qlen > 1) bottom_up = true;
      const bool in_cluster = g->params.cluster_bfs && qlen <= kClusterMaxVerts &&
                              g->ctr_host->fmaxdeg <= kClusterMaxDeg;
      if (!bottom_up && g->params.persistent_bfs && fedges > 0 &&
          (in_cluster || (qlen <= kPersistMaxVerts && fedges <= kPersistMaxEdges &&
                          g->ctr_host->fmaxdeg <= kPersistMaxDeg))) {
        int32_t next_lvl = lvl;
        uint64_t next_len = 0;
        bool next_in_b = false;
        if (in_cluster)
          TC_TRY(run_cluster(g, q, nq, qlen, lvl, st, &next_lvl, &next_len, &next_in_b));
        else
          TC_TRY(run_persistent(g, q, nq, qlen, lvl, st, &next_lvl, &next_len, &next_in_b));
        g->stats.bfs_steps += (uint32_t)(next_lvl - lvl);
        unexplored -= (long double)fedges;  // the first step's edges; later ones are small
        prev_frontier = next_len;
        if (next_in_b) {
          uint32_t* t = q;
          q = nq;
          nq = t;
        }
        qlen = next_len;
        if (qlen == 0) {
          lvl = next_lvl - 1;
          break;
        }
        lvl = next_lvl;
        continue;
      }
    }
    TC_TRY(reset_next(g, st));
    uint64_t found;
    if (!bottom_up) {
      if (fedges > 0) {
        k_bfs_td<<<grid_for(fedges, kTdEdgesPerBlock, sms * 8), kTdBlock, 0, st>>>(
            g->row_ptr, g->col, g->level, q, qlen, g->qoff, lvl + 1, nq, g->ctr); TC_LAUNCHED();
        TC_CUDA_TRY(cudaGetLastError());
      }
      TC_TRY(read_counters(g, st));
      found = g->ctr_host->next_n;
      uint32_t* t = q;
      q = nq;
      nq = t;
      qlen = found;
    } else {
      k_bfs_bu<<<sms * 8, kBuBlock, 0, st>>>(g->row_ptr, g->col, g->level, n, lvl, g->ctr); TC_LAUNCHED();
      TC_CUDA_TRY(cudaGetLastError());
      TC_TRY(read_counters(g, st));
      found = g->ctr_host->next_n;
      g->stats.bottom_up_steps++;
      if (found > 0 && found < n / beta && found < prev_frontier) {
        TC_TRY(reset_next(g, st));
        k_collect_level<<<sms * 8, 256, 0, st>>>(g->level, n, lvl + 1, q, g->ctr); TC_LAUNCHED();
        TC_CUDA_TRY(cudaGetLastError());
        TC_TRY(read_counters(g, st));
        qlen = g->ctr_host->next_n;
        bottom_up = false;
      }
    }
    g->stats.bfs_steps++;
    unexplored -= (long double)fedges;
    prev_frontier = found;
    if (found == 0) break;
    ++lvl;
  }
  *levels_out = (uint32_t)lvl + 1;
  return TC_OK;
}

}  // namespace

tc_status run_bfs(tc_graph* g, uint32_t root, cudaStream_t st) {
  TC_CUDA_TRY(cudaMemsetAsync(g->level, 0xFF, sizeof(int32_t) * g->n, st));
  k_set_root<<<1, 1, 0, st>>>(g->level, g->queue_a, root); TC_LAUNCHED();
  TC_CUDA_TRY(cudaGetLastError());
  return run_bfs_from_queue(g, 1, st);
}

tc_status run_bfs_from_queue(tc_graph* g, uint64_t k, cudaStream_t st) {
  const uint32_t n = g->n;
  const int sms = num_sms();
  g->stats.bfs_steps = 0;
  g->stats.bottom_up_steps = 0;
  g->stats.restarted = 0;
  TC_CUDA_TRY(cudaMemsetAsync(g->ctr, 0, sizeof(DevCounters), st));
  uint32_t levels = 0;
  TC_TRY(level_loop(g, k, st, &levels));
  g->stats.num_levels = levels;

  // restart phase
  TC_CUDA_TRY(cudaMemsetAsync(&g->ctr->unvisited, 0, sizeof(unsigned long long), st));
  k_count_unvisited<<<sms * 8, 256, 0, st>>>(g->level, n, g->ctr); TC_LAUNCHED();
  TC_CUDA_TRY(cudaGetLastError());
  TC_TRY(read_counters(g, st));
  if (g->ctr_host->unvisited == 0) return TC_OK;
  g->stats.restarted = 1;
  k_cc_init<<<sms * 8, 256, 0, st>>>(g->parent, n); TC_LAUNCHED();
  k_cc_hook<<<sms * 16, 256, 0, st>>>(g->row_ptr, g->col, g->level, g->parent, n); TC_LAUNCHED();
  TC_TRY(reset_next(g, st));
  k_cc_seed<<<sms * 8, 256, 0, st>>>(g->parent, g->level, n, g->queue_a, g->ctr); TC_LAUNCHED();
  TC_CUDA_TRY(cudaGetLastError());
  TC_TRY(read_counters(g, st));
  uint32_t more = 0;
  TC_TRY(level_loop(g, g->ctr_host->next_n, st, &more));
  return TC_OK;
}

}  // namespace tc

// Internal declarations of libtc (CUDA, sm_103a).  Not part of the ABI.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "../../include/tc.h"

namespace tc {

constexpr int kWarp = 32;
constexpr uint32_t kNoLevel = 0xFFFFFFFFu;  // level word of an unvisited vertex (-1)

// Device-side error word values (bit flags, OR-ed by kernels).
enum : uint32_t { kErrVertexRange = 1u, kErrTimeout = 2u, kErrOverflow = 4u, kErrBounds = 8u };

// Checked builds (-DTC_CHECKED, the stand-in for a memory checker): kernels
// test the preconditions of their data-dependent accesses, record a failure
// in the error word (the count then returns TC_ERR_CUDA) and skip the access
// instead of trapping.  In normal builds the checks compile away.
#ifdef TC_CHECKED
constexpr bool kChecked = true;
#else
constexpr bool kChecked = false;
#endif

// Counters that kernels accumulate and the host reads back with one copy.
struct DevCounters {
  unsigned long long tri;        // T
  unsigned long long c1;         // apex on another level
  unsigned long long c2;         // apex on the same level
  unsigned long long num_cover;  // |S|
  unsigned long long num_large;  // cover edges sent to the owner-hash path
  unsigned long long num_medium; // cover edges sent to the warp merge
  unsigned long long next_n;     // BFS: vertices discovered this step
  unsigned long long next_m;     // BFS: sum of their degrees
  unsigned long long scan_total; // total of the last device-wide scan
  unsigned long long items;      // owner-hash work items
  unsigned long long item_cursor;// dynamic work counter
  unsigned long long unvisited;  // vertices still unvisited
  unsigned long long listed;     // triangle listing: triangles found so far (output cursor)
  unsigned long long plen[3];    // persistent BFS: frontier lengths, one slot per level mod 3
  unsigned long long pedges[3];  // persistent BFS: degree sums of those frontiers
  unsigned int pmaxdeg[3];       // persistent BFS: largest degree in those frontiers
  unsigned int fmaxdeg;          // largest degree of the current frontier (host-driven steps)
  unsigned int bar_count;        // grid barrier: blocks arrived
  unsigned int bar_gen;          // grid barrier: generation
  unsigned int p_level;          // persistent BFS: level of the frontier it stopped at
  unsigned int p_slot;           // ... its length slot
  unsigned int p_buf;            // ... which queue holds it (0: first, 1: second)
  unsigned int err;              // kErr* flags
  unsigned int dmax;             // largest degree
  unsigned int dmax_vertex;      // smallest id of largest degree
  unsigned int pad;
};

// Scratch for the device-wide exclusive scan (reduce-then-scan, recursive).
struct ScanScratch {
  unsigned long long* sums = nullptr;  // block totals, all recursion levels
  size_t capacity = 0;                 // entries in sums
};

}  // namespace tc

// The opaque handle.  Every array is device memory owned by the handle.
struct tc_graph {
  uint32_t n = 0;
  uint64_t m = 0;          // undirected edges
  uint64_t nnz = 0;        // 2m
  uint32_t d_max = 0;
  uint32_t maxdeg_vertex = 0;
  unsigned long long* row_ptr = nullptr;  // [n+1]
  uint32_t* col = nullptr;                // [nnz]
  uint32_t* erow = nullptr;               // [nnz] row of each entry (the CSR's rows as COO)

  // per-count state, sized at creation so a count allocates nothing
  int32_t* level = nullptr;      // [n]
  uint32_t* queue_a = nullptr;   // [n]  frontier queues
  uint32_t* queue_b = nullptr;   // [n]
  unsigned long long* qoff = nullptr;  // [n+1] frontier degree offsets
  unsigned long long* ooff = nullptr;  // [n+1] owner bucket offsets
  uint32_t* parent = nullptr;    // [n]  union-find parents (restart components)
  uint32_t* fdeg = nullptr;      // [n]  degrees of frontier vertices
  uint32_t* ocount = nullptr;    // [n]  cover edges per owner
  uint32_t* ofill = nullptr;     // [n]  owner bucket fill cursors
  unsigned long long* ioff = nullptr;  // [n+1] work-item offsets per owner
  uint32_t* item_owner = nullptr;      // [item_cap] owner of each hash work item
  unsigned long long item_cap = 0;
  uint2* cover = nullptr;        // [m]  all cover edges (u < v)
  uint2* large = nullptr;        // [m]  (owner, streamer) of owner-hash cover edges
  uint2* medium = nullptr;       // [m]  (u, v) cover edges of the warp-merge bin
  uint32_t* ostream = nullptr;   // [m]  streamers bucketed by owner
  uint32_t* lcol = nullptr;      // [nnz] rows reordered [same-level | other-level] per count
  unsigned long long* lsplit = nullptr;  // [n] start of the other-level part of each row
  unsigned long long* obeg = nullptr;  // [n+1] oriented adjacency A+() (forward counts), on first use
  uint32_t* ocol = nullptr;            // [m]
  uint32_t* tile_row = nullptr;  // [tile_cap] row of each tile of a long row (level split)
  uint32_t* tile_cnt = nullptr;  // [tile_cap] other-level entries per tile
  unsigned long long tile_cap = 0;
  tc::DevCounters* ctr = nullptr;      // device counters
  tc::DevCounters* ctr_host = nullptr; // pinned mirror
  tc::ScanScratch scan;
  cudaEvent_t ev[6] = {nullptr, nullptr, nullptr, nullptr, nullptr, nullptr};

  // batch mode: this handle is the disjoint union of batch_k graphs; vertex v
  // belongs to graph g with voff[g] <= v < voff[g+1], whose count goes to gcount[g]
  uint32_t batch_k = 0;
  const unsigned long long* voff = nullptr;  // device, batch_k + 1
  unsigned long long* gcount = nullptr;      // device, batch_k

  tc_params params;
  tc_stats stats;
  bool counted = false;
  uint32_t last_root = 0;
  // pooled: device memory comes stream-ordered from the library's pool and is
  // returned without synchronising the device (batches built from edge lists,
  // which a serving loop creates and destroys while other work runs); the
  // counter mirror is then pageable host memory (freeing pinned memory would
  // synchronise the device)
  bool pooled = false;
};

namespace tc {

// ---- helpers shared by the .cu files ------------------------------------

#define TC_CUDA_TRY(expr)                                  \
  do {                                                     \
    cudaError_t _e = (expr);                               \
    if (_e != cudaSuccess) {                               \
      tc::set_last_cuda_error(_e);                         \
      return (_e == cudaErrorMemoryAllocation) ? TC_ERR_OOM : TC_ERR_CUDA; \
    }                                                      \
  } while (0)

#define TC_TRY(expr)                 \
  do {                               \
    tc_status _s = (expr);           \
    if (_s != TC_OK) return _s;      \
  } while (0)

void set_last_cuda_error(cudaError_t e);

// Kernel launches made by the library on this host thread (for tc_stats).
extern thread_local uint32_t g_launches;
#define TC_LAUNCHED() (++tc::g_launches)

inline unsigned grid_for(uint64_t work, unsigned per_block, unsigned cap = 1u << 20) {
  uint64_t g = (work + per_block - 1) / per_block;
  if (g < 1) g = 1;
  if (g > cap) g = cap;
  return (unsigned)g;
}

int num_sms();

// Device memory of handle g (g may be NULL: plain).  A pooled handle's memory
// is taken from the library's per-device pool in stream order on `st` and
// freed in stream order (cudaFreeAsync); other memory uses cudaMalloc /
// cudaFree.  dev_free ignores NULL.
cudaError_t dev_malloc(const tc_graph* g, void** p, size_t bytes, cudaStream_t st);
void dev_free(const tc_graph* g, void* p, cudaStream_t st);
template <typename T>
cudaError_t dev_alloc(const tc_graph* g, T** p, size_t count, cudaStream_t st) {
  *p = nullptr;
  return dev_malloc(g, reinterpret_cast<void**>(p), sizeof(T) * (count ? count : 1), st);
}
// A non-blocking stream of the current device owned by the library, on which
// destroy calls return pooled memory (every call on a handle has finished its
// work before it returns, so nothing is pending on that memory).
cudaStream_t free_stream();

// Device-wide exclusive scan of `count` values (uint32 or uint64 input) into
// uint64 offsets out[0..count]; out[count] holds the total.  `in` and `out`
// may alias only for the uint64 variant.
tc_status exclusive_scan_u32(const uint32_t* in, unsigned long long* out, uint64_t count,
                             ScanScratch& s, cudaStream_t st);
tc_status exclusive_scan_u64(const unsigned long long* in, unsigned long long* out,
                             uint64_t count, ScanScratch& s, cudaStream_t st);
size_t scan_scratch_entries(uint64_t max_count);

// Phases (implemented in the .cu files of the same name).
// Several graphs' edge lists in one array: edges [ein[i], ein[i+1]) belong to
// graph i, whose local ids must be < nvert[i] and become voff[i] + id.
struct EdgeGroups {
  const unsigned long long* ein;   // device, k + 1
  const unsigned long long* voff;  // device, k + 1
  const uint32_t* nvert;           // device, k
  uint32_t k;
};
tc_status build_csr(tc_graph* g, const uint32_t* d_src, const uint32_t* d_dst, uint64_t E,
                    cudaStream_t st, const EdgeGroups* groups = nullptr);
tc_status run_bfs(tc_graph* g, uint32_t root, cudaStream_t st);
// Stable LSD radix sort of N uint64 keys below 2^bits (8-bit digits).  The
// sorted keys end in *keys; *tmp (N entries) is scratch, and the two pointers
// may come back swapped.  Synchronises `st`.
tc_status sort_keys(unsigned long long** keys, unsigned long long** tmp, uint64_t N, int bits,
                    cudaStream_t st);
int key_bits(uint32_t n);
// BFS from the k roots already stored in queue_a (all at level 0, level[] set
// to -1 elsewhere by the caller), then the restart rule.
tc_status run_bfs_from_queue(tc_graph* g, uint64_t k, cudaStream_t st);
tc_status alloc_count_state(tc_graph* g, cudaStream_t st);
void free_graph(tc_graph* g);
void params_default(tc_params* p);

// Graph of vertex (or entry) x in a batch: the largest g < nb with off[g] <= x.
__device__ __forceinline__ uint32_t batch_graph_of(const unsigned long long* off, uint32_t lo,
                                                   uint32_t hi, unsigned long long x) {
  while (lo < hi) {
    const uint32_t mid = lo + (hi - lo + 1) / 2;
    if (off[mid] <= x) lo = mid; else hi = mid - 1;
  }
  return lo;
}
tc_status run_cover_and_count(tc_graph* g, cudaStream_t st);
// A batch union's graphs counted in one persistent launch, one graph per block
// (k_batch_graphs): roots[g] is graph g's root as a union id, order[] the
// graphs in the order blocks take them; counts to gcount[g], totals to u->ctr.
tc_status run_batch_graphs(tc_graph* u, const unsigned long long* voff, const uint32_t* roots,
                           const uint32_t* order, uint32_t k, unsigned long long* gcount,
                           cudaStream_t st);
// g->erow[j] = the row of adjacency entry j (after the CSR is built; once per
// graph: the per-count entry loops read it instead of searching row_ptr).
tc_status fill_entry_rows(tc_graph* g, cudaStream_t st);
// TC_OK if owner-hash blocks of `hash_block` threads with chunks of `chunk`
// entries fit the device's shared memory per block, else TC_ERR_INVALID_ARG.
tc_status owner_hash_fits(uint32_t chunk, uint32_t hash_block);
// Algorithm Forward (degree orientation) over the whole graph; counters in g->ctr.
tc_status run_forward_count(tc_graph* g, cudaStream_t st);
// Algorithm CETC-Seq-S after run_bfs: c1 = T1, c2 = 3 T0, tri = T0 + T1.
tc_status run_split_count(tc_graph* g, cudaStream_t st);
// Where a listing count puts its triangles: up to cap triples (u, v, w) in
// tri[3 cap] (device; NULL: none) and per-vertex counts in vcount[n] (device,
// zeroed by the caller; NULL: none).
struct EmitSink {
  uint32_t* tri;
  unsigned long long cap;
  unsigned long long* vcount;
};
// run_cover_and_count with every counted triangle also emitted to `sink`
// (single graphs only; the medium bin is not used).
tc_status run_cover_and_list(tc_graph* g, const EmitSink& sink, cudaStream_t st);
// |S| after run_bfs (resets g->ctr).
tc_status run_count_horizontal(tc_graph* g, cudaStream_t st, unsigned long long* num_cover);

// ---- device helpers -----------------------------------------------------

// True (and the failure recorded) when `bad` holds in a checked build; always
// false in a normal build.
template <typename Counters>
__device__ __forceinline__ bool check_failed(bool bad, Counters* ctr) {
  if (kChecked && bad) {
    atomicOr(&ctr->err, (unsigned)kErrBounds);
    return true;
  }
  return false;
}

__device__ __forceinline__ unsigned lane_id() { return threadIdx.x & 31u; }

template <typename T>
__device__ __forceinline__ T warp_sum(T v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// Inclusive warp scan.
template <typename T>
__device__ __forceinline__ T warp_inclusive_scan(T v) {
  const unsigned lane = lane_id();
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    T t = __shfl_up_sync(0xffffffffu, v, o);
    if (lane >= (unsigned)o) v += t;
  }
  return v;
}

// Block-wide exclusive scan; all threads of the block call it.  `tmp` holds
// blockDim.x / 32 + 1 entries.  Returns the exclusive prefix; *total gets the sum.
template <typename T>
__device__ __forceinline__ T block_exclusive_scan(T v, T* tmp, T* total) {
  const unsigned lane = lane_id(), warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
  T inc = warp_inclusive_scan(v);
  if (lane == 31) tmp[warp] = inc;
  __syncthreads();
  if (warp == 0) {
    T w = lane < nw ? tmp[lane] : T(0);
    T wi = warp_inclusive_scan(w);
    if (lane < nw) tmp[lane] = wi - w;
    if (lane == nw - 1) tmp[nw] = wi;
  }
  __syncthreads();
  T out = tmp[warp] + inc - v;
  *total = tmp[nw];
  __syncthreads();
  return out;
}

// Block-wide sum delivered to every thread. `tmp` holds blockDim.x/32 + 1 entries.
template <typename T>
__device__ __forceinline__ T block_sum(T v, T* tmp) {
  T total;
  block_exclusive_scan(v, tmp, &total);
  return total;
}

}  // namespace tc

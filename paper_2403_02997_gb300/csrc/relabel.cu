// Degree ordering: the pre-processing of Algorithms CETC-Seq-D and CETC-Seq-SD
// (Section "Experimental Results"), which reorders the vertices in decreasing
// order of their degrees (Section "Related Work", on Algorithm Forward).
//
//   1. k_rank_keys      key(v) = ((d_max - d(v)) << kb) | v, so an ascending
//                       sort takes the vertices by decreasing degree, ties by
//                       increasing id;
//   2. sort_keys        the CSR build's stable LSD radix sort;
//   3. k_new_ids        new_of_old[v] = the position of v's key;
//   4. k_relabel_edges  every CSR entry (u, v) becomes (new(u), new(v));
//   5. build_csr        the relabelled list (each edge appears twice, and the
//                       build's canonicalisation keeps one) becomes the new
//                       graph's CSR, rows sorted by new id.
#include <cstring>
#include <new>

#include "tc_internal.cuh"

namespace tc {

namespace {

__global__ void k_rank_keys(const unsigned long long* __restrict__ row_ptr, uint32_t n,
                            uint32_t d_max, int kb, unsigned long long* __restrict__ keys) {
  for (uint64_t v = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; v < n;
       v += (uint64_t)gridDim.x * blockDim.x) {
    const unsigned long long d = row_ptr[v + 1] - row_ptr[v];
    keys[v] = ((unsigned long long)(d_max - d) << kb) | v;
  }
}

__global__ void k_new_ids(const unsigned long long* __restrict__ sorted, uint32_t n, int kb,
                          uint32_t* __restrict__ new_of_old, uint32_t* __restrict__ old_of_new) {
  const unsigned long long mask = (1ull << kb) - 1ull;
  for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (uint64_t)gridDim.x * blockDim.x) {
    const uint32_t v = (uint32_t)(sorted[i] & mask);
    new_of_old[v] = (uint32_t)i;
    old_of_new[i] = v;
  }
}

// One warp per row u: the row's entries become (new(u), new(v)) at the same
// positions.
__global__ void k_relabel_edges(const unsigned long long* __restrict__ row_ptr,
                                const uint32_t* __restrict__ col, uint32_t n,
                                const uint32_t* __restrict__ new_of_old,
                                uint32_t* __restrict__ src, uint32_t* __restrict__ dst) {
  const unsigned lane = lane_id();
  const uint64_t warps = (uint64_t)gridDim.x * blockDim.x / 32;
  for (uint64_t u = ((uint64_t)blockIdx.x * blockDim.x + threadIdx.x) / 32; u < n; u += warps) {
    const uint32_t nu = new_of_old[u];
    for (unsigned long long j = row_ptr[u] + lane; j < row_ptr[u + 1]; j += 32) {
      src[j] = nu;
      dst[j] = new_of_old[col[j]];
    }
  }
}

}  // namespace

}  // namespace tc

using namespace tc;

extern "C" tc_status tc_graph_relabel_degree(const tc_graph* g, void* stream, tc_graph** out,
                                             uint32_t* host_old_of_new) {
  if (!g || !out) return TC_ERR_INVALID_ARG;
  *out = nullptr;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  const uint32_t n = g->n;
  const int sms = num_sms();
  unsigned long long *keys = nullptr, *tmp = nullptr;
  uint32_t *new_of_old = nullptr, *old_of_new = nullptr, *src = nullptr, *dst = nullptr;
  tc_status s = TC_OK;
  do {
    if (n > 0) {
      const int kb = key_bits(n);
      const int bits = kb + key_bits(g->d_max + 2);
      if (cudaMalloc(&keys, sizeof(unsigned long long) * n) != cudaSuccess ||
          cudaMalloc(&tmp, sizeof(unsigned long long) * n) != cudaSuccess ||
          cudaMalloc(&new_of_old, sizeof(uint32_t) * n) != cudaSuccess ||
          cudaMalloc(&old_of_new, sizeof(uint32_t) * n) != cudaSuccess) {
        s = TC_ERR_OOM;
        break;
      }
      k_rank_keys<<<grid_for(n, 256, sms * 16), 256, 0, st>>>(g->row_ptr, n, g->d_max, kb, keys); TC_LAUNCHED();
      if ((s = sort_keys(&keys, &tmp, n, bits, st)) != TC_OK) break;
      k_new_ids<<<grid_for(n, 256, sms * 16), 256, 0, st>>>(keys, n, kb, new_of_old, old_of_new); TC_LAUNCHED();
      if (g->nnz > 0) {
        if (cudaMalloc(&src, sizeof(uint32_t) * g->nnz) != cudaSuccess ||
            cudaMalloc(&dst, sizeof(uint32_t) * g->nnz) != cudaSuccess) {
          s = TC_ERR_OOM;
          break;
        }
        k_relabel_edges<<<sms * 16, 256, 0, st>>>(g->row_ptr, g->col, n, new_of_old, src, dst); TC_LAUNCHED();
      }
      if (cudaGetLastError() != cudaSuccess) {
        s = TC_ERR_CUDA;
        break;
      }
      if (host_old_of_new &&
          cudaMemcpyAsync(host_old_of_new, old_of_new, sizeof(uint32_t) * n,
                          cudaMemcpyDeviceToHost, st) != cudaSuccess) {
        s = TC_ERR_CUDA;
        break;
      }
    }
    // the new handle: the relabelled entries, canonicalised like any edge list
    s = tc_graph_create(src, dst, g->nnz, n, 1, stream, out);
  } while (0);
  cudaStreamSynchronize(st);
  cudaFree(keys);
  cudaFree(tmp);
  cudaFree(new_of_old);
  cudaFree(old_of_new);
  cudaFree(src);
  cudaFree(dst);
  if (s == TC_OK && *out) (*out)->params = g->params;
  return s;
}

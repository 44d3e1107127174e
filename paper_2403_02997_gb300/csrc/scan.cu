// Device-wide exclusive scan (reduce-then-scan), used for CSR offsets, frontier
// offsets, owner buckets and work-item offsets.  Three passes per level:
// tile totals, a scan of the totals (recursive), and the tile scans.
#include "tc_internal.cuh"

namespace tc {

namespace {
constexpr int kScanBlock = 512;
constexpr int kScanItems = 8;
constexpr uint64_t kScanTile = (uint64_t)kScanBlock * kScanItems;

template <typename Tin>
__global__ void __launch_bounds__(kScanBlock) k_tile_reduce(const Tin* __restrict__ in,
                                                            uint64_t count,
                                                            unsigned long long* __restrict__ sums) {
  __shared__ unsigned long long tmp[kScanBlock / 32 + 1];
  const uint64_t base = (uint64_t)blockIdx.x * kScanTile;
  unsigned long long s = 0;
#pragma unroll
  for (int k = 0; k < kScanItems; ++k) {
    uint64_t i = base + (uint64_t)k * kScanBlock + threadIdx.x;
    if (i < count) s += (unsigned long long)in[i];
  }
  s = block_sum(s, tmp);
  if (threadIdx.x == 0) sums[blockIdx.x] = s;
}

// out[i] = offs[tile] + sum(in[tile_start .. i)); the thread holding the last
// element also writes out[count].  Each thread reads all its items before it
// writes, so in == out is allowed.
template <typename Tin>
__global__ void __launch_bounds__(kScanBlock) k_tile_scan(const Tin* in, unsigned long long* out,
                                                          uint64_t count,
                                                          const unsigned long long* offs) {
  __shared__ unsigned long long tmp[kScanBlock / 32 + 1];
  const uint64_t base = (uint64_t)blockIdx.x * kScanTile + (uint64_t)threadIdx.x * kScanItems;
  unsigned long long v[kScanItems];
  unsigned long long s = 0;
#pragma unroll
  for (int k = 0; k < kScanItems; ++k) {
    uint64_t i = base + k;
    v[k] = i < count ? (unsigned long long)in[i] : 0ull;
    s += v[k];
  }
  unsigned long long total;
  unsigned long long run = block_exclusive_scan(s, tmp, &total);
  if (offs) run += offs[blockIdx.x];
#pragma unroll
  for (int k = 0; k < kScanItems; ++k) {
    uint64_t i = base + k;
    if (i < count) {
      out[i] = run;
      run += v[k];
      if (i == count - 1) out[count] = run;
    }
  }
}

__global__ void k_write_zero(unsigned long long* p) { *p = 0ull; }

template <typename Tin>
tc_status scan_level(const Tin* in, unsigned long long* out, uint64_t count,
                     unsigned long long* sums, size_t sums_cap, cudaStream_t st) {
  if (count == 0) {
    k_write_zero<<<1, 1, 0, st>>>(out); TC_LAUNCHED();
    TC_CUDA_TRY(cudaGetLastError());
    return TC_OK;
  }
  const uint64_t nb = (count + kScanTile - 1) / kScanTile;
  if (nb == 1) {
    k_tile_scan<Tin><<<1, kScanBlock, 0, st>>>(in, out, count, nullptr); TC_LAUNCHED();
    TC_CUDA_TRY(cudaGetLastError());
    return TC_OK;
  }
  if (nb + 1 > sums_cap || nb > 0x7FFFFFFFull) return TC_ERR_OVERFLOW;
  k_tile_reduce<Tin><<<(unsigned)nb, kScanBlock, 0, st>>>(in, count, sums); TC_LAUNCHED();
  TC_CUDA_TRY(cudaGetLastError());
  TC_TRY(scan_level<unsigned long long>(sums, sums, nb, sums + nb + 1, sums_cap - (nb + 1), st));
  k_tile_scan<Tin><<<(unsigned)nb, kScanBlock, 0, st>>>(in, out, count, sums); TC_LAUNCHED();
  TC_CUDA_TRY(cudaGetLastError());
  return TC_OK;
}
}  // namespace

size_t scan_scratch_entries(uint64_t max_count) {
  size_t total = 0;
  uint64_t c = max_count;
  while (true) {
    uint64_t nb = (c + kScanTile - 1) / kScanTile;
    if (nb <= 1) break;
    total += nb + 1;
    c = nb;
  }
  return total + 16;
}

tc_status exclusive_scan_u32(const uint32_t* in, unsigned long long* out, uint64_t count,
                             ScanScratch& s, cudaStream_t st) {
  return scan_level<uint32_t>(in, out, count, s.sums, s.capacity, st);
}

tc_status exclusive_scan_u64(const unsigned long long* in, unsigned long long* out,
                             uint64_t count, ScanScratch& s, cudaStream_t st) {
  return scan_level<unsigned long long>(in, out, count, s.sums, s.capacity, st);
}

}  // namespace tc

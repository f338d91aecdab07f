// Exclusive int64 prefix sum for the variable-layer numbering: with a
// per-entity column size, Algorithm 1's counter at the start of entity i's
// column is the sum of the sizes of the entities before it.  Three passes:
// per-tile sums, one CTA scanning the tile sums, and a per-tile scan that
// adds the tile's start.  data has n + 1 entries; data[n] receives the total.
#include "ext_internal.cuh"

namespace {

constexpr int kThreads = 1024;
constexpr int kPer = 4;
constexpr int kTile = kThreads * kPer;

// exclusive scan of one value per thread across the CTA; returns the total
__device__ int64_t block_exclusive_scan(int64_t v, int64_t &excl) {
  __shared__ int64_t warp_tot[kThreads / 32];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  int64_t x = v;
#pragma unroll
  for (int d = 1; d < 32; d <<= 1) {
    const int64_t y = __shfl_up_sync(0xffffffffu, x, d);
    if (lane >= d) x += y;
  }
  __syncthreads();  // warp_tot may still be read by a previous call
  if (lane == 31) warp_tot[warp] = x;
  __syncthreads();
  if (warp == 0) {
    int64_t w = warp_tot[lane];
#pragma unroll
    for (int d = 1; d < 32; d <<= 1) {
      const int64_t y = __shfl_up_sync(0xffffffffu, w, d);
      if (lane >= d) w += y;
    }
    warp_tot[lane] = w;  // inclusive over warps
  }
  __syncthreads();
  const int64_t before = warp == 0 ? 0 : warp_tot[warp - 1];
  excl = before + x - v;
  return warp_tot[kThreads / 32 - 1];
}

__global__ void __launch_bounds__(kThreads) k_scan_tiles(const int64_t *data, int64_t n, int64_t *sums) {
  const int64_t base = (int64_t)blockIdx.x * kTile + (int64_t)threadIdx.x * kPer;
  int64_t v = 0;
#pragma unroll
  for (int i = 0; i < kPer; ++i)
    if (base + i < n) v += data[base + i];
  int64_t excl;
  const int64_t tot = block_exclusive_scan(v, excl);
  if (threadIdx.x == 0) sums[blockIdx.x] = tot;
}

__global__ void __launch_bounds__(kThreads) k_scan_sums(int64_t *sums, int64_t nt, int64_t *total) {
  int64_t carry = 0;
  for (int64_t c0 = 0; c0 < nt; c0 += kThreads) {
    const int64_t i = c0 + threadIdx.x;
    const int64_t v = i < nt ? sums[i] : 0;
    int64_t excl;
    const int64_t tot = block_exclusive_scan(v, excl);
    if (i < nt) sums[i] = carry + excl;
    carry += tot;
  }
  if (threadIdx.x == 0) *total = carry;
}

__global__ void __launch_bounds__(kThreads) k_scan_apply(int64_t *data, int64_t n, const int64_t *sums) {
  const int64_t base = (int64_t)blockIdx.x * kTile + (int64_t)threadIdx.x * kPer;
  int64_t v[kPer], t = 0;
#pragma unroll
  for (int i = 0; i < kPer; ++i) {
    v[i] = base + i < n ? data[base + i] : 0;
    t += v[i];
  }
  int64_t excl;
  block_exclusive_scan(t, excl);
  int64_t run = sums[blockIdx.x] + excl;
#pragma unroll
  for (int i = 0; i < kPer; ++i)
    if (base + i < n) {
      data[base + i] = run;
      run += v[i];
    }
}

}  // namespace

int64_t scan_scratch_elems(int64_t n) { return (n + kTile - 1) / kTile + 1; }

cudaError_t launch_scan_i64(int64_t *data, int64_t n, int64_t *scratch, cudaStream_t s) {
  const int64_t nt = (n + kTile - 1) / kTile;
  if (nt == 0) return cudaMemsetAsync(data, 0, sizeof(int64_t), s);
  if (nt > 0x7fffffff) return cudaErrorInvalidValue;
  k_scan_tiles<<<(unsigned)nt, kThreads, 0, s>>>(data, n, scratch);
  k_scan_sums<<<1, kThreads, 0, s>>>(scratch, nt, data + n);
  k_scan_apply<<<(unsigned)nt, kThreads, 0, s>>>(data, n, scratch);
  return cudaGetLastError();
}

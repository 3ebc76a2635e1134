// Device-wide exclusive scan of int32 counts (stream compaction offsets).
// Two launches: per-tile scan (writing the tile totals), then add-back, where
// every tile sums the totals of the tiles before it (integer sums: exact in
// any order).  out has n + 1 entries; out[n] is the total.
#include "ebr_kernels.cuh"
#include "lookback.cuh"

namespace ebr {

constexpr int SCAN_T = 256;
constexpr int SCAN_ITEMS = 4;
constexpr int SCAN_TILE = SCAN_T * SCAN_ITEMS;

__global__ void __launch_bounds__(SCAN_T) k_scan_tiles(const int* __restrict__ in, int* __restrict__ out,
                                                       int n, int* __restrict__ tile_sum) {
  pdl_enter();
  __shared__ int sh[32];
  long long base = (long long)blockIdx.x * SCAN_TILE + threadIdx.x * SCAN_ITEMS;
  int v[SCAN_ITEMS];
  int local = 0;
#pragma unroll
  for (int q = 0; q < SCAN_ITEMS; ++q) {
    long long i = base + q;
    v[q] = i < n ? in[i] : 0;
    local += v[q];
  }
  int total;
  int ex = block_excl_scan(local, sh, total);
#pragma unroll
  for (int q = 0; q < SCAN_ITEMS; ++q) {
    long long i = base + q;
    if (i < n) out[i] = ex;
    ex += v[q];
  }
  if (threadIdx.x == 0) tile_sum[blockIdx.x] = total;
}

__global__ void __launch_bounds__(SCAN_T) k_scan_sums(int* __restrict__ tile_sum, int ntiles,
                                                      int* __restrict__ out, int n) {
  pdl_enter();
  __shared__ int sh[32];
  int carry = 0;
  for (int base = 0; base < ntiles; base += SCAN_T) {
    int i = base + threadIdx.x;
    int v = i < ntiles ? tile_sum[i] : 0;
    int total;
    int ex = block_excl_scan(v, sh, total);
    if (i < ntiles) tile_sum[i] = carry + ex;
    carry += total;
  }
  if (threadIdx.x == 0) out[n] = carry;
}

__global__ void __launch_bounds__(SCAN_T) k_scan_add(int* __restrict__ out, int n,
                                                     const int* __restrict__ tile_sum, int ntiles) {
  pdl_enter();
  __shared__ int sh[32];
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  // offset of this tile: the totals of the tiles before it (one more for the
  // last tile, whose sum is the grand total out[n])
  const int upto = blockIdx.x == ntiles - 1 ? ntiles : blockIdx.x;
  int part = 0;
  for (int i = threadIdx.x; i < upto; i += SCAN_T) part += tile_sum[i];
  part = __reduce_add_sync(0xffffffffu, part);
  if (lane == 0) sh[w] = part;
  __syncthreads();
  int before = 0, total = 0;
  for (int q = 0; q < SCAN_T / 32; ++q) total += sh[q];
  if (blockIdx.x == ntiles - 1) {
    before = total - tile_sum[ntiles - 1];
    if (threadIdx.x == 0) out[n] = total;
  } else {
    before = total;
  }
  long long base = (long long)blockIdx.x * SCAN_TILE + threadIdx.x * SCAN_ITEMS;
#pragma unroll
  for (int q = 0; q < SCAN_ITEMS; ++q) {
    long long i = base + q;
    if (i < n) out[i] += before;
  }
}

size_t scan_temp_bytes(int n) {
  int ntiles = (n + SCAN_TILE - 1) / SCAN_TILE;
  return sizeof(int) * (size_t)(ntiles > 0 ? ntiles : 1);
}

void launch_scan(const int* in, int* out, int n, void* temp, cudaStream_t s) {
  int ntiles = (n + SCAN_TILE - 1) / SCAN_TILE;
  int* ts = static_cast<int*>(temp);
  if (n <= 0) {
    launch(k_scan_sums, 1, SCAN_T, 0, s, ts, 0, out, 0);
    return;
  }
  launch(k_scan_tiles, ntiles, SCAN_T, 0, s, in, out, n, ts);
  launch(k_scan_add, ntiles, SCAN_T, 0, s, out, n, ts, ntiles);
}

}  // namespace ebr

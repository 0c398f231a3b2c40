// Exclusive prefix sums over int64 arrays (three-phase: tile scan, scan of
// tile totals, add-back), used by the CSR update and work-list builders.
#include "common.cuh"

namespace grest {

namespace {
constexpr int kScanThreads = 1024;
constexpr int kScanItems = 4;
constexpr int kScanTile = kScanThreads * kScanItems;

__device__ __forceinline__ int64_t warp_incl_scan(int64_t v) {
  const int lane = threadIdx.x & 31;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    int64_t t = __shfl_up_sync(0xffffffffu, v, o);
    if (lane >= o) v += t;
  }
  return v;
}

// Block-wide exclusive scan of one value per thread; returns the block total.
__device__ int64_t block_excl_scan(int64_t v, int64_t* excl) {
  __shared__ int64_t wsum[kScanThreads / 32];
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  int64_t inc = warp_incl_scan(v);
  if (lane == 31) wsum[wid] = inc;
  __syncthreads();
  if (wid == 0) {
    int64_t t = (lane < kScanThreads / 32) ? wsum[lane] : 0;
    t = warp_incl_scan(t);
    if (lane < kScanThreads / 32) wsum[lane] = t;
  }
  __syncthreads();
  int64_t before = wid ? wsum[wid - 1] : 0;
  *excl = before + inc - v;
  int64_t total = wsum[kScanThreads / 32 - 1];
  __syncthreads();
  return total;
}

__global__ void __launch_bounds__(kScanThreads) k_scan_tiles(const int64_t* __restrict__ in, int64_t* out,
                                                             int64_t n, int64_t* tile_sum) {
  const int64_t base = (int64_t)blockIdx.x * kScanTile + (int64_t)threadIdx.x * kScanItems;
  int64_t v[kScanItems];
  int64_t s = 0;
#pragma unroll
  for (int i = 0; i < kScanItems; ++i) {
    v[i] = (base + i < n) ? in[base + i] : 0;
    s += v[i];
  }
  int64_t excl;
  int64_t total = block_excl_scan(s, &excl);
#pragma unroll
  for (int i = 0; i < kScanItems; ++i) {
    if (base + i < n) out[base + i] = excl;
    excl += v[i];
  }
  if (threadIdx.x == 0) tile_sum[blockIdx.x] = total;
}

__global__ void k_scan_add(int64_t* out, int64_t n, const int64_t* tile_off) {
  const int64_t i = (int64_t)blockIdx.x * kScanTile + threadIdx.x;
  const int64_t add = tile_off[blockIdx.x];
  for (int j = 0; j < kScanItems; ++j) {
    int64_t k = i + (int64_t)j * kScanThreads;
    if (k < n) out[k] += add;
  }
}

__global__ void k_scan_total(int64_t* out, int64_t n, const int64_t* tile_off, int64_t ntiles) {
  out[n] = tile_off[ntiles];
}

}  // namespace

size_t scan_temp_bytes(int64_t n) {
  size_t bytes = 0;
  while (true) {
    int64_t nt = (n + kScanTile - 1) / kScanTile;
    bytes += (size_t)(nt + 1) * sizeof(int64_t);
    if (nt <= 1) break;
    n = nt;
  }
  return bytes + 256;
}

int exclusive_scan_i64(const int64_t* in, int64_t* out, int64_t n, void* temp, cudaStream_t s) {
  if (n <= 0) {
    cudaMemsetAsync(out, 0, sizeof(int64_t), s);
    return 0;
  }
  int64_t nt = (n + kScanTile - 1) / kScanTile;
  int64_t* tiles = reinterpret_cast<int64_t*>(temp);
  k_scan_tiles<<<(unsigned)nt, kScanThreads, 0, s>>>(in, out, n, tiles);
  if (nt == 1) {  // a single tile: its total is the grand total
    k_scan_total<<<1, 1, 0, s>>>(out, n, tiles, 0);
    return 2;
  }
  // tiles[0..nt) -> exclusive offsets in place, total in tiles[nt]
  int k = exclusive_scan_i64(tiles, tiles, nt, tiles + nt + 1, s);
  k_scan_add<<<(unsigned)nt, kScanThreads, 0, s>>>(out, n, tiles);
  k_scan_total<<<1, 1, 0, s>>>(out, n, tiles, nt);
  return k + 3;
}

}  // namespace grest

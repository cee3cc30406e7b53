// scan.cu — device-wide exclusive prefix sum of u64 (reduce, scan the block
// sums recursively, then scan each block with its offset).  Used for event
// offsets per packet, radix-sort digit offsets and output compaction.
#include "internal.cuh"

namespace thapi {

namespace {

constexpr int kT = 256;
constexpr int kIpt = 8;
constexpr int kTile = kT * kIpt;

__device__ __forceinline__ uint64_t warp_incl_scan(uint64_t v) {
  const int lane = threadIdx.x & 31;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    uint64_t u = __shfl_up_sync(0xffffffffu, v, o);
    if (lane >= o) v += u;
  }
  return v;
}

// Block-wide exclusive scan of one value per thread; *total = block total.
__device__ __forceinline__ uint64_t block_excl_scan(uint64_t v, uint64_t *total) {
  __shared__ uint64_t wsum[kT / 32];
  __shared__ uint64_t tot;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  uint64_t inc = warp_incl_scan(v);
  if (lane == 31) wsum[warp] = inc;
  __syncthreads();
  if (warp == 0) {
    uint64_t w = lane < kT / 32 ? wsum[lane] : 0;
    uint64_t wi = warp_incl_scan(w);
    if (lane < kT / 32) wsum[lane] = wi - w;
    if (lane == 31) tot = wi;
  }
  __syncthreads();
  *total = tot;
  return wsum[warp] + inc - v;
}

__global__ void k_block_sums(const uint64_t *d, uint64_t n, uint64_t *sums) {
  uint64_t base = (uint64_t)blockIdx.x * kTile;
  uint64_t s = 0;
#pragma unroll
  for (int k = 0; k < kIpt; ++k) {
    uint64_t i = base + (uint64_t)k * kT + threadIdx.x;
    if (i < n) s += d[i];
  }
  for (int o = 16; o > 0; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o);
  __shared__ uint64_t ws[kT / 32];
  if ((threadIdx.x & 31) == 0) ws[threadIdx.x >> 5] = s;
  __syncthreads();
  if (threadIdx.x == 0) {
    uint64_t t = 0;
    for (int w = 0; w < kT / 32; ++w) t += ws[w];
    sums[blockIdx.x] = t;
  }
}

// Exclusive scan of each tile plus offs[block]; the grand total goes to *total (if set)
// from the last block.
__global__ void k_block_apply(uint64_t *d, uint64_t n, const uint64_t *offs, uint64_t *total) {
  __shared__ uint64_t tile[kTile];
  uint64_t base = (uint64_t)blockIdx.x * kTile;
#pragma unroll
  for (int k = 0; k < kIpt; ++k) {
    uint64_t i = base + (uint64_t)k * kT + threadIdx.x;
    tile[k * kT + threadIdx.x] = i < n ? d[i] : 0;
  }
  __syncthreads();
  uint64_t v[kIpt];
  uint64_t s = 0;
#pragma unroll
  for (int k = 0; k < kIpt; ++k) {
    v[k] = tile[threadIdx.x * kIpt + k];
    s += v[k];
  }
  uint64_t btot;
  uint64_t excl = block_excl_scan(s, &btot);
  uint64_t off = (offs ? offs[blockIdx.x] : 0) + excl;
#pragma unroll
  for (int k = 0; k < kIpt; ++k) {
    tile[threadIdx.x * kIpt + k] = off;
    off += v[k];
  }
  __syncthreads();
#pragma unroll
  for (int k = 0; k < kIpt; ++k) {
    uint64_t i = base + (uint64_t)k * kT + threadIdx.x;
    if (i < n) d[i] = tile[k * kT + threadIdx.x];
  }
  if (total && blockIdx.x == gridDim.x - 1 && threadIdx.x == 0) *total = (offs ? offs[blockIdx.x] : 0) + btot;
}

}  // namespace

void scan_exclusive_u64(uint64_t *data, uint64_t n, uint64_t *total_dev, Scratch &sc, cudaStream_t s) {
  if (n == 0) {
    if (total_dev) cudaMemsetAsync(total_dev, 0, sizeof(uint64_t), s);
    return;
  }
  uint64_t nb = (n + kTile - 1) / kTile;
  if (nb == 1) {
    k_block_apply<<<1, kT, 0, s>>>(data, n, nullptr, total_dev);
    count_launches(1);
    return;
  }
  uint64_t *sums = static_cast<uint64_t *>(sc.get(nb * sizeof(uint64_t)));
  if (!sums) return;
  k_block_sums<<<(unsigned)nb, kT, 0, s>>>(data, n, sums);
  scan_exclusive_u64(sums, nb, total_dev, sc, s);
  k_block_apply<<<(unsigned)nb, kT, 0, s>>>(data, n, sums, nullptr);
  count_launches(2);
}

}  // namespace thapi

// radix.cu — stable LSD radix sort of (u64 key, u32 value) pairs, 8-bit
// digits.  Per pass: tile digit histograms, one exclusive scan over the
// (digit-major, tile-minor) histogram, then a stable scatter in which each
// warp ranks its items with match-any and the CTA combines the warps' counts.
// Used to group packets by stream (stable in file order) and to order
// timeline intervals by start time (stable over stream order).
#include "internal.cuh"

namespace thapi {

namespace {

constexpr int kBits = 8;
constexpr int kBins = 1 << kBits;
constexpr int kT = 256;
constexpr int kWarps = kT / 32;
constexpr int kRounds = 16;                   // 32-item rounds per warp
constexpr int kTile = kWarps * 32 * kRounds;  // 4096 items

__global__ void __launch_bounds__(kT) k_hist(const uint64_t *keys, uint64_t n, int shift, uint64_t *hist,
                                              uint64_t ntiles) {
  __shared__ uint32_t h[kBins];
  for (int b = threadIdx.x; b < kBins; b += kT) h[b] = 0;
  __syncthreads();
  uint64_t base = (uint64_t)blockIdx.x * kTile;
  for (int k = threadIdx.x; k < kTile; k += kT) {
    uint64_t i = base + k;
    if (i < n) atomicAdd(&h[(uint32_t)(keys[i] >> shift) & (kBins - 1)], 1u);
  }
  __syncthreads();
  for (int b = threadIdx.x; b < kBins; b += kT) hist[(uint64_t)b * ntiles + blockIdx.x] = h[b];
}

__global__ void __launch_bounds__(kT) k_scatter(const uint64_t *kin, const uint32_t *vin, uint64_t *kout,
                                                 uint32_t *vout, uint64_t n, int shift, const uint64_t *offs,
                                                 uint64_t ntiles) {
  __shared__ uint32_t wcount[kWarps][kBins];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  for (int b = lane; b < kBins; b += 32) wcount[warp][b] = 0;
  __syncwarp();
  const uint64_t wbase = (uint64_t)blockIdx.x * kTile + (uint64_t)warp * 32 * kRounds;
  const uint32_t lt = (1u << lane) - 1u;
  uint32_t local[kRounds];
  uint32_t dig[kRounds];
#pragma unroll
  for (int r = 0; r < kRounds; ++r) {
    uint64_t i = wbase + (uint64_t)r * 32 + lane;
    bool valid = i < n;
    uint32_t d = valid ? ((uint32_t)(kin[i] >> shift) & (kBins - 1)) : kBins + lane;
    uint32_t peers = __match_any_sync(0xffffffffu, d);
    uint32_t rank = __popc(peers & lt);
    uint32_t before = valid ? wcount[warp][d] : 0;
    __syncwarp();
    if (valid && rank == 0) wcount[warp][d] = before + __popc(peers);
    __syncwarp();
    local[r] = before + rank;
    dig[r] = d;
  }
  __syncthreads();
  // exclusive prefix over warps for each digit
  for (int b = threadIdx.x; b < kBins; b += kT) {
    uint32_t run = 0;
#pragma unroll
    for (int w = 0; w < kWarps; ++w) {
      uint32_t t = wcount[w][b];
      wcount[w][b] = run;
      run += t;
    }
  }
  __syncthreads();
#pragma unroll
  for (int r = 0; r < kRounds; ++r) {
    uint64_t i = wbase + (uint64_t)r * 32 + lane;
    if (i < n) {
      uint32_t d = dig[r];
      uint64_t pos = offs[(uint64_t)d * ntiles + blockIdx.x] + wcount[warp][d] + local[r];
      kout[pos] = kin[i];
      vout[pos] = vin[i];
    }
  }
}

}  // namespace

void radix_sort_pairs(uint64_t *keys, uint32_t *vals, uint64_t *keys_alt, uint32_t *vals_alt, uint64_t n, int bits,
                      bool *result_in_alt, Scratch &sc, cudaStream_t s) {
  *result_in_alt = false;
  if (n <= 1 || bits <= 0) return;
  uint64_t ntiles = (n + kTile - 1) / kTile;
  uint64_t *hist = static_cast<uint64_t *>(sc.get(ntiles * kBins * sizeof(uint64_t)));
  if (!hist) return;
  uint64_t *ki = keys, *ko = keys_alt;
  uint32_t *vi = vals, *vo = vals_alt;
  bool alt = false;
  for (int shift = 0; shift < bits; shift += kBits) {
    k_hist<<<(unsigned)ntiles, kT, 0, s>>>(ki, n, shift, hist, ntiles);
    scan_exclusive_u64(hist, ntiles * kBins, nullptr, sc, s);
    k_scatter<<<(unsigned)ntiles, kT, 0, s>>>(ki, vi, ko, vo, n, shift, hist, ntiles);
    count_launches(2);
    uint64_t *tk = ki;
    ki = ko;
    ko = tk;
    uint32_t *tv = vi;
    vi = vo;
    vo = tv;
    alt = !alt;
  }
  *result_in_alt = alt;
}

}  // namespace thapi

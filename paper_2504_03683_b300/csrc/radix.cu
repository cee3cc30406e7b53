// radix.cu — stable LSD radix sort of (key, u32 value) pairs, 8-bit digits,
// keys u32 or u64.  Below 2^20 items, per pass: tile digit histograms
// (warp-aggregated), one exclusive scan over the (digit-major, tile-minor)
// histogram, then a stable scatter.  From 2^20 items on (the one-sweep
// form): all passes' global digit histograms in one read of the keys, then
// one kernel per pass whose tiles find their offsets by decoupled look-back
// over the tiles before them (bounded waits).  Either way a tile is loaded
// into registers, ranked per warp (one ballot per digit bit), laid out digit
// by digit in shared memory, and written out in runs of equal digits so that
// stores coalesce.  The last pass can gather the
// final records (out[pos] = rec[value]) instead of writing (key, value).
// Used to group packets by stream (stable in file order) and to order
// timeline intervals by start time (stable over stream order).
#include <algorithm>

#include "internal.cuh"

namespace thapi {

namespace {

constexpr int kBits = 8;
constexpr int kBins = 1 << kBits;
constexpr int kT = 256;
constexpr int kWarps = kT / 32;
constexpr int kRounds = 16;                   // 32-item rounds per warp
constexpr int kTile = kWarps * 32 * kRounds;  // 4096 items

// Lanes of the warp whose digit equals this lane's (valid lanes only): one
// ballot per digit bit, fewer issue slots than a match on the digit.
__device__ __forceinline__ uint32_t same_digit(uint32_t d, bool valid) {
  uint32_t peers = __ballot_sync(0xffffffffu, valid);
#pragma unroll
  for (int bit = 0; bit < kBits; ++bit) {
    const uint32_t m = __ballot_sync(0xffffffffu, (d >> bit) & 1u);
    peers &= ((d >> bit) & 1u) ? m : ~m;
  }
  return peers;
}

template <class K>
__global__ void __launch_bounds__(kT) k_hist(const K *keys, uint64_t n, int shift, uint64_t *hist, uint64_t ntiles) {
  __shared__ uint32_t h[kBins];
  for (int b = threadIdx.x; b < kBins; b += kT) h[b] = 0;
  __syncthreads();
  const int lane = threadIdx.x & 31;
  const uint64_t base = (uint64_t)blockIdx.x * kTile;
  for (int k = threadIdx.x; k < kTile; k += kT) {
    const uint64_t i = base + k;
    const bool in = i < n;
    const uint32_t d = in ? (uint32_t)(keys[i] >> shift) & (kBins - 1) : 0u;
    const uint32_t peers = same_digit(d, in);
    if (in && (peers & ((1u << lane) - 1u)) == 0) atomicAdd(&h[d], (uint32_t)__popc(peers));
  }
  __syncthreads();
  for (int b = threadIdx.x; b < kBins; b += kT) hist[(uint64_t)b * ntiles + blockIdx.x] = h[b];
}

template <class K>
__global__ void __launch_bounds__(kT) k_scatter(const K *kin, const uint32_t *vin, K *kout, uint32_t *vout, uint64_t n,
                                                 int shift, const uint64_t *offs, uint64_t ntiles,
                                                 const thapi_interval *rec, thapi_interval *rec_out) {
  extern __shared__ __align__(16) uint8_t smem[];
  K *s_key = reinterpret_cast<K *>(smem);
  uint32_t *s_val = reinterpret_cast<uint32_t *>(smem + sizeof(K) * kTile);
  __shared__ uint32_t wcount[kWarps][kBins];
  __shared__ uint32_t dstart[kBins];  // first tile-local index of each digit
  __shared__ uint64_t dglob[kBins];   // first global index of each digit for this tile
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  for (int b = lane; b < kBins; b += 32) wcount[warp][b] = 0;
  __syncwarp();
  const uint64_t wbase = (uint64_t)blockIdx.x * kTile + (uint64_t)warp * 32 * kRounds;
  const uint32_t lt = (1u << lane) - 1u;
  K key[kRounds];
  uint32_t val[kRounds];
#pragma unroll
  for (int r = 0; r < kRounds; ++r) {
    const uint64_t i = wbase + (uint64_t)r * 32 + lane;
    key[r] = i < n ? kin[i] : (K)0;
    val[r] = i < n ? vin[i] : 0u;
  }
  uint32_t local[kRounds];
#pragma unroll
  for (int r = 0; r < kRounds; ++r) {
    const uint64_t i = wbase + (uint64_t)r * 32 + lane;
    const bool valid = i < n;
    const uint32_t d = valid ? ((uint32_t)(key[r] >> shift) & (kBins - 1)) : 0u;
    const uint32_t peers = same_digit(d, valid);
    const uint32_t rank = __popc(peers & lt);
    const uint32_t before = valid ? wcount[warp][d] : 0u;
    __syncwarp();
    if (valid && rank == 0) wcount[warp][d] = before + __popc(peers);
    __syncwarp();
    local[r] = before + rank;
  }
  __syncthreads();
  // per digit: exclusive prefix over warps, the tile's count, and its global start
  for (int b = threadIdx.x; b < kBins; b += kT) {
    uint32_t run = 0;
#pragma unroll
    for (int w = 0; w < kWarps; ++w) {
      const uint32_t t = wcount[w][b];
      wcount[w][b] = run;
      run += t;
    }
    dstart[b] = run;  // temporarily the tile count of digit b
    dglob[b] = offs[(uint64_t)b * ntiles + blockIdx.x];
  }
  __syncthreads();
  if (warp == 0) {  // exclusive scan of the tile's digit counts
    uint32_t carry = 0;
    for (int b0 = 0; b0 < kBins; b0 += 32) {
      const uint32_t c = dstart[b0 + lane];
      uint32_t inc = c;
#pragma unroll
      for (int o = 1; o < 32; o <<= 1) {
        const uint32_t u = __shfl_up_sync(0xffffffffu, inc, o);
        if (lane >= o) inc += u;
      }
      dstart[b0 + lane] = carry + inc - c;
      carry += __shfl_sync(0xffffffffu, inc, 31);
    }
  }
  __syncthreads();
  // lay the tile out digit by digit in shared memory
#pragma unroll
  for (int r = 0; r < kRounds; ++r) {
    const uint64_t i = wbase + (uint64_t)r * 32 + lane;
    if (i < n) {
      const uint32_t d = (uint32_t)(key[r] >> shift) & (kBins - 1);
      const uint32_t at = dstart[d] + wcount[warp][d] + local[r];
      s_key[at] = key[r];
      s_val[at] = val[r];
    }
  }
  __syncthreads();
  // write runs of equal digits to consecutive global positions
  const uint64_t rest = n - (uint64_t)blockIdx.x * kTile;
  const uint64_t tile_n = rest < (uint64_t)kTile ? rest : (uint64_t)kTile;
  for (uint32_t j = threadIdx.x; j < tile_n; j += kT) {
    const K k = s_key[j];
    const uint32_t d = (uint32_t)(k >> shift) & (kBins - 1);
    const uint64_t pos = dglob[d] + (j - dstart[d]);
    if (rec_out) {
      rec_out[pos] = rec[s_val[j]];
    } else {
      kout[pos] = k;
      vout[pos] = s_val[j];
    }
  }
}

// ---------------------------------------------------------------- one sweep
// Large inputs: every pass's global digit histogram in one read of the keys,
// then one kernel per pass.  Tiles take ids in launch order from a counter;
// a tile publishes its per-digit counts (AGGREGATE), sums its predecessors'
// counts walking back until one has published its INCLUSIVE prefix, and
// publishes its own; a tile waits only on tiles that took their ids before
// it and publish their counts before they wait, so the walk always ends.
// Every poll is bounded all the same; a wait that runs out sets *err and the
// sort reports a timeout.
constexpr uint64_t kAggr = 1ull << 62, kIncl = 2ull << 62, kValMask = (1ull << 62) - 1;
constexpr uint32_t kSpinLimit = 1u << 22;
constexpr uint64_t kOneSweepMin = 1ull << 20;  // items; smaller sorts keep the per-pass histograms

template <class K>
__global__ void __launch_bounds__(kT) k_os_hist(const K *keys, uint64_t n, int passes, uint32_t *ghist) {
  __shared__ uint32_t h[8][kBins];
  for (int b = threadIdx.x; b < 8 * kBins; b += kT) (&h[0][0])[b] = 0;
  __syncthreads();
  for (uint64_t i = (uint64_t)blockIdx.x * kT + threadIdx.x; i < n; i += (uint64_t)gridDim.x * kT) {
    const K k = keys[i];
    for (int p = 0; p < passes; ++p) atomicAdd(&h[p][(uint32_t)(k >> (p * kBits)) & (kBins - 1)], 1u);
  }
  __syncthreads();
  for (int b = threadIdx.x; b < passes * kBins; b += kT) {
    const uint32_t v = (&h[0][0])[b];
    if (v) atomicAdd(&ghist[b], v);
  }
}

// gbase[p][d] = exclusive prefix of pass p's digit counts (one block, a thread per digit)
__global__ void __launch_bounds__(kBins) k_os_scan(const uint32_t *ghist, int passes, uint64_t *gbase) {
  __shared__ uint64_t w[kBins / 32];
  const int d = threadIdx.x, lane = d & 31, warp = d >> 5;
  for (int p = 0; p < passes; ++p) {
    const uint64_t c = ghist[p * kBins + d];
    uint64_t inc = c;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const uint64_t u = __shfl_up_sync(0xffffffffu, inc, o);
      if (lane >= o) inc += u;
    }
    if (lane == 31) w[warp] = inc;
    __syncthreads();
    uint64_t base = 0;
    for (int k = 0; k < warp; ++k) base += w[k];
    gbase[p * kBins + d] = base + inc - c;
    __syncthreads();
  }
}

// Items of a tile are addressed by 32-bit offsets from the tile's first item;
// vin null: the values are the items' indexes (the first pass of a sort whose
// values start as 0, 1, 2, ...).  The write-out handles kOut items per thread
// at a time, their loads (and, gathering, their records) in flight together.
constexpr int kOut = 8;
static_assert(kTile % (kT * kOut) == 0, "whole write-out rounds");

template <class K>
__global__ void __launch_bounds__(kT) k_os_pass(const K *kin, const uint32_t *vin, K *kout, uint32_t *vout, uint64_t n,
                                                 int shift, const uint64_t *gbase, unsigned long long *status,
                                                 unsigned *tile_ctr, unsigned *err, const thapi_interval *rec,
                                                 thapi_interval *rec_out) {
  static_assert(kT == kBins, "a thread per digit in the look-back");
  extern __shared__ __align__(16) uint8_t smem[];
  K *s_key = reinterpret_cast<K *>(smem);
  uint32_t *s_val = reinterpret_cast<uint32_t *>(smem + sizeof(K) * kTile);
  __shared__ uint32_t wcount[kWarps][kBins];
  __shared__ uint32_t dstart[kBins];
  __shared__ unsigned long long doff[kBins];  // output position of tile slot j of digit d: doff[d] + j
  __shared__ uint32_t s_tile;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  if (threadIdx.x == 0) s_tile = atomicAdd(tile_ctr, 1u);
  for (int b = lane; b < kBins; b += 32) wcount[warp][b] = 0;
  __syncthreads();
  const uint64_t tile = s_tile;
  const uint64_t tbase = tile * kTile;
  const uint32_t tile_n = (uint32_t)(n - tbase < (uint64_t)kTile ? n - tbase : (uint64_t)kTile);
  const K *tk = kin + tbase;
  const uint32_t wfirst = (uint32_t)warp * 32 * kRounds + (uint32_t)lane;
  const uint32_t lt = (1u << lane) - 1u;
  K key[kRounds];
  uint32_t val[kRounds], local[kRounds];
#pragma unroll
  for (int r = 0; r < kRounds; ++r) {
    const uint32_t i = wfirst + (uint32_t)r * 32;
    key[r] = i < tile_n ? tk[i] : (K)0;
    val[r] = i < tile_n ? (vin ? vin[tbase + i] : (uint32_t)(tbase + i)) : 0u;
  }
#pragma unroll
  for (int r = 0; r < kRounds; ++r) {
    const bool valid = wfirst + (uint32_t)r * 32 < tile_n;
    const uint32_t d = valid ? ((uint32_t)(key[r] >> shift) & (kBins - 1)) : 0u;
    const uint32_t peers = same_digit(d, valid);
    const uint32_t rank = __popc(peers & lt);
    const uint32_t before = valid ? wcount[warp][d] : 0u;
    __syncwarp();
    if (valid && rank == 0) wcount[warp][d] = before + __popc(peers);
    __syncwarp();
    local[r] = before + rank;
  }
  __syncthreads();
  uint64_t dglob;  // this thread's digit: first output position of the tile's items of that digit
  {  // digit b = threadIdx.x: prefix over warps, publish, look back
    const int b = threadIdx.x;
    uint32_t run = 0;
#pragma unroll
    for (int w = 0; w < kWarps; ++w) {
      const uint32_t t = wcount[w][b];
      wcount[w][b] = run;
      run += t;
    }
    dstart[b] = run;
    unsigned long long *mine = status + tile * kBins + b;
    uint64_t excl = 0;
    if (tile == 0) {
      atomicExch(mine, kIncl | run);
    } else {
      atomicExch(mine, kAggr | run);
      // walk back kLook tiles per round (their loads in flight together), in
      // order; an entry not yet published is polled again from there
      constexpr int kLook = 8;
      int64_t j = (int64_t)tile - 1;
      uint32_t spins = 0;
      bool done = false;
      while (!done && j >= 0) {
        uint64_t v[kLook];
#pragma unroll
        for (int u = 0; u < kLook; ++u)
          v[u] = j - u >= 0 ? *reinterpret_cast<volatile unsigned long long *>(status + (uint64_t)(j - u) * kBins + b)
                            : kIncl;
        int used = kLook;
#pragma unroll
        for (int u = 0; u < kLook; ++u) {
          if (used < kLook || done) continue;
          const uint64_t f = v[u] & ~kValMask;
          if (f == 0) {  // not published yet: poll again from this entry
            used = u;
            continue;
          }
          excl += v[u] & kValMask;
          if (f == kIncl) done = true;
        }
        if (used < kLook && ++spins > kSpinLimit) {
          atomicExch(err, 1u);
          break;
        }
        j -= used;
      }
      atomicExch(mine, kIncl | (excl + run));
    }
    dglob = gbase[b] + excl;
  }
  __syncthreads();
  if (warp == 0) {  // exclusive scan of the tile's digit counts
    uint32_t carry = 0;
    for (int b0 = 0; b0 < kBins; b0 += 32) {
      const uint32_t c = dstart[b0 + lane];
      uint32_t inc = c;
#pragma unroll
      for (int o = 1; o < 32; o <<= 1) {
        const uint32_t u = __shfl_up_sync(0xffffffffu, inc, o);
        if (lane >= o) inc += u;
      }
      dstart[b0 + lane] = carry + inc - c;
      carry += __shfl_sync(0xffffffffu, inc, 31);
    }
  }
  __syncthreads();
  doff[threadIdx.x] = dglob - dstart[threadIdx.x];
#pragma unroll
  for (int r = 0; r < kRounds; ++r) {
    if (wfirst + (uint32_t)r * 32 < tile_n) {
      const uint32_t d = (uint32_t)(key[r] >> shift) & (kBins - 1);
      const uint32_t at = dstart[d] + wcount[warp][d] + local[r];
      s_key[at] = key[r];
      s_val[at] = val[r];
    }
  }
  __syncthreads();
  // runs of equal digits to consecutive output positions
  for (uint32_t j0 = threadIdx.x; j0 < tile_n; j0 += kT * kOut) {
    uint64_t pos[kOut];
    uint32_t v[kOut];
    K k[kOut];
#pragma unroll
    for (int u = 0; u < kOut; ++u) {
      const uint32_t j = j0 + (uint32_t)u * kT;
      if (j < tile_n) {
        k[u] = s_key[j];
        v[u] = s_val[j];
        pos[u] = doff[(uint32_t)(k[u] >> shift) & (kBins - 1)] + j;
      }
    }
    if (rec_out) {
      thapi_interval g[kOut];
#pragma unroll
      for (int u = 0; u < kOut; ++u)
        if (j0 + (uint32_t)u * kT < tile_n) g[u] = rec[v[u]];
#pragma unroll
      for (int u = 0; u < kOut; ++u)
        if (j0 + (uint32_t)u * kT < tile_n) rec_out[pos[u]] = g[u];
    } else {
#pragma unroll
      for (int u = 0; u < kOut; ++u)
        if (j0 + (uint32_t)u * kT < tile_n) {
          kout[pos[u]] = k[u];
          vout[pos[u]] = v[u];
        }
    }
  }
}

// Returns false when a look-back wait ran out (then sc.failed = 2).
template <class K>
bool sort_onesweep(K *keys, uint32_t *vals, K *keys_alt, uint32_t *vals_alt, uint64_t n, int bits,
                   bool *result_in_alt, const thapi_interval *rec, thapi_interval *rec_out, bool iota, Scratch &sc,
                   cudaStream_t s) {
  const int passes = (bits + kBits - 1) / kBits;
  const uint64_t ntiles = (n + kTile - 1) / kTile;
  uint32_t *ghist = static_cast<uint32_t *>(sc.get(8 * kBins * sizeof(uint32_t)));
  uint64_t *gbase = static_cast<uint64_t *>(sc.get(8 * kBins * sizeof(uint64_t)));
  unsigned long long *status = static_cast<unsigned long long *>(sc.get(ntiles * kBins * sizeof(uint64_t)));
  unsigned *ctr = static_cast<unsigned *>(sc.get(16 * sizeof(unsigned)));
  if (sc.failed) return true;
  unsigned *err = ctr + 8;
  cudaMemsetAsync(ghist, 0, 8 * kBins * sizeof(uint32_t), s);
  cudaMemsetAsync(ctr, 0, 16 * sizeof(unsigned), s);
  const unsigned hgrid = (unsigned)std::min<uint64_t>((n + kT - 1) / kT, 148ull * 8);
  k_os_hist<K><<<hgrid, kT, 0, s>>>(keys, n, passes, ghist);
  k_os_scan<<<1, kBins, 0, s>>>(ghist, passes, gbase);
  count_launches(2);
  const size_t smem = (sizeof(K) + sizeof(uint32_t)) * kTile;
  cudaFuncSetAttribute(k_os_pass<K>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  K *ki = keys, *ko = keys_alt;
  uint32_t *vi = vals, *vo = vals_alt;
  bool alt = false;
  const bool gather = rec_out != nullptr;
  for (int p = 0; p < passes; ++p) {
    const bool last = p == passes - 1;
    cudaMemsetAsync(status, 0, ntiles * kBins * sizeof(uint64_t), s);
    k_os_pass<K><<<(unsigned)ntiles, kT, smem, s>>>(ki, p == 0 && iota ? nullptr : vi, ko, vo, n, p * kBits,
                                                     gbase + p * kBins, status, ctr + p, err, rec,
                                                     last && gather ? rec_out : nullptr);
    count_launches(1);
    if (last && gather) break;
    K *tk = ki;
    ki = ko;
    ko = tk;
    uint32_t *tv = vi;
    vi = vo;
    vo = tv;
    alt = !alt;
  }
  *result_in_alt = alt;
  unsigned h_err = 0;
  if (cudaMemcpyAsync(&h_err, err, sizeof(h_err), cudaMemcpyDeviceToHost, s) != cudaSuccess ||
      cudaStreamSynchronize(s) != cudaSuccess || h_err) {
    sc.failed = 2;
    return false;
  }
  return true;
}

// iota: the values are the items' indexes 0, 1, 2, ... (vals is not read
// before the first pass writes it).
template <class K>
void sort_impl(K *keys, uint32_t *vals, K *keys_alt, uint32_t *vals_alt, uint64_t n, int bits, bool *result_in_alt,
               const thapi_interval *rec, thapi_interval *rec_out, bool iota, Scratch &sc, cudaStream_t s) {
  *result_in_alt = false;
  const bool gather = rec_out != nullptr;
  if (n == 0) return;
  if (bits <= 0) {
    if (gather) {
      if (iota)
        cudaMemcpyAsync(rec_out, rec, n * sizeof(thapi_interval), cudaMemcpyDeviceToDevice, s);
      else
        launch_timeline_gather(rec, vals, n, rec_out, s);
    }
    return;
  }
  if (n >= kOneSweepMin) {
    sort_onesweep<K>(keys, vals, keys_alt, vals_alt, n, bits, result_in_alt, rec, rec_out, iota, sc, s);
    return;
  }
  if (iota) launch_iota_u32(vals, n, s);
  const uint64_t ntiles = (n + kTile - 1) / kTile;
  uint64_t *hist = static_cast<uint64_t *>(sc.get(ntiles * kBins * sizeof(uint64_t)));
  if (!hist) return;
  const size_t smem = (sizeof(K) + sizeof(uint32_t)) * kTile;
  cudaFuncSetAttribute(k_scatter<K>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  K *ki = keys, *ko = keys_alt;
  uint32_t *vi = vals, *vo = vals_alt;
  bool alt = false;
  for (int shift = 0; shift < bits; shift += kBits) {
    const bool last = shift + kBits >= bits;
    k_hist<K><<<(unsigned)ntiles, kT, 0, s>>>(ki, n, shift, hist, ntiles);
    scan_exclusive_u64(hist, ntiles * kBins, nullptr, sc, s);
    k_scatter<K><<<(unsigned)ntiles, kT, smem, s>>>(ki, vi, ko, vo, n, shift, hist, ntiles, rec,
                                                     last && gather ? rec_out : nullptr);
    count_launches(2);
    if (last && gather) break;
    K *tk = ki;
    ki = ko;
    ko = tk;
    uint32_t *tv = vi;
    vi = vo;
    vo = tv;
    alt = !alt;
  }
  *result_in_alt = alt;
}

}  // namespace

void radix_sort_pairs(uint64_t *keys, uint32_t *vals, uint64_t *keys_alt, uint32_t *vals_alt, uint64_t n, int bits,
                      bool *result_in_alt, Scratch &sc, cudaStream_t s) {
  sort_impl<uint64_t>(keys, vals, keys_alt, vals_alt, n, bits, result_in_alt, nullptr, nullptr, false, sc, s);
}

void radix_sort_pairs32(uint32_t *keys, uint32_t *vals, uint32_t *keys_alt, uint32_t *vals_alt, uint64_t n, int bits,
                        bool *result_in_alt, Scratch &sc, cudaStream_t s) {
  sort_impl<uint32_t>(keys, vals, keys_alt, vals_alt, n, bits, result_in_alt, nullptr, nullptr, false, sc, s);
}

// Sorts the keys stably and writes rec_out[i] = rec[index of the i-th smallest
// key]; vals and vals_alt are work space.
void radix_sort_gather(uint64_t *keys, uint32_t *vals, uint64_t *keys_alt, uint32_t *vals_alt, uint64_t n, int bits,
                       const thapi_interval *rec, thapi_interval *rec_out, Scratch &sc, cudaStream_t s) {
  bool alt = false;
  if (bits <= 32) {
    sort_impl<uint32_t>(reinterpret_cast<uint32_t *>(keys), vals, reinterpret_cast<uint32_t *>(keys_alt), vals_alt, n,
                        bits, &alt, rec, rec_out, true, sc, s);
  } else {
    sort_impl<uint64_t>(keys, vals, keys_alt, vals_alt, n, bits, &alt, rec, rec_out, true, sc, s);
  }
}

}  // namespace thapi

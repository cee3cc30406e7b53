// bucket.cu — timeline order by bucketing on start time.
//
// The compacted interval records are in (stream, entry position) order and
// each stream's records are sorted by start, so the records of one stream
// that fall in one start bucket are a contiguous run.  With B buckets on the
// high bits of the start offset and S streams, the compaction counts the
// records of each (bucket, stream) cell and notes the cell's first record
// (one atomic pair per cell and warp).  Then one CTA per bucket:
//  1. reads its S cells, then the cells' runs of records into shared memory
//     in (stream, position) order, a thread per record (its cell from a
//     binary search of the cell starts), four loads in flight;
//  2. sorts the items (low key bits, position) in shared memory: each item
//     takes a rank in its bin of the key's top 9 bits from a shared-memory
//     atomic and lands at its bin's start plus that rank; the ranks follow no
//     order, so a thread per bin then insertion-sorts its bin by item value
//     (about c / 512 items when the starts spread over the bucket).  Items
//     are unique, so equal starts keep the (stream, position) order.  A
//     bucket with a bin over kBinMax items (clustered starts) is sorted by
//     stable LSD radix passes instead (9-bit digits, warp ranks from one
//     ballot per digit bit);
//  3. writes the records out in that order with coalesced stores, at the
//     bucket's offset (an exclusive scan of the bucket sizes).
// The result is the order (start, stream, entry position).  A cell's records
// are contiguous only while each stream's starts never decrease (an absolute
// timestamp may go back): every record read is checked to lie in its bucket,
// which holds exactly when the cell is contiguous.  A failed check, too many
// cells or a bucket over kCap records make the caller fall back to the radix
// sort.
#include <algorithm>

#include "internal.cuh"

namespace thapi {

namespace {

constexpr uint64_t kCoarse = 4096;          // bucket size aimed at (the mean lands between half and all of it)
constexpr uint64_t kMaxCells = 1ull << 26;  // (bucket, stream) cells
constexpr uint32_t kMaxStreams = 2048;      // cells of one bucket held in shared memory
constexpr uint32_t kCap = 4096;             // records of one bucket sorted in shared memory
constexpr int kDigit = 9;
constexpr uint32_t kBins = 1u << kDigit;
constexpr int kThreads = 512;
constexpr int kWarps = kThreads / 32;
constexpr uint32_t kRounds = kCap / kThreads;  // 32-record rounds per warp and radix pass
constexpr uint32_t kBinMax = 32;               // items of one bin the insertion sort takes
static_assert(kThreads == (int)kBins, "one thread per digit in the digit scan");
static_assert(kMaxStreams == 4 * kThreads, "four cells per thread in the cell scan");

// Shared memory of k_bucket_sort for item type IT.
template <class IT>
constexpr uint32_t sort_smem() {
  return (uint32_t)(kCap * sizeof(thapi_interval) + 2 * kCap * sizeof(IT) +
                    (kWarps * kBins + kBins + kWarps + 2 * kMaxStreams + 1) * sizeof(uint32_t));
}

__global__ void k_bucket_sizes(const uint32_t *cnt, uint32_t nb, uint32_t S, uint64_t *size) {
  const uint32_t lane = threadIdx.x & 31;
  const uint32_t b = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;  // one warp per bucket
  if (b >= nb) return;
  uint32_t c = 0;
  for (uint32_t r = lane; r < S; r += 32) c += cnt[(uint64_t)b * S + r];
  c = __reduce_add_sync(0xffffffffu, c);
  if (lane == 0) size[b] = c;
}

__global__ void k_bucket_max(const uint64_t *size, uint32_t nb, unsigned long long *out) {
  uint32_t m = 0;
  for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < nb; i += gridDim.x * blockDim.x)
    m = max(m, (uint32_t)size[i]);
  m = __reduce_max_sync(0xffffffffu, m);
  if ((threadIdx.x & 31) == 0 && m) atomicMax(out, (unsigned long long)m);
}

// One CTA per bucket (strided).  IT items: low key bits << QSH | position.
template <class IT>
__global__ void __launch_bounds__(kThreads, 1) k_bucket_sort(const uint32_t *cnt, const uint32_t *first,
                                                             const uint64_t *bstart, const uint64_t *bsize,
                                                             uint32_t nb, uint32_t S, int shift, uint64_t t_min,
                                                             const thapi_interval *__restrict__ rec,
                                                             thapi_interval *__restrict__ out, unsigned int *fail) {
  constexpr int QSH = sizeof(IT) == 4 ? 12 : 32;  // position bits (kCap <= 2^12)
  constexpr IT QMASK = ((IT)1 << QSH) - 1;
  extern __shared__ __align__(16) uint8_t smem[];
  thapi_interval *srec = reinterpret_cast<thapi_interval *>(smem);
  IT *ia = reinterpret_cast<IT *>(smem + kCap * sizeof(thapi_interval));
  IT *ib = ia + kCap;
  uint32_t *wcount = reinterpret_cast<uint32_t *>(ib + kCap);  // [kWarps][kBins]
  uint32_t *dstart = wcount + kWarps * kBins;                  // [kBins]
  uint32_t *wsum = dstart + kBins;                             // [kWarps]
  uint32_t *cpre = wsum + kWarps;                              // [S + 1] cell starts in the bucket
  uint32_t *cfirst = cpre + kMaxStreams + 1;                   // [S] first record of each cell
  const uint32_t tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const uint32_t lt = (1u << lane) - 1u;
  const uint64_t kmask = shift >= 64 ? ~0ull : ((1ull << shift) - 1);
  // the next bucket's cells (thread t: entries 4t .. 4t+3) are loaded while
  // the current one is sorted
  uint32_t ncnt[4], nfirst[4], nc = 0;
  uint64_t nst = 0;
  auto fetch = [&](uint32_t b) {
    if (b >= nb) return;
    nc = (uint32_t)bsize[b];
    nst = bstart[b];
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      const uint32_t r = tid * 4 + q;
      ncnt[q] = r < S ? cnt[(uint64_t)b * S + r] : 0u;
      nfirst[q] = r < S ? first[(uint64_t)b * S + r] : 0u;
    }
  };
  fetch(blockIdx.x);
  uint32_t pw = 1;  // largest power of two below S (at least 1)
  while ((pw << 1) < S) pw <<= 1;
  for (uint32_t b = blockIdx.x; b < nb; b += gridDim.x) {
    const uint32_t c = nc;
    const uint64_t st = nst;
    uint32_t loc[4];
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      loc[q] = ncnt[q];
      if (tid * 4 + q < S) cfirst[tid * 4 + q] = nfirst[q];
    }
    fetch(b + gridDim.x);
    if (c == 0) continue;
    // cells of this bucket: exclusive scan of the counts
    {
      uint32_t sum = 0;
#pragma unroll
      for (int q = 0; q < 4; ++q) sum += loc[q];
      uint32_t inc = sum;
#pragma unroll
      for (int o = 1; o < 32; o <<= 1) {
        const uint32_t u = __shfl_up_sync(0xffffffffu, inc, o);
        if (lane >= (uint32_t)o) inc += u;
      }
      if (lane == 31) wsum[warp] = inc;
      __syncthreads();
      uint32_t run = inc - sum;
      for (uint32_t w = 0; w < warp; ++w) run += wsum[w];
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        const uint32_t r = tid * 4 + q;
        if (r < S) cpre[r] = run;
        run += loc[q];
      }
      if (tid == 0) cpre[S] = c;
    }
    __syncthreads();
    // records of the bucket in (cell, position) order: thread per record, its
    // cell found by a binary search of the cell starts (the largest cell start
    // not above it belongs to a non-empty cell), so that neighbouring threads
    // read neighbouring records of a cell; all of a thread's records in flight
    auto put = [&](uint32_t q, const thapi_interval &v) {
      srec[q] = v;
      const uint64_t key = v.start_ns - t_min;
      if ((key >> shift) != b && !(b == nb - 1 && (key >> shift) > b)) atomicExch(fail, 1u);  // cell not contiguous
      const uint64_t kl = (key - ((uint64_t)b << shift)) & kmask;
      ia[q] = ((IT)kl << QSH) | (IT)q;
    };
    {
      // branchless steps of decreasing powers of two, a thread's searches interleaved
      uint32_t lo[kRounds];
#pragma unroll
      for (uint32_t u = 0; u < kRounds; ++u) lo[u] = 0;
      for (uint32_t k = pw; k; k >>= 1) {
#pragma unroll
        for (uint32_t u = 0; u < kRounds; ++u) {
          const uint32_t t = lo[u] + k;
          if (t < S && cpre[t] <= tid + u * kThreads) lo[u] = t;
        }
      }
      uint64_t g[kRounds];
      thapi_interval v[kRounds];
#pragma unroll
      for (uint32_t u = 0; u < kRounds; ++u) {
        const uint32_t q = tid + u * kThreads;
        g[u] = q < c ? (uint64_t)cfirst[lo[u]] + (q - cpre[lo[u]]) : 0;
      }
#pragma unroll
      for (uint32_t u = 0; u < kRounds; ++u)
        if (tid + u * kThreads < c) v[u] = rec[g[u]];
#pragma unroll
      for (uint32_t u = 0; u < kRounds; ++u)
        if (tid + u * kThreads < c) put(tid + u * kThreads, v[u]);
    }
    // bins of the key's top bits: counts and ranks from shared-memory atomics
    const int dsh = shift > kDigit ? shift - kDigit : 0;
    uint32_t *bcnt = wcount;  // [kBins]
    bcnt[tid] = 0;
    __syncthreads();
    IT bv[kRounds];
    uint32_t brk[kRounds];
#pragma unroll
    for (uint32_t r = 0; r < kRounds; ++r) {
      const uint32_t q = tid + r * kThreads;
      if (q < c) {
        bv[r] = ia[q];
        brk[r] = atomicAdd(&bcnt[(uint32_t)((bv[r] >> QSH) >> dsh)], 1u);
      }
    }
    __syncthreads();
    {
      const uint32_t mine = bcnt[tid];
      uint32_t inc = mine;
#pragma unroll
      for (int o = 1; o < 32; o <<= 1) {
        const uint32_t u = __shfl_up_sync(0xffffffffu, inc, o);
        if (lane >= (uint32_t)o) inc += u;
      }
      if (lane == 31) wsum[warp] = inc;
      __syncthreads();
      uint32_t wbase = 0;
      for (uint32_t w = 0; w < warp; ++w) wbase += wsum[w];
      dstart[tid] = wbase + inc - mine;
    }
    IT *src = ia;
    const bool crowded = __syncthreads_or(bcnt[tid] > kBinMax);
    if (!crowded) {
#pragma unroll
      for (uint32_t r = 0; r < kRounds; ++r) {
        const uint32_t q = tid + r * kThreads;
        if (q < c) ib[dstart[(uint32_t)((bv[r] >> QSH) >> dsh)] + brk[r]] = bv[r];
      }
      __syncthreads();
      // insertion sort of bin tid by item value (items are unique)
      const uint32_t b0 = dstart[tid], nbin = bcnt[tid];
      for (uint32_t i = 1; i < nbin; ++i) {
        const IT x = ib[b0 + i];
        uint32_t j = i;
        for (; j > 0; --j) {
          const IT y = ib[b0 + j - 1];
          if (y < x) break;
          ib[b0 + j] = y;
        }
        ib[b0 + j] = x;
      }
      __syncthreads();
      src = ib;
    }
    // stable LSD radix on the key bits above QSH (buckets with a crowded bin)
    const uint32_t chunk = ((c + kThreads - 1) / kThreads) * 32;  // items per warp
    const uint32_t lo = warp * chunk, hi = min(lo + chunk, c);
    IT *dst = ib;
    for (int sh = QSH; crowded && sh < QSH + shift; sh += kDigit) {
      for (uint32_t d = lane; d < kBins; d += 32) wcount[warp * kBins + d] = 0;
      __syncwarp();
      IT v[kRounds];
      uint32_t loc[kRounds], dg[kRounds];
#pragma unroll
      for (uint32_t r = 0; r < kRounds; ++r) {
        const uint32_t i = lo + r * 32 + lane;
        const bool in = i < hi;
        v[r] = in ? src[i] : (IT)0;
        const uint32_t d = (uint32_t)(v[r] >> sh) & (kBins - 1);
        // lanes holding the same digit: one ballot per digit bit
        uint32_t peers = __ballot_sync(0xffffffffu, in);
#pragma unroll
        for (int bit = 0; bit < kDigit; ++bit) {
          const uint32_t m = __ballot_sync(0xffffffffu, (d >> bit) & 1u);
          peers &= ((d >> bit) & 1u) ? m : ~m;
        }
        const uint32_t before = in ? wcount[warp * kBins + d] : 0u;
        __syncwarp();
        if (in && (peers & lt) == 0) wcount[warp * kBins + d] = before + __popc(peers);
        __syncwarp();
        loc[r] = before + __popc(peers & lt);
        dg[r] = d;
      }
      __syncthreads();
      uint32_t tot = 0;  // digit tid: exclusive prefix over warps (in place) and the digit total
#pragma unroll
      for (int w = 0; w < kWarps; ++w) {
        const uint32_t t = wcount[w * kBins + tid];
        wcount[w * kBins + tid] = tot;
        tot += t;
      }
      uint32_t inc = tot;
#pragma unroll
      for (int o = 1; o < 32; o <<= 1) {
        const uint32_t u = __shfl_up_sync(0xffffffffu, inc, o);
        if (lane >= (uint32_t)o) inc += u;
      }
      if (lane == 31) wsum[warp] = inc;
      __syncthreads();
      uint32_t wbase = 0;
      for (uint32_t w = 0; w < warp; ++w) wbase += wsum[w];
      dstart[tid] = wbase + inc - tot;
      __syncthreads();
#pragma unroll
      for (uint32_t r = 0; r < kRounds; ++r) {
        const uint32_t i = lo + r * 32 + lane;
        if (i < hi) dst[dstart[dg[r]] + wcount[warp * kBins + dg[r]] + loc[r]] = v[r];
      }
      __syncthreads();
      IT *t = src;
      src = dst;
      dst = t;
    }
    // out as 8-byte words, consecutive threads on consecutive words
    const unsigned long long *sw = reinterpret_cast<const unsigned long long *>(srec);
    unsigned long long *ow = reinterpret_cast<unsigned long long *>(out + st);
    for (uint32_t w = tid; w < 3 * c; w += kThreads) {
      const uint32_t p = w / 3;
      ow[w] = sw[3 * (uint32_t)(src[p] & QMASK) + (w - 3 * p)];
    }
    __syncthreads();
  }
}

}  // namespace

bool bucket_plan(uint64_t n, int bits, uint32_t S, Scratch &sc, cudaStream_t s, BucketCells *bc) {
  *bc = BucketCells{};
  if (n < 2 || bits <= 0 || n >= 0xFFFFFFFFull || S == 0 || S > kMaxStreams) return false;
  int k1 = 0;
  while ((n >> k1) > kCoarse && k1 < bits && ((uint64_t)S << (k1 + 1)) <= kMaxCells) ++k1;
  if (bits - k1 > 32) k1 = bits - 32;  // the low key bits must fit 32 bits
  if (((uint64_t)S << k1) > kMaxCells) return false;
  const uint64_t cells = (uint64_t)S << k1;
  bc->cnt = static_cast<uint32_t *>(sc.get(cells * sizeof(uint32_t)));
  bc->first = static_cast<uint32_t *>(sc.get(cells * sizeof(uint32_t)));
  if (!bc->cnt || !bc->first) return false;
  cudaMemsetAsync(bc->cnt, 0, cells * sizeof(uint32_t), s);
  cudaMemsetAsync(bc->first, 0xFF, cells * sizeof(uint32_t), s);
  bc->shift = bits - k1;
  bc->nb = 1u << k1;
  bc->S = S;
  return true;
}

bool bucket_run(const BucketCells &bc, uint64_t t_min, uint64_t n, const thapi_interval *rec, thapi_interval *out,
                Scratch &sc, cudaStream_t s, int num_sms) {
  if (!bc.cnt) return false;
  uint64_t *bsize = static_cast<uint64_t *>(sc.get((uint64_t)bc.nb * sizeof(uint64_t)));
  uint64_t *bstart = static_cast<uint64_t *>(sc.get((uint64_t)bc.nb * sizeof(uint64_t)));
  unsigned long long *maxv = static_cast<unsigned long long *>(sc.get(2 * sizeof(unsigned long long)));
  if (!bsize || !bstart || !maxv) return false;
  unsigned int *fail = reinterpret_cast<unsigned int *>(maxv + 1);
  cudaMemsetAsync(maxv, 0, 2 * sizeof(unsigned long long), s);
  k_bucket_sizes<<<(unsigned)(((uint64_t)bc.nb * 32 + 255) / 256), 256, 0, s>>>(bc.cnt, bc.nb, bc.S, bsize);
  k_bucket_max<<<(unsigned)std::min<uint32_t>((bc.nb + 255) / 256, 1024u), 256, 0, s>>>(bsize, bc.nb, maxv);
  count_launches(2);
  if (cudaMemcpyAsync(bstart, bsize, (uint64_t)bc.nb * sizeof(uint64_t), cudaMemcpyDeviceToDevice, s) != cudaSuccess)
    return false;
  scan_exclusive_u64(bstart, bc.nb, nullptr, sc, s);
  unsigned long long mx = 0;
  if (cudaMemcpyAsync(&mx, maxv, sizeof(mx), cudaMemcpyDeviceToHost, s) != cudaSuccess ||
      cudaStreamSynchronize(s) != cudaSuccess)
    return false;
  if (mx > kCap) return false;
  const unsigned grid = (unsigned)std::max<uint64_t>(1, std::min<uint64_t>(bc.nb, (uint64_t)num_sms));
  if (bc.shift + 12 <= 32) {
    auto fn = k_bucket_sort<uint32_t>;
    if (cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sort_smem<uint32_t>()) !=
        cudaSuccess)
      return false;
    fn<<<grid, kThreads, sort_smem<uint32_t>(), s>>>(bc.cnt, bc.first, bstart, bsize, bc.nb, bc.S, bc.shift, t_min,
                                                      rec, out, fail);
  } else {
    auto fn = k_bucket_sort<uint64_t>;
    if (cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sort_smem<uint64_t>()) !=
        cudaSuccess)
      return false;
    fn<<<grid, kThreads, sort_smem<uint64_t>(), s>>>(bc.cnt, bc.first, bstart, bsize, bc.nb, bc.S, bc.shift, t_min,
                                                      rec, out, fail);
  }
  count_launches(1);
  unsigned int failed = 1;
  if (cudaGetLastError() != cudaSuccess ||
      cudaMemcpyAsync(&failed, fail, sizeof(failed), cudaMemcpyDeviceToHost, s) != cudaSuccess ||
      cudaStreamSynchronize(s) != cudaSuccess)
    return false;
  return failed == 0 && !sc.failed;
}

}  // namespace thapi

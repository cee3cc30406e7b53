// window.cu — time-window queries over a resident timeline (the timeline view
// of a time range, Sec. 3.6), without scratch that grows with the timeline.
//
// The timeline is in start order.  An interval belongs to the window [t0, t1)
// iff start < t1 and end >= t0.  The intervals with start < t1 are a prefix,
// [0, hi) with hi = lower_bound(start >= t1).  For the other condition a
// block index is kept per trace: for each block of kWinBlock intervals, the
// largest end over that block and every block before it (a prefix maximum,
// nondecreasing).  No interval before the first block whose prefix maximum
// reaches t0 can end at or after t0, so the window lies in
// [lo, hi) with lo = that block's first index, and a query reads only that
// range (its width plus the intervals of calls still open at t0), not the
// timeline up to t1.
//
// A query is two launches on a fixed grid: k_win_count finds lo and hi with
// warp-cooperative 32-way searches (about six rounds of loads for 10^8
// intervals) and counts the matches of each CTA's chunk of [lo, hi);
// k_win_write turns the per-CTA counts into offsets and writes the matches in
// timeline order, when they fit the caller's capacity, straight to the
// destination (device memory, or pinned host memory the device can reach).
// Its working memory is one WinWork record per query in flight.
#include <algorithm>

#include "internal.cuh"

namespace thapi {

namespace {

constexpr uint32_t kFullMask = 0xffffffffu;

// First index in [0, n) whose key is >= target (n if none), for
// nondecreasing keys key(i); one warp, 32 probes per round.
template <class Key>
__device__ uint64_t warp_lower_bound(uint64_t n, uint64_t target, Key key) {
  const uint32_t lane = threadIdx.x & 31;
  uint64_t a = 0, b = n;  // keys below a are < target, keys from b on are >= target
  while (b - a > 32) {
    const uint64_t step = (b - a + 31) / 32;
    const uint64_t p = a + (uint64_t)lane * step;
    const bool in = p < b;
    const bool less = in && key(p) < target;
    const uint32_t bal = __ballot_sync(kFullMask, less);
    const uint32_t inb = __ballot_sync(kFullMask, in);
    const uint32_t c = __popc(bal);  // the lanes whose probe is below target form a prefix
    const uint64_t na = c ? a + (uint64_t)(c - 1) * step + 1 : a;
    const uint64_t nb = (c < (uint32_t)__popc(inb)) ? a + (uint64_t)c * step : b;
    a = na;
    b = nb;
  }
  const uint64_t p = a + lane;
  const bool less = p < b && key(p) < target;
  return a + __popc(__ballot_sync(kFullMask, less));
}

__global__ void k_win_blockmax(const thapi_interval *tl, uint64_t n, uint64_t *bmax) {
  __shared__ unsigned long long part[8];
  const uint64_t b0 = (uint64_t)blockIdx.x * kWinBlock;
  const uint64_t b1 = min(b0 + kWinBlock, n);
  unsigned long long m = 0;
  for (uint64_t i = b0 + threadIdx.x; i < b1; i += blockDim.x) m = max(m, (unsigned long long)tl[i].end_ns);
  for (int o = 16; o; o >>= 1) m = max(m, __shfl_down_sync(kFullMask, m, o));
  if ((threadIdx.x & 31) == 0) part[threadIdx.x >> 5] = m;
  __syncthreads();
  if (threadIdx.x == 0) {
    for (uint32_t k = 1; k < blockDim.x / 32; ++k) m = max(m, part[k]);
    bmax[blockIdx.x] = m;
  }
}

// In-place running maximum of bmax[0..nb), one CTA of 1024 threads: each
// thread scans a contiguous chunk, then the chunk maxima are scanned.
__global__ void k_win_prefix(uint64_t *bmax, uint64_t nb) {
  __shared__ unsigned long long carry[1024];
  const uint64_t per = (nb + blockDim.x - 1) / blockDim.x;
  const uint64_t a = min((uint64_t)threadIdx.x * per, nb), b = min(a + per, nb);
  unsigned long long m = 0;
  for (uint64_t i = a; i < b; ++i) m = max(m, (unsigned long long)bmax[i]);
  carry[threadIdx.x] = m;
  __syncthreads();
  for (uint32_t o = 1; o < blockDim.x; o <<= 1) {  // inclusive max scan of the chunk maxima
    const unsigned long long v = threadIdx.x >= o ? carry[threadIdx.x - o] : 0ull;
    __syncthreads();
    carry[threadIdx.x] = max(carry[threadIdx.x], v);
    __syncthreads();
  }
  unsigned long long run = threadIdx.x ? carry[threadIdx.x - 1] : 0ull;
  for (uint64_t i = a; i < b; ++i) {
    run = max(run, (unsigned long long)bmax[i]);
    bmax[i] = run;
  }
}

__device__ __forceinline__ void chunk_of(uint64_t lo, uint64_t hi, uint32_t g, uint32_t G, uint64_t *c0,
                                         uint64_t *c1) {
  const uint64_t r = hi > lo ? hi - lo : 0;
  uint64_t per = (r + G - 1) / G;
  per = max(per, (uint64_t)kWinBlock);
  *c0 = min(lo + (uint64_t)g * per, max(hi, lo));
  *c1 = min(*c0 + per, max(hi, lo));
}

__global__ void __launch_bounds__(256) k_win_count(const thapi_interval *tl, uint64_t n, const uint64_t *bmax,
                                                   uint64_t nb, uint64_t t0, uint64_t t1, WinWork *w) {
  __shared__ uint64_t s_lo, s_hi;
  __shared__ unsigned long long part[8];
  const uint32_t warp = threadIdx.x >> 5;
  if (warp == 0) {
    const uint64_t hi = warp_lower_bound(n, t1, [&](uint64_t i) { return (uint64_t)tl[i].start_ns; });
    if ((threadIdx.x & 31) == 0) s_hi = hi;
  } else if (warp == 1) {
    const uint64_t lb = warp_lower_bound(nb, t0, [&](uint64_t j) { return bmax[j]; });
    if ((threadIdx.x & 31) == 0) s_lo = min(lb * (uint64_t)kWinBlock, n);
  }
  __syncthreads();
  const uint64_t lo = s_lo, hi = s_hi;
  uint64_t c0, c1;
  chunk_of(lo, hi, blockIdx.x, gridDim.x, &c0, &c1);
  unsigned long long cnt = 0;
  for (uint64_t i = c0 + threadIdx.x; i < c1; i += blockDim.x) cnt += tl[i].end_ns >= t0 ? 1u : 0u;
  for (int o = 16; o; o >>= 1) cnt += __shfl_down_sync(kFullMask, cnt, o);
  if ((threadIdx.x & 31) == 0) part[warp] = cnt;
  __syncthreads();
  if (threadIdx.x == 0) {
    for (uint32_t k = 1; k < blockDim.x / 32; ++k) cnt += part[k];
    w->cnt[blockIdx.x] = cnt;
    if (blockIdx.x == 0) {
      w->lo = lo;
      w->hi = hi;
    }
  }
}

__global__ void __launch_bounds__(256) k_win_write(const thapi_interval *tl, uint64_t t0, const WinWork *w,
                                                   thapi_interval *out, uint64_t cap, unsigned long long *total_out) {
  __shared__ unsigned long long s_off, s_tot;
  __shared__ uint32_t wcnt[8];
  const uint32_t lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  if (warp == 0) {  // this CTA's offset and the total, from the per-CTA counts
    unsigned long long off = 0, tot = 0;
    for (uint32_t k = lane; k < gridDim.x; k += 32) {
      const unsigned long long c = w->cnt[k];
      tot += c;
      off += k < blockIdx.x ? c : 0ull;
    }
    for (int o = 16; o; o >>= 1) {
      off += __shfl_down_sync(kFullMask, off, o);
      tot += __shfl_down_sync(kFullMask, tot, o);
    }
    if (lane == 0) {
      s_off = off;
      s_tot = tot;
      if (blockIdx.x == 0) *total_out = tot;
    }
  }
  __syncthreads();
  if (s_tot > cap || !out) return;
  uint64_t c0, c1;
  chunk_of(w->lo, w->hi, blockIdx.x, gridDim.x, &c0, &c1);
  unsigned long long base = s_off;
  for (uint64_t t = c0; t < c1; t += blockDim.x) {  // tiles of 256 in order
    const uint64_t i = t + threadIdx.x;
    const bool act = i < c1;
    uint64_t q0 = 0, q1 = 0, q2 = 0;
    if (act) {
      const unsigned long long *src = reinterpret_cast<const unsigned long long *>(tl + i);
      q0 = src[0];
      q1 = src[1];
      q2 = src[2];
    }
    const bool m = act && q1 >= t0;
    const uint32_t bal = __ballot_sync(kFullMask, m);
    if (lane == 0) wcnt[warp] = __popc(bal);
    __syncthreads();
    uint32_t before = 0, all = 0;
    for (uint32_t k = 0; k < blockDim.x / 32; ++k) {
      before += k < warp ? wcnt[k] : 0u;
      all += wcnt[k];
    }
    if (m) {
      unsigned long long *dst =
          reinterpret_cast<unsigned long long *>(out + base + before + __popc(bal & ((1u << lane) - 1u)));
      dst[0] = q0;
      dst[1] = q1;
      dst[2] = q2;
    }
    base += all;
    __syncthreads();  // wcnt is rewritten by the next tile
  }
}

}  // namespace

void launch_win_index(const thapi_interval *tl, uint64_t n, uint64_t *bmax, cudaStream_t s) {
  if (!n) return;
  const uint64_t nb = (n + kWinBlock - 1) / kWinBlock;
  k_win_blockmax<<<(unsigned)nb, 256, 0, s>>>(tl, n, bmax);
  k_win_prefix<<<1, 1024, 0, s>>>(bmax, nb);
  count_launches(2);
}

void launch_win_query(const thapi_interval *tl, uint64_t n, const uint64_t *bmax, uint64_t t0, uint64_t t1,
                      WinWork *w, uint32_t grid, thapi_interval *out, uint64_t cap, unsigned long long *total_out,
                      cudaStream_t s) {
  const uint64_t nb = (n + kWinBlock - 1) / kWinBlock;
  grid = std::max<uint32_t>(1, std::min<uint32_t>(grid, kWinCtas));
  k_win_count<<<grid, 256, 0, s>>>(tl, n, bmax, nb, t0, t1, w);
  k_win_write<<<grid, 256, 0, s>>>(tl, t0, w, out, cap, total_out);
  count_launches(2);
}

}  // namespace thapi

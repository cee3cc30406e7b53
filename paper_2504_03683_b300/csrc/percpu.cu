// percpu.cu — pairing the threads of per-CPU buffers.
//
// LTTng keeps one ring buffer per CPU (Sec. 3.1), so a buffer interleaves the
// events of every thread that ran on that CPU, each event naming its thread
// (vpid / vtid context, Sec. 3.2), and a thread that migrates leaves its
// events in several buffers.  A thread is (host, vpid, vtid); its events from
// all buffers, ordered by (ts, stream, position), are paired with one call
// stack.  Here, over the records k_percpu_decode wrote for every ENTRY and
// EXIT of those buffers:
//  1. stable LSD radix sorts by position, then ts, then (vpid, vtid), then
//     host give the order (host, vpid, vtid, ts, position);
//  2. thread boundaries, thread numbers (a scan of the boundaries) and a
//     segmented scan of the depth monoid (sum, min-prefix) give every event
//     its clamped depth before it, pre = S - min(0, min prefix S); an exit
//     with pre = 0 is unmatched, an entry's level is pre, an exit's pre - 1;
//  3. a stable sort by (thread, level) puts every entry right before the exit
//     that pops it (nothing at that level happens between them), so pairs
//     are neighbours: equal functions make an interval (written into the
//     entry's slot, tallied on the thread's cells), different ones a
//     mismatched pair; an entry with no exit after it is unmatched;
//  4. with self time on, the parent of a pair at level L > 0 is the last
//     record of the (thread, L - 1) run before its entry (binary search); a
//     parent that is a pair takes the child's duration, and each pair's self
//     time (duration less its children's) is tallied per thread.
#include <algorithm>

#include "device_util.cuh"
#include "internal.cuh"

namespace thapi {

namespace {

using dev::DM;
using dev::d_op;

constexpr int kT = 256;
constexpr int kSegThreads = 1024;

unsigned blocks(uint64_t n, int t = kT) { return (unsigned)((n + t - 1) / t); }

// key of the i-th record in the current order: 0 position, 1 ts - t_min, 2 thread, 3 host
__global__ void k_pc_key(const PcRec *rec, const uint32_t *perm, uint64_t m, int which, uint64_t t_min,
                         uint64_t *key, uint32_t *val) {
  const uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= m) return;
  const uint32_t j = perm ? perm[i] : (uint32_t)i;
  const PcRec &r = rec[j];
  key[i] = which == 0 ? r.gpos : which == 1 ? r.ts - t_min : which == 2 ? r.thread : r.host;
  if (!perm) val[i] = (uint32_t)i;
}

__global__ void k_pc_gather(const PcRec *rec, const uint32_t *perm, uint64_t m, PcRec *out) {
  const uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < m) out[i] = rec[perm[i]];
}

__device__ __forceinline__ bool same_thread(const PcRec &a, const PcRec &b) {
  return a.host == b.host && a.thread == b.thread;
}

__global__ void k_pc_heads(const PcRec *r, uint64_t m, uint64_t *head) {
  const uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < m) head[i] = (i == 0 || !same_thread(r[i - 1], r[i])) ? 1u : 0u;
}

// excl: exclusive scan of the heads.  Thread keys at the heads.
__global__ void k_pc_keys(const PcRec *r, const uint64_t *excl, uint64_t m, uint32_t *keys) {
  const uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= m) return;
  if (i == 0 || !same_thread(r[i - 1], r[i])) {
    const uint64_t t = excl[i];
    keys[3 * t] = r[i].host;
    keys[3 * t + 1] = (uint32_t)(r[i].thread >> 32);
    keys[3 * t + 2] = (uint32_t)r[i].thread;
  }
}

// Segmented monoid (head, DM): (ha, a) . (hb, b) = (ha | hb, hb ? b : a.b).
struct SegDM {
  uint32_t h;
  DM d;
};
__device__ __forceinline__ SegDM seg_op(SegDM a, SegDM b) { return b.h ? b : SegDM{a.h, d_op(a.d, b.d)}; }

// Inclusive segmented scan of one block (kSegThreads elements, one per thread).
__device__ __forceinline__ SegDM block_scan(SegDM x, SegDM *wagg) {
  const uint32_t lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const uint32_t uh = __shfl_up_sync(0xffffffffu, x.h, o);
    const int us = __shfl_up_sync(0xffffffffu, x.d.s, o), um = __shfl_up_sync(0xffffffffu, x.d.m, o);
    if (lane >= (uint32_t)o) x = seg_op(SegDM{uh, DM{us, um}}, x);
  }
  if (lane == 31) wagg[warp] = x;
  __syncthreads();
  if (warp == 0) {
    SegDM y = lane < kSegThreads / 32 ? wagg[lane] : SegDM{0u, DM{0, 0}};
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const uint32_t uh = __shfl_up_sync(0xffffffffu, y.h, o);
      const int us = __shfl_up_sync(0xffffffffu, y.d.s, o), um = __shfl_up_sync(0xffffffffu, y.d.m, o);
      if (lane >= (uint32_t)o) y = seg_op(SegDM{uh, DM{us, um}}, y);
    }
    if (lane < kSegThreads / 32) wagg[lane] = y;  // inclusive over warps
  }
  __syncthreads();
  if (warp > 0) x = seg_op(wagg[warp - 1], x);
  return x;
}

__device__ __forceinline__ SegDM element(const PcRec *r, uint64_t i, uint64_t m) {
  if (i >= m) return SegDM{1u, DM{0, 0}};
  const int e = r[i].kind == kEntry ? 1 : -1;
  const bool h = i == 0 || !same_thread(r[i - 1], r[i]);
  return SegDM{h ? 1u : 0u, DM{e, min(0, e)}};
}

// Per block: inclusive scan; the block's aggregate to agg[b].
__global__ void __launch_bounds__(kSegThreads) k_seg_local(const PcRec *r, uint64_t m, SegDM *agg) {
  __shared__ SegDM wagg[kSegThreads / 32];
  const uint64_t i = (uint64_t)blockIdx.x * kSegThreads + threadIdx.x;
  const SegDM x = block_scan(element(r, i, m), wagg);
  if (threadIdx.x == kSegThreads - 1) agg[blockIdx.x] = x;
}

// One CTA: exclusive scan of the block aggregates, in chunks of kSegThreads;
// agg[b] becomes the carry into block b.
__global__ void __launch_bounds__(kSegThreads) k_seg_blocks(SegDM *agg, uint64_t nb) {
  __shared__ SegDM wagg[kSegThreads / 32];
  __shared__ SegDM incs[kSegThreads];
  __shared__ SegDM carry;
  if (threadIdx.x == 0) carry = SegDM{0u, DM{0, 0}};
  __syncthreads();
  for (uint64_t c0 = 0; c0 < nb; c0 += kSegThreads) {
    const uint64_t i = c0 + threadIdx.x;
    const SegDM v = i < nb ? agg[i] : SegDM{0u, DM{0, 0}};
    const SegDM inc = block_scan(v, wagg);
    incs[threadIdx.x] = inc;
    __syncthreads();
    const SegDM ex = threadIdx.x > 0 ? incs[threadIdx.x - 1] : SegDM{0u, DM{0, 0}};
    const SegDM cin = carry;
    __syncthreads();  // carry and incs read by all
    if (i < nb) agg[i] = seg_op(cin, ex);
    if (threadIdx.x == kSegThreads - 1) carry = seg_op(cin, inc);
    __syncthreads();
  }
}

// pre = clamped depth before each event; key (thread << 32 | level), or ~0 for
// an unmatched exit; the largest level to *lmax.
__global__ void __launch_bounds__(kSegThreads) k_seg_apply(const PcRec *r, uint64_t m, const SegDM *carry,
                                                           const uint64_t *excl, uint64_t *key, uint32_t *val,
                                                           unsigned long long *lmax, unsigned long long *diag) {
  __shared__ SegDM wagg[kSegThreads / 32];
  __shared__ SegDM incs[kSegThreads];
  const uint64_t i = (uint64_t)blockIdx.x * kSegThreads + threadIdx.x;
  const SegDM x = element(r, i, m);
  const SegDM inc = block_scan(x, wagg);
  incs[threadIdx.x] = inc;
  __syncthreads();
  uint32_t lvl = 0;
  if (i < m) {
    SegDM ex = threadIdx.x > 0 ? incs[threadIdx.x - 1] : SegDM{0u, DM{0, 0}};
    ex = seg_op(carry[blockIdx.x], ex);
    const DM before = x.h ? DM{0, 0} : ex.d;
    const uint32_t pre = (uint32_t)(before.s - before.m);
    const bool entry = r[i].kind == kEntry;
    val[i] = (uint32_t)i;
    if (!entry && pre == 0) {
      key[i] = ~0ull;
      atomicAdd(&diag[dUnExit], 1ull);
    } else {
      lvl = entry ? pre : pre - 1;
      key[i] = (excl[i] + (x.h ? 1 : 0) - 1) << 32 | lvl;
    }
  }
  lvl = __reduce_max_sync(0xffffffffu, lvl);
  if ((threadIdx.x & 31) == 0 && lvl) atomicMax(lmax, (unsigned long long)lvl);
}

// (thread << 32 | level) -> (thread << lb | level); unmatched exits above every key
__global__ void k_pc_pack(uint64_t *key, uint64_t m, int lb, uint64_t unmatched_key) {
  const uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= m) return;
  const uint64_t k = key[i];
  key[i] = k == ~0ull ? unmatched_key : (k >> 32) << lb | (k & 0xFFFFFFFFull);
}

__global__ void k_pc_pair(const PcRec *r, const uint64_t *key, const uint32_t *val, uint64_t m,
                          uint64_t unmatched_key, int lb, uint32_t F, Cell *cells, thapi_interval *slots,
                          uint32_t *sum_nvalid, unsigned long long *diag) {
  const uint64_t k = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
  unsigned long long pairs = 0, mism = 0, unent = 0;
  if (k < m && key[k] != unmatched_key && r[val[k]].kind == kEntry) {
    const PcRec &en = r[val[k]];
    if (k + 1 < m && key[k + 1] == key[k] && r[val[k + 1]].kind == kExit) {
      const PcRec &ex = r[val[k + 1]];
      if (ex.func != en.func) {
        ++mism;
      } else {
        ++pairs;
        const uint64_t t = key[k] >> lb;
        const uint32_t lvl = (uint32_t)(key[k] & ((1ull << lb) - 1));
        const uint64_t dur = ex.ts - en.ts;
        Cell &c = cells[t * F + en.func];
        atomicAdd(&c.count, 1ull);
        atomicAdd(&c.total, (unsigned long long)dur);
        atomicMin(&c.mn, (unsigned long long)dur);
        atomicMax(&c.mx, (unsigned long long)dur);
        if (ex.err) atomicAdd(&c.err, 1ull);
        if (slots) {
          unsigned long long *q = reinterpret_cast<unsigned long long *>(slots + en.slot);
          q[0] = en.ts;
          q[1] = ex.ts;
          q[2] = 0xFFFFFFFFull | ((unsigned long long)en.func << 32) |
                 ((unsigned long long)(lvl < 255 ? lvl : 255) << 48) |
                 ((unsigned long long)(kIvValid | (ex.err ? kIvErr : 0)) << 56);
          atomicAdd(&sum_nvalid[en.pos], 1u);
        }
      }
    } else {
      ++unent;
    }
  }
  for (int o = 16; o > 0; o >>= 1) {
    pairs += __shfl_down_sync(0xffffffffu, pairs, o);
    mism += __shfl_down_sync(0xffffffffu, mism, o);
    unent += __shfl_down_sync(0xffffffffu, unent, o);
  }
  if ((threadIdx.x & 31) == 0) {
    if (pairs) atomicAdd(&diag[dPairs], pairs);
    if (mism) atomicAdd(&diag[dMismatch], mism);
    if (unent) atomicAdd(&diag[dUnEntry], unent);
  }
}

// An entry at sorted position k that its neighbour closes with the same function.
__device__ __forceinline__ bool is_pair(const PcRec *r, const uint64_t *key, const uint32_t *val, uint64_t m,
                                        uint64_t k) {
  if (k + 1 >= m || key[k + 1] != key[k]) return false;
  const PcRec &en = r[val[k]], &ex = r[val[k + 1]];
  return en.kind == kEntry && ex.kind == kExit && en.func == ex.func;
}

// Self time: the parent of the pair at k (level L > 0) is the entry open at
// depth L - 1 when k's entry is pushed, the last record of the (thread, L - 1)
// run before it in thread order; it takes the child's duration when it is a
// pair itself.
__global__ void k_pc_child(const PcRec *r, const uint64_t *key, const uint32_t *val, uint64_t m,
                           uint64_t unmatched_key, int lb, unsigned long long *child) {
  const uint64_t k = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= m) return;
  const uint64_t kk = key[k];
  if (kk == unmatched_key || (kk & ((1ull << lb) - 1)) == 0 || !is_pair(r, key, val, m, k)) return;
  const uint64_t target = kk - 1;
  const uint32_t pos = val[k];
  uint64_t lo = 0, hi = k;
  while (lo < hi) {
    const uint64_t mid = (lo + hi) >> 1;
    const uint64_t km = key[mid];
    if (km < target || (km == target && val[mid] < pos))
      lo = mid + 1;
    else
      hi = mid;
  }
  if (lo == 0 || key[lo - 1] != target || !is_pair(r, key, val, m, lo - 1)) return;
  atomicAdd(&child[lo - 1], (unsigned long long)(r[val[k + 1]].ts - r[val[k]].ts));
}

__global__ void k_pc_self(const PcRec *r, const uint64_t *key, const uint32_t *val, uint64_t m,
                          uint64_t unmatched_key, int lb, uint32_t F, const unsigned long long *child, Cell *cells) {
  const uint64_t k = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= m || key[k] == unmatched_key || !is_pair(r, key, val, m, k)) return;
  const PcRec &en = r[val[k]], &ex = r[val[k + 1]];
  const unsigned long long self = (ex.ts - en.ts) - child[k];
  Cell &c = cells[(key[k] >> lb) * F + en.func];
  atomicAdd(&c.count, 1ull);
  atomicAdd(&c.total, self);
  atomicMin(&c.mn, self);
  atomicMax(&c.mx, self);
  if (ex.err) atomicAdd(&c.err, 1ull);
}

}  // namespace

int percpu_pair(PcRec *rec, uint64_t m, uint64_t t_min, int ts_bits, uint32_t F, thapi_interval *slots,
                uint32_t *sum_nvalid, unsigned long long *diag, uint64_t *word, bool self_on, Scratch &sc,
                cudaStream_t s, PcPairOut *out) {
  *out = PcPairOut{};
  if (m == 0) return THAPI_OK;
  uint64_t *k1 = static_cast<uint64_t *>(sc.get(m * sizeof(uint64_t)));
  uint64_t *k2 = static_cast<uint64_t *>(sc.get(m * sizeof(uint64_t)));
  uint32_t *v1 = static_cast<uint32_t *>(sc.get(m * sizeof(uint32_t)));
  uint32_t *v2 = static_cast<uint32_t *>(sc.get(m * sizeof(uint32_t)));
  PcRec *r2 = static_cast<PcRec *>(sc.get(m * sizeof(PcRec)));
  uint64_t *head = static_cast<uint64_t *>(sc.get(m * sizeof(uint64_t)));
  if (sc.failed) return THAPI_E_NOMEM;
  // 1. order (host, vpid, vtid, ts, position): stable sorts from the last key to the first
  uint32_t *perm = nullptr;
  const int bits[4] = {32, std::max(1, std::min(64, ts_bits)), 64, 32};
  for (int which = 0; which < 4; ++which) {
    uint32_t *vin = perm ? perm : v1;
    uint32_t *valt = vin == v1 ? v2 : v1;
    k_pc_key<<<blocks(m), kT, 0, s>>>(rec, perm, m, which, t_min, k1, v1);
    bool alt = false;
    radix_sort_pairs(k1, vin, k2, valt, m, bits[which], &alt, sc, s);
    if (sc.failed) return THAPI_E_NOMEM;
    perm = alt ? valt : vin;
  }
  k_pc_gather<<<blocks(m), kT, 0, s>>>(rec, perm, m, r2);
  // 2. threads, their keys and the clamped depths
  k_pc_heads<<<blocks(m), kT, 0, s>>>(r2, m, head);
  scan_exclusive_u64(head, m, word, sc, s);
  if (sc.failed) return THAPI_E_NOMEM;
  uint64_t T = 0;
  if (cudaMemcpyAsync(&T, word, sizeof(T), cudaMemcpyDeviceToHost, s) != cudaSuccess ||
      cudaStreamSynchronize(s) != cudaSuccess)
    return THAPI_E_CUDA;
  out->threads = T;
  out->keys = static_cast<uint32_t *>(sc.get(3 * T * sizeof(uint32_t)));
  out->cells = static_cast<Cell *>(sc.get(T * F * sizeof(Cell)));
  const uint64_t nb = (m + kSegThreads - 1) / kSegThreads;
  SegDM *agg = static_cast<SegDM *>(sc.get(nb * sizeof(SegDM)));
  if (sc.failed) return THAPI_E_NOMEM;
  k_pc_keys<<<blocks(m), kT, 0, s>>>(r2, head, m, out->keys);
  launch_tally_init(out->cells, T * F, s);
  k_seg_local<<<(unsigned)nb, kSegThreads, 0, s>>>(r2, m, agg);
  k_seg_blocks<<<1, kSegThreads, 0, s>>>(agg, nb);
  if (cudaMemsetAsync(word + 1, 0, sizeof(uint64_t), s) != cudaSuccess) return THAPI_E_CUDA;
  k_seg_apply<<<(unsigned)nb, kSegThreads, 0, s>>>(r2, m, agg, head, k1, v1,
                                                   reinterpret_cast<unsigned long long *>(word + 1), diag);
  uint64_t lmax = 0;
  if (cudaMemcpyAsync(&lmax, word + 1, sizeof(lmax), cudaMemcpyDeviceToHost, s) != cudaSuccess ||
      cudaStreamSynchronize(s) != cudaSuccess)
    return THAPI_E_CUDA;
  // 3. (thread, level) order in tb + lb bits (T < 2^32 and levels < 2^32: at most 64), then neighbours pair
  int tb = 1, lb = 1;
  while ((1ull << tb) <= T) ++tb;
  while (lb < 32 && (lmax >> lb)) ++lb;
  const uint64_t unmatched = T << lb;  // above every (thread, level) key
  k_pc_pack<<<blocks(m), kT, 0, s>>>(k1, m, lb, unmatched);
  bool alt = false;
  radix_sort_pairs(k1, v1, k2, v2, m, tb + lb, &alt, sc, s);
  if (sc.failed) return THAPI_E_NOMEM;
  const uint64_t *key = alt ? k2 : k1;
  const uint32_t *val = alt ? v2 : v1;
  k_pc_pair<<<blocks(m), kT, 0, s>>>(r2, key, val, m, unmatched, lb, F, out->cells, slots, sum_nvalid, diag);
  count_launches(15);
  if (self_on) {  // 4. self time: children's durations to their parents, then the self tally
    unsigned long long *child = static_cast<unsigned long long *>(sc.get(m * sizeof(uint64_t)));
    out->self_cells = static_cast<Cell *>(sc.get(T * F * sizeof(Cell)));
    if (sc.failed) return THAPI_E_NOMEM;
    if (cudaMemsetAsync(child, 0, m * sizeof(uint64_t), s) != cudaSuccess) return THAPI_E_CUDA;
    launch_tally_init(out->self_cells, T * F, s);
    k_pc_child<<<blocks(m), kT, 0, s>>>(r2, key, val, m, unmatched, lb, child);
    k_pc_self<<<blocks(m), kT, 0, s>>>(r2, key, val, m, unmatched, lb, F, child, out->self_cells);
    count_launches(2);
  }
  return cudaGetLastError() == cudaSuccess ? THAPI_OK : THAPI_E_CUDA;
}

}  // namespace thapi

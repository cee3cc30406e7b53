// percpu.cu — pairing the threads of per-CPU buffers.
//
// LTTng keeps one ring buffer per CPU (Sec. 3.1), so a buffer interleaves the
// events of every thread that ran on that CPU, each event naming its thread
// (vpid / vtid context, Sec. 3.2), and a thread that migrates leaves its
// events in several buffers.  A thread is (host, vpid, vtid); its events from
// all buffers, ordered by (ts, stream, position), are paired with one call
// stack.  Here, over the records k_percpu_decode wrote at the per-CPU event
// positions (in (stream, position) order; positions of other events marked):
//  1. thread numbers: a table of (host, vpid, vtid) fingerprints (one insert
//     per distinct thread of a warp), then a scan of its used slots; every
//     record looks its thread up and checks the full key.  One stable radix
//     sort by (thread number, ts) of the position-ordered records gives the
//     thread order (thread, ts, stream, position).  When the table would fill
//     or two keys share a fingerprint, stable sorts by ts, (vpid, vtid) and
//     host give it instead, and thread numbers come from a scan of the thread
//     boundaries;
//  2. a segmented scan of the depth monoid (sum, min-prefix) per thread gives
//     every event its clamped depth before it, pre = S - min(0, min prefix
//     S); an exit with pre = 0 is unmatched, an entry's level is pre, an
//     exit's pre - 1;
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

// Records arrive in position order (each at its packet's per-CPU event base
// plus its index in the packet); positions of other events hold kNone.

// Per order position: its packet's events if it is a per-CPU buffer, else 0.
__global__ void k_pc_count(const PkDesc *desc, uint64_t n, uint64_t *out) {
  const uint64_t w = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (w < n) {
    const PkDesc d = dev::load_desc(desc + w);
    out[w] = d.group == kPerCpuGroup ? d.nev : 0u;
  }
}

// Thread table: open addressing on a 64-bit fingerprint of (host, vpid,
// vtid), the full key kept beside it and checked when records look it up.
__device__ __forceinline__ uint64_t thread_fp(uint32_t host, uint64_t thread) {
  uint64_t z = thread ^ ((uint64_t)host * 0x9E3779B97F4A7C15ull);
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  z ^= z >> 31;
  return z ? z : 1u;
}

// One insert per distinct thread of the warp, at most kProbes probes; flags
// bit 0: the table is too full (more than half its slots, or a probe run
// past kProbes), and the fallback order is taken.
constexpr uint32_t kProbes = 1024;
__global__ void k_thr_insert(const PcRec *rec, uint64_t m, unsigned long long *tfp, uint32_t *tkey, uint32_t mask,
                             unsigned long long *count, unsigned long long *flags) {
  const uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const bool valid = i < m && rec[i].kind != kPcNone;
  const uint32_t host = valid ? rec[i].host : 0u;
  const uint64_t thread = valid ? rec[i].thread : 0ull;
  const unsigned long long fp = valid ? thread_fp(host, thread) : 0ull;
  const uint32_t peers = __match_any_sync(0xffffffffu, fp);
  if (!valid || (threadIdx.x & 31) != (uint32_t)(__ffs(peers) - 1)) return;
  if (*reinterpret_cast<volatile unsigned long long *>(flags) & 1ull) return;
  uint32_t h = (uint32_t)fp & mask;
  for (uint32_t probe = 0; probe < kProbes; ++probe, h = (h + 1) & mask) {
    unsigned long long cur = tfp[h];
    if (cur == 0) {
      cur = atomicCAS(&tfp[h], 0ull, fp);
      if (cur == 0) {
        tkey[3 * h] = host;
        tkey[3 * h + 1] = (uint32_t)(thread >> 32);
        tkey[3 * h + 2] = (uint32_t)thread;
        if (atomicAdd(count, 1ull) + 1 > (mask + 1ull) / 2) atomicOr(flags, 1ull);
        return;
      }
    }
    if (cur == fp) return;
  }
  atomicOr(flags, 1ull);
}

__global__ void k_thr_used(const unsigned long long *tfp, uint64_t cap, uint64_t *used) {
  const uint64_t h = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (h < cap) used[h] = tfp[h] != 0 ? 1u : 0u;
}

// dense: exclusive scan of the used slots (dense thread numbers, slot order)
__global__ void k_thr_keys(const unsigned long long *tfp, const uint32_t *tkey, const uint64_t *dense, uint64_t cap,
                           uint32_t *keys) {
  const uint64_t h = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (h >= cap || tfp[h] == 0) return;
  const uint64_t t = dense[h];
  keys[3 * t] = tkey[3 * h];
  keys[3 * t + 1] = tkey[3 * h + 1];
  keys[3 * t + 2] = tkey[3 * h + 2];
}

// Sort key (thread number << tsb | ts - t_min); kNone positions get T << tsb
// (after every record).  flags bit 1: a fingerprint matched another key.
__global__ void k_pc_tkey(const PcRec *rec, uint64_t m, const unsigned long long *tfp, const uint32_t *tkey,
                          const uint64_t *dense, uint32_t mask, int tsb, uint64_t t_min, uint64_t T, uint64_t *key,
                          uint32_t *val, uint32_t *tid, unsigned long long *flags) {
  const uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= m) return;
  val[i] = (uint32_t)i;
  const PcRec r = rec[i];
  if (r.kind == kPcNone) {
    key[i] = T << tsb;
    return;
  }
  const unsigned long long fp = thread_fp(r.host, r.thread);
  uint32_t h = (uint32_t)fp & mask;
  uint32_t probe = 0;
  while (probe < kProbes && tfp[h] != fp && tfp[h] != 0) {
    h = (h + 1) & mask;
    ++probe;
  }
  if (probe >= kProbes || tfp[h] != fp || tkey[3 * h] != r.host || tkey[3 * h + 1] != (uint32_t)(r.thread >> 32) ||
      tkey[3 * h + 2] != (uint32_t)r.thread) {
    atomicOr(flags, 2ull);
    key[i] = T << tsb;
    return;
  }
  const uint64_t t = dense[h];
  tid[i] = (uint32_t)t;
  key[i] = t << tsb | (r.ts - t_min);
}

// Sorted records with the thread number in place of (host, vpid, vtid).
// Also tk[i] = thread number << 1 | (ENTRY): all the depth scan reads.
__global__ void k_pc_gather_t(const PcRec *rec, const uint32_t *perm, const uint32_t *tid, uint64_t m, PcRec *out,
                              uint32_t *tk) {
  const uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= m) return;
  const uint32_t j = perm[i];
  PcRec r = rec[j];
  r.thread = tid[j];
  r.host = 0;
  out[i] = r;
  tk[i] = tid[j] << 1 | (r.kind == kEntry ? 1u : 0u);
}

// Fallback order (table full or a fingerprint clash): stable sorts by ts,
// then (vpid, vtid), then host (kNone positions last).
__global__ void k_pc_key(const PcRec *rec, const uint32_t *perm, uint64_t m, int which, uint64_t t_min,
                         uint64_t *key, uint32_t *val) {
  const uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= m) return;
  const uint32_t j = perm ? perm[i] : (uint32_t)i;
  const PcRec &r = rec[j];
  const bool none = r.kind == kPcNone;
  key[i] = which == 1 ? (none ? 0 : r.ts - t_min) : which == 2 ? (none ? 0 : r.thread)
                                                               : (none ? (1ull << 32) : r.host);
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

// Fallback: excl = exclusive scan of the heads; thread keys at the heads and
// every record's thread number (to tnum).
__global__ void k_pc_keys(const PcRec *r, const uint64_t *excl, uint64_t m, uint32_t *keys, uint32_t *tnum) {
  const uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= m) return;
  const bool head = i == 0 || !same_thread(r[i - 1], r[i]);
  const uint64_t t = excl[i] + (head ? 1 : 0) - 1;
  tnum[i] = (uint32_t)t;
  if (head) {
    keys[3 * t] = r[i].host;
    keys[3 * t + 1] = (uint32_t)(r[i].thread >> 32);
    keys[3 * t + 2] = (uint32_t)r[i].thread;
  }
}

__global__ void k_pc_renumber(PcRec *r, const uint32_t *tnum, uint64_t m, uint32_t *tk) {
  const uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= m) return;
  r[i].thread = tnum[i];
  r[i].host = 0;
  tk[i] = tnum[i] << 1 | (r[i].kind == kEntry ? 1u : 0u);
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

// tk: thread number << 1 | (ENTRY), in thread order
__device__ __forceinline__ SegDM element(const uint32_t *tk, uint64_t i, uint64_t m) {
  if (i >= m) return SegDM{1u, DM{0, 0}};
  const uint32_t v = tk[i];
  const int e = (v & 1u) ? 1 : -1;
  const bool h = i == 0 || (tk[i - 1] >> 1) != (v >> 1);
  return SegDM{h ? 1u : 0u, DM{e, min(0, e)}};
}

// Per block: inclusive scan; the block's aggregate to agg[b].
__global__ void __launch_bounds__(kSegThreads) k_seg_local(const uint32_t *r, uint64_t m, SegDM *agg) {
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
__global__ void __launch_bounds__(kSegThreads) k_seg_apply(const uint32_t *r, uint64_t m, const SegDM *carry,
                                                           uint64_t *key, uint32_t *val, unsigned long long *lmax,
                                                           unsigned long long *diag) {
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
    const bool entry = (r[i] & 1u) != 0;
    val[i] = (uint32_t)i;
    if (!entry && pre == 0) {
      key[i] = ~0ull;
      atomicAdd(&diag[dUnExit], 1ull);
    } else {
      lvl = entry ? pre : pre - 1;
      key[i] = (uint64_t)(r[i] >> 1) << 32 | lvl;  // the thread number
    }
  }
  lvl = __reduce_max_sync(0xffffffffu, lvl);
  // one word for the whole grid: read first, write only a new maximum
  if ((threadIdx.x & 31) == 0 && lvl > *reinterpret_cast<volatile unsigned long long *>(lmax))
    atomicMax(lmax, (unsigned long long)lvl);
}

// (thread << 32 | level) -> (thread << lb | level); unmatched exits above every key
__global__ void k_pc_pack(uint64_t *key, uint64_t m, int lb, uint64_t unmatched_key) {
  const uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= m) return;
  const uint64_t k = key[i];
  key[i] = k == ~0ull ? unmatched_key : (k >> 32) << lb | (k & 0xFFFFFFFFull);
}

// A grid-stride loop over chunks of kT positions (chunks spread as in
// spread()); counters summed per thread and added once per block.
__global__ void k_pc_pair(const PcRec *r, const uint64_t *key, const uint32_t *val, uint64_t m,
                          uint64_t unmatched_key, int lb, uint32_t F, Cell *cells, thapi_interval *slots,
                          uint32_t *sum_nvalid, unsigned long long *diag) {
  __shared__ CellPart scr[kT];
  __shared__ unsigned long long part[kT / 32][3];
  const uint32_t lane = threadIdx.x & 31;
  const uint64_t nchunks = (m + kT - 1) / kT;
  unsigned long long pairs = 0, mism = 0, unent = 0;
  for (uint64_t c = blockIdx.x; c < nchunks; c += gridDim.x) {
    const uint64_t k = spread(c, nchunks) * kT + threadIdx.x;
    bool ok = false;
    uint64_t cell = 0;
    unsigned long long dur = 0;
    bool err = false;
    uint32_t pos = 0;
    if (k < m && key[k] != unmatched_key && r[val[k]].kind == kEntry) {
      const PcRec en = r[val[k]];
      if (k + 1 < m && key[k + 1] == key[k] && r[val[k + 1]].kind == kExit) {
        const PcRec ex = r[val[k + 1]];
        if (ex.func != en.func) {
          ++mism;
        } else {
          ++pairs;
          ok = true;
          const uint64_t t = key[k] >> lb;
          const uint32_t lvl = (uint32_t)(key[k] & ((1ull << lb) - 1));
          dur = ex.ts - en.ts;
          err = ex.err != 0;
          cell = t * F + en.func;
          pos = en.pos;
          if (slots) {
            unsigned long long *q = reinterpret_cast<unsigned long long *>(slots + en.slot);
            q[0] = en.ts;
            q[1] = ex.ts;
            q[2] = 0xFFFFFFFFull | ((unsigned long long)en.func << 32) |
                   ((unsigned long long)(lvl < 255 ? lvl : 255) << 48) |
                   ((unsigned long long)(kIvValid | (err ? kIvErr : 0)) << 56);
          }
        }
      } else {
        ++unent;
      }
    }
    warp_tally(cells, cell, ok, dur, err, scr + (threadIdx.x & ~31u));
    if (slots) {  // intervals per packet: one add per distinct packet of the warp
      const uint32_t peers = __match_any_sync(0xffffffffu, ok ? pos : 0xFFFFFFFFu);
      if (ok && lane == (uint32_t)(__ffs(peers) - 1)) atomicAdd(&sum_nvalid[pos], (uint32_t)__popc(peers));
    }
  }
  for (int o = 16; o > 0; o >>= 1) {
    pairs += __shfl_down_sync(0xffffffffu, pairs, o);
    mism += __shfl_down_sync(0xffffffffu, mism, o);
    unent += __shfl_down_sync(0xffffffffu, unent, o);
  }
  if (lane == 0) {
    part[threadIdx.x >> 5][0] = pairs;
    part[threadIdx.x >> 5][1] = mism;
    part[threadIdx.x >> 5][2] = unent;
  }
  __syncthreads();
  if (threadIdx.x < 3) {
    unsigned long long v = 0;
    for (int w = 0; w < kT / 32; ++w) v += part[w][threadIdx.x];
    if (v) atomicAdd(&diag[threadIdx.x == 0 ? dPairs : threadIdx.x == 1 ? dMismatch : dUnEntry], v);
  }
}

// An entry at sorted position k that its neighbour closes with the same function.
__device__ __forceinline__ bool is_pair(const PcRec *r, const uint64_t *key, const uint32_t *val, uint64_t m,
                                        uint64_t k) {
  if (k + 1 >= m || key[k + 1] != key[k]) return false;
  const PcRec &en = r[val[k]], &ex = r[val[k + 1]];
  return en.kind == kEntry && ex.kind == kExit && en.func == ex.func;
}

// First index in [lo, hi) whose (key, val) is not below (tk, tv).
__device__ __forceinline__ uint64_t lower_kv(const uint64_t *key, const uint32_t *val, uint64_t lo, uint64_t hi,
                                             uint64_t tk, uint32_t tv) {
  while (lo < hi) {
    const uint64_t mid = (lo + hi) >> 1;
    const uint64_t km = key[mid];
    if (km < tk || (km == tk && val[mid] < tv))
      lo = mid + 1;
    else
      hi = mid;
  }
  return lo;
}

// Self time: the parent of the pair at k (level L > 0) is the entry open at
// depth L - 1 when k's entry is pushed, the last record of the (thread, L - 1)
// run before it in thread order; it takes the child's duration when it is a
// pair itself (a binary search over the positions before k).
__global__ void k_pc_child(const PcRec *r, const uint64_t *key, const uint32_t *val, uint64_t m,
                           uint64_t unmatched_key, int lb, unsigned long long *child) {
  const uint64_t k = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= m) return;
  const uint64_t kk = key[k];
  if (kk == unmatched_key || (kk & ((1ull << lb) - 1)) == 0 || !is_pair(r, key, val, m, k)) return;
  const uint64_t target = kk - 1;
  const uint64_t lo = lower_kv(key, val, 0, k, target, val[k]);
  if (lo == 0 || key[lo - 1] != target || !is_pair(r, key, val, m, lo - 1)) return;
  atomicAdd(&child[lo - 1], (unsigned long long)(r[val[k + 1]].ts - r[val[k]].ts));
}

__global__ void k_pc_self(const PcRec *r, const uint64_t *key, const uint32_t *val, uint64_t m,
                          uint64_t unmatched_key, int lb, uint32_t F, const unsigned long long *child, Cell *cells) {
  __shared__ CellPart scr[kT];
  const uint64_t k = spread(blockIdx.x, gridDim.x) * blockDim.x + threadIdx.x;
  const bool ok = k < m && key[k] != unmatched_key && is_pair(r, key, val, m, k);
  uint64_t cell = 0;
  unsigned long long self = 0;
  bool err = false;
  if (ok) {
    const PcRec &en = r[val[k]], &ex = r[val[k + 1]];
    self = (ex.ts - en.ts) - child[k];
    cell = (key[k] >> lb) * F + en.func;
    err = ex.err != 0;
  }
  warp_tally(cells, cell, ok, self, err, scr + (threadIdx.x & ~31u));
}

}  // namespace

// n device words to the host (one wait)
static bool read_words(const uint64_t *d, uint64_t *h, int n, cudaStream_t s) {
  return cudaMemcpyAsync(h, d, n * sizeof(uint64_t), cudaMemcpyDeviceToHost, s) == cudaSuccess &&
         cudaStreamSynchronize(s) == cudaSuccess;
}

namespace {
__global__ void k_pc_bytes(const PkDesc *desc, const uint32_t *sum_nslot, uint64_t n, unsigned long long *out) {
  __shared__ unsigned long long part[kT / 32][2];
  unsigned long long rd = 0, en = 0;
  for (uint64_t w = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; w < n; w += (uint64_t)gridDim.x * blockDim.x) {
    const PkDesc d = dev::load_desc(desc + w);
    if (d.group == kPerCpuGroup) {
      rd += kPacketHeader + d.content;
      en += sum_nslot[w];
    }
  }
  for (int o = 16; o > 0; o >>= 1) {
    rd += __shfl_down_sync(0xffffffffu, rd, o);
    en += __shfl_down_sync(0xffffffffu, en, o);
  }
  if ((threadIdx.x & 31) == 0) {
    part[threadIdx.x >> 5][0] = rd;
    part[threadIdx.x >> 5][1] = en;
  }
  __syncthreads();
  if (threadIdx.x < 2) {
    unsigned long long v = 0;
    for (int k = 0; k < kT / 32; ++k) v += part[k][threadIdx.x];
    if (v) atomicAdd(&out[threadIdx.x], v);
  }
}
}  // namespace

void launch_pc_bytes(const PkDesc *desc, const uint32_t *sum_nslot, uint64_t n, unsigned long long *out,
                     cudaStream_t s) {
  if (!n) return;
  k_pc_bytes<<<(unsigned)std::min<uint64_t>(blocks(n), 256), kT, 0, s>>>(desc, sum_nslot, n, out);
  count_launches(1);
}

void launch_pc_count(const PkDesc *desc, uint64_t n, uint64_t *out, cudaStream_t s) {
  if (!n) return;
  k_pc_count<<<blocks(n), kT, 0, s>>>(desc, n, out);
  count_launches(1);
}

int percpu_pair(PcRec *rec, uint64_t m_all, uint64_t m, uint64_t t_min, int ts_bits, uint32_t F,
                thapi_interval *slots, uint32_t *sum_nvalid, unsigned long long *diag, bool self_on, int num_sms,
                Scratch &sc, cudaStream_t s, PcPairOut *out) {
  *out = PcPairOut{};
  if (m == 0) return THAPI_OK;
  uint64_t *k1 = static_cast<uint64_t *>(sc.get(m_all * sizeof(uint64_t)));
  uint64_t *k2 = static_cast<uint64_t *>(sc.get(m_all * sizeof(uint64_t)));
  uint32_t *v1 = static_cast<uint32_t *>(sc.get(m_all * sizeof(uint32_t)));
  uint32_t *v2 = static_cast<uint32_t *>(sc.get(m_all * sizeof(uint32_t)));
  uint32_t *tid = static_cast<uint32_t *>(sc.get(m_all * sizeof(uint32_t)));
  PcRec *r2 = static_cast<PcRec *>(sc.get(m * sizeof(PcRec)));
  uint32_t *tk = static_cast<uint32_t *>(sc.get(m * sizeof(uint32_t)));
  uint64_t *word = static_cast<uint64_t *>(sc.get(4 * sizeof(uint64_t)));  // threads, level, flags
  constexpr uint32_t kTabCap = 1u << 16, kTabMask = kTabCap - 1;
  unsigned long long *tfp = static_cast<unsigned long long *>(sc.get(kTabCap * sizeof(uint64_t)));
  uint32_t *tkey = static_cast<uint32_t *>(sc.get(3ull * kTabCap * sizeof(uint32_t)));
  uint64_t *used = static_cast<uint64_t *>(sc.get(kTabCap * sizeof(uint64_t)));
  if (sc.failed) return THAPI_E_NOMEM;
  unsigned long long *flags = reinterpret_cast<unsigned long long *>(word + 2);
  const int tsb = std::max(1, std::min(64, ts_bits));
  uint64_t h[4] = {0, 0, 0, 0};
  if (cudaMemsetAsync(word, 0, 4 * sizeof(uint64_t), s) != cudaSuccess ||
      cudaMemsetAsync(tfp, 0, kTabCap * sizeof(uint64_t), s) != cudaSuccess)
    return THAPI_E_CUDA;
  // 1. thread numbers from a table of (host, vpid, vtid), then one stable sort
  //    by (thread number, ts) of the position-ordered records
  k_thr_insert<<<blocks(m_all), kT, 0, s>>>(rec, m_all, tfp, tkey, kTabMask,
                                            reinterpret_cast<unsigned long long *>(word + 3), flags);
  k_thr_used<<<blocks(kTabCap), kT, 0, s>>>(tfp, kTabCap, used);
  scan_exclusive_u64(used, kTabCap, word, sc, s);
  count_launches(2);
  if (sc.failed) return THAPI_E_NOMEM;
  if (!read_words(word, h, 3, s)) return THAPI_E_CUDA;
  uint64_t T = h[0];
  int tb = 1;
  while ((1ull << tb) <= T) ++tb;
  bool ordered = false;
  if (!(h[2] & 1) && tb + tsb <= 64) {
    out->keys = static_cast<uint32_t *>(sc.get(3 * T * sizeof(uint32_t)));
    if (sc.failed) return THAPI_E_NOMEM;
    k_thr_keys<<<blocks(kTabCap), kT, 0, s>>>(tfp, tkey, used, kTabCap, out->keys);
    k_pc_tkey<<<blocks(m_all), kT, 0, s>>>(rec, m_all, tfp, tkey, used, kTabMask, tsb, t_min, T, k1, v1, tid, flags);
    count_launches(2);
    bool alt = false;
    radix_sort_pairs(k1, v1, k2, v2, m_all, tb + tsb, &alt, sc, s);
    if (sc.failed) return THAPI_E_NOMEM;
    if (!read_words(word + 2, h + 2, 1, s)) return THAPI_E_CUDA;
    if (!(h[2] & 2)) {  // no fingerprint clash: the first m sorted positions are the records
      k_pc_gather_t<<<blocks(m), kT, 0, s>>>(rec, alt ? v2 : v1, tid, m, r2, tk);
      count_launches(1);
      ordered = true;
    }
  }
  if (!ordered) {  // fallback: stable sorts by ts, (vpid, vtid), host over position order
    uint32_t *perm = nullptr;
    const int bits[4] = {0, tsb, 64, 33};
    for (int which = 1; which < 4; ++which) {
      uint32_t *vin = perm ? perm : v1;
      uint32_t *valt = vin == v1 ? v2 : v1;
      k_pc_key<<<blocks(m_all), kT, 0, s>>>(rec, perm, m_all, which, t_min, k1, v1);
      count_launches(1);
      bool alt = false;
      radix_sort_pairs(k1, vin, k2, valt, m_all, bits[which], &alt, sc, s);
      if (sc.failed) return THAPI_E_NOMEM;
      perm = alt ? valt : vin;
    }
    k_pc_gather<<<blocks(m), kT, 0, s>>>(rec, perm, m, r2);
    uint64_t *head = k2;  // free again: heads, then their exclusive scan
    k_pc_heads<<<blocks(m), kT, 0, s>>>(r2, m, head);
    scan_exclusive_u64(head, m, word, sc, s);
    count_launches(2);
    if (sc.failed) return THAPI_E_NOMEM;
    if (!read_words(word, h, 1, s)) return THAPI_E_CUDA;
    T = h[0];
    if (T >= (1ull << 31)) return THAPI_E_UNSUPPORTED;  // thread numbers fit 31 bits of the scan words
    tb = 1;
    while ((1ull << tb) <= T) ++tb;
    out->keys = static_cast<uint32_t *>(sc.get(3 * T * sizeof(uint32_t)));
    if (sc.failed) return THAPI_E_NOMEM;
    k_pc_keys<<<blocks(m), kT, 0, s>>>(r2, head, m, out->keys, tid);
    k_pc_renumber<<<blocks(m), kT, 0, s>>>(r2, tid, m, tk);
    count_launches(2);
  }
  out->threads = T;
  out->cells = static_cast<Cell *>(sc.get(T * F * sizeof(Cell)));
  const uint64_t nb = (m + kSegThreads - 1) / kSegThreads;
  SegDM *agg = static_cast<SegDM *>(sc.get(nb * sizeof(SegDM)));
  if (sc.failed) return THAPI_E_NOMEM;
  launch_tally_init(out->cells, T * F, s);
  k_seg_local<<<(unsigned)nb, kSegThreads, 0, s>>>(tk, m, agg);
  k_seg_blocks<<<1, kSegThreads, 0, s>>>(agg, nb);
  if (cudaMemsetAsync(word + 1, 0, sizeof(uint64_t), s) != cudaSuccess) return THAPI_E_CUDA;
  k_seg_apply<<<(unsigned)nb, kSegThreads, 0, s>>>(tk, m, agg, k1, v1,
                                                   reinterpret_cast<unsigned long long *>(word + 1), diag);
  uint64_t lmax = 0;
  if (cudaMemcpyAsync(&lmax, word + 1, sizeof(lmax), cudaMemcpyDeviceToHost, s) != cudaSuccess ||
      cudaStreamSynchronize(s) != cudaSuccess)
    return THAPI_E_CUDA;
  // 3. (thread, level) order in tb + lb bits (T < 2^32 and levels < 2^32: at most 64), then neighbours pair
  int lb = 1;
  while (lb < 32 && (lmax >> lb)) ++lb;
  const uint64_t unmatched = T << lb;  // above every (thread, level) key
  k_pc_pack<<<blocks(m), kT, 0, s>>>(k1, m, lb, unmatched);
  bool alt = false;
  radix_sort_pairs(k1, v1, k2, v2, m, tb + lb, &alt, sc, s);
  if (sc.failed) return THAPI_E_NOMEM;
  const uint64_t *key = alt ? k2 : k1;
  const uint32_t *val = alt ? v2 : v1;
  const unsigned pgrid = (unsigned)std::min<uint64_t>(blocks(m), (uint64_t)std::max(num_sms, 1) * 8);
  k_pc_pair<<<pgrid, kT, 0, s>>>(r2, key, val, m, unmatched, lb, F, out->cells, slots, sum_nvalid, diag);
  count_launches(5);
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

// self.cu — self (exclusive) time of the calls of per-thread streams.
//
// The layering analysis of the paper (Sec. 4.3) separates the time a call
// spends itself from the time of the calls it makes (hipDeviceSynchronize
// over the zeEventHostSynchronize spin).  A call's self time is its duration
// less the durations of the calls paired directly inside it.  With self time
// on, the pairing kernels leave per interval slot the event positions of the
// entry and of its exit and the entry's depth (SelfSlot).  Over the valid host
// intervals of per-thread streams:
//  1. a warp per packet compacts them in slot order (stream, entry position),
//     finishing each depth with the depth carried into the packet;
//  2. a stable radix sort by (stream, level) keeps entry order inside each
//     (stream, level) run;
//  3. the direct parent of an interval at level L > 0 is the entry open at
//     depth L - 1 when its own entry is pushed: within the (stream, L - 1)
//     run, the last interval whose entry comes first, provided its exit comes
//     after.  That run ends where the interval's own run starts (no key lies
//     between them), and a table of run starts by key bounds the search.  When that open entry is no interval (mismatched or never
//     closed), the run's last earlier interval closed before it was pushed,
//     so the test fails and no call takes the child's duration;
//  4. self = duration - the children's durations (u64), tallied per
//     (group, function) like the inclusive tally.
// Per-CPU buffers are paired, and their self time taken, in percpu.cu.
#include <algorithm>

#include "internal.cuh"

namespace thapi {

namespace {

constexpr int kT = 256;

struct SelfRec {
  uint64_t entry_pos, exit_pos, dur;
  uint32_t cell;  // group * n_funcs + function; ~0u: not a host call of a per-thread stream
  uint32_t err;
};

unsigned blocks(uint64_t n) { return (unsigned)((n + kT - 1) / kT); }

// Same walk as the timeline compaction (a warp per packet, valid slots in
// order at out_base): key = stream << 32 | absolute level, or ~0 for slots
// that take no part (device intervals, per-CPU buffers).
__global__ void k_self_compact(const thapi_interval *slots, const SelfSlot *side, const uint64_t *evbase,
                               const uint32_t *nslot, const uint64_t *out_base, const uint32_t *A,
                               const uint32_t *order, const uint32_t *pk_stream, const uint32_t *stream_group,
                               uint32_t F, uint64_t n_order, SelfRec *rec, uint64_t *key, uint32_t *val,
                               unsigned long long *lmax) {
  const uint32_t lane = threadIdx.x & 31;
  const uint64_t wg = ((uint64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const uint64_t nw = ((uint64_t)gridDim.x * blockDim.x) >> 5;
  uint32_t mx = 0;
  // one chunk of slots and the next packet's fields are loaded ahead
  uint64_t n_sb = 0, n_ob = 0;
  uint32_t n_n = 0, n_a = 0, n_stream = 0;
  auto fields = [&](uint64_t i) {
    if (i >= n_order) return;
    n_sb = evbase[i];
    n_n = nslot[i];
    n_a = A[i];
    n_stream = pk_stream[order[i]];
    n_ob = out_base[i];
  };
  fields(wg);
  for (uint64_t i = wg; i < n_order; i += nw) {
    const uint64_t sb = n_sb;
    const uint32_t n = n_n;
    const uint32_t a = n_a;
    const uint32_t stream = n_stream;
    const uint32_t group = stream_group[stream];
    uint64_t ob = n_ob;
    fields(i + nw);
    thapi_interval nxt{};
    bool n_in = lane < n;
    if (n_in) nxt = slots[sb + lane];
    for (uint32_t c = 0; c < n; c += 32) {
      const bool in = n_in;
      thapi_interval iv = nxt;
      n_in = c + 32 + lane < n;
      if (n_in) nxt = slots[sb + c + 32 + lane];
      const bool valid = in && (iv.flags & kIvValid) != 0;
      const uint32_t bal = __ballot_sync(0xffffffffu, valid);
      if (valid) {
        const uint64_t at = ob + __popc(bal & ((1u << lane) - 1u));
        SelfRec r{0, 0, 0, ~0u, 0};
        uint64_t k = ~0ull;
        if (group != kPerCpuGroup && !(iv.flags & kIvDevice)) {
          const SelfSlot ss = side[sb + c + lane];
          uint32_t lvl;
          if (ss.level & kSelfAbs) {
            lvl = ss.level & ~kSelfAbs;
          } else {
            const uint32_t npend = iv.stream_id;  // pending exits before the entry in its packet
            lvl = (a > npend ? a - npend : 0u) + ss.level;
          }
          r.entry_pos = ss.entry_pos;
          r.exit_pos = ss.exit_pos;
          r.dur = iv.end_ns - iv.start_ns;
          r.cell = group * F + iv.func_id;
          r.err = (iv.flags & kIvErr) ? 1u : 0u;
          k = (uint64_t)stream << 32 | lvl;
          mx = max(mx, lvl);
        }
        rec[at] = r;
        key[at] = k;
        val[at] = (uint32_t)at;
      }
      ob += __popc(bal);
    }
  }
  mx = __reduce_max_sync(0xffffffffu, mx);
  if (lane == 0 && mx) atomicMax(lmax, (unsigned long long)mx);
}

// (stream << 32 | level) -> (stream << lb | level); the others above every key
__global__ void k_self_pack(uint64_t *key, uint64_t n, int lb, uint64_t sentinel) {
  const uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const uint64_t k = key[i];
  key[i] = k == ~0ull ? sentinel : (k >> 32) << lb | (k & 0xFFFFFFFFull);
}

__global__ void k_self_spos(const SelfRec *rec, const uint32_t *val, uint64_t n, uint64_t *spos) {
  const uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) spos[i] = rec[val[i]].entry_pos;
}

// First index in [lo, hi) whose (key, pos) is not below (tk, tp).
template <class P>
__device__ __forceinline__ uint64_t lower_kp(const uint64_t *key, const P *pos, uint64_t lo, uint64_t hi, uint64_t tk,
                                             uint64_t tp) {
  while (lo < hi) {
    const uint64_t mid = (lo + hi) >> 1;
    const uint64_t km = key[mid];
    if (km < tk || (km == tk && (uint64_t)pos[mid] < tp))
      lo = mid + 1;
    else
      hi = mid;
  }
  return lo;
}

// run_start[key] = the first sorted index of key's run (the table holds ~0
// for keys without a run).
__global__ void k_self_runs(const uint64_t *key, uint64_t n, uint64_t sentinel, uint64_t *run_start) {
  const uint64_t k = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= n) return;
  const uint64_t kk = key[k];
  if (kk < sentinel && (k == 0 || key[k - 1] != kk)) run_start[kk] = k;
}

// The parent of the interval at k, if it is one: the last entry of the
// (stream, level - 1) run before it in entry order, a binary search of that
// run's positions (neighbouring lanes share its first steps in cache).
__global__ void k_self_child_runs(const uint64_t *key, const uint32_t *val, const uint64_t *spos, const SelfRec *rec,
                                  const uint64_t *run_start, uint64_t n, int lb, uint64_t sentinel,
                                  unsigned long long *child) {
  const uint64_t k = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= n) return;
  const uint64_t kk = key[k];
  if (kk >= sentinel || (kk & ((1ull << lb) - 1)) == 0) return;
  uint64_t lo = run_start[kk - 1];
  if (lo == ~0ull) return;  // no interval one level up on this stream
  uint64_t hi = run_start[kk];
  const uint64_t p0 = lo, pos = spos[k];
  while (lo < hi) {  // the first of the run's positions not below pos
    const uint64_t mid = (lo + hi) >> 1;
    if (spos[mid] < pos)
      lo = mid + 1;
    else
      hi = mid;
  }
  if (lo == p0) return;
  const uint32_t pj = val[lo - 1];
  if (rec[pj].exit_pos > pos) atomicAdd(&child[pj], (unsigned long long)rec[val[k]].dur);
}

// Sorted order: the parent of the interval at k, if it is one, is the last
// entry of the (stream, level - 1) run before it in entry order (a binary
// search over the positions before k; neighbouring lanes share its first
// steps in cache).  For key spaces too large for a table of run starts.
__global__ void k_self_child(const uint64_t *key, const uint32_t *val, const uint64_t *spos, const SelfRec *rec,
                             uint64_t n, int lb, uint64_t sentinel, unsigned long long *child) {
  const uint64_t k = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= n) return;
  const uint64_t kk = key[k];
  if (kk >= sentinel || (kk & ((1ull << lb) - 1)) == 0) return;
  const uint64_t target = kk - 1, pos = spos[k];
  const uint64_t lo = lower_kp(key, spos, 0, k, target, pos);
  if (lo == 0) return;
  const uint64_t jp = lo - 1;
  if (key[jp] != target) return;
  const uint32_t pj = val[jp];
  if (rec[pj].exit_pos > pos) atomicAdd(&child[pj], (unsigned long long)rec[val[k]].dur);
}

__global__ void k_self_tally(const SelfRec *rec, const unsigned long long *child, uint64_t n, Cell *cells) {
  __shared__ CellPart scr[kT];
  const uint64_t i = spread(blockIdx.x, gridDim.x) * blockDim.x + threadIdx.x;
  SelfRec r{0, 0, 0, ~0u, 0};
  unsigned long long self = 0;
  if (i < n) {
    r = rec[i];
    self = r.dur - child[i];
  }
  warp_tally(cells, r.cell, r.cell != ~0u, self, r.err != 0, scr + (threadIdx.x & ~31u));
}

}  // namespace

int self_time(const SelfIn &in, Cell *cells, uint64_t *word, Scratch &sc, cudaStream_t s) {
  const uint64_t n = in.n_iv;
  if (n == 0) return THAPI_OK;
  SelfRec *rec = static_cast<SelfRec *>(sc.get(n * sizeof(SelfRec)));
  uint64_t *k1 = static_cast<uint64_t *>(sc.get(n * sizeof(uint64_t)));
  uint64_t *k2 = static_cast<uint64_t *>(sc.get(n * sizeof(uint64_t)));
  uint32_t *v1 = static_cast<uint32_t *>(sc.get(n * sizeof(uint32_t)));
  uint32_t *v2 = static_cast<uint32_t *>(sc.get(n * sizeof(uint32_t)));
  uint64_t *spos = static_cast<uint64_t *>(sc.get(n * sizeof(uint64_t)));
  unsigned long long *child = static_cast<unsigned long long *>(sc.get(n * sizeof(uint64_t)));
  if (sc.failed) return THAPI_E_NOMEM;
  if (cudaMemsetAsync(word, 0, sizeof(uint64_t), s) != cudaSuccess ||
      cudaMemsetAsync(child, 0, n * sizeof(uint64_t), s) != cudaSuccess)
    return THAPI_E_CUDA;
  const uint64_t warps = std::max<uint64_t>(1, std::min<uint64_t>(in.n_order, (uint64_t)in.num_sms * 64));
  k_self_compact<<<(unsigned)((warps * 32 + kT - 1) / kT), kT, 0, s>>>(
      in.slots, in.side, in.evbase, in.nslot, in.obase, in.A, in.order, in.pk_stream, in.stream_group, in.n_funcs,
      in.n_order, rec, k1, v1, reinterpret_cast<unsigned long long *>(word));
  uint64_t lmax = 0;
  if (cudaMemcpyAsync(&lmax, word, sizeof(lmax), cudaMemcpyDeviceToHost, s) != cudaSuccess ||
      cudaStreamSynchronize(s) != cudaSuccess)
    return THAPI_E_CUDA;
  int lb = 1, sb = 1;
  while (lb < 32 && (lmax >> lb)) ++lb;
  while ((1ull << sb) <= (uint64_t)in.n_streams) ++sb;  // the sentinel n_streams must fit
  const uint64_t sentinel = (uint64_t)in.n_streams << lb;
  k_self_pack<<<blocks(n), kT, 0, s>>>(k1, n, lb, sentinel);
  bool alt = false;
  radix_sort_pairs(k1, v1, k2, v2, n, sb + lb, &alt, sc, s);
  if (sc.failed) return THAPI_E_NOMEM;
  const uint64_t *key = alt ? k2 : k1;
  const uint32_t *val = alt ? v2 : v1;
  k_self_spos<<<blocks(n), kT, 0, s>>>(rec, val, n, spos);
  // a table of run starts when the keys (stream, level) are few next to the intervals
  uint64_t *run_start = sentinel <= std::max<uint64_t>(n, 1u << 20) ? static_cast<uint64_t *>(
                                                                          sc.get(sentinel * sizeof(uint64_t)))
                                                                    : nullptr;
  if (run_start) {
    if (cudaMemsetAsync(run_start, 0xFF, sentinel * sizeof(uint64_t), s) != cudaSuccess) return THAPI_E_CUDA;
    k_self_runs<<<blocks(n), kT, 0, s>>>(key, n, sentinel, run_start);
    k_self_child_runs<<<blocks(n), kT, 0, s>>>(key, val, spos, rec, run_start, n, lb, sentinel, child);
    count_launches(1);
  } else {
    sc.failed = 0;  // the table was optional
    k_self_child<<<blocks(n), kT, 0, s>>>(key, val, spos, rec, n, lb, sentinel, child);
  }
  k_self_tally<<<blocks(n), kT, 0, s>>>(rec, child, n, cells);
  count_launches(5);
  return cudaGetLastError() == cudaSuccess ? THAPI_OK : THAPI_E_CUDA;
}

}  // namespace thapi

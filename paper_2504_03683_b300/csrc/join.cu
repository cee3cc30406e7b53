// join.cu — device-activity pairing.
//
// The paper's GPU profiling code records when each command a host API call
// submits starts and ends on the device (Sec. 3.3), and the timeline shows
// those device rows beside the host calls (Sec. 3.6).  In a trace these are
// DEV_BEGIN / DEV_END events carrying a 64-bit command id, and the host
// call's ENTRY carries the same id.  Per command id c, with B, E and H the
// numbers of its DEV_BEGIN, DEV_END and host ENTRY events: c is a device pair
// when B = E = 1 and its end is not before its begin; a pair with H = 1
// becomes a device interval [begin, end] on the begin's stream, labelled with
// the host call's function; H = 0 (unjoined) and H > 1 (ambiguous) pairs are
// counted and dropped.
//
// The analysis kernels write one record per event carrying a command id.
// Here every record claims (or finds) the table entry of its id by linear
// probing from a hash of the id and counts itself there (the first DEV_END
// and the first host record also leave their timestamp / function); then one
// pass over the DEV_BEGIN records reads each command's entry and writes the
// device interval into the begin's slot, tallies it on the device-stream
// group's cells and counts it in its packet's valid intervals.  Counts are
// order-independent and the data left by "first" records is only used when
// that record is the only one of its kind, so the result does not depend on
// the order the records were written in.
#include "internal.cuh"

namespace thapi {

namespace {

constexpr int kThreads = 256;

// Finaliser of SplitMix64 (Steele, Lea & Flood, "Fast splittable
// pseudorandom number generators", OOPSLA 2014): a bijective mix of the id.
__device__ __forceinline__ uint64_t mix_id(uint64_t z) {
  z = (z ^ (z >> 30)) * 0xbf58476d1ce4e5b9ull;
  z = (z ^ (z >> 27)) * 0x94d049bb133111ebull;
  return z ^ (z >> 31);
}

// Index of the entry holding `key` (claimed if absent), or ~0 after
// `limit` probes without finding it or a free entry.  The zero id lives in
// the extra entry past the table (0 marks a free entry).
__device__ __forceinline__ uint64_t find_or_claim(CmdEntry *tab, uint64_t mask, uint64_t key, uint64_t limit) {
  if (key == 0) return mask + 1;
  uint64_t i = mix_id(key) & mask;
  for (uint64_t n = 0; n < limit; ++n) {
    unsigned long long cur = __ldcg(&tab[i].key);
    if (cur == key) return i;
    if (cur == 0) {
      cur = atomicCAS(&tab[i].key, 0ull, (unsigned long long)key);
      if (cur == 0 || cur == key) return i;
    }
    i = (i + 1) & mask;
  }
  return ~0ull;
}

// Index of the entry holding `key` (present), or ~0.
__device__ __forceinline__ uint64_t find(const CmdEntry *tab, uint64_t mask, uint64_t key, uint64_t limit) {
  if (key == 0) return mask + 1;
  uint64_t i = mix_id(key) & mask;
  for (uint64_t n = 0; n < limit; ++n) {
    const unsigned long long cur = __ldcg(&tab[i].key);
    if (cur == key) return i;
    if (cur == 0) return ~0ull;
    i = (i + 1) & mask;
  }
  return ~0ull;
}

__global__ void __launch_bounds__(kThreads) k_cmd_insert(JoinParams p) {
  const uint64_t n = p.nb + p.ne + p.nh;
  const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
  bool over = false;
  for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride) {
    uint64_t key;
    int kind;
    if (i < p.nb) {
      key = p.b[i].cmd;
      kind = 0;
    } else if (i < p.nb + p.ne) {
      key = p.e[i - p.nb].cmd;
      kind = 1;
    } else {
      key = p.h[i - p.nb - p.ne].cmd;
      kind = 2;
    }
    const uint64_t at = find_or_claim(p.tab, p.mask, key, p.probe_limit);
    if (at == ~0ull) {
      over = true;
      continue;
    }
    CmdEntry &e = p.tab[at];
    if (kind == 0) {
      atomicAdd(&e.nb, 1u);
    } else if (kind == 1) {
      if (atomicAdd(&e.ne, 1u) == 0u) e.te = p.e[i - p.nb].ts;
    } else {
      if (atomicAdd(&e.nh, 1u) == 0u) e.func = p.h[i - p.nb - p.ne].func;
    }
  }
  if (__any_sync(0xffffffffu, over) && (threadIdx.x & 31) == 0) atomicExch(&p.out[5], 1ull);
}

__global__ void __launch_bounds__(kThreads) k_cmd_emit(JoinParams p) {
  const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
  unsigned long long pairs = 0, joined = 0, unjoined = 0, ambiguous = 0, nh_pairs = 0;
  for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < p.nb; i += stride) {
    const CmdBegin r = p.b[i];
    const uint64_t at = find(p.tab, p.mask, r.cmd, p.mask + 1);
    if (at == ~0ull) continue;  // not reached: every begin record has its entry
    const CmdEntry e = p.tab[at];
    if (e.nb != 1u || e.ne != 1u || e.te < r.ts) continue;
    ++pairs;
    nh_pairs += e.nh;
    if (e.nh == 0u) {
      ++unjoined;
    } else if (e.nh > 1u) {
      ++ambiguous;
    } else {
      ++joined;
      const uint64_t dur = e.te - r.ts;
      if (p.slots) {
        unsigned long long *q = reinterpret_cast<unsigned long long *>(p.slots + r.slot);
        q[0] = r.ts;
        q[1] = e.te;
        // no pending-exit count (its level stays 0), the host call's function, level 0, valid device interval
        q[2] = 0xFFFFFFFFull | ((unsigned long long)(e.func & 0xFFFFu) << 32) |
               ((unsigned long long)(kIvValid | kIvDevice) << 56);
        atomicAdd(&p.sum_nvalid[r.pos], 1u);
      }
      Cell &c = p.dcells[(uint64_t)r.group * p.n_funcs + e.func];
      atomicAdd(&c.count, 1ull);
      atomicAdd(&c.total, (unsigned long long)dur);
      atomicMin(&c.mn, (unsigned long long)dur);
      atomicMax(&c.mx, (unsigned long long)dur);
    }
  }
  for (int o = 16; o > 0; o >>= 1) {
    pairs += __shfl_down_sync(0xffffffffu, pairs, o);
    joined += __shfl_down_sync(0xffffffffu, joined, o);
    unjoined += __shfl_down_sync(0xffffffffu, unjoined, o);
    ambiguous += __shfl_down_sync(0xffffffffu, ambiguous, o);
    nh_pairs += __shfl_down_sync(0xffffffffu, nh_pairs, o);
  }
  if ((threadIdx.x & 31) == 0) {
    if (pairs) atomicAdd(&p.out[0], pairs);
    if (joined) atomicAdd(&p.out[1], joined);
    if (unjoined) atomicAdd(&p.out[2], unjoined);
    if (ambiguous) atomicAdd(&p.out[3], ambiguous);
    if (nh_pairs) atomicAdd(&p.out[4], nh_pairs);
  }
}

unsigned grid_for(uint64_t n, int num_sms) {
  const uint64_t want = (n + kThreads - 1) / kThreads;
  const uint64_t most = (uint64_t)num_sms * 8;
  return (unsigned)(want < most ? (want ? want : 1) : most);
}

}  // namespace

void launch_cmd_insert(const JoinParams &jp, int num_sms, cudaStream_t s) {
  const uint64_t n = jp.nb + jp.ne + jp.nh;
  if (!n) return;
  k_cmd_insert<<<grid_for(n, num_sms), kThreads, 0, s>>>(jp);
  count_launches(1);
}

void launch_cmd_emit(const JoinParams &jp, int num_sms, cudaStream_t s) {
  if (!jp.nb) return;
  k_cmd_emit<<<grid_for(jp.nb, num_sms), kThreads, 0, s>>>(jp);
  count_launches(1);
}

}  // namespace thapi

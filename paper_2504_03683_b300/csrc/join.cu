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
// probing from a hash of the id and adds itself there: counts per kind, and
// the sums of the DEV_END timestamps and of the host functions, which are
// the timestamp and the function whenever the count is one (the only case
// that uses them).  Then one pass over the DEV_BEGIN records reads each
// command's entry and writes the device interval into the begin's slot,
// tallies it on the device-stream group's cells and counts it in its
// packet's valid intervals.  Everything stored is a sum, so the result does
// not depend on the order the records were written in.
#include <algorithm>

#include "internal.cuh"

namespace thapi {

namespace {

constexpr int kThreads = 256;


// Index of the entry holding `key` (claimed if absent), or ~0 after
// `limit` probes without finding it or a free entry.  Each probe is one
// compare-and-swap of 0 -> key.  The zero id lives in the extra entry past
// the table (0 marks a free entry).
__device__ __forceinline__ uint64_t find_or_claim(CmdEntry *tab, uint64_t mask, uint64_t key, uint64_t limit) {
  if (key == 0) return mask + 1;
  uint64_t i = cmd_hash(key) & mask;
  for (uint64_t n = 0; n < limit; ++n) {
    const unsigned long long cur = atomicCAS(&tab[i].key, 0ull, (unsigned long long)key);
    if (cur == 0 || cur == key) return i;
    i = (i + 1) & mask;
  }
  return ~0ull;
}

// Index of the entry holding `key` (present), or ~0.
__device__ __forceinline__ uint64_t find(const CmdEntry *tab, uint64_t mask, uint64_t key, uint64_t limit) {
  if (key == 0) return mask + 1;
  uint64_t i = cmd_hash(key) & mask;
  for (uint64_t n = 0; n < limit; ++n) {
    const unsigned long long cur = __ldcg(&tab[i].key);
    if (cur == key) return i;
    if (cur == 0) return ~0ull;
    i = (i + 1) & mask;
  }
  return ~0ull;
}

// Every record finds or claims its id's entry and adds itself with
// fire-and-forget reductions: counts, the end timestamp, the host function
// (sums, which are the value itself when the count is one).
__global__ void __launch_bounds__(kThreads) k_cmd_insert(JoinParams p) {
  const uint64_t n = p.nb + p.ne + p.nh;
  const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
  bool over = false;
  for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride) {
    uint64_t key, val = 0;
    int kind;
    if (i < p.nb) {
      key = p.b[i].cmd;
      kind = 0;
    } else if (i < p.nb + p.ne) {
      const CmdEnd r = p.e[i - p.nb];
      key = r.cmd;
      val = r.ts;
      kind = 1;
    } else {
      const CmdHost r = p.h[i - p.nb - p.ne];
      key = r.cmd;
      val = r.func;
      kind = 2;
    }
    const uint64_t at = find_or_claim(p.tab, p.mask, key, p.probe_limit);
    if (at == ~0ull) {
      over = true;
      continue;
    }
    CmdEntry &e = p.tab[at];
    if (kind == 0) {
      atomicAdd(&e.nbe, 1ull);
    } else if (kind == 1) {
      atomicAdd(&e.nbe, 1ull << 32);
      atomicAdd(&e.te, (unsigned long long)val);
    } else {
      atomicAdd(&e.nhf, 1ull | ((unsigned long long)val << 32));
    }
  }
  if (__any_sync(0xffffffffu, over) && (threadIdx.x & 31) == 0) atomicExch(&p.out[5], 1ull);
}

// One thread per DEV_BEGIN record (warp-aligned so a warp's lanes agree on
// the loop): the command's entry decides pair / join; a joined pair writes
// its interval into the begin's slot and is tallied.  The begins of one
// packet are consecutive records, so their packet's interval count is raised
// once per packet and warp.
__global__ void __launch_bounds__(kThreads) k_cmd_emit(JoinParams p) {
  const uint32_t lane = threadIdx.x & 31;
  const uint64_t wstride = (uint64_t)gridDim.x * blockDim.x;
  unsigned long long pairs = 0, joined = 0, unjoined = 0, ambiguous = 0, nh_pairs = 0;
  for (uint64_t i0 = ((uint64_t)blockIdx.x * blockDim.x + threadIdx.x) & ~31ull; i0 < p.nb; i0 += wstride) {
    const uint64_t i = i0 + lane;
    bool ok = false;
    uint32_t pos = 0xFFFFFFFFu;
    if (i < p.nb) {
      const CmdBegin r = p.b[i];
      const uint64_t at = find(p.tab, p.mask, r.cmd, p.mask + 1);
      if (at != ~0ull) {  // always: every begin record has its entry
        const CmdEntry e = p.tab[at];
        const uint32_t nb = (uint32_t)e.nbe, ne = (uint32_t)(e.nbe >> 32), nh = (uint32_t)e.nhf;
        if (nb == 1u && ne == 1u && e.te >= r.ts) {
          ++pairs;
          nh_pairs += nh;
          if (nh == 0u) {
            ++unjoined;
          } else if (nh > 1u) {
            ++ambiguous;
          } else {
            ++joined;
            ok = true;
            pos = r.pos;
            const uint32_t func = (uint32_t)(e.nhf >> 32);
            const uint64_t dur = e.te - r.ts;
            if (p.slots) {
              unsigned long long *q = reinterpret_cast<unsigned long long *>(p.slots + r.slot);
              q[0] = r.ts;
              q[1] = e.te;
              // no pending-exit count (its level stays 0), the host call's function, level 0, valid device interval
              q[2] = 0xFFFFFFFFull | ((unsigned long long)(func & 0xFFFFu) << 32) |
                     ((unsigned long long)(kIvValid | kIvDevice) << 56);
            }
            Cell &c = p.dcells[(uint64_t)r.group * p.n_funcs + func];
            atomicAdd(&c.count, 1ull);
            atomicAdd(&c.total, (unsigned long long)dur);
            atomicMin(&c.mn, (unsigned long long)dur);
            atomicMax(&c.mx, (unsigned long long)dur);
          }
        }
      }
    }
    if (p.slots) {
      const uint32_t peers = __match_any_sync(0xffffffffu, pos);
      if (ok && lane == (uint32_t)(__ffs(peers) - 1)) atomicAdd(&p.sum_nvalid[pos], (uint32_t)__popc(peers));
    }
  }
  for (int o = 16; o > 0; o >>= 1) {
    pairs += __shfl_down_sync(0xffffffffu, pairs, o);
    joined += __shfl_down_sync(0xffffffffu, joined, o);
    unjoined += __shfl_down_sync(0xffffffffu, unjoined, o);
    ambiguous += __shfl_down_sync(0xffffffffu, ambiguous, o);
    nh_pairs += __shfl_down_sync(0xffffffffu, nh_pairs, o);
  }
  if (lane == 0) {
    if (pairs) atomicAdd(&p.out[0], pairs);
    if (joined) atomicAdd(&p.out[1], joined);
    if (unjoined) atomicAdd(&p.out[2], unjoined);
    if (ambiguous) atomicAdd(&p.out[3], ambiguous);
    if (nh_pairs) atomicAdd(&p.out[4], nh_pairs);
  }
}

// ------------------------------------------------------ partitioned join
// The records are grouped by the top bits of the id's hash (the analysis
// counted them per partition), so that all records of one id land in one
// partition; a CTA then takes a partition at a time with its table in shared
// memory: keys and a 64-bit state per entry,
//   bits 0-1 / 2-3 / 4-5: begin / end / host records (0, 1, 2 = more),
//   bits 8-27: the (first) end record's index, bits 28-47: the (first) host
//   record's index, both within the partition, bit 63: a device pair.
// The first index is only read when its count is one, so the order in which
// the records arrive does not matter.
constexpr uint32_t kTab = 4096;  // most entries of the shared-memory table (+1 for the zero id)
constexpr int kJoinThreads = 256;
constexpr unsigned long long kPairBit = 1ull << 63;
static_assert(kPartMaxRecords < kTab, "a partition's distinct ids always fit the table");

__global__ void k_part_prep(PartPlan pp, uint32_t P) {
  const uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
  uint32_t m = 0;
  if (i < 3ull * P) pp.base[i] = pp.hist[i];
  if (i < P) m = pp.hist[i] + pp.hist[P + i] + pp.hist[2ull * P + i];
  m = __reduce_max_sync(0xffffffffu, m);
  if ((threadIdx.x & 31) == 0 && m) atomicMax(pp.max_records, (unsigned long long)m);
}

__global__ void k_part_cursor(PartPlan pp, uint32_t P) {
  const uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < 3ull * P) pp.cursor[i] = pp.base[i];
}

__global__ void __launch_bounds__(kThreads) k_part_scatter(JoinParams p, PartPlan pp, uint32_t P) {
  const uint64_t n = p.nb + p.ne + p.nh;
  const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
  for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride) {
    if (i < p.nb) {
      const CmdBegin r = p.b[i];
      const uint64_t at = atomicAdd(&pp.cursor[cmd_part(r.cmd, pp.part_bits)], 1ull);
      if (at < p.nb) pp.pb[at] = r;
    } else if (i < p.nb + p.ne) {
      const CmdEnd r = p.e[i - p.nb];
      const uint64_t at = atomicAdd(&pp.cursor[P + cmd_part(r.cmd, pp.part_bits)], 1ull) - p.nb;
      if (at < p.ne) pp.pe[at] = r;
    } else {
      const CmdHost r = p.h[i - p.nb - p.ne];
      const uint64_t at = atomicAdd(&pp.cursor[2ull * P + cmd_part(r.cmd, pp.part_bits)], 1ull) - p.nb - p.ne;
      if (at < p.nh) pp.ph[at] = r;
    }
  }
}

// Entry of `key` in a partition table of `mask` + 1 entries (claimed if
// absent; the zero id has entry T, past the largest table).  ~0u if the table
// had no room (never with at most T / 2 records).
__device__ __forceinline__ uint32_t sm_claim(unsigned long long *skey, uint32_t mask, uint32_t T, uint64_t key) {
  if (key == 0) return T;
  uint32_t i = (uint32_t)cmd_hash(key) & mask;
  for (uint32_t n = 0; n <= mask; ++n) {
    const unsigned long long cur = atomicCAS(&skey[i], 0ull, (unsigned long long)key);
    if (cur == 0 || cur == key) return i;
    i = (i + 1) & mask;
  }
  return ~0u;
}

__device__ __forceinline__ uint32_t sm_find(const unsigned long long *skey, uint32_t mask, uint32_t T, uint64_t key) {
  if (key == 0) return T;
  uint32_t i = (uint32_t)cmd_hash(key) & mask;
  for (uint32_t n = 0; n <= mask; ++n) {
    const unsigned long long cur = skey[i];
    if (cur == key) return i;
    if (cur == 0) return ~0u;
    i = (i + 1) & mask;
  }
  return ~0u;
}

// Counts one record of `kind` (0 begin, 1 end, 2 host) in the entry's state;
// the first end / host record also leaves its index.
__device__ __forceinline__ void sm_count(unsigned long long *st, int kind, uint32_t idx) {
  unsigned long long old = *st;
  for (int it = 0; it < 4 * kJoinThreads; ++it) {  // one contender wins each round
    const uint32_t c = (uint32_t)(old >> (2 * kind)) & 3u;
    if (c >= 2) return;  // saturated
    unsigned long long nw = old + (1ull << (2 * kind));
    if (c == 0 && kind == 1) nw |= (unsigned long long)idx << 8;
    if (c == 0 && kind == 2) nw |= (unsigned long long)idx << 28;
    const unsigned long long cur = atomicCAS(st, old, nw);
    if (cur == old) return;
    old = cur;
  }
}

// T: table entries, a power of two at least twice the largest partition's
// records (so that a CTA's shared memory, and with it the CTAs per SM,
// follows the partition size).
__global__ void __launch_bounds__(kJoinThreads) k_part_join(JoinParams p, PartPlan pp, uint32_t P, uint32_t T) {
  extern __shared__ unsigned long long jsm[];
  unsigned long long *skey = jsm, *sst = jsm + T + 1;
  __shared__ unsigned long long red[kJoinThreads / 32][5];
  const uint32_t tid = threadIdx.x;
  unsigned long long pairs = 0, joined = 0, unjoined = 0, ambiguous = 0, h_in_pairs = 0;
  bool over = false;
  for (uint32_t part = blockIdx.x; part < P; part += gridDim.x) {
    const uint64_t b0 = pp.base[part], b1 = pp.base[part + 1];
    const uint64_t e0 = pp.base[P + part] - p.nb, e1 = pp.base[P + part + 1] - p.nb;
    const uint64_t h0 = pp.base[2ull * P + part] - p.nb - p.ne, h1 = pp.base[2ull * P + part + 1] - p.nb - p.ne;
    const uint32_t n_rec = (uint32_t)((b1 - b0) + (e1 - e0) + (h1 - h0));
    uint32_t tcap = 64;
    while (tcap < 2 * n_rec && tcap < T) tcap <<= 1;
    const uint32_t mask = tcap - 1;
    for (uint32_t k = tid; k < tcap; k += kJoinThreads) skey[k] = sst[k] = 0;
    if (tid == 0) skey[T] = sst[T] = 0;
    __syncthreads();
    // count every record of the partition
    for (uint64_t i = e0 + tid; i < e1; i += kJoinThreads) {
      const uint32_t at = sm_claim(skey, mask, T, pp.pe[i].cmd);
      if (at == ~0u) { over = true; continue; }
      sm_count(&sst[at], 1, (uint32_t)(i - e0));
    }
    for (uint64_t i = h0 + tid; i < h1; i += kJoinThreads) {
      const uint32_t at = sm_claim(skey, mask, T, pp.ph[i].cmd);
      if (at == ~0u) { over = true; continue; }
      sm_count(&sst[at], 2, (uint32_t)(i - h0));
    }
    for (uint64_t i = b0 + tid; i < b1; i += kJoinThreads) {
      const uint32_t at = sm_claim(skey, mask, T, pp.pb[i].cmd);
      if (at == ~0u) { over = true; continue; }
      sm_count(&sst[at], 0, 0);
    }
    __syncthreads();
    // every begin: pair? joined? then its interval, tally and packet count
    for (uint64_t i = b0 + tid; i < b1; i += kJoinThreads) {
      const CmdBegin r = pp.pb[i];
      const uint32_t at = sm_find(skey, mask, T, r.cmd);
      if (at == ~0u) continue;  // not reached: counted above
      const unsigned long long st = sst[at];
      if ((st & 3u) != 1u || ((st >> 2) & 3u) != 1u) continue;
      const uint64_t te = pp.pe[e0 + ((st >> 8) & 0xFFFFFu)].ts;
      if (te < r.ts) continue;
      atomicOr(&sst[at], kPairBit);
      ++pairs;
      const uint32_t nh = (uint32_t)(st >> 4) & 3u;
      if (nh == 0u) {
        ++unjoined;
      } else if (nh > 1u) {
        ++ambiguous;
      } else {
        ++joined;
        const uint32_t func = pp.ph[h0 + ((st >> 28) & 0xFFFFFu)].func;
        if (p.slots) {
          unsigned long long *q = reinterpret_cast<unsigned long long *>(p.slots + r.slot);
          q[0] = r.ts;
          q[1] = te;
          q[2] = 0xFFFFFFFFull | ((unsigned long long)(func & 0xFFFFu) << 32) |
                 ((unsigned long long)(kIvValid | kIvDevice) << 56);
          atomicAdd(&p.sum_nvalid[r.pos], 1u);
        }
        const uint64_t dur = te - r.ts;
        Cell &c = p.dcells[(uint64_t)r.group * p.n_funcs + func];
        atomicAdd(&c.count, 1ull);
        atomicAdd(&c.total, (unsigned long long)dur);
        atomicMin(&c.mn, (unsigned long long)dur);
        atomicMax(&c.mx, (unsigned long long)dur);
      }
    }
    __syncthreads();
    // host records whose id is a device pair
    for (uint64_t i = h0 + tid; i < h1; i += kJoinThreads) {
      const uint32_t at = sm_find(skey, mask, T, pp.ph[i].cmd);
      if (at != ~0u && (sst[at] & kPairBit)) ++h_in_pairs;
    }
    __syncthreads();  // the table is cleared for the next partition
  }
  // block totals, five atomics per CTA
  const uint32_t lane = tid & 31, warp = tid >> 5;
  unsigned long long v[5] = {pairs, joined, unjoined, ambiguous, h_in_pairs};
#pragma unroll
  for (int k = 0; k < 5; ++k) {
    for (int o = 16; o > 0; o >>= 1) v[k] += __shfl_down_sync(0xffffffffu, v[k], o);
    if (lane == 0) red[warp][k] = v[k];
  }
  __syncthreads();
  if (tid < 5) {
    unsigned long long t = 0;
    for (int w = 0; w < kJoinThreads / 32; ++w) t += red[w][tid];
    if (t) atomicAdd(&p.out[tid], t);
  }
  if (__syncthreads_or(over) && tid == 0) atomicExch(&p.out[5], 1ull);
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

void launch_part_prep(const PartPlan &pp, cudaStream_t s) {
  const uint32_t P = 1u << pp.part_bits;
  k_part_prep<<<(unsigned)((3ull * P + 255) / 256), 256, 0, s>>>(pp, P);
  count_launches(1);
}

void launch_part_scatter(const JoinParams &jp, const PartPlan &pp, int num_sms, cudaStream_t s) {
  const uint32_t P = 1u << pp.part_bits;
  k_part_cursor<<<(unsigned)((3ull * P + 255) / 256), 256, 0, s>>>(pp, P);
  count_launches(1);
  const uint64_t n = jp.nb + jp.ne + jp.nh;
  if (!n) return;
  k_part_scatter<<<grid_for(n, num_sms), kThreads, 0, s>>>(jp, pp, P);
  count_launches(1);
}

void launch_part_join(const JoinParams &jp, const PartPlan &pp, uint64_t max_records, cudaStream_t s) {
  const uint32_t P = 1u << pp.part_bits;
  uint32_t T = 64;
  while (T < 2 * max_records && T < kTab) T <<= 1;
  const size_t smem = 2ull * (T + 1) * sizeof(unsigned long long);
  int dev = 0, sms = 0, per_sm = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  cudaFuncSetAttribute(k_part_join, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_part_join, kJoinThreads, smem);
  const uint64_t grid = std::min<uint64_t>(P, (uint64_t)std::max(1, sms) * std::max(1, per_sm));
  k_part_join<<<(unsigned)grid, kJoinThreads, smem, s>>>(jp, pp, P, T);
  count_launches(1);
}

}  // namespace thapi

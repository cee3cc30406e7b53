// analyze_warp.cu — decode + in-packet pairing + tally, one warp per packet.
//
// A CTA holds NW independent warps that share the class table.  The CTA
// takes a contiguous run of the stream-ordered packet list and its warps take
// the run's packets in turn.  Each warp stages its packet with a TMA bulk copy
// (mbarrier completion) and then works on it alone:
//
//  1. boundaries: every lane walks a 32*(BW-1)+1-word segment speculatively from the
//     segment start, marking the offsets it visits; the warp stitches the
//     segments (a lane assumes its entry offset is its predecessor's
//     speculative exit; the first lane whose exit breaks that assumption hands
//     its successor the right entry, one ballot round per such lane).  The
//     marks are then exactly the event starts of the chain from offset 0, and
//     they are compacted into the packet's event offsets, in order.
//  2. validation, 32 events at a time (one per lane): format checks and a
//     warp scan of the depth monoid (sum, min-prefix), carried across the
//     batches, giving the packet's depth range;
//  3. pairing, 32 events at a time: warp scans of the timestamp monoid
//     (has_abs, value), the depth monoid and the entry count give each
//     event's timestamp, depths before/after and entry rank.  An exit at
//     depth h after it closes the latest earlier entry at height h: in its
//     batch (the highest earlier lane of the same height, from match-any), or
//     else the packet's latest entry at h kept in a per-height table (written
//     by the last entry of each height in each batch).  An exit whose height is
//     below every depth reached so far pops an entry of an earlier packet: it
//     is a pending exit.  The table rows left at the end, heights from the
//     minimum depth up to the final depth, are the packet's open entries.
//     Pending exits and open entries form the packet's frontier, resolved
//     across packets by frontier.cu.
// Every lane runs the same instructions on its event; pairs are tallied with
// fire-and-forget global reductions on the (group, function) cells and their
// interval slots are written at once.  Packets with more than kEvMax events or
// a depth range over kHeights go to the CTA kernel of analyze.cu (appended to
// the fallback list).
#include <algorithm>

#include "device_util.cuh"
#include "internal.cuh"

namespace thapi {

namespace {
using namespace dev;

constexpr uint32_t kEvMax = 1024;       // events of one packet the warp path takes
constexpr uint32_t kHeights = 32;       // per-height table rows (depth range of a packet)
constexpr uint32_t kClsMax = 4096;      // class rows held in shared memory
constexpr uint32_t kChunk = 2048;       // frontier items grabbed per global atomic
constexpr uint32_t kMaxWarps = 16;      // warps per CTA
// Per-lane pairing (the fast path): each lane's pending exits and open
// entries, 8 bytes each, in the warp's table and offset area (2,560 bytes =
// 32 lanes x kLaneSlots, lane-interleaved so that lanes at any slot hit
// distinct banks)
constexpr uint32_t kLaneSlots = (kHeights * 16u + kEvMax * 2u) / (32u * 8u);
constexpr uint32_t kFull = 0xffffffffu;

__host__ __device__ inline uint32_t rup(uint32_t v, uint32_t a) { return (v + a - 1u) / a * a; }

struct WLayout {
  uint32_t off_off, off_tab, off_bar, warp_bytes;  // within one warp's block
  uint32_t off_ctab, off_cfn, total;               // CTA-wide
};

__host__ __device__ inline WLayout wlayout(uint32_t P, uint32_t NW, uint32_t NC) {
  WLayout L;
  // 16-byte granules (what the bulk copies and the mbarrier need): with 16 KB
  // packets 12 warps and up to ~700 classes fit one SM's shared memory
  uint32_t o = rup(P + 48u, 16u);  // packet (header + content) and a zeroed tail
  L.off_tab = o;
  o += kHeights * 16u;  // per-height table: entry timestamp, entry metadata
  L.off_off = o;
  o += kEvMax * 2u;
  L.off_bar = o;
  o += 16u;
  L.warp_bytes = rup(o, 16u);
  o = L.warp_bytes * NW;
  L.off_ctab = o;
  o += rup((NC + 1u) * 4u, 16u);
  L.off_cfn = o;
  o += rup(NC * 2u, 16u);
  L.total = rup(o, 128u);
  return L;
}

// Shared-memory class row: fixed words (14 bits) | kind << 14 (3) | (result word + 1) << 17 (14)
//   | carries a command id (device pairing on) << 31.
__device__ __forceinline__ uint32_t row_fixedw(uint32_t r) { return r & 0x3FFFu; }
__device__ __forceinline__ uint32_t row_kind(uint32_t r) { return (r >> 14) & 7u; }
__device__ __forceinline__ int32_t row_resw(uint32_t r) { return (int32_t)((r >> 17) & 0x3FFFu) - 1; }

// Event chain step from word offset o.  An offset whose class id is out of
// range is no event start: the chain moves to the next offset whose class id
// is in range, at most four words on (the offsets a one-word-at-a-time walk
// would pass through and land on, so every in-range offset it reaches is the
// same).  Reads up to C[o + 4].  HW: header words (2; 4 in per-CPU buffers,
// whose events carry vpid / vtid).
template <uint32_t HW = 2>
__device__ __forceinline__ uint32_t step(const uint32_t *C, uint32_t o, const uint32_t *ctab, uint32_t NC) {
  const uint32_t w0 = C[o], w1 = C[o + 1], w2 = C[o + 2], w3 = C[o + 3], w4 = C[o + 4];
  const uint32_t c = w1 & 0xFFFFu;
  const bool ok = c < NC;
  const uint32_t r = ctab[ok ? c : NC];
  const uint32_t len = HW + ((w0 >> 26) & 2u) + row_fixedw(r) + (((w1 >> 16) + 3u) >> 2);
  const uint32_t skip = (w2 & 0xFFFFu) < NC ? 1u : (w3 & 0xFFFFu) < NC ? 2u : (w4 & 0xFFFFu) < NC ? 3u : 4u;
  return o + (ok ? len : skip);
}

// Walks from o while o < b, marking the offsets visited; returns at the first
// offset already marked in `stop`.
template <int BW, uint32_t HW = 2>
__device__ __forceinline__ uint32_t walk_to(const uint32_t *C, uint32_t o, uint32_t a, uint32_t b, const Bits<BW> &stop,
                                            Bits<BW> &marks, const uint32_t *ctab, uint32_t NC) {
  while (o < b) {
    if (stop.test(o - a)) return o;
    marks.set(o - a);
    o = step<HW>(C, o, ctab, NC);
  }
  return o;
}

// Event starts of segment [a, b) when its chain enters at y: the speculative
// marks from where the chain meets them, plus the offsets walked before that.
// Returns the chain's exit offset.
template <int BW, uint32_t HW = 2>
__device__ __forceinline__ uint32_t resolve_seg(const uint32_t *C, uint32_t y, uint32_t a, uint32_t b,
                                                const Bits<BW> &spec, uint32_t spec_x, Bits<BW> &bits,
                                                const uint32_t *ctab, uint32_t NC) {
  if (y == a && a < b) {
    bits = spec;
    return spec_x;
  }
  if (y >= b) {
    bits.clear();
    return y;
  }
  Bits<BW> walked;
  walked.clear();
  const uint32_t m = walk_to<BW, HW>(C, y, a, b, spec, walked, ctab, NC);
  if (m < b) {
    bits = spec;
    bits.keep_from(m - a);
    bits.merge(walked);
    return spec_x;
  }
  bits = walked;
  return m;
}

// The set marks of a lane's bitmap in increasing order, one per next():
// the words sit in a shift register (static indexes keep them in registers)
// so that one loop body serves every word.
template <int BW>
struct MarkIter {
  uint32_t w[BW];
  uint32_t base;
  __device__ __forceinline__ MarkIter(const Bits<BW> &b, uint32_t a) : base(a) {
#pragma unroll
    for (int k = 0; k < BW; ++k) w[k] = b.w[k];
  }
  // the next marked offset (only while marks are left)
  __device__ __forceinline__ uint32_t next() {
    while (w[0] == 0) {
#pragma unroll
      for (int k = 0; k + 1 < BW; ++k) w[k] = w[k + 1];
      w[BW - 1] = 0;
      base += 32;
    }
    const uint32_t o = base + (uint32_t)(__ffs(w[0]) - 1);
    w[0] &= w[0] - 1;
    return o;
  }
};

// Marks set in increasing offset order: the word being filled is kept
// apart and pushed into a shift register when the offsets pass it (after BW
// pushes the words are in order), instead of a select over every word per
// mark.
template <int BW>
struct MarkFill {
  uint32_t w[BW];
  uint32_t cur = 0, lim = 32, pushed = 0;
  __device__ __forceinline__ MarkFill() {
#pragma unroll
    for (int k = 0; k < BW; ++k) w[k] = 0;
  }
  __device__ __forceinline__ void push() {
#pragma unroll
    for (int k = 0; k + 1 < BW; ++k) w[k] = w[k + 1];
    w[BW - 1] = cur;
    cur = 0;
    lim += 32;
    ++pushed;
  }
  __device__ __forceinline__ void set(uint32_t rel) {  // rel: nondecreasing, < 32 * BW
    while (rel >= lim) push();
    cur |= 1u << (rel & 31u);
  }
  __device__ __forceinline__ void finish(Bits<BW> &out) {
    while (pushed < (uint32_t)BW) push();
#pragma unroll
    for (int k = 0; k < BW; ++k) out.w[k] = w[k];
  }
};

// Interval slot (24 bytes at a multiple of 24 from a 16-byte aligned base):
// one 16-byte and one 8-byte store, the 16-byte one on whichever half is
// aligned.
__device__ __forceinline__ void put_interval(thapi_interval *dst, uint64_t start, uint64_t end, uint32_t np,
                                             uint32_t fn, uint32_t lvl, uint32_t flags) {
  unsigned long long *q = reinterpret_cast<unsigned long long *>(dst);
  const unsigned long long w2 = (unsigned long long)np | ((unsigned long long)fn << 32) |
                                ((unsigned long long)lvl << 48) | ((unsigned long long)flags << 56);
  const bool lo16 = (reinterpret_cast<uintptr_t>(dst) & 15u) == 0;
  *reinterpret_cast<ulonglong2 *>(lo16 ? q : q + 1) = lo16 ? make_ulonglong2(start, end) : make_ulonglong2(end, w2);
  q[lo16 ? 2 : 0] = lo16 ? w2 : start;
}

// Entry metadata: func | rank << 16 | level << 32 | depth below the packet start << 40.
__device__ __forceinline__ uint64_t entry_meta(uint32_t fn, uint32_t rank, uint32_t lvl, uint32_t np) {
  return (uint64_t)fn | ((uint64_t)rank << 16) | ((uint64_t)lvl << 32) | ((uint64_t)np << 40);
}

// Inclusive warp scans.
__device__ __forceinline__ DM scan_dm(DM x, uint32_t lane) {
#pragma unroll
  for (int q = 1; q < 32; q <<= 1) {
    const int us = __shfl_up_sync(kFull, x.s, q), um = __shfl_up_sync(kFull, x.m, q);
    if (lane >= (uint32_t)q) x = d_op(DM{us, um}, x);
  }
  return x;
}
__device__ __forceinline__ TsM scan_ts(TsM x, uint32_t lane) {
#pragma unroll
  for (int q = 1; q < 32; q <<= 1) {
    const uint32_t uh = __shfl_up_sync(kFull, x.has, q);
    const uint64_t uv = __shfl_up_sync(kFull, x.v, q);
    if (lane >= (uint32_t)q) x = ts_op(TsM{uh, uv}, x);
  }
  return x;
}

// DEV: device-activity records wanted (p.cmd.counts set); the kernel without
// them carries none of that code.
template <int BW, bool DEV, bool SIDE>
__global__ void __launch_bounds__(kMaxWarps * 32) k_analyze_warp(AnalyzeParams p, uint32_t NW, unsigned int *status) {
  extern __shared__ __align__(128) uint8_t sm[];
  constexpr uint32_t SEGW = 32u * (BW - 1) + 1;  // odd: lane k's segment starts in shared-memory bank k
  const uint32_t lane = threadIdx.x & 31;
  const uint32_t warp = threadIdx.x >> 5;
  const uint32_t lt = (1u << lane) - 1u;
  const uint32_t gt = ~((2u << lane) - 1u);
  const uint32_t F = p.n_funcs;
  const uint32_t NC = p.n_classes;
  const WLayout L = wlayout(p.P, NW, NC);
  uint8_t *wb = sm + warp * L.warp_bytes;
  uint8_t *buf = wb;
  uint32_t *C = reinterpret_cast<uint32_t *>(buf + kPacketHeader);
  uint64_t *tab_ts = reinterpret_cast<uint64_t *>(wb + L.off_tab);  // [height - minimum depth]
  uint64_t *tab_md = tab_ts + kHeights;
  uint16_t *s_off = reinterpret_cast<uint16_t *>(wb + L.off_off);
  uint64_t *bar = reinterpret_cast<uint64_t *>(wb + L.off_bar);
  uint32_t *ctab = reinterpret_cast<uint32_t *>(sm + L.off_ctab);
  uint16_t *cfn = reinterpret_cast<uint16_t *>(sm + L.off_cfn);

  uint64_t w_begin = (uint64_t)blockIdx.x * p.per_cta;
  uint64_t w_end = (w_begin + p.per_cta < p.n_order) ? w_begin + p.per_cta : p.n_order;
  if (p.run_start) {  // runs of about equal cost
    w_begin = p.run_start[blockIdx.x];
    w_end = p.run_start[blockIdx.x + 1];
  }
  if (w_begin >= w_end) return;  // uniform over the CTA
  auto pos_of = [&](uint64_t w) -> uint64_t { return p.poslist ? p.poslist[w] : w; };

  constexpr bool dev_on = DEV;
  for (uint32_t c = threadIdx.x; c <= NC; c += blockDim.x) {
    if (c < NC) {
      const uint64_t r = p.classes[c];
      const uint32_t k = cls_kind(r);
      const bool carries = dev_on && cls_cmdw(r) >= 0 && (k == kEntry || k == kDevBegin || k == kDevEnd);
      ctab[c] = cls_fixedw(r) | (k << 14) | ((uint32_t)(cls_resw(r) + 1) << 17) | (carries ? 1u << 31 : 0u);
      cfn[c] = (uint16_t)cls_func(r);
    } else {
      ctab[c] = 0;
    }
  }
  if (lane == 0) {
    mbar_init(bar, 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  __syncthreads();

  auto issue = [&](const PkDesc &d) {
    const uint32_t bytes = align16(kPacketHeader + d.content);
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    mbar_expect_tx(bar, bytes);
    bulk_copy_g2s(buf, packet_at(p.packets, p.pk_addr, d.pk, p.P), bytes, bar);
  };

  uint64_t fr_base = 0;
  uint32_t fr_left = 0;  // lane 0: current frontier chunk
  unsigned long long n_mismatch = 0, n_other = 0, n_pairs = 0, n_events = 0, n_disc = 0, n_pk = 0, n_slots = 0;
  unsigned long long n_dev = 0;  // DEV_BEGIN / DEV_END events (device pairing on)
  uint64_t tmin = ~0ull, tmax = 0;
  uint32_t phase = 0;
  bool issued = false;  // a copy is in flight into buf
  bool timed_out = false;

  // room for a packet's frontier items, from lane 0's chunk (~0: none, the host retries)
  auto grab_frontier = [&](uint32_t need) -> uint64_t {
    uint64_t fb = 0;
    if (lane == 0 && need) {
      if (need > fr_left) {
        const uint32_t grab = need > kChunk ? need : kChunk;
        fr_base = atomicAdd(p.frontier_top, (unsigned long long)grab);
        fr_left = grab;
        if (fr_base + grab > p.frontier_cap) fr_left = 0;  // overflow: the host retries with more room
      }
      if (need <= fr_left) {
        fb = fr_base;
        fr_base += need;
        fr_left -= need;
      } else {
        fb = ~0ull;
      }
    }
    return __shfl_sync(kFull, fb, 0);
  };

  uint64_t w = w_begin + warp;
  PkDesc dcur{}, dnext{};

  // Per-lane pairing of one packet whose events are valid, carry no absolute
  // timestamp, have deltas summing below 2^32 and need at most kLaneSlots
  // slots per lane.  Each lane walks its own events in order with a call
  // stack of its own: an exit pops the lane's latest open entry or, on an
  // empty stack, is a pending exit of the lane.  A lane's slots hold its
  // pending exits (at most one per new minimum depth, so they come first),
  // then its stack.  Timestamps are relative to the packet's ts_begin.
  // Afterwards, the k-th pending exit of a lane that starts at depth D closes
  // height D - 1 - k: it pairs with the open entry at that height of the
  // latest earlier lane that has one (per-height lane masks from ballots),
  // and with none it pops below the packet's start (a frontier item).  The
  // latest lane's open entry at each height from the packet's minimum depth
  // to its final depth is an open entry of the packet.  The running minimum
  // depth when an exit closes an entry equals the one when the entry was
  // made (the depth stays above the entry's height in between), which gives
  // the interval's packet-relative level and depth below the packet start.
  auto pair_lanes = [&](const PkDesc &d, uint64_t pos, bool has_next, DM dc, DM ex, DM ld, const Bits<BW> &bits,
                        uint32_t a, uint32_t e0, uint32_t cnt, uint32_t c_tot, uint32_t ecnt, uint64_t dsum) {
    const int dmin = dc.m;
    const uint32_t P_p = (uint32_t)(-dmin), O_p = (uint32_t)(dc.s - dmin);
    const uint64_t fbase = grab_frontier(P_p + O_p);
    thapi_interval *const pslots = p.slots ? p.slots + d.evbase : nullptr;
    Cell *const gcells = p.tally + (uint64_t)d.group * F;
    uint2 *const stk = reinterpret_cast<uint2 *>(wb + L.off_tab);  // [slot][lane]
    // lane prefixes: the slot rank of the lane's first entry and the time
    // before its first event (entries in bits 40.., deltas below)
    const uint64_t own = ((uint64_t)ecnt << 40) | dsum;
    uint64_t inc = own;
#pragma unroll
    for (int q = 1; q < 32; q <<= 1) {
      const uint64_t u = __shfl_up_sync(kFull, inc, q);
      if (lane >= (uint32_t)q) inc += u;
    }
    const uint64_t exs = inc - own;
    const uint32_t n_ent = (uint32_t)(__shfl_sync(kFull, inc, 31) >> 40);
    uint32_t rank = (uint32_t)(exs >> 40);
    uint32_t trel = (uint32_t)exs;  // the deltas of the whole packet sum below 2^32
    const int D = ex.s, Mex = ex.m;  // depth at the lane's start, running minimum before it
    uint32_t valid = 0, mism = 0, other = 0;
    // one pair: entry (time, slot rank, function) closed by an exit; post =
    // depth after the exit, bm = running minimum depth before it
    auto pair = [&](uint32_t ets, uint32_t erank, uint32_t efn, uint32_t xts, uint32_t xfn, uint32_t err, int post,
                    int bm) {
      uint32_t flags = 0;
      if (efn == xfn) {
        ++valid;
        flags = kIvValid | err;
        const unsigned long long dur = (unsigned long long)(xts - ets);
        Cell &cell = gcells[xfn];
        atomicAdd(&cell.count, 1ull);
        atomicAdd(&cell.total, dur);
        atomicMin(&cell.mn, dur);
        atomicMax(&cell.mx, dur);
        if (err) atomicAdd(&cell.err, 1ull);
      } else {
        ++mism;  // mismatched pair: no interval
      }
      if (pslots)
        put_interval(pslots + erank, d.tsb + ets, d.tsb + xts, (uint32_t)(-bm), efn, (uint32_t)min(post - bm, 255),
                     flags);
    };
    int sd = 0, md = 0;     // the lane's depth and running minimum, relative to its start
    uint32_t sp = 0, np = 0;  // open entries on the lane's stack; pending exits below them
    uint32_t e = e0;          // event index in the packet
    const uint32_t first_delta = C[0] & kDeltaMask;  // the packet's first event starts at word 0
    MarkIter<BW> it(bits, a);
    for (uint32_t left = cnt; left; --left) {
      const uint32_t oo = it.next();
      const uint32_t w0 = C[oo], w1 = C[oo + 1];
      const uint32_t c = w1 & 0xFFFFu;
      const uint32_t r = ctab[c];
      const uint32_t kd = row_kind(r);
      const uint32_t fn = cfn[c];
      trel += w0 & kDeltaMask;
      const bool is_e = kd == kEntry, is_x = kd == kExit;
      const bool pop = is_x && sp != 0, pend = is_x && sp == 0;
      const int32_t rw = row_resw(r);
      const uint32_t err = (is_x && rw >= 0 && C[oo + 2 + (uint32_t)max(rw, 0)] != 0) ? 1u : 0u;
      // an entry pushes at np + sp, a pop reads np + sp - 1, a pending exit writes np (sp = 0)
      const uint32_t slot = (np + sp - (pop ? 1u : 0u)) * 32 + lane;
      uint2 q = make_uint2(0u, 0u);
      if (pop) q = stk[slot];
      if (is_e || pend) stk[slot] = make_uint2(trel, fn | ((is_e ? rank : (e | (err << 15))) << 16));
      sd += is_e ? 1 : (is_x ? -1 : 0);
      if (pop) pair(q.x, q.y >> 16, q.y & 0xFFFFu, trel, fn, err, D + sd, min(Mex, D + md));
      sp += is_e ? 1u : 0u;
      sp -= pop ? 1u : 0u;
      np += pend ? 1u : 0u;
      rank += is_e ? 1u : 0u;
      md = pend ? sd : md;
      other += (!is_e && !is_x) ? 1u : 0u;
      ++e;
    }
    const uint32_t tlast = trel;
    __syncwarp();  // every lane's slots are written; the packet bytes are no longer needed
    if (lane == 0 && has_next && dcur.group != kPerCpuGroup) issue(dcur);
    issued = has_next && dcur.group != kPerCpuGroup;
    // heights indexed from the packet's minimum depth; the lane's open entries are [lo, hi)
    const int lo = D + ld.m - dmin, hi = D + ld.s - dmin;
    const int hn = __reduce_max_sync(kFull, hi);
    uint32_t hmask = 0;  // lane u: the lanes with an open entry at height index u
    for (int u = 0; u < hn; ++u) {
      const uint32_t bal = __ballot_sync(kFull, lo <= u && u < hi);
      if (lane == (uint32_t)u) hmask = bal;
    }
    const uint32_t maxp = __reduce_max_sync(kFull, np);
    for (uint32_t k = 0; k < maxp; ++k) {
      const bool act = k < np;
      const int h = D - 1 - (int)k;  // the height this pending exit closes
      const int u = act ? h - dmin : 0;
      const uint32_t lu = __shfl_sync(kFull, hmask, u);
      const uint32_t cand = act ? (lu & lt) : 0u;
      const int j = cand ? 31 - __clz(cand) : (int)lane;
      const int lo_j = __shfl_sync(kFull, lo, j);
      const uint32_t np_j = __shfl_sync(kFull, np, j);
      if (act) {
        const uint2 x = stk[k * 32 + lane];
        const uint32_t xfn = x.y & 0xFFFFu, xe = (x.y >> 16) & 0x7FFFu, xerr = x.y >> 31;
        if (cand) {
          const uint2 q = stk[(np_j + (uint32_t)(u - lo_j)) * 32 + (uint32_t)j];
          pair(q.x, q.y >> 16, q.y & 0xFFFFu, x.x, xfn, xerr, h, min(Mex, D - (int)k));
        } else if (fbase != ~0ull) {  // it pops below the packet's start
          Frontier fr;
          fr.ts = d.tsb + x.x;
          fr.aux = xe;
          fr.func = (uint16_t)xfn;
          fr.flags = (uint16_t)xerr;
          p.frontier[fbase + (uint64_t)(-h - 1)] = fr;
        }
      }
    }
    {  // the packet's open entries, one height per lane
      const uint32_t ow = lane < O_p ? hmask : 0u;
      const int j = ow ? 31 - __clz(ow) : (int)lane;
      const int lo_j = __shfl_sync(kFull, lo, j);
      const uint32_t np_j = __shfl_sync(kFull, np, j);
      if (ow) {
        const uint2 q = stk[(np_j + (lane - (uint32_t)lo_j)) * 32 + (uint32_t)j];
        const uint32_t orank = q.y >> 16, ofn = q.y & 0xFFFFu;
        if (fbase != ~0ull) {
          Frontier fr;
          fr.ts = d.tsb + q.x;
          fr.aux = pslots ? orank : 0xFFFFFFFFu;
          fr.func = (uint16_t)ofn;
          fr.flags = 0;
          p.frontier[fbase + P_p + lane] = fr;
        }
        if (pslots) put_interval(pslots + orank, d.tsb + q.x, 0, (uint32_t)(-dmin), ofn, min(lane, 255u), kIvOpen);
      }
    }
    __syncwarp();  // the slots are read before the next packet's offsets reuse the area
    n_mismatch += mism;
    n_pairs += valid;
    n_other += other;
    if (c_tot) {  // timestamps never decrease here: the packet's first and last event bound them
      tmin = min(tmin, d.tsb + first_delta);
      tmax = max(tmax, d.tsb + tlast);
    }
    const uint32_t vsum = __reduce_add_sync(kFull, valid);
    if (lane == 0) {
      p.sum_pend[pos] = P_p;
      p.sum_open[pos] = O_p;
      p.sum_fbase[pos] = fbase;
      p.sum_nslot[pos] = n_ent;
      p.sum_nvalid[pos] = vsum;
      n_events += c_tot;
      if (p.slots) n_slots += n_ent;
      n_disc += d.disc;
      n_pk += 1;
    }
  };
  if (w < w_end) {
    dcur = load_desc(p.desc + pos_of(w));
    dnext = dcur;
    if (w + NW < w_end) dnext = load_desc(p.desc + pos_of(w + NW));
    issued = dcur.group != kPerCpuGroup;  // per-CPU buffers are not staged here (percpu.cu takes them)
    if (lane == 0 && issued) issue(dcur);
  }
  __syncwarp();

  for (; w < w_end; w += NW) {
    const PkDesc d = dcur;
    const uint64_t pos = pos_of(w);
    const bool has_next = w + NW < w_end;
    dcur = dnext;  // next packet's descriptor (its copy is issued once the buffer is free)
    if (w + 2 * NW < w_end) dnext = load_desc(p.desc + pos_of(w + 2 * NW));
    if (d.group == kPerCpuGroup) {  // a per-CPU buffer: no copy was issued; percpu.cu pairs its threads
      if (lane == 0) {
        p.sum_pend[pos] = 0;
        p.sum_open[pos] = 0;
        p.sum_fbase[pos] = 0;
        p.sum_nslot[pos] = 0;
        p.sum_nvalid[pos] = 0;
        if (has_next && dcur.group != kPerCpuGroup) issue(dcur);
      }
      issued = has_next && dcur.group != kPerCpuGroup;
      __syncwarp();
      continue;
    }
    const bool ok_wait = mbar_wait_bounded(bar, phase);
    if (__any_sync(kFull, !ok_wait)) {
      timed_out = true;
      break;
    }
    phase ^= 1u;
    issued = false;
    const uint32_t W = d.content >> 2;
    if (lane < 8) C[W + lane] = 0;
    __syncwarp();

    // ---- 1. boundaries
    const uint32_t a = lane * SEGW;
    const uint32_t b = min(a + SEGW, W);
    Bits<BW> spec, bits;
    uint32_t o = a;
    {
      MarkFill<BW> mf;
      while (o < b) {
        mf.set(o - a);
        o = step(C, o, ctab, NC);
      }
      mf.finish(spec);
    }
    const uint32_t spec_x = a < b ? o : a;
    const bool succ_live = a + SEGW < W;
    uint32_t ent = __shfl_up_sync(kFull, spec_x, 1);
    if (lane == 0) ent = 0;
    uint32_t x = resolve_seg<BW>(C, ent, a, b, spec, spec_x, bits, ctab, NC);
    for (int r = 0; r < 32; ++r) {
      const uint32_t next_ent = __shfl_down_sync(kFull, ent, 1);
      const uint32_t bal = __ballot_sync(kFull, lane < 31 && succ_live && x != next_ent);
      if (!bal) break;
      const int k = __ffs(bal) - 1;
      const uint32_t xk = __shfl_sync(kFull, x, k);
      if (lane == (uint32_t)k + 1) {
        ent = xk;
        x = resolve_seg<BW>(C, ent, a, b, spec, spec_x, bits, ctab, NC);
      }
    }
    const uint32_t cnt = bits.count();
    uint32_t cinc = cnt;
#pragma unroll
    for (int q = 1; q < 32; q <<= 1) {
      const uint32_t u = __shfl_up_sync(kFull, cinc, q);
      if (lane >= (uint32_t)q) cinc += u;
    }
    const uint32_t c_tot = __shfl_sync(kFull, cinc, 31);
    bool fallback = c_tot > kEvMax || d.nev > kEvMax;
    // ---- 2. compaction and validation: each lane stores its events' offsets
    // in order and checks them, folding the depth monoid (sum, min-prefix) and
    // the highest depth of its events
    uint32_t ekey = 0xFFFFFFFFu;  // event index << 3 | code of the first bad event
    DM ld{0, 0};
    int lmax = 0;
    uint32_t nrec = 0;  // device-activity records of the lane's events: begin | end << 10 | host << 20
    // for per-lane pairing: the lane's entries, the sum of its timestamp deltas, an EXT event seen
    uint32_t ecnt = 0;
    uint64_t dsum = 0;
    bool lext = false;
    int lneed = 0;  // most slots the lane's pending exits and stack take at once: max(depth - 2 min)
    if (!fallback) {
      uint32_t e = cinc - cnt;
      // one event: its error code (0 if none) and depth step
      // (rec: its device-activity record, counted in nrec's fields)
      auto check = [&](uint32_t oo, uint32_t &code, int &dv, uint32_t &rec, uint32_t &dl) {
        const uint32_t w0 = C[oo], w1 = C[oo + 1];
        dl = w0;
        const uint32_t c = w1 & 0xFFFFu;
        const bool ext = (w0 & kExtBit) != 0;
        const uint32_t r = ctab[c < NC ? c : NC];
        const uint32_t sz = 2u + (ext ? 2u : 0u) + row_fixedw(r) + (((w1 >> 16) + 3u) >> 2);
        code = oo + 2 > W ? THAPI_E_TRUNCATED
               : ((w0 >> 28) != 0 || c >= NC || (ext && (w0 & kDeltaMask) != 0)) ? THAPI_E_FORMAT
               : oo + sz > W ? THAPI_E_TRUNCATED : 0u;
        const uint32_t kd = row_kind(r);
        dv = code ? 0 : kd == kEntry ? 1 : (kd == kExit ? -1 : 0);
        rec = (dev_on && !code && (r >> 31))
                  ? (kd == kDevBegin ? 1u : kd == kDevEnd ? (1u << 10) : kd == kEntry ? (1u << 20) : 0u)
                  : 0u;
      };
      auto fold = [&](uint32_t code, int dv, uint32_t rec, uint32_t dl) {
        nrec += rec;
        ecnt += dv > 0 ? 1u : 0u;
        dsum += dl & kDeltaMask;
        lext = lext || (dl & kExtBit) != 0;
        if (code) ekey = min(ekey, (e << 3) | code);
        ld.s += dv;
        ld.m = min(ld.m, ld.s);
        lmax = max(lmax, ld.s);
        lneed = max(lneed, ld.s - 2 * ld.m);
        ++e;
      };
      MarkIter<BW> it(bits, a);
      for (uint32_t left = cnt; left;) {  // two events per iteration: their loads overlap
        const uint32_t oo0 = it.next();
        const bool two = left > 1;
        const uint32_t oo1 = two ? it.next() : oo0;
        left -= two ? 2u : 1u;
        s_off[e] = (uint16_t)oo0;
        if (two) s_off[e + 1] = (uint16_t)oo1;
        uint32_t c0, c1, r0, r1, l0, l1;
        int d0, d1;
        check(oo0, c0, d0, r0, l0);
        check(oo1, c1, d1, r1, l1);
        fold(c0, d0, r0, l0);
        if (two) fold(c1, d1, r1, l1);
      }
    }
    __syncwarp();
    const uint32_t nb = fallback ? 0u : (c_tot + 31) >> 5;  // batches of 32 events
    // the packet's depth range: exclusive scan of the lanes' depth monoids
    DM dc, ex;
    int dmax;
    {
      DM inc = scan_dm(ld, lane);
      ex = DM{__shfl_up_sync(kFull, inc.s, 1), __shfl_up_sync(kFull, inc.m, 1)};
      if (lane == 0) ex = DM{0, 0};
      dc = DM{__shfl_sync(kFull, inc.s, 31), __shfl_sync(kFull, inc.m, 31)};
      dmax = __reduce_max_sync(kFull, ex.s + lmax);
    }
    const uint32_t gkey = __reduce_min_sync(kFull, ekey);
    const bool bad = !fallback && (gkey != 0xFFFFFFFFu || c_tot != d.nev);
    fallback = fallback || (!bad && (uint32_t)(dmax - dc.m) > kHeights);
    if (bad || fallback) {
      if (lane == 0) {
        if (bad)
          atomicMin(p.content_err, gkey != 0xFFFFFFFFu ? err_key(d.pk, gkey >> 3, gkey & 7u)
                                                       : err_key(d.pk, c_tot, THAPI_E_FORMAT));
        else  // the CTA kernel takes it
          p.dense_list[atomicAdd(p.dense_count, 1ull)] = (uint32_t)pos;
      }
      __syncwarp();
      if (lane == 0 && has_next && dcur.group != kPerCpuGroup) issue(dcur);
      issued = has_next && dcur.group != kPerCpuGroup;
      continue;
    }

    // ---- 3a. per-lane pairing, for packets without absolute timestamps, with
    // a span below 2^32 ns and nesting shallow enough for the lanes' slots
    if constexpr (!DEV && !SIDE) {
      uint64_t dtot = dsum;
#pragma unroll
      for (int q = 16; q; q >>= 1) dtot += __shfl_xor_sync(kFull, dtot, q);
      const bool fast = !__any_sync(kFull, lext) && dtot < (1ull << 32) &&
                        !__any_sync(kFull, lneed > (int)kLaneSlots);
      if (fast) {
        pair_lanes(d, pos, has_next, dc, ex, ld, bits, a, cinc - cnt, cnt, c_tot, ecnt, dsum);
        continue;
      }
    }

    // ---- 3. pairing, 32 events at a time
    const int dmin = dc.m;  // minimum depth (packet-relative, <= 0); heights are indexed from it
    const uint32_t P_p = (uint32_t)(-dmin);
    const uint32_t O_p = (uint32_t)(dc.s - dmin);
    // the packet's device-activity records, reserved at once (bases per kind)
    unsigned long long rbase_b = 0, rbase_e = 0, rbase_h = 0;
    if (dev_on) {
      const uint32_t nb_p = __reduce_add_sync(kFull, nrec & 0x3FFu);
      const uint32_t ne_p = __reduce_add_sync(kFull, (nrec >> 10) & 0x3FFu);
      const uint32_t nh_p = __reduce_add_sync(kFull, nrec >> 20);
      if (lane == 0) {
        if (nb_p) rbase_b = atomicAdd(&p.cmd.counts[0], (unsigned long long)nb_p);
        if (ne_p) rbase_e = atomicAdd(&p.cmd.counts[1], (unsigned long long)ne_p);
        if (nh_p) rbase_h = atomicAdd(&p.cmd.counts[2], (unsigned long long)nh_p);
      }
    }
    const uint64_t fbase = grab_frontier(P_p + O_p);
    if (dev_on) {
      rbase_b = __shfl_sync(kFull, rbase_b, 0);
      rbase_e = __shfl_sync(kFull, rbase_e, 0);
      rbase_h = __shfl_sync(kFull, rbase_h, 0);
    }
    thapi_interval *const pslots = p.slots ? p.slots + d.evbase : nullptr;
    Cell *const gcells = p.tally + (uint64_t)d.group * F;
    uint32_t valid = 0, mism = 0;
    uint64_t tcur = d.tsb;  // timestamp of the last event so far
    DM dp{0, 0};            // depth monoid of the batches so far
    uint32_t rank_c = 0;  // slot owners so far: entries, and command-carrying DEV_BEGINs
    uint32_t pend_c = 0;  // pending exits so far
    // the next batch's offsets, header words and class row are loaded one batch ahead
    uint32_t n_oo, n_w0, n_w1, n_r;
    auto prefetch = [&](uint32_t bt) {
      const uint32_t e = bt * 32 + lane;
      n_oo = e < c_tot ? s_off[min(e, c_tot - 1)] : W;
      n_w0 = C[n_oo];
      n_w1 = C[n_oo + 1];
      n_r = ctab[e < c_tot ? (n_w1 & 0xFFFFu) : NC];
    };
    if (nb) prefetch(0);
    for (uint32_t bt = 0; bt < nb; ++bt) {
      const uint32_t e = bt * 32 + lane;
      const bool act = e < c_tot;
      const uint32_t oo = n_oo, w0 = n_w0, w1 = n_w1, r = n_r;
      if (bt + 1 < nb) prefetch(bt + 1);
      const uint32_t c = act ? (w1 & 0xFFFFu) : NC;
      const bool ext = (w0 & kExtBit) != 0;
      const uint32_t kd = act ? row_kind(r) : kSample;
      const uint32_t fn = cfn[min(c, NC - 1)];
      const bool is_entry = kd == kEntry, is_exit = kd == kExit;
      const int32_t rw = row_resw(r);
      const uint32_t err =
          (is_exit && rw >= 0 && C[min(oo + 2 + (ext ? 2u : 0u) + (uint32_t)max(rw, 0), W)] != 0) ? 1u : 0u;
      // depths from the entry/exit ballots, relative to the batch start; the
      // match on batch-relative heights (equal iff the heights are) needs nothing else
      const int dv = is_entry ? 1 : (is_exit ? -1 : 0);
      const uint32_t ebal = __ballot_sync(kFull, is_entry), xbal = __ballot_sync(kFull, is_exit);
      const uint32_t le = lt | (1u << lane);
      const int s_in = (int)__popc(ebal & le) - (int)__popc(xbal & le);
      const uint32_t key =
          is_entry ? (uint32_t)(s_in - dv + 64) : is_exit ? (uint32_t)(s_in + 64) : (0x80000000u | lane);
      const uint32_t peers = __match_any_sync(kFull, key);
      // timestamps (32-bit deltas) and the running minimum depth in one set of scan rounds
      const bool any_ext = __any_sync(kFull, act && ext);
      uint32_t x = act ? (w0 & kDeltaMask) : 0u;
      int m_in = min(s_in, 0);
#pragma unroll
      for (int q = 1; q < 32; q <<= 1) {
        const uint32_t u = __shfl_up_sync(kFull, x, q);
        const int um = __shfl_up_sync(kFull, m_in, q);
        if (lane >= (uint32_t)q) {
          x += u;
          m_in = min(m_in, um);
        }
      }
      uint64_t t, t_last;
      if (any_ext) {  // an absolute timestamp in the batch: the (has_abs, value) monoid
        const uint64_t xts = (uint64_t)C[min(oo + 2, W)] | ((uint64_t)C[min(oo + 3, W)] << 32);
        t = ts_op(TsM{1u, tcur}, scan_ts(TsM{act && ext ? 1u : 0u, !act ? 0ull : ext ? xts : (w0 & kDeltaMask)}, lane)).v;
        if (act) {
          tmin = min(tmin, t);
          tmax = max(tmax, t);
        }
        t_last = __shfl_sync(kFull, t, 31);
      } else {
        t = tcur + x;
        // nondecreasing over the batch (lane 0 holds an event): its ends bound it
        t_last = tcur + __shfl_sync(kFull, x, 31);
        tmin = min(tmin, tcur + __shfl_sync(kFull, x, 0));
        tmax = max(tmax, t_last);
      }
      int m_ex = __shfl_up_sync(kFull, m_in, 1);
      if (lane == 0) m_ex = 0;
      const DM before{dp.s + s_in - dv, min(dp.m, dp.s + m_ex)};  // depth and running minimum before the event
      const int post = before.s + dv;                              // depth after the event
      // a DEV_BEGIN with a command id owns an interval slot too (its device interval)
      const bool hcmd = (r >> 31) != 0;
      const bool rec_b = hcmd && kd == kDevBegin;
      const uint32_t bbal = dev_on ? __ballot_sync(kFull, rec_b) : 0u;
      const uint32_t obal = ebal | bbal;
      const uint32_t rank = rank_c + __popc(obal & lt);
      const uint64_t meta = entry_meta(fn, rank, (uint32_t)min(before.s - before.m, 255), (uint32_t)(-before.m));
      const uint32_t cand = is_exit ? (peers & ebal & lt) : 0u;
      const int src = cand ? 31 - __clz(cand) : (int)lane;
      const uint64_t ets_b = __shfl_sync(kFull, t, src), em_b = __shfl_sync(kFull, meta, src);
      const bool from_tab = is_exit && !cand && post >= before.m;
      const bool pend = is_exit && !cand && post < before.m;
      uint64_t ets = ets_b, em = em_b;
      if (from_tab) {
        ets = tab_ts[post - dmin];
        em = tab_md[post - dmin];
      }
      if (cand || from_tab) {  // one pair: entry (ets, em) closed by this exit
        const uint32_t efn = (uint32_t)(em & 0xFFFFu);
        uint32_t flags = 0;
        if (efn == fn) {
          ++valid;
          flags = kIvValid | err;
          const uint64_t dur = t - ets;
          Cell &cell = gcells[fn];
          atomicAdd(&cell.count, 1ull);
          atomicAdd(&cell.total, (unsigned long long)dur);
          atomicMin(&cell.mn, (unsigned long long)dur);
          atomicMax(&cell.mx, (unsigned long long)dur);
          if (err) atomicAdd(&cell.err, 1ull);
          if (SIDE) {  // self time: the exit's position and the entry's exact packet-relative depth
            SelfSlot &ss = p.side[d.evbase + ((em >> 16) & 0xFFFFu)];
            ss.exit_pos = d.evbase + e;
            ss.level = (uint32_t)(post - before.m);
          }
        } else {
          ++mism;  // mismatched pair: no interval
        }
        if (pslots)
          put_interval(pslots + ((em >> 16) & 0xFFFFu), ets, t, (uint32_t)((em >> 40) & 0xFFFFu), efn,
                       (uint32_t)((em >> 32) & 0xFFu), flags);
      }
      if (SIDE && is_entry) p.side[d.evbase + rank].entry_pos = d.evbase + e;
      const uint32_t pbal = __ballot_sync(kFull, pend);
      if (pend && fbase != ~0ull) {
        Frontier fr;
        fr.ts = t;
        fr.aux = e;
        fr.func = (uint16_t)fn;
        fr.flags = (uint16_t)err;
        p.frontier[fbase + pend_c + __popc(pbal & lt)] = fr;
      }
      if (dev_on) {  // device-activity records of the batch, at the packet's reserved bases
        n_dev += (kd == kDevBegin || kd == kDevEnd) ? 1u : 0u;
        const bool rec_e = hcmd && kd == kDevEnd, rec_h = hcmd && is_entry;
        const uint32_t xb = __ballot_sync(kFull, rec_e), hb = __ballot_sync(kFull, rec_h);
        if (rec_b || rec_e || rec_h) {
          const uint32_t q = min(oo + 2u + (ext ? 2u : 0u) + (uint32_t)cls_cmdw(p.classes[c]), W);
          const uint64_t id = (uint64_t)C[q] | ((uint64_t)C[min(q + 1u, W)] << 32);
          atomicAdd(&p.cmd.hist[((rec_b ? 0u : rec_e ? 1u : 2u) << p.cmd.part_bits) + cmd_part(id, p.cmd.part_bits)],
                    1u);
          if (rec_b) {
            const uint64_t k = rbase_b + __popc(bbal & lt);
            if (k < p.cmd.cap_b) p.cmd.b[k] = CmdBegin{id, t, d.evbase + rank, d.group, (uint32_t)pos};
            if (pslots) put_interval(pslots + rank, t, 0, 0xFFFFFFFFu, 0, 0, 0);  // invalid until joined
          } else if (rec_e) {
            const uint64_t k = rbase_e + __popc(xb & lt);
            if (k < p.cmd.cap_e) p.cmd.e[k] = CmdEnd{id, t};
          } else {
            const uint64_t k = rbase_h + __popc(hb & lt);
            if (k < p.cmd.cap_h) p.cmd.h[k] = CmdHost{id, fn, 0u};
          }
        }
        rbase_b += __popc(bbal);
        rbase_e += __popc(xb);
        rbase_h += __popc(hb);
      }
      __syncwarp();  // the table is read above before the batch's entries update it
      if (is_entry && (peers & ebal & gt) == 0) {  // the batch's last entry at its height
        tab_ts[before.s - dmin] = t;
        tab_md[before.s - dmin] = meta;
      }
      __syncwarp();
      n_other += (act && !is_entry && !is_exit) ? 1u : 0u;
      tcur = t_last;
      dp = d_op(dp, DM{(int)__popc(ebal) - (int)__popc(xbal), __shfl_sync(kFull, m_in, 31)});
      rank_c += __popc(obal);
      pend_c += __popc(pbal);
    }
    __syncwarp();
    // the packet bytes are no longer needed: stage the next packet now
    if (lane == 0 && has_next && dcur.group != kPerCpuGroup) issue(dcur);
    issued = has_next && dcur.group != kPerCpuGroup;
    // the table rows from the minimum depth up to the final depth are the open entries
    for (uint32_t k = lane; k < O_p; k += 32) {
      const uint64_t ots = tab_ts[k], om = tab_md[k];
      const uint32_t orank = (uint32_t)((om >> 16) & 0xFFFFu);
      if (fbase != ~0ull) {
        Frontier fr;
        fr.ts = ots;
        fr.aux = pslots ? orank : 0xFFFFFFFFu;
        fr.func = (uint16_t)(om & 0xFFFFu);
        fr.flags = 0;
        p.frontier[fbase + P_p + k] = fr;
      }
      if (pslots)
        put_interval(pslots + orank, ots, 0, (uint32_t)((om >> 40) & 0xFFFFu), (uint32_t)(om & 0xFFFFu),
                     (uint32_t)((om >> 32) & 0xFFu), kIvOpen);
    }
    n_mismatch += mism;
    n_pairs += valid;
    const uint32_t vsum = __reduce_add_sync(kFull, valid);
    if (lane == 0) {
      p.sum_pend[pos] = P_p;
      p.sum_open[pos] = O_p;
      p.sum_fbase[pos] = fbase;
      p.sum_nslot[pos] = rank_c;
      p.sum_nvalid[pos] = vsum;
      n_events += c_tot;
      if (p.slots) n_slots += rank_c;
      n_disc += d.disc;
      n_pk += 1;
    }
    __syncwarp();
  }

  if (timed_out) {
    if (issued) (void)mbar_wait_bounded(bar, phase);
    if (lane == 0) atomicExch(status, (unsigned)THAPI_E_TIMEOUT);
  }

  for (int off = 16; off > 0; off >>= 1) {
    n_mismatch += __shfl_down_sync(kFull, n_mismatch, off);
    n_other += __shfl_down_sync(kFull, n_other, off);
    n_pairs += __shfl_down_sync(kFull, n_pairs, off);
    n_dev += __shfl_down_sync(kFull, n_dev, off);
    tmin = min(tmin, __shfl_down_sync(kFull, tmin, off));
    tmax = max(tmax, __shfl_down_sync(kFull, tmax, off));
  }
  if (lane == 0) {
    if (n_mismatch) atomicAdd(&p.diag[dMismatch], n_mismatch);
    if (n_other) atomicAdd(&p.diag[dOther], n_other);
    if (n_pairs) atomicAdd(&p.diag[dPairs], n_pairs);
    if (n_dev) atomicAdd(&p.diag[dDevEvents], n_dev);
    if (tmin != ~0ull) atomicMin(&p.tminmax[0], (unsigned long long)tmin);
    if (tmax) atomicMax(&p.tminmax[1], (unsigned long long)tmax);
    if (n_events) atomicAdd(&p.diag[dEvents], n_events);
    if (n_disc) atomicAdd(&p.diag[dDiscarded], n_disc);
    if (n_pk) atomicAdd(&p.diag[dPackets], n_pk);
    if (n_slots && p.slots_written) atomicAdd(p.slots_written, n_slots);
  }
}

template <int BW>
cudaError_t launch_w(const AnalyzeParams &p, const WarpPlan &wp, uint32_t grid, cudaStream_t s, unsigned *status) {
  auto fn = p.cmd.counts ? (p.side ? k_analyze_warp<BW, true, true> : k_analyze_warp<BW, true, false>)
                         : (p.side ? k_analyze_warp<BW, false, true> : k_analyze_warp<BW, false, false>);
  cudaError_t e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)wp.smem);
  if (e != cudaSuccess) return e;
  fn<<<grid, wp.nw * 32, wp.smem, s>>>(p, wp.nw, status);
  count_launches(1);
  return cudaGetLastError();
}

// Bitmap words per lane segment for packets of P bytes (0: too large for the
// warp kernel).  A lane's segment is 32 * (BW - 1) + 1 words: an odd length,
// so that the 32 segments start in 32 different shared-memory banks (with
// 32 * k words they would all start in bank 0, and lanes walking events of
// one size would stay in the same bank in lock step).
int warp_bw(uint32_t P) {
  const uint32_t wmax = (P - kPacketHeader) / 4;
  if (wmax <= 32u * 33) return 2;
  if (wmax <= 32u * 65) return 3;
  if (wmax <= 32u * 129) return 5;
  if (wmax <= 32u * 257) return 9;
  return 0;
}

// ---------------------------------------------------------------- decode
// Every event of every packet as a record (thapi_event) at its global event
// index: the same boundary walk, stitch and checks as the analysis, then 32
// events per batch with the timestamp monoid scanned across the batches.  No
// pairing.  Plain coalesced loads stage the packet (one warp per packet).
constexpr uint32_t kDecodeWarps = 16;  // at most; shared memory sets the count (11 warps of 16 KB packets)

__host__ __device__ inline uint32_t decode_warp_bytes(uint32_t P) {
  return rup(P + 48u, 128u) + rup(((P - kPacketHeader) / 8u + 1u) * 2u, 128u);
}

// One packet of the decode (HW header words: 2, or 4 in per-CPU buffers).
template <int BW, uint32_t HW>
__device__ __forceinline__ void decode_packet(const DecodeParams &p, const PkDesc &d, uint8_t *buf, uint16_t *s_off,
                                              const uint32_t *ctab, uint32_t lane) {
  constexpr uint32_t SEGW = 32u * (BW - 1) + 1;
  const uint32_t NC = p.n_classes;
  uint32_t *C = reinterpret_cast<uint32_t *>(buf + kPacketHeader);
  const uint32_t W = d.content >> 2;
  {  // stage header + content
    const uint4 *src = reinterpret_cast<const uint4 *>(packet_at(p.packets, p.pk_addr, d.pk, p.P));
    uint4 *dst = reinterpret_cast<uint4 *>(buf);
    const uint32_t n16 = align16(kPacketHeader + d.content) / 16u;
    for (uint32_t k = lane; k < n16; k += 32) dst[k] = __ldg(src + k);  // packets are read-only here
  }
  __syncwarp();
  if (lane < 8) C[W + lane] = 0;
  __syncwarp();
  // boundaries (as in the analysis kernel)
  const uint32_t a = lane * SEGW;
  const uint32_t b = min(a + SEGW, W);
  Bits<BW> spec, bits;
  spec.clear();
  uint32_t o = a;
  while (o < b) {
    spec.set(o - a);
    o = step<HW>(C, o, ctab, NC);
  }
  const uint32_t spec_x = a < b ? o : a;
  const bool succ_live = a + SEGW < W;
  uint32_t ent = __shfl_up_sync(kFull, spec_x, 1);
  if (lane == 0) ent = 0;
  uint32_t x = resolve_seg<BW, HW>(C, ent, a, b, spec, spec_x, bits, ctab, NC);
  for (int r = 0; r < 32; ++r) {
    const uint32_t next_ent = __shfl_down_sync(kFull, ent, 1);
    const uint32_t bal = __ballot_sync(kFull, lane < 31 && succ_live && x != next_ent);
    if (!bal) break;
    const int k = __ffs(bal) - 1;
    const uint32_t xk = __shfl_sync(kFull, x, k);
    if (lane == (uint32_t)k + 1) {
      ent = xk;
      x = resolve_seg<BW, HW>(C, ent, a, b, spec, spec_x, bits, ctab, NC);
    }
  }
  const uint32_t cnt = bits.count();
  uint32_t cinc = cnt;
#pragma unroll
  for (int q = 1; q < 32; q <<= 1) {
    const uint32_t u = __shfl_up_sync(kFull, cinc, q);
    if (lane >= (uint32_t)q) cinc += u;
  }
  const uint32_t c_tot = __shfl_sync(kFull, cinc, 31);
  // offsets in order, with the format and truncation checks
  uint32_t ekey = 0xFFFFFFFFu;
  {
    uint32_t e = cinc - cnt;
#pragma unroll
    for (int k = 0; k < BW; ++k) {
      uint32_t m = bits.w[k];
      while (m) {
        const uint32_t oo = a + k * 32 + (__ffs(m) - 1);
        m &= m - 1;
        s_off[e] = (uint16_t)oo;
        const uint32_t w0 = C[oo], w1 = C[oo + 1];
        const uint32_t c = w1 & 0xFFFFu;
        const bool ext = (w0 & kExtBit) != 0;
        const uint32_t r = ctab[c < NC ? c : NC];
        const uint32_t sz = HW + (ext ? 2u : 0u) + row_fixedw(r) + (((w1 >> 16) + 3u) >> 2);
        const uint32_t code = oo + HW > W ? THAPI_E_TRUNCATED
                              : ((w0 >> 28) != 0 || c >= NC || (ext && (w0 & kDeltaMask) != 0)) ? THAPI_E_FORMAT
                              : oo + sz > W ? THAPI_E_TRUNCATED : 0u;
        if (code) ekey = min(ekey, (e << 3) | code);
        ++e;
      }
    }
  }
  __syncwarp();
  const uint32_t gkey = __reduce_min_sync(kFull, ekey);
  if (gkey != 0xFFFFFFFFu || c_tot != d.nev) {
    if (lane == 0)
      atomicMin(p.content_err, gkey != 0xFFFFFFFFu ? err_key(d.pk, gkey >> 3, gkey & 7u)
                                                   : err_key(d.pk, c_tot, THAPI_E_FORMAT));
    __syncwarp();
    return;
  }
  // the stream's pid / tid (per-thread streams) or each event's vpid / vtid (per-CPU buffers)
  const uint32_t spid = HW == 2 ? p.group_keys[3ull * d.group + 1] : 0u;
  const uint32_t stid = HW == 2 ? p.group_keys[3ull * d.group + 2] : 0u;
  // records, 32 events at a time
  uint64_t tcur = d.tsb;
  for (uint32_t e0 = 0; e0 < c_tot; e0 += 32) {
    const uint32_t e = e0 + lane;
    const bool act = e < c_tot;
    const uint32_t oo = act ? s_off[e] : W;
    const uint32_t w0 = C[oo], w1 = C[oo + 1];
    const bool ext = act && (w0 & kExtBit) != 0;
    const uint32_t c = act ? (w1 & 0xFFFFu) : 0u;
    const uint64_t xts = (uint64_t)C[min(oo + HW, W)] | ((uint64_t)C[min(oo + HW + 1, W)] << 32);
    const TsM tm = ts_op(TsM{1u, tcur}, scan_ts(TsM{ext ? 1u : 0u, !act ? 0ull : ext ? xts : (w0 & kDeltaMask)}, lane));
    const uint64_t t = tm.v;
    tcur = __shfl_sync(kFull, t, 31);
    if (act) {
      const uint64_t r = p.classes[c];
      const uint32_t base = oo + HW + (ext ? 2u : 0u);
      const int32_t rw = cls_resw(r), cw = cls_cmdw(r);
      thapi_event ev;
      ev.ts = t;
      ev.cmd = cw >= 0 ? ((uint64_t)C[min(base + cw, W)] | ((uint64_t)C[min(base + cw + 1, W)] << 32)) : 0ull;
      ev.stream_id = d.stream;
      ev.class_id = (uint16_t)c;
      ev.var_len = (uint16_t)(w1 >> 16);
      ev.result = rw >= 0 ? (int32_t)C[min(base + rw, W)] : 0;
      ev.ext = ext ? 1 : 0;
      ev.kind = (uint8_t)cls_kind(r);
      ev.func_id = (uint16_t)cls_func(r);
      ev.vpid = HW == 2 ? spid : C[oo + 2];
      ev.vtid = HW == 2 ? stid : C[oo + 3];
      p.out[d.evbase + e] = ev;
    }
  }
  __syncwarp();
}

template <int BW>
__global__ void __launch_bounds__(kDecodeWarps * 32) k_decode_warp(DecodeParams p, uint32_t NW) {
  extern __shared__ __align__(128) uint8_t sm[];
  const uint32_t lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const uint32_t NC = p.n_classes;
  const uint32_t wbytes = decode_warp_bytes(p.P);
  uint8_t *buf = sm + warp * wbytes;
  uint16_t *s_off = reinterpret_cast<uint16_t *>(buf + rup(p.P + 48u, 128u));
  uint32_t *ctab = reinterpret_cast<uint32_t *>(sm + NW * wbytes);
  for (uint32_t c = threadIdx.x; c <= NC; c += blockDim.x) {
    if (c < NC) {
      const uint64_t r = p.classes[c];
      ctab[c] = cls_fixedw(r) | (cls_kind(r) << 14) | ((uint32_t)(cls_resw(r) + 1) << 17);
    } else {
      ctab[c] = 0;
    }
  }
  __syncthreads();
  for (uint64_t w = (uint64_t)blockIdx.x * NW + warp; w < p.n_order; w += (uint64_t)gridDim.x * NW) {
    const PkDesc d = load_desc(p.desc + w);
    if (d.group == kPerCpuGroup)
      decode_packet<BW, 4>(p, d, buf, s_off, ctab, lane);
    else
      decode_packet<BW, 2>(p, d, buf, s_off, ctab, lane);
  }
}

template <int BW>
cudaError_t launch_dw(const DecodeParams &p, uint32_t nw, uint32_t grid, cudaStream_t s) {
  const uint32_t smem = nw * decode_warp_bytes(p.P) + rup((p.n_classes + 1u) * 4u, 16u);
  cudaError_t e = cudaFuncSetAttribute(k_decode_warp<BW>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  k_decode_warp<BW><<<grid, nw * 32, smem, s>>>(p, nw);
  count_launches(1);
  return cudaGetLastError();
}

// ------------------------------------------------------------ per-CPU decode
// The events of per-CPU buffers (16-byte headers: tsw, class, var_len, vpid,
// vtid): the same boundary walk, stitch and checks with 4 header words, then
// 32 events per batch: every ENTRY and EXIT becomes a PcRec (at a range
// reserved once per packet), every ENTRY owns an interval slot (written
// invalid; percpu.cu fills the paired ones).
template <int BW>
__global__ void __launch_bounds__(kDecodeWarps * 32) k_percpu_decode(PcParams p, uint32_t NW) {
  extern __shared__ __align__(128) uint8_t sm[];
  constexpr uint32_t SEGW = 32u * (BW - 1) + 1;
  constexpr uint32_t HW = 4;
  const uint32_t lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const uint32_t lt = (1u << lane) - 1u;
  const uint32_t NC = p.n_classes;
  const uint32_t wbytes = decode_warp_bytes(p.P);
  uint8_t *buf = sm + warp * wbytes;
  uint32_t *C = reinterpret_cast<uint32_t *>(buf + kPacketHeader);
  uint16_t *s_off = reinterpret_cast<uint16_t *>(buf + rup(p.P + 48u, 128u));
  uint32_t *ctab = reinterpret_cast<uint32_t *>(sm + NW * wbytes);
  for (uint32_t c = threadIdx.x; c <= NC; c += blockDim.x) {
    if (c < NC) {
      const uint64_t r = p.classes[c];
      ctab[c] = cls_fixedw(r) | (cls_kind(r) << 14) | ((uint32_t)(cls_resw(r) + 1) << 17);
    } else {
      ctab[c] = 0;
    }
  }
  __syncthreads();
  unsigned long long n_ev = 0, n_pk = 0, n_disc = 0, n_other = 0;
  uint64_t tmin = ~0ull, tmax = 0;
  for (uint64_t w = (uint64_t)blockIdx.x * NW + warp; w < p.n_order; w += (uint64_t)gridDim.x * NW) {
    const PkDesc d = load_desc(p.desc + w);
    if (d.group != kPerCpuGroup) continue;  // uniform over the warp
    const uint32_t W = d.content >> 2;
    {
      const uint4 *src = reinterpret_cast<const uint4 *>(packet_at(p.packets, p.pk_addr, d.pk, p.P));
      uint4 *dst = reinterpret_cast<uint4 *>(buf);
      const uint32_t n16 = align16(kPacketHeader + d.content) / 16u;
      for (uint32_t k = lane; k < n16; k += 32) dst[k] = __ldg(src + k);  // packets are read-only here
    }
    __syncwarp();
    if (lane < 8) C[W + lane] = 0;
    __syncwarp();
    const uint32_t a = lane * SEGW;
    const uint32_t b = min(a + SEGW, W);
    Bits<BW> spec, bits;
    spec.clear();
    uint32_t o = a;
    while (o < b) {
      spec.set(o - a);
      o = step<HW>(C, o, ctab, NC);
    }
    const uint32_t spec_x = a < b ? o : a;
    const bool succ_live = a + SEGW < W;
    uint32_t ent = __shfl_up_sync(kFull, spec_x, 1);
    if (lane == 0) ent = 0;
    uint32_t x = resolve_seg<BW, HW>(C, ent, a, b, spec, spec_x, bits, ctab, NC);
    for (int r = 0; r < 32; ++r) {
      const uint32_t next_ent = __shfl_down_sync(kFull, ent, 1);
      const uint32_t bal = __ballot_sync(kFull, lane < 31 && succ_live && x != next_ent);
      if (!bal) break;
      const int k = __ffs(bal) - 1;
      const uint32_t xk = __shfl_sync(kFull, x, k);
      if (lane == (uint32_t)k + 1) {
        ent = xk;
        x = resolve_seg<BW, HW>(C, ent, a, b, spec, spec_x, bits, ctab, NC);
      }
    }
    const uint32_t cnt = bits.count();
    uint32_t cinc = cnt;
#pragma unroll
    for (int q = 1; q < 32; q <<= 1) {
      const uint32_t u = __shfl_up_sync(kFull, cinc, q);
      if (lane >= (uint32_t)q) cinc += u;
    }
    const uint32_t c_tot = __shfl_sync(kFull, cinc, 31);
    uint32_t ekey = 0xFFFFFFFFu, nrec = 0;
    {
      uint32_t e = cinc - cnt;
#pragma unroll
      for (int k = 0; k < BW; ++k) {
        uint32_t m = bits.w[k];
        while (m) {
          const uint32_t oo = a + k * 32 + (__ffs(m) - 1);
          m &= m - 1;
          s_off[e] = (uint16_t)oo;
          const uint32_t w0 = C[oo], w1 = C[oo + 1];
          const uint32_t c = w1 & 0xFFFFu;
          const bool ext = (w0 & kExtBit) != 0;
          const uint32_t r = ctab[c < NC ? c : NC];
          const uint32_t sz = HW + (ext ? 2u : 0u) + row_fixedw(r) + (((w1 >> 16) + 3u) >> 2);
          const uint32_t code = oo + HW > W ? THAPI_E_TRUNCATED
                                : ((w0 >> 28) != 0 || c >= NC || (ext && (w0 & kDeltaMask) != 0)) ? THAPI_E_FORMAT
                                : oo + sz > W ? THAPI_E_TRUNCATED : 0u;
          if (code) ekey = min(ekey, (e << 3) | code);
          const uint32_t kd = row_kind(r);
          nrec += (!code && (kd == kEntry || kd == kExit)) ? 1u : 0u;
          ++e;
        }
      }
    }
    __syncwarp();
    const uint32_t gkey = __reduce_min_sync(kFull, ekey);
    if (gkey != 0xFFFFFFFFu || c_tot != d.nev) {
      if (lane == 0)
        atomicMin(p.content_err, gkey != 0xFFFFFFFFu ? err_key(d.pk, gkey >> 3, gkey & 7u)
                                                     : err_key(d.pk, c_tot, THAPI_E_FORMAT));
      __syncwarp();
      continue;
    }
    const uint32_t nrec_p = __reduce_add_sync(kFull, nrec);
    if (lane == 0 && nrec_p) atomicAdd(p.count, (unsigned long long)nrec_p);
    const uint64_t rbase = p.pc_base[w];  // the packet's events at their positions
    const uint32_t host = p.stream_host[d.stream];
    uint64_t tcur = d.tsb;
    uint32_t rank_e = 0;
    for (uint32_t e0 = 0; e0 < c_tot; e0 += 32) {
      const uint32_t e = e0 + lane;
      const bool act = e < c_tot;
      const uint32_t oo = act ? s_off[e] : W;
      const uint32_t w0 = C[oo], w1 = C[oo + 1];
      const bool ext = act && (w0 & kExtBit) != 0;
      const uint32_t c = act ? (w1 & 0xFFFFu) : 0u;
      const uint64_t xts = (uint64_t)C[min(oo + HW, W)] | ((uint64_t)C[min(oo + HW + 1, W)] << 32);
      const uint64_t t =
          ts_op(TsM{1u, tcur}, scan_ts(TsM{ext ? 1u : 0u, !act ? 0ull : ext ? xts : (w0 & kDeltaMask)}, lane)).v;
      tcur = __shfl_sync(kFull, t, 31);
      const uint64_t r = act ? p.classes[c] : 0ull;
      const uint32_t kd = act ? cls_kind(r) : kSample;
      const bool is_e = kd == kEntry, is_x = kd == kExit;
      const uint32_t eb = __ballot_sync(kFull, is_e);
      if (act) {
        tmin = min(tmin, t);
        tmax = max(tmax, t);
        if (!is_e && !is_x) ++n_other;
      }
      if (act && !is_e && !is_x) {  // no call event: the position holds kPcNone
        PcRec rec{};
        rec.kind = kPcNone;
        if (rbase + e < p.cap) p.rec[rbase + e] = rec;
      }
      if (is_e || is_x) {
        const uint32_t base = oo + HW + (ext ? 2u : 0u);
        const int32_t rw = cls_resw(r);
        PcRec rec;
        rec.ts = t;
        rec.thread = ((uint64_t)C[oo + 2] << 32) | C[oo + 3];
        rec.host = host;
        rec.slot = (uint32_t)(d.evbase + rank_e + __popc(eb & lt));
        rec.pos = (uint32_t)w;
        rec.func = (uint16_t)cls_func(r);
        rec.kind = (uint8_t)kd;
        rec.err = (is_x && rw >= 0 && C[min(base + rw, W)] != 0) ? 1 : 0;
        if (rbase + e < p.cap) p.rec[rbase + e] = rec;
        if (is_e && p.slots) {  // the entry's slot, invalid until paired
          unsigned long long *q = reinterpret_cast<unsigned long long *>(p.slots + rec.slot);
          q[0] = t;
          q[1] = 0;
          q[2] = 0xFFFFFFFFull;
        }
      }
      rank_e += __popc(eb);
    }
    if (lane == 0) {
      p.sum_nslot[w] = rank_e;
      n_ev += c_tot;
      n_pk += 1;
      n_disc += d.disc;
    }
    __syncwarp();
  }
  for (int off = 16; off > 0; off >>= 1) {
    n_other += __shfl_down_sync(kFull, n_other, off);
    tmin = min(tmin, __shfl_down_sync(kFull, tmin, off));
    tmax = max(tmax, __shfl_down_sync(kFull, tmax, off));
  }
  if (lane == 0) {
    if (n_ev) atomicAdd(&p.diag[dEvents], n_ev);
    if (n_pk) atomicAdd(&p.diag[dPackets], n_pk);
    if (n_disc) atomicAdd(&p.diag[dDiscarded], n_disc);
    if (n_other) atomicAdd(&p.diag[dOther], n_other);
    if (tmin != ~0ull) atomicMin(&p.tminmax[0], (unsigned long long)tmin);
    if (tmax) atomicMax(&p.tminmax[1], (unsigned long long)tmax);
  }
}

template <int BW>
cudaError_t launch_pc(const PcParams &p, uint32_t nw, uint32_t grid, cudaStream_t s) {
  const uint32_t smem = nw * decode_warp_bytes(p.P) + rup((p.n_classes + 1u) * 4u, 16u);
  cudaError_t e = cudaFuncSetAttribute(k_percpu_decode<BW>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  k_percpu_decode<BW><<<grid, nw * 32, smem, s>>>(p, nw);
  count_launches(1);
  return cudaGetLastError();
}

}  // namespace

// Chooses warps per CTA and CTAs per SM for the warp kernel (false: the CTA
// kernel takes every packet of this trace).
bool plan_analyze_warp(uint32_t P, uint32_t n_classes, int smem_optin, int smem_per_sm, WarpPlan *out) {
  if (!warp_bw(P) || n_classes > kClsMax) return false;
  WarpPlan best{};
  for (uint32_t nw = 1; nw <= kMaxWarps; ++nw) {
    const uint32_t smem = wlayout(P, nw, n_classes).total;
    if ((int)smem > smem_optin) break;
    const uint32_t ctas = std::min<uint32_t>(32u / nw, (uint32_t)(smem_per_sm / (int)(smem + 1024)));
    if (ctas * nw > best.ctas_per_sm * best.nw) {
      best.nw = nw;
      best.ctas_per_sm = ctas;
      best.smem = smem;
    }
  }
  if (!best.nw) return false;
  *out = best;
  return true;
}

cudaError_t launch_analyze_warp(const AnalyzeParams &p, const WarpPlan &wp, uint32_t grid, cudaStream_t s,
                                unsigned *status) {
  switch (warp_bw(p.P)) {
    case 2: return launch_w<2>(p, wp, grid, s, status);
    case 3: return launch_w<3>(p, wp, grid, s, status);
    case 5: return launch_w<5>(p, wp, grid, s, status);
    case 9: return launch_w<9>(p, wp, grid, s, status);
    default: return cudaErrorInvalidValue;
  }
}

uint64_t analyze_warp_frontier_slack(uint64_t warps) { return warps * kChunk; }

// Warps per CTA of the decode kernel (0: not supported for this packet size).
uint32_t decode_warps(uint32_t P, uint32_t n_classes, int smem_optin) {
  if (!warp_bw(P) || n_classes > kClsMax) return 0;
  const uint32_t fixed = rup((n_classes + 1u) * 4u, 16u), per = decode_warp_bytes(P);
  if ((uint32_t)smem_optin < fixed + per) return 0;
  return std::min<uint32_t>(kDecodeWarps, ((uint32_t)smem_optin - fixed) / per);
}

cudaError_t launch_percpu_decode(const PcParams &p, uint32_t nw, uint32_t grid, cudaStream_t s) {
  switch (warp_bw(p.P)) {
    case 2: return launch_pc<2>(p, nw, grid, s);
    case 3: return launch_pc<3>(p, nw, grid, s);
    case 5: return launch_pc<5>(p, nw, grid, s);
    case 9: return launch_pc<9>(p, nw, grid, s);
    default: return cudaErrorInvalidValue;
  }
}

cudaError_t launch_decode_warp(const DecodeParams &p, uint32_t nw, uint32_t grid, cudaStream_t s) {
  switch (warp_bw(p.P)) {
    case 2: return launch_dw<2>(p, nw, grid, s);
    case 3: return launch_dw<3>(p, nw, grid, s);
    case 5: return launch_dw<5>(p, nw, grid, s);
    case 9: return launch_dw<9>(p, nw, grid, s);
    default: return cudaErrorInvalidValue;
  }
}

namespace {

// A packet's cost in events: its events plus the boundary walk, stitch and
// compaction, which take about as long as pairing kPacketCost events.
constexpr uint64_t kPacketCost = 384;

__global__ void k_cost_split(const uint64_t *evbase, uint64_t n, uint64_t total_events, uint32_t grid,
                             uint32_t *run_start) {
  const uint32_t c = blockIdx.x * blockDim.x + threadIdx.x;
  if (c > grid) return;
  if (c == grid) {
    run_start[c] = (uint32_t)n;
    return;
  }
  const uint64_t total = total_events + kPacketCost * n;
  const uint64_t target = total / grid * c + total % grid * c / grid;
  uint64_t lo = 0, hi = n;  // first i with evbase[i] + kPacketCost * i >= target
  while (lo < hi) {
    const uint64_t mid = (lo + hi) / 2;
    if (evbase[mid] + kPacketCost * mid < target)
      lo = mid + 1;
    else
      hi = mid;
  }
  run_start[c] = (uint32_t)lo;
}

}  // namespace

void launch_cost_split(const uint64_t *evbase, uint64_t n, uint64_t total_events, uint32_t grid, uint32_t *run_start,
                       cudaStream_t s) {
  k_cost_split<<<(grid + 1 + 127) / 128, 128, 0, s>>>(evbase, n, total_events, grid, run_start);
  count_launches(1);
}

}  // namespace thapi

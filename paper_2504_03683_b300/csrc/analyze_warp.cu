// analyze_warp.cu — decode + in-packet pairing + tally, one warp per packet.
//
// A CTA holds NW independent warps that share the class table.  The CTA
// takes a contiguous run of the stream-ordered packet list and its warps take
// the run's packets in turn.  Pairs are tallied with fire-and-forget global
// reductions on the (group, function) cells: on this part those cost the SM
// less than shared-memory atomics, whose latency sits on the decode chain.  Each warp stages its packet
// with a TMA bulk copy (mbarrier completion) and then works on it alone:
//
//  1. boundaries: every lane walks a 32*BW-word segment speculatively from
//     the segment start, marking the offsets it visits; the warp stitches
//     the segments (a lane assumes its entry offset is its predecessor's
//     speculative exit; the first lane whose exit breaks that assumption
//     hands its successor the right entry, one ballot round per such lane).
//     The marks are then exactly the event starts of the chain from offset 0.
//  2. the event offsets are compacted and dealt out in equal runs, one run per
//     lane, so that every lane decodes the same number of events (stored
//     transposed: the i-th event of every lane's run sits in one 64-byte row);
//  3. validation and per-lane summaries (entries, timestamp monoid, depth
//     monoid, stack slots used), then warp shuffle scans of the summaries;
//  4. decode with a per-lane call stack: entries are pushed, exits pop the
//     lane's own entries (pairs are tallied and their interval slots written
//     at once), exits on an empty lane stack are kept as lane-pending;
//  5. merge of the lane frontiers with the bracket monoid
//     (p1,o1).(p2,o2) = (p1 + max(p2-o1,0), o2 + max(o1-p2,0)): the k-th
//     pending exit of lane i pops height A_i-1-k, held by the latest earlier
//     lane whose base is <= that height (found from per-height ballots);
//     what no lane of the packet pops is the packet's frontier (pending exits,
//     open entries), resolved across packets by frontier.cu.
// Packets with more than kEvMax events, or whose lanes need more than kStack
// stack slots, are appended to the fallback list for the CTA kernel.
#include <algorithm>

#include "device_util.cuh"
#include "internal.cuh"

namespace thapi {

namespace {
using namespace dev;

constexpr int kStack = 12;             // lane stack slots (pending exits below open entries)
constexpr uint32_t kEvMax = 1024;      // events of one packet the warp path takes
constexpr uint32_t kClsMax = 4096;     // class rows held in shared memory
constexpr uint32_t kHMax = 64;         // heights with a precomputed owner mask
constexpr uint32_t kChunk = 2048;      // frontier items grabbed per global atomic
constexpr uint32_t kMaxWarps = 16;     // warps per CTA

__host__ __device__ inline uint32_t rup(uint32_t v, uint32_t a) { return (v + a - 1u) / a * a; }

struct WLayout {
  uint32_t off_stk, off_off, off_bpc, off_hm, off_bar, warp_bytes;  // within one warp's block
  uint32_t off_ctab, off_cfn, total;                                // CTA-wide
};

__host__ __device__ inline WLayout wlayout(uint32_t P, uint32_t NW, uint32_t NC) {
  WLayout L;
  uint32_t o = rup(P + 48u, 128u);  // packet (header + content) and a zeroed tail
  L.off_stk = o;
  o += kStack * 32u * 16u;  // slot timestamps, slot metadata
  L.off_off = o;
  o += kEvMax * 2u;
  L.off_bpc = o;
  o += 32u * 4u;
  L.off_hm = o;
  o += kHMax * 4u;
  L.off_bar = o;
  o += 16u;
  L.warp_bytes = rup(o, 128u);
  o = L.warp_bytes * NW;
  L.off_ctab = o;
  o += rup((NC + 1u) * 4u, 16u);
  L.off_cfn = o;
  o += rup(NC * 2u, 16u);
  L.total = rup(o, 128u);
  return L;
}

// Shared-memory class row: fixed words (14 bits) | kind << 14 (3) | (result word + 1) << 17 (15).
__device__ __forceinline__ uint32_t row_fixedw(uint32_t r) { return r & 0x3FFFu; }
__device__ __forceinline__ uint32_t row_kind(uint32_t r) { return (r >> 14) & 7u; }
__device__ __forceinline__ int32_t row_resw(uint32_t r) { return (int32_t)(r >> 17) - 1; }

// Event chain step from word offset o; class ids out of range step one word.
__device__ __forceinline__ uint32_t step(const uint32_t *C, uint32_t o, const uint32_t *ctab, uint32_t NC) {
  const uint32_t w0 = C[o], w1 = C[o + 1];
  const uint32_t c = w1 & 0xFFFFu;
  const bool ok = c < NC;
  const uint32_t r = ctab[ok ? c : NC];
  const uint32_t len = 2u + ((w0 >> 26) & 2u) + row_fixedw(r) + (((w1 >> 16) + 3u) >> 2);
  return o + (ok ? len : 1u);
}

// Walks from o while o < b, marking the offsets visited; with STOP, returns at
// the first offset already marked in `stop`.
template <bool STOP, int BW>
__device__ __forceinline__ uint32_t walk(const uint32_t *C, uint32_t o, uint32_t a, uint32_t b, const Bits<BW> &stop,
                                         Bits<BW> &marks, const uint32_t *ctab, uint32_t NC) {
  while (o < b) {
    if (STOP && stop.test(o - a)) return o;
    marks.set(o - a);
    o = step(C, o, ctab, NC);
  }
  return o;
}

// (p, o) bracket monoid
__device__ __forceinline__ void bm(uint32_t &p1, uint32_t &o1, uint32_t p2, uint32_t o2) {
  const uint32_t np = p1 + (p2 > o1 ? p2 - o1 : 0u);
  const uint32_t no = o2 + (o1 > p2 ? o1 - p2 : 0u);
  p1 = np;
  o1 = no;
}

// Interval slot, written as three 8-byte words.
__device__ __forceinline__ void put_interval(thapi_interval *dst, uint64_t start, uint64_t end, uint32_t np,
                                             uint32_t fn, uint32_t lvl, uint32_t flags) {
  unsigned long long *q = reinterpret_cast<unsigned long long *>(dst);
  q[0] = start;
  q[1] = end;
  q[2] = (unsigned long long)np | ((unsigned long long)fn << 32) | ((unsigned long long)lvl << 48) |
         ((unsigned long long)flags << 56);
}

// Open-entry slot metadata: func | rank << 16 | level << 32 | pending-before << 40.
// Pending-exit slot metadata: func | error << 16.
__device__ __forceinline__ uint64_t open_meta(uint32_t fn, uint32_t rank, uint32_t lvl, uint32_t np) {
  return (uint64_t)fn | ((uint64_t)rank << 16) | ((uint64_t)lvl << 32) | ((uint64_t)np << 40);
}

template <int BW>
__global__ void __launch_bounds__(kMaxWarps * 32) k_analyze_warp(AnalyzeParams p, uint32_t NW, unsigned int *status) {
  extern __shared__ __align__(128) uint8_t sm[];
  constexpr uint32_t SEGW = 32u * BW;
  const int lane = threadIdx.x & 31;
  const uint32_t warp = threadIdx.x >> 5;
  const uint32_t F = p.n_funcs;
  const uint32_t NC = p.n_classes;
  const WLayout L = wlayout(p.P, NW, NC);
  uint8_t *wb = sm + warp * L.warp_bytes;
  uint8_t *buf = wb;
  uint32_t *C = reinterpret_cast<uint32_t *>(buf + kPacketHeader);
  uint64_t *stk_ts = reinterpret_cast<uint64_t *>(wb + L.off_stk);
  uint64_t *stk_md = stk_ts + kStack * 32;
  uint16_t *s_off = reinterpret_cast<uint16_t *>(wb + L.off_off);
  uint32_t *s_bpc = reinterpret_cast<uint32_t *>(wb + L.off_bpc);
  uint32_t *s_hm = reinterpret_cast<uint32_t *>(wb + L.off_hm);
  uint64_t *bar = reinterpret_cast<uint64_t *>(wb + L.off_bar);
  uint32_t *ctab = reinterpret_cast<uint32_t *>(sm + L.off_ctab);
  uint16_t *cfn = reinterpret_cast<uint16_t *>(sm + L.off_cfn);

  const uint64_t w_begin = (uint64_t)blockIdx.x * p.per_cta;
  const uint64_t w_end = (w_begin + p.per_cta < p.n_order) ? w_begin + p.per_cta : p.n_order;
  if (w_begin >= w_end) return;  // uniform over the CTA
  auto pos_of = [&](uint64_t w) -> uint64_t { return p.poslist ? p.poslist[w] : w; };

  for (uint32_t c = threadIdx.x; c <= NC; c += blockDim.x) {
    if (c < NC) {
      const uint64_t r = p.classes[c];
      ctab[c] = cls_fixedw(r) | (cls_kind(r) << 14) | ((uint32_t)(cls_resw(r) + 1) << 17);
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
    bulk_copy_g2s(buf, p.packets + (uint64_t)d.pk * p.P, bytes, bar);
  };

  uint64_t fr_base = 0;
  uint32_t fr_left = 0;  // lane 0: current frontier chunk
  unsigned long long n_mismatch = 0, n_other = 0, n_pairs = 0, n_events = 0, n_disc = 0, n_pk = 0, n_slots = 0;
  uint64_t tmin = ~0ull, tmax = 0;
  uint32_t phase = 0;
  bool issued = false;  // a copy is in flight into buf
  bool timed_out = false;

  uint64_t w = w_begin + warp;
  PkDesc dcur{}, dnext{};
  if (w < w_end) {
    dcur = load_desc(p.desc + pos_of(w));
    dnext = dcur;
    if (w + NW < w_end) dnext = load_desc(p.desc + pos_of(w + NW));
    if (lane == 0) issue(dcur);
    issued = true;
  }
  __syncwarp();

  for (; w < w_end; w += NW) {
    const PkDesc d = dcur;
    const uint64_t pos = pos_of(w);
    const bool has_next = w + NW < w_end;
    dcur = dnext;  // next packet's descriptor (its copy is issued once the buffer is free)
    if (w + 2 * NW < w_end) dnext = load_desc(p.desc + pos_of(w + 2 * NW));
    const bool ok_wait = mbar_wait_bounded(bar, phase);
    if (__any_sync(0xffffffffu, !ok_wait)) {
      timed_out = true;
      break;
    }
    phase ^= 1u;
    issued = false;
    const uint32_t W = d.content >> 2;
    if (lane < 4) C[W + lane] = 0;
    __syncwarp();

    // ---- 1. boundaries
    const uint32_t a = (uint32_t)lane * SEGW;
    const uint32_t b = min(a + SEGW, W);
    Bits<BW> spec;
    spec.clear();
    const uint32_t spec_x = a < b ? walk<false, BW>(C, a, a, b, spec, spec, ctab, NC) : a;
    Bits<BW> bits;
    auto resolve = [&](uint32_t y) -> uint32_t {
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
      const uint32_t m = walk<true, BW>(C, y, a, b, spec, walked, ctab, NC);
      if (m < b) {
        bits = spec;
        bits.keep_from(m - a);
        bits.merge(walked);
        return spec_x;
      }
      bits = walked;
      return m;
    };
    const bool succ_live = a + SEGW < W;
    uint32_t ent = __shfl_up_sync(0xffffffffu, spec_x, 1);
    if (lane == 0) ent = 0;
    uint32_t x = resolve(ent);
    for (int r = 0; r < 32; ++r) {
      const uint32_t next_ent = __shfl_down_sync(0xffffffffu, ent, 1);
      const uint32_t bal = __ballot_sync(0xffffffffu, lane < 31 && succ_live && x != next_ent);
      if (!bal) break;
      const int k = __ffs(bal) - 1;
      const uint32_t xk = __shfl_sync(0xffffffffu, x, k);
      if (lane == k + 1) {
        ent = xk;
        x = resolve(ent);
      }
    }

    // ---- 2. compact the event offsets
    const uint32_t cnt = bits.count();
    uint32_t cinc = cnt;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const uint32_t u = __shfl_up_sync(0xffffffffu, cinc, o);
      if (lane >= o) cinc += u;
    }
    const uint32_t c_tot = __shfl_sync(0xffffffffu, cinc, 31);
    bool fallback = c_tot > kEvMax || d.nev > kEvMax;
    bool bad = false;
    uint32_t e0 = 0, e1 = 0;
    if (!fallback) {
      // event e is the (e % per)-th of lane e / per's run: s_off[(e % per) * 32 + e / per]
      const uint32_t per = (c_tot + 31u) >> 5;
      const uint32_t inv = per ? (65536u + per - 1u) / per : 0u;  // e / per = (e * inv) >> 16 for e < 1024
      uint32_t e = cinc - cnt;
#pragma unroll
      for (int k = 0; k < BW; ++k) {
        uint32_t m = bits.w[k];
        while (m) {
          const uint32_t q = (e * inv) >> 16;
          s_off[(e - q * per) * 32 + q] = (uint16_t)(a + k * 32 + (__ffs(m) - 1));
          m &= m - 1;
          ++e;
        }
      }
      e0 = min((uint32_t)lane * per, c_tot);
      e1 = min(e0 + per, c_tot);
    }
    __syncwarp();

    // ---- 3. validation + lane summaries over events [e0, e1)
    uint32_t n_entry = 0;
    TsM tsum{0, 0};
    DM dsum{0, 0};
    int slots_used = 0;
    uint32_t ekey = 0xFFFFFFFFu;  // event index << 3 | code of the first bad event
    for (uint32_t e = e0; e < e1; ++e) {
      const uint32_t oo = s_off[(e - e0) * 32 + (uint32_t)lane];
      const uint32_t w0 = C[oo], w1 = C[oo + 1];
      const uint32_t c = w1 & 0xFFFFu;
      const bool ext = (w0 & kExtBit) != 0;
      const uint32_t r = ctab[c < NC ? c : NC];
      const uint32_t sz = 2u + (ext ? 2u : 0u) + row_fixedw(r) + (((w1 >> 16) + 3u) >> 2);
      uint32_t code = 0;
      if (oo + 2 > W)
        code = THAPI_E_TRUNCATED;
      else if ((w0 >> 28) != 0 || c >= NC || (ext && (w0 & kDeltaMask) != 0))
        code = THAPI_E_FORMAT;
      else if (oo + sz > W)
        code = THAPI_E_TRUNCATED;
      if (code) {
        if (ekey == 0xFFFFFFFFu) ekey = (e << 3) | code;
      } else {
        const uint32_t kd = row_kind(r);
        const int dv = kd == kEntry ? 1 : (kd == kExit ? -1 : 0);
        n_entry += kd == kEntry ? 1u : 0u;
        dsum.s += dv;
        dsum.m = min(dsum.m, dsum.s);
        slots_used = max(slots_used, dsum.s - 2 * dsum.m);  // pending exits + open entries
        if (ext) {
          tsum.has = 1;
          tsum.v = (uint64_t)C[oo + 2] | ((uint64_t)C[oo + 3] << 32);
        } else {
          tsum.v += w0 & kDeltaMask;
        }
      }
    }
    // warp scans (exclusive) of entries, timestamps, depth
    uint32_t ei = n_entry;
    TsM ti = tsum;
    DM di = dsum;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const uint32_t ue = __shfl_up_sync(0xffffffffu, ei, o);
      const uint32_t uh = __shfl_up_sync(0xffffffffu, ti.has, o);
      const uint64_t uv = __shfl_up_sync(0xffffffffu, ti.v, o);
      const int us = __shfl_up_sync(0xffffffffu, di.s, o);
      const int um = __shfl_up_sync(0xffffffffu, di.m, o);
      if (lane >= o) {
        ei += ue;
        ti = ts_op(TsM{uh, uv}, ti);
        di = d_op(DM{us, um}, di);
      }
    }
    const uint32_t e_tot = __shfl_sync(0xffffffffu, ei, 31);
    const int dtot_s = __shfl_sync(0xffffffffu, di.s, 31), dtot_m = __shfl_sync(0xffffffffu, di.m, 31);
    uint32_t e_ex = __shfl_up_sync(0xffffffffu, ei, 1);
    uint32_t hex = __shfl_up_sync(0xffffffffu, ti.has, 1);
    uint64_t vex = __shfl_up_sync(0xffffffffu, ti.v, 1);
    int sex = __shfl_up_sync(0xffffffffu, di.s, 1), mex = __shfl_up_sync(0xffffffffu, di.m, 1);
    if (lane == 0) {
      e_ex = 0;
      hex = 0;
      vex = 0;
      sex = 0;
      mex = 0;
    }
    const uint32_t gkey = __reduce_min_sync(0xffffffffu, ekey);
    if (!fallback) {
      bad = gkey != 0xFFFFFFFFu || c_tot != d.nev;
      fallback = !bad && __any_sync(0xffffffffu, slots_used > kStack);
    }
    if (bad || fallback) {
      if (lane == 0) {
        if (bad)
          atomicMin(p.content_err, gkey != 0xFFFFFFFFu ? err_key(d.pk, gkey >> 3, gkey & 7u)
                                                       : err_key(d.pk, c_tot, THAPI_E_FORMAT));
        else  // the CTA kernel takes it
          p.dense_list[atomicAdd(p.dense_count, 1ull)] = (uint32_t)pos;
      }
      __syncwarp();
      if (lane == 0 && has_next) issue(dcur);
      issued = has_next;
      continue;
    }

    // ---- 4. decode with per-lane call stacks
    const uint32_t P_p = (uint32_t)(-dtot_m);
    const uint32_t O_p = (uint32_t)(dtot_s - dtot_m);
    uint64_t fbase = 0;
    if (lane == 0) {
      const uint32_t need = P_p + O_p;
      if (need) {
        if (need > fr_left) {
          const uint32_t grab = need > kChunk ? need : kChunk;
          fr_base = atomicAdd(p.frontier_top, (unsigned long long)grab);
          fr_left = grab;
          if (fr_base + grab > p.frontier_cap) fr_left = 0;  // overflow: the host retries with more room
        }
        if (need <= fr_left) {
          fbase = fr_base;
          fr_base += need;
          fr_left -= need;
        } else {
          fbase = ~0ull;
        }
      }
    }
    fbase = __shfl_sync(0xffffffffu, fbase, 0);
    thapi_interval *const pslots = p.slots ? p.slots + d.evbase : nullptr;
    Cell *const gcells = p.tally + (uint64_t)d.group * F;
    auto tally = [&](uint32_t fn, uint64_t dur, uint32_t err) {
      Cell &cell = gcells[fn];
      atomicAdd(&cell.count, 1ull);
      atomicAdd(&cell.total, (unsigned long long)dur);
      atomicMin(&cell.mn, (unsigned long long)dur);
      atomicMax(&cell.mx, (unsigned long long)dur);
      if (err) atomicAdd(&cell.err, 1ull);
    };
    uint32_t valid = 0, mism = 0;
    // one pair: entry (ets, metadata em) closed by an exit (xts, xfn, xerr)
    auto emit = [&](uint64_t ets, uint64_t em, uint64_t xts, uint32_t xfn, uint32_t xerr) {
      const uint32_t efn = (uint32_t)(em & 0xFFFFu);
      uint32_t flags = 0;
      if (efn == xfn) {
        ++valid;
        flags = kIvValid | xerr;
        tally(xfn, xts - ets, xerr);
      } else {
        ++mism;  // mismatched pair: no interval
      }
      if (pslots)
        put_interval(pslots + ((em >> 16) & 0xFFFFu), ets, xts, (uint32_t)((em >> 40) & 0xFFFFu), efn,
                     (uint32_t)((em >> 32) & 0xFFu), flags);
    };
    uint64_t t = hex ? vex : d.tsb + vex;
    int depth = sex;   // packet-relative depth before the next event
    int runmin = mex;  // packet-relative running minimum of the depth (<= 0)
    uint32_t rank = e_ex;
    uint32_t top = 0, pc = 0;
    bool first = true;
    const uint32_t n_run = e1 - e0;
    uint32_t oo_n = 0, w0_n = 0, w1_n = 0;  // next event of the run, loaded one step ahead
    if (n_run) {
      oo_n = s_off[lane];
      w0_n = C[oo_n];
      w1_n = C[oo_n + 1];
    }
    for (uint32_t i = 0; i < n_run; ++i) {
      const uint32_t oo = oo_n, w0 = w0_n, w1 = w1_n;
      if (i + 1 < n_run) {
        oo_n = s_off[(i + 1) * 32 + (uint32_t)lane];
        w0_n = C[oo_n];
        w1_n = C[oo_n + 1];
      }
      const uint32_t c = w1 & 0xFFFFu;
      const bool ext = (w0 & kExtBit) != 0;
      const uint32_t r = ctab[c];
      const uint32_t kd = row_kind(r);
      const uint32_t fn = cfn[c];
      const uint64_t tn = ext ? ((uint64_t)C[oo + 2] | ((uint64_t)C[oo + 3] << 32)) : t + (w0 & kDeltaMask);
      if (ext || first || tn < t) {  // a new nondecreasing run of timestamps
        if (!first) tmax = max(tmax, t);
        tmin = min(tmin, tn);
        first = false;
      }
      t = tn;
      if (kd == kEntry) {
        const uint32_t si = (pc + top) * 32 + (uint32_t)lane;
        stk_ts[si] = t;
        stk_md[si] = open_meta(fn, rank, (uint32_t)min(depth - runmin, 255), (uint32_t)(-runmin));
        ++top;
        ++rank;
        ++depth;
      } else if (kd == kExit) {
        const int32_t rw = row_resw(r);
        const uint32_t err = (rw >= 0 && C[oo + 2 + (ext ? 2 : 0) + rw] != 0) ? 1u : 0u;
        --depth;
        runmin = min(runmin, depth);
        if (top) {
          --top;
          const uint32_t si = (pc + top) * 32 + (uint32_t)lane;
          emit(stk_ts[si], stk_md[si], t, fn, err);
        } else {
          const uint32_t si = pc * 32 + (uint32_t)lane;
          stk_ts[si] = t;
          stk_md[si] = (uint64_t)fn | ((uint64_t)err << 16);
          ++pc;
        }
      } else {
        ++n_other;
      }
    }
    if (!first) tmax = max(tmax, t);
    __syncwarp();
    // the packet bytes are no longer needed: stage the next packet now
    if (lane == 0 && has_next) issue(dcur);
    issued = has_next;

    // ---- 5. warp merge of the lane frontiers
    uint32_t sp = pc, so = top;  // inclusive bracket-monoid scan over lanes
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const uint32_t up = __shfl_up_sync(0xffffffffu, sp, o);
      const uint32_t uo = __shfl_up_sync(0xffffffffu, so, o);
      if (lane >= o) {
        uint32_t tp = up, to = uo;
        bm(tp, to, sp, so);
        sp = tp;
        so = to;
      }
    }
    uint32_t pb = __shfl_up_sync(0xffffffffu, sp, 1), A = __shfl_up_sync(0xffffffffu, so, 1);
    if (lane == 0) {
      pb = 0;
      A = 0;
    }
    const uint32_t base = A > pc ? A - pc : 0u;
    s_bpc[lane] = base | (pc << 16);
    uint32_t later;  // min base of the lanes after me
    {
      uint32_t suf = base;
#pragma unroll
      for (int o = 1; o < 32; o <<= 1) {
        const uint32_t u = __shfl_down_sync(0xffffffffu, suf, o);
        if (lane + o < 32) suf = min(suf, u);
      }
      later = __shfl_down_sync(0xffffffffu, suf, 1);
      if (lane == 31) later = 0xFFFFFFFFu;
    }
    // owner masks: bit j of s_hm[h] is set when lane j's base is <= h
    const uint32_t hq = __reduce_max_sync(0xffffffffu, pc ? A : 0u);
    const bool masks = hq <= kHMax;
    if (masks)
      for (uint32_t h = 0; h < hq; ++h) {
        const uint32_t m = __ballot_sync(0xffffffffu, base <= h);
        if (lane == 0) s_hm[h] = m;
      }
    __syncwarp();
    // my pending exits: pop earlier lanes' opens, the rest leave the packet
    for (uint32_t k = 0; k < pc; ++k) {
      const uint32_t si = k * 32 + (uint32_t)lane;
      const uint64_t xts = stk_ts[si];
      const uint64_t xm = stk_md[si];
      const uint32_t xfn = (uint32_t)(xm & 0xFFFFu), xerr = (uint32_t)((xm >> 16) & 1u);
      if (k < A) {
        const uint32_t h = A - 1 - k;
        int j;
        if (masks) {
          j = 31 - __clz(s_hm[h] & ((1u << lane) - 1u));
        } else {
          j = lane - 1;
          while (j > 0 && (s_bpc[j] & 0xFFFFu) > h) --j;
        }
        const uint32_t bj = s_bpc[j];
        const uint32_t it = ((bj >> 16) + h - (bj & 0xFFFFu)) * 32 + (uint32_t)j;
        emit(stk_ts[it], stk_md[it], xts, xfn, xerr);
      } else if (fbase != ~0ull) {
        Frontier fr;
        fr.ts = xts;
        fr.aux = xerr;
        fr.func = (uint16_t)xfn;
        fr.flags = 0;
        p.frontier[fbase + pb + (k - A)] = fr;
      }
    }
    // my opens that no later lane pops leave the packet
    for (uint32_t i = 0; i < top; ++i) {
      const uint32_t h = base + i;
      if (h >= later) break;
      const uint32_t si = (pc + i) * 32 + (uint32_t)lane;
      const uint64_t ots = stk_ts[si];
      const uint64_t om = stk_md[si];
      const uint32_t orank = (uint32_t)((om >> 16) & 0xFFFFu);
      if (fbase != ~0ull) {
        Frontier fr;
        fr.ts = ots;
        fr.aux = pslots ? orank : 0xFFFFFFFFu;
        fr.func = (uint16_t)(om & 0xFFFFu);
        fr.flags = 0;
        p.frontier[fbase + P_p + h] = fr;
      }
      if (pslots)
        put_interval(pslots + orank, ots, 0, (uint32_t)((om >> 40) & 0xFFFFu), (uint32_t)(om & 0xFFFFu),
                     (uint32_t)((om >> 32) & 0xFFu), kIvOpen);
    }
    n_mismatch += mism;
    n_pairs += valid;
    const uint32_t vsum = __reduce_add_sync(0xffffffffu, valid);
    if (lane == 0) {
      p.sum_pend[pos] = P_p;
      p.sum_open[pos] = O_p;
      p.sum_fbase[pos] = fbase;
      p.sum_nslot[pos] = e_tot;
      p.sum_nvalid[pos] = vsum;
      n_events += c_tot;
      if (p.slots) n_slots += e_tot;
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
    n_mismatch += __shfl_down_sync(0xffffffffu, n_mismatch, off);
    n_other += __shfl_down_sync(0xffffffffu, n_other, off);
    n_pairs += __shfl_down_sync(0xffffffffu, n_pairs, off);
    tmin = min(tmin, __shfl_down_sync(0xffffffffu, tmin, off));
    tmax = max(tmax, __shfl_down_sync(0xffffffffu, tmax, off));
  }
  if (lane == 0) {
    if (n_mismatch) atomicAdd(&p.diag[dMismatch], n_mismatch);
    if (n_other) atomicAdd(&p.diag[dOther], n_other);
    if (n_pairs) atomicAdd(&p.diag[dPairs], n_pairs);
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
  auto fn = k_analyze_warp<BW>;
  cudaError_t e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)wp.smem);
  if (e != cudaSuccess) return e;
  fn<<<grid, wp.nw * 32, wp.smem, s>>>(p, wp.nw, status);
  count_launches(1);
  return cudaGetLastError();
}

int warp_bw(uint32_t P) {
  const uint32_t wmax = (P - kPacketHeader) / 4;
  if (wmax <= 32u * 32) return 1;
  if (wmax <= 64u * 32) return 2;
  if (wmax <= 128u * 32) return 4;
  if (wmax <= 256u * 32) return 8;
  return 0;
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
    case 1: return launch_w<1>(p, wp, grid, s, status);
    case 2: return launch_w<2>(p, wp, grid, s, status);
    case 4: return launch_w<4>(p, wp, grid, s, status);
    case 8: return launch_w<8>(p, wp, grid, s, status);
    default: return cudaErrorInvalidValue;
  }
}

uint64_t analyze_warp_frontier_slack(uint64_t warps) { return warps * kChunk; }

}  // namespace thapi

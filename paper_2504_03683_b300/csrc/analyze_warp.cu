// analyze_warp.cu — decode + in-packet pairing + tally, one warp per packet.
//
// Each persistent CTA is one warp and walks a contiguous run of the
// stream-ordered packet list; the next packet is staged with a TMA bulk copy
// (mbarrier completion) as soon as the current packet's bytes are decoded.
// Every lane owns a 32*BW-word segment of the packet:
//
//  1. boundaries: each lane walks its segment speculatively from the segment
//     start (marking the offsets it visits), then the warp stitches the
//     segments: a lane assumes its entry offset is its predecessor's
//     speculative exit; the first lane whose exit breaks that assumption
//     hands its successor the right entry (one ballot round per such lane).
//     The marks are then exactly the event starts of the chain from offset 0.
//  2. validation and per-lane summaries (events, entries, timestamp monoid,
//     depth monoid, deepest local stack), then warp shuffle scans: each lane
//     learns its first event index, timestamp and depth.
//  3. decode with a per-lane call stack: entries are pushed, exits pop the
//     lane's own entries (pairs are tallied and their interval slots written
//     at once); exits on an empty lane stack are lane-pending, entries left
//     are lane-open.
//  4. warp merge of the lane frontiers with the bracket monoid
//     (p1,o1).(p2,o2) = (p1 + max(p2-o1,0), o2 + max(o1-p2,0)): the k-th
//     pending exit of lane j pops height A_j-1-k, held by the latest earlier
//     lane whose base is <= that height; what no lane of the packet pops
//     becomes the packet's frontier (pending exits, open entries) for
//     frontier.cu.
// Packets whose lane stacks would exceed kStack entries go to the CTA kernel
// of analyze.cu (pushed on the fallback list).
#include "device_util.cuh"
#include "internal.cuh"

namespace thapi {

namespace {
using namespace dev;

constexpr int kStack = 8;                 // per-lane stack / pending capacity
constexpr uint32_t kChunk = 2048;         // frontier items grabbed per global atomic
constexpr int kTallySmemMax = 512;

struct WLayout {
  uint32_t off_buf, off_ots, off_pts, off_ofn, off_orank, off_onp, off_pfn, off_olvl, off_perr, off_base, off_tally,
      total;
};

__host__ __device__ inline WLayout wlayout(uint32_t P, uint32_t n_funcs, bool tally_smem) {
  WLayout L;
  uint32_t o = 16;  // mbarrier
  L.off_buf = 128;
  o = L.off_buf + P + 48;  // packet + zeroed tail
  o = (o + 15u) & ~15u;
  L.off_ots = o;
  o += 32 * kStack * 8;
  L.off_pts = o;
  o += 32 * kStack * 8;
  L.off_ofn = o;
  o += 32 * kStack * 2;
  L.off_orank = o;
  o += 32 * kStack * 2;
  L.off_onp = o;
  o += 32 * kStack * 2;
  L.off_pfn = o;
  o += 32 * kStack * 2;
  L.off_olvl = o;
  o += 32 * kStack;
  L.off_perr = o;
  o += 32 * kStack;
  L.off_base = o;
  o += 32 * 4;
  o = (o + 15u) & ~15u;
  L.off_tally = o;
  if (tally_smem) o += n_funcs * 24 + 16;
  L.total = (o + 127u) & ~127u;
  return L;
}

// Event chain step from offset o (unknown class ids step one word).
__device__ __forceinline__ uint32_t step_from(const uint32_t *C, uint32_t o, const uint64_t *cls, uint32_t ncls) {
  const uint32_t w0 = C[o], w1 = C[o + 1];
  const uint32_t c = w1 & 0xFFFFu;
  if (c >= ncls) return o + 1;
  return o + 2 + ((w0 >> 26) & 2u) + cls_fixedw(__ldg(cls + c)) + (((w1 >> 16) + 3u) >> 2);
}

template <int BW>
__device__ __forceinline__ uint32_t walk(const uint32_t *C, uint32_t o, uint32_t a, uint32_t b, const Bits<BW> *stop,
                                         Bits<BW> &marks, const uint64_t *cls, uint32_t ncls) {
  while (o < b) {
    if (stop && stop->test(o - a)) return o;
    marks.set(o - a);
    o = step_from(C, o, cls, ncls);
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

template <int BW, bool TALLY_SMEM>
__global__ void __launch_bounds__(32) k_analyze_warp(AnalyzeParams p, unsigned int *status) {
  extern __shared__ __align__(128) uint8_t sm[];
  constexpr uint32_t SEGW = 32u * BW;
  const int lane = threadIdx.x;
  const uint32_t F = p.n_funcs;
  const uint32_t NC = p.n_classes;
  const WLayout L = wlayout(p.P, F, TALLY_SMEM);
  uint64_t *bar = reinterpret_cast<uint64_t *>(sm);
  uint8_t *buf = sm + L.off_buf;
  uint32_t *C = reinterpret_cast<uint32_t *>(buf + kPacketHeader);
  uint64_t *o_ts = reinterpret_cast<uint64_t *>(sm + L.off_ots);
  uint64_t *p_ts = reinterpret_cast<uint64_t *>(sm + L.off_pts);
  uint16_t *o_fn = reinterpret_cast<uint16_t *>(sm + L.off_ofn);
  uint16_t *o_rank = reinterpret_cast<uint16_t *>(sm + L.off_orank);
  uint16_t *o_np = reinterpret_cast<uint16_t *>(sm + L.off_onp);
  uint16_t *p_fn = reinterpret_cast<uint16_t *>(sm + L.off_pfn);
  uint8_t *o_lvl = sm + L.off_olvl;
  uint8_t *p_err = sm + L.off_perr;
  uint32_t *s_base = reinterpret_cast<uint32_t *>(sm + L.off_base);
  uint32_t *t_cnt = reinterpret_cast<uint32_t *>(sm + L.off_tally);
  uint32_t *t_err = t_cnt + F;
  uint32_t *t_mn = t_err + F;
  uint32_t *t_mx = t_mn + F;
  unsigned long long *t_tot = reinterpret_cast<unsigned long long *>(sm + L.off_tally + ((F * 16u + 15u) & ~15u));

  const uint64_t w_begin = (uint64_t)blockIdx.x * p.per_cta;
  const uint64_t w_end = (w_begin + p.per_cta < p.n_order) ? w_begin + p.per_cta : p.n_order;
  if (w_begin >= w_end) return;
  auto pos_of = [&](uint64_t w) -> uint64_t { return p.poslist ? p.poslist[w] : w; };

  if (TALLY_SMEM)
    for (uint32_t f = lane; f < F; f += 32) {
      t_cnt[f] = 0;
      t_err[f] = 0;
      t_mn[f] = 0xFFFFFFFFu;
      t_mx[f] = 0;
      t_tot[f] = 0;
    }
  auto issue = [&](const PkDesc &d) {
    const uint32_t bytes = align16(kPacketHeader + d.content);
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    mbar_expect_tx(bar, bytes);
    bulk_copy_g2s(buf, p.packets + (uint64_t)d.pk * p.P, bytes, bar);
  };
  PkDesc dcur = load_desc(p.desc + pos_of(w_begin));
  PkDesc dnext = dcur;
  if (w_begin + 1 < w_end) dnext = load_desc(p.desc + pos_of(w_begin + 1));
  if (lane == 0) {
    mbar_init(bar, 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    issue(dcur);
  }
  __syncwarp();

  uint64_t fr_base = 0;
  uint32_t fr_left = 0;  // lane 0: current frontier chunk
  unsigned long long n_mismatch = 0, n_other = 0, n_pairs = 0, n_events = 0, n_disc = 0, n_pk = 0, n_slots = 0;
  uint64_t tmin = ~0ull, tmax = 0;
  uint32_t phase = 0;
  bool issued = true;  // a copy is in flight into buf
  bool timed_out = false;

  for (uint64_t w = w_begin; w < w_end; ++w) {
    const PkDesc d = dcur;
    const uint64_t pos = pos_of(w);
    const bool has_next = w + 1 < w_end;
    dcur = dnext;  // next packet's descriptor (issued below once the buffer is free)
    if (w + 2 < w_end) dnext = load_desc(p.desc + pos_of(w + 2));
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
    const uint32_t spec_x = a < b ? walk<BW>(C, a, a, b, nullptr, spec, p.classes, NC) : a;
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
      const uint32_t m = walk<BW>(C, y, a, b, &spec, walked, p.classes, NC);
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

    // ---- 2. validation + lane summaries
    const uint32_t cnt = bits.count();
    uint32_t n_entry = 0;
    TsM tsum{0, 0};
    DM dsum{0, 0};
    int maxh = 0;
    uint32_t ekey = 0xFFFFFFFFu;  // local index << 3 | code of the first bad event
    {
      uint32_t local = 0;
#pragma unroll
      for (int k = 0; k < BW; ++k) {
        uint32_t m = bits.w[k];
        while (m) {
          const uint32_t oo = a + k * 32 + (__ffs(m) - 1);
          m &= m - 1;
          uint32_t code = 0;
          const uint32_t w0 = C[oo], w1 = C[oo + 1];
          const uint32_t c = w1 & 0xFFFFu;
          uint64_t cr = 0;
          const bool ext = (w0 & kExtBit) != 0;
          if (oo + 2 > W) {
            code = THAPI_E_TRUNCATED;
          } else if ((w0 >> 28) != 0 || c >= NC || (ext && (w0 & kDeltaMask) != 0)) {
            code = THAPI_E_FORMAT;
          } else {
            cr = __ldg(p.classes + c);
            const uint32_t sz = 2 + (ext ? 2 : 0) + cls_fixedw(cr) + (((w1 >> 16) + 3u) >> 2);
            if (oo + sz > W) code = THAPI_E_TRUNCATED;
          }
          if (code) {
            if (ekey == 0xFFFFFFFFu) ekey = (local << 3) | code;
          } else {
            const uint32_t kd = cls_kind(cr);
            const int e = kd == kEntry ? 1 : (kd == kExit ? -1 : 0);
            n_entry += kd == kEntry ? 1u : 0u;
            dsum.s += e;
            dsum.m = min(dsum.m, dsum.s);
            maxh = max(maxh, dsum.s - dsum.m);
            if (ext) {
              tsum.has = 1;
              tsum.v = (uint64_t)C[oo + 2] | ((uint64_t)C[oo + 3] << 32);
            } else {
              tsum.v += w0 & kDeltaMask;
            }
          }
          ++local;
        }
      }
    }
    // warp scans (exclusive) of counts, timestamps, depth
    uint32_t ci = cnt | (n_entry << 16);
    TsM ti = tsum;
    DM di = dsum;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const uint32_t uc = __shfl_up_sync(0xffffffffu, ci, o);
      const uint32_t uh = __shfl_up_sync(0xffffffffu, ti.has, o);
      const uint64_t uv = __shfl_up_sync(0xffffffffu, ti.v, o);
      const int us = __shfl_up_sync(0xffffffffu, di.s, o);
      const int um = __shfl_up_sync(0xffffffffu, di.m, o);
      if (lane >= o) {
        ci += uc;
        ti = ts_op(TsM{uh, uv}, ti);
        di = d_op(DM{us, um}, di);
      }
    }
    const uint32_t c_tot2 = __shfl_sync(0xffffffffu, ci, 31);
    const int dtot_s = __shfl_sync(0xffffffffu, di.s, 31), dtot_m = __shfl_sync(0xffffffffu, di.m, 31);
    uint32_t cex2 = __shfl_up_sync(0xffffffffu, ci, 1);
    uint32_t hex = __shfl_up_sync(0xffffffffu, ti.has, 1);
    uint64_t vex = __shfl_up_sync(0xffffffffu, ti.v, 1);
    int sex = __shfl_up_sync(0xffffffffu, di.s, 1), mex = __shfl_up_sync(0xffffffffu, di.m, 1);
    if (lane == 0) {
      cex2 = 0;
      hex = 0;
      vex = 0;
      sex = 0;
      mex = 0;
    }
    const uint32_t c_ex = cex2 & 0xFFFFu, e_ex = cex2 >> 16;
    const uint32_t c_tot = c_tot2 & 0xFFFFu, e_tot = c_tot2 >> 16;
    const uint32_t gkey = __reduce_min_sync(0xffffffffu, ekey == 0xFFFFFFFFu ? 0xFFFFFFFFu : ekey + (c_ex << 3));
    const bool counts_ok = c_tot == d.nev;
    const bool deep = __any_sync(0xffffffffu, maxh > kStack || -dsum.m > kStack);
    const bool bad = gkey != 0xFFFFFFFFu || !counts_ok;
    if (bad || deep) {
      if (lane == 0) {
        if (bad)
          atomicMin(p.content_err, gkey != 0xFFFFFFFFu ? err_key(d.pk, gkey >> 3, gkey & 7u)
                                                       : err_key(d.pk, c_tot, THAPI_E_FORMAT));
        else  // lane stacks too small for this packet: the CTA kernel takes it
          p.dense_list[atomicAdd(p.dense_count, 1ull)] = (uint32_t)pos;
      }
      __syncwarp();
      if (lane == 0 && has_next) issue(dcur);
      issued = has_next;
    } else {

    // ---- 3. decode with per-lane call stacks
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
    const TsM t_ex = TsM{hex, vex};
    uint64_t t = t_ex.has ? t_ex.v : d.tsb + t_ex.v;
    int depth = sex;  // packet-relative depth before the next event
    int runmin = mex;  // packet-relative running minimum of the depth (<= 0)
    uint32_t rank = e_ex;
    uint32_t top = 0, pc = 0;
    uint32_t valid = 0, mism = 0;
    const uint32_t sb = (uint32_t)lane;  // stack entry i of this lane lives at i * 32 + lane
#pragma unroll
    for (int kk = 0; kk < BW; ++kk) {
      uint32_t m = bits.w[kk];
      while (m) {
        const uint32_t oo = a + kk * 32 + (__ffs(m) - 1);
        m &= m - 1;
        const uint32_t w0 = C[oo], w1 = C[oo + 1];
        const bool ext = (w0 & kExtBit) != 0;
        const uint64_t cr = __ldg(p.classes + (w1 & 0xFFFFu));
        const uint32_t kd = cls_kind(cr);
        const uint32_t fn = cls_func(cr);
        t = ext ? ((uint64_t)C[oo + 2] | ((uint64_t)C[oo + 3] << 32)) : t + (w0 & kDeltaMask);
        tmin = min(tmin, t);
        tmax = max(tmax, t);
        if (kd == kEntry) {
          o_ts[top * 32 + sb] = t;
          o_fn[top * 32 + sb] = (uint16_t)fn;
          o_rank[top * 32 + sb] = (uint16_t)rank;
          o_lvl[top * 32 + sb] = (uint8_t)min(depth - runmin, 255);
          o_np[top * 32 + sb] = (uint16_t)(-runmin);
          ++top;
          ++rank;
          ++depth;
        } else if (kd == kExit) {
          const int32_t rw = cls_resw(cr);
          const uint32_t err = (rw >= 0 && C[oo + 2 + (ext ? 2 : 0) + rw] != 0) ? 1u : 0u;
          --depth;
          runmin = min(runmin, depth);
          if (top) {
            --top;
            const uint64_t ets = o_ts[top * 32 + sb];
            const uint32_t efn = o_fn[top * 32 + sb];
            thapi_interval iv;
            iv.start_ns = ets;
            iv.end_ns = t;
            iv.stream_id = o_np[top * 32 + sb];
            iv.func_id = (uint16_t)efn;
            iv.level = o_lvl[top * 32 + sb];
            if (efn == fn) {
              ++valid;
              iv.flags = (uint8_t)(kIvValid | err);
              const uint64_t dur = t - ets;
              if (TALLY_SMEM && dur < (1ull << 32)) {
                atomicAdd(&t_cnt[fn], 1u);
                atomicAdd(&t_tot[fn], (unsigned long long)dur);
                atomicMin(&t_mn[fn], (uint32_t)dur);
                atomicMax(&t_mx[fn], (uint32_t)dur);
                if (err) atomicAdd(&t_err[fn], 1u);
              } else {
                Cell &cell = p.tally[(uint64_t)d.group * F + fn];
                atomicAdd(&cell.count, 1ull);
                atomicAdd(&cell.total, (unsigned long long)dur);
                atomicMin(&cell.mn, (unsigned long long)dur);
                atomicMax(&cell.mx, (unsigned long long)dur);
                if (err) atomicAdd(&cell.err, 1ull);
              }
            } else {
              iv.flags = 0;  // mismatched pair: no interval
              ++mism;
            }
            if (p.slots) p.slots[d.evbase + o_rank[top * 32 + sb]] = iv;
          } else {
            p_ts[pc * 32 + sb] = t;
            p_fn[pc * 32 + sb] = (uint16_t)fn;
            p_err[pc * 32 + sb] = (uint8_t)err;
            ++pc;
          }
        } else {
          ++n_other;
        }
      }
    }
    __syncwarp();
    // the packet bytes are no longer needed: stage the next packet now
    if (lane == 0 && has_next) issue(dcur);
    issued = has_next;

    // ---- 4. warp merge of the lane frontiers
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
    s_base[lane] = base;
    uint32_t later = base;  // min base of the lanes after me
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
    __syncwarp();
    // my pending exits: pop earlier lanes' opens, the rest leave the packet
    for (uint32_t k = 0; k < pc; ++k) {
      const uint64_t xts = p_ts[k * 32 + sb];
      const uint32_t xfn = p_fn[k * 32 + sb];
      const uint32_t xerr = p_err[k * 32 + sb];
      if (k < A) {
        const uint32_t h = A - 1 - k;
        int j = lane - 1;
        while (j > 0 && s_base[j] > h) --j;
        const uint32_t it = (h - s_base[j]) * 32 + (uint32_t)j;
        const uint64_t ets = o_ts[it];
        const uint32_t efn = o_fn[it];
        thapi_interval iv;
        iv.start_ns = ets;
        iv.end_ns = xts;
        iv.stream_id = o_np[it];
        iv.func_id = (uint16_t)efn;
        iv.level = o_lvl[it];
        if (efn == xfn) {
          ++valid;
          iv.flags = (uint8_t)(kIvValid | xerr);
          const uint64_t dur = xts - ets;
          if (TALLY_SMEM && dur < (1ull << 32)) {
            atomicAdd(&t_cnt[xfn], 1u);
            atomicAdd(&t_tot[xfn], (unsigned long long)dur);
            atomicMin(&t_mn[xfn], (uint32_t)dur);
            atomicMax(&t_mx[xfn], (uint32_t)dur);
            if (xerr) atomicAdd(&t_err[xfn], 1u);
          } else {
            Cell &cell = p.tally[(uint64_t)d.group * F + xfn];
            atomicAdd(&cell.count, 1ull);
            atomicAdd(&cell.total, (unsigned long long)dur);
            atomicMin(&cell.mn, (unsigned long long)dur);
            atomicMax(&cell.mx, (unsigned long long)dur);
            if (xerr) atomicAdd(&cell.err, 1ull);
          }
        } else {
          iv.flags = 0;
          ++mism;
        }
        if (p.slots) p.slots[d.evbase + o_rank[it]] = iv;
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
      const uint32_t it = i * 32 + sb;
      if (fbase != ~0ull) {
        Frontier fr;
        fr.ts = o_ts[it];
        fr.aux = p.slots ? (uint32_t)o_rank[it] : 0xFFFFFFFFu;
        fr.func = o_fn[it];
        fr.flags = 0;
        p.frontier[fbase + P_p + h] = fr;
      }
      if (p.slots) {
        thapi_interval iv;
        iv.start_ns = o_ts[it];
        iv.end_ns = 0;
        iv.stream_id = o_np[it];
        iv.func_id = o_fn[it];
        iv.level = o_lvl[it];
        iv.flags = kIvOpen;
        p.slots[d.evbase + o_rank[it]] = iv;
      }
    }
    n_mismatch += mism;
    const uint32_t vsum = __reduce_add_sync(0xffffffffu, valid);
    n_pairs += valid;
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
    }  // analysed in the warp
    // ---- 5. flush the lane-shared tally when the stream changes
    if (TALLY_SMEM && (!has_next || dcur.stream != d.stream)) {
      __syncwarp();
      for (uint32_t f = lane; f < F; f += 32) {
        const uint32_t c = t_cnt[f];
        if (c) {
          Cell &cell = p.tally[(uint64_t)d.group * F + f];
          atomicAdd(&cell.count, (unsigned long long)c);
          atomicAdd(&cell.total, t_tot[f]);
          atomicMin(&cell.mn, (unsigned long long)t_mn[f]);
          atomicMax(&cell.mx, (unsigned long long)t_mx[f]);
          if (t_err[f]) atomicAdd(&cell.err, (unsigned long long)t_err[f]);
          t_cnt[f] = 0;
          t_err[f] = 0;
          t_mn[f] = 0xFFFFFFFFu;
          t_mx[f] = 0;
          t_tot[f] = 0;
        }
      }
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
    atomicAdd(&p.diag[dEvents], n_events);
    atomicAdd(&p.diag[dDiscarded], n_disc);
    atomicAdd(&p.diag[dPackets], n_pk);
    if (n_slots && p.slots_written) atomicAdd(p.slots_written, n_slots);
  }
}

template <int BW, bool TS>
cudaError_t launch_w(const AnalyzeParams &p, uint32_t grid, uint32_t smem, cudaStream_t s, unsigned *status) {
  auto fn = k_analyze_warp<BW, TS>;
  cudaError_t e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  fn<<<grid, 32, smem, s>>>(p, status);
  count_launches(1);
  return cudaGetLastError();
}

}  // namespace

// Bitmap words per lane for packets of P bytes (0: too large for the warp kernel).
int analyze_warp_bw(uint32_t P) {
  const uint32_t wmax = (P - kPacketHeader) / 4;
  if (wmax <= 32u * 32) return 1;
  if (wmax <= 64u * 32) return 2;
  if (wmax <= 128u * 32) return 4;
  if (wmax <= 256u * 32) return 8;
  return 0;
}

uint32_t analyze_warp_smem_bytes(uint32_t P, uint32_t n_funcs) {
  return wlayout(P, n_funcs, n_funcs <= kTallySmemMax).total;
}

// One warp per CTA; packets the warp kernel cannot take are appended to
// p.dense_list for the CTA kernel.
cudaError_t launch_analyze_warp(const AnalyzeParams &p, uint32_t grid, cudaStream_t s, unsigned *status) {
  const bool ts = p.n_funcs <= kTallySmemMax;
  const uint32_t smem = analyze_warp_smem_bytes(p.P, p.n_funcs);
  switch (analyze_warp_bw(p.P)) {
    case 1: return ts ? launch_w<1, true>(p, grid, smem, s, status) : launch_w<1, false>(p, grid, smem, s, status);
    case 2: return ts ? launch_w<2, true>(p, grid, smem, s, status) : launch_w<2, false>(p, grid, smem, s, status);
    case 4: return ts ? launch_w<4, true>(p, grid, smem, s, status) : launch_w<4, false>(p, grid, smem, s, status);
    case 8: return ts ? launch_w<8, true>(p, grid, smem, s, status) : launch_w<8, false>(p, grid, smem, s, status);
    default: return cudaErrorInvalidValue;
  }
}

}  // namespace thapi

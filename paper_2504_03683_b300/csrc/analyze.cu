// analyze.cu — fused decode + in-packet pairing + tally: one CTA per packet.
//
// Each persistent CTA (128 threads) walks a contiguous run of the
// stream-ordered packet list.  Packets are staged into shared memory with
// cp.async.bulk (TMA bulk copy, mbarrier completion), double-buffered so the
// next packet is in flight while the current one is analysed; the packet
// descriptors are loaded one packet further ahead.
//
//  1. boundaries: event sizes depend on the class and var_len, so finding
//     where events start is a serial chain.  Every thread walks its own
//     32-word segment speculatively from the segment start (crossing runs of
//     unknown class ids in one jump), marking the offsets it visits.  Chains
//     started anywhere merge within a few events, so a thread's speculative
//     exit is usually already the true one.  Stitching: each lane assumes its
//     entry is its predecessor's speculative exit; the first lane whose exit
//     breaks that assumption passes the right entry on (a warp ballot per
//     fix), and a warp whose guessed entry was wrong is redone.  The result is
//     exactly the chain from offset 0.
//  2. validation of every true event in the documented check order, and
//     per-thread summaries.
//  3. decode: timestamps by a CTA-wide scan of (has-absolute, sum) over the
//     deltas seeded with ts_begin (EXT events reset it), depth by a scan of
//     the (sum, min-prefix) monoid over +1 entry / -1 exit; events go to a
//     shared-memory table {ts, post-depth|kind|err, func}.
//  4. in-packet matching: an entry at depth r pairs with the first later event
//     whose post-depth is <= r (necessarily its exit); per-thread and
//     per-warp minima of the depth let a search skip whole thread ranges.
//     Entries with no exit in the packet are "open", exits that reach a new
//     minimum are "pending" — both go to a per-packet frontier that
//     frontier.cu resolves across packets.  Matched pairs are tallied per
//     function in shared memory (a CTA's packets belong to one stream at a
//     time) and flushed to the global (group, function) table when the stream
//     changes.  Every entry gets an interval slot (dense per packet in entry
//     order) for the timeline.
#include "device_util.cuh"
#include "internal.cuh"

namespace thapi {

namespace {
using namespace dev;

constexpr int kT = 128;
constexpr int kWarps = kT / 32;
constexpr int kClsSmemMax = 1024;
constexpr int kTallySmemMax = 512;
constexpr uint32_t kFrontierChunk = 2048;

struct ScanSmem {
  uint32_t c[kWarps];
  TsM t[kWarps];
  DM d[kWarps];
};

// CTA-wide exclusive scans of three per-thread summaries (c: events in the
// low 16 bits + entries in the high 16 bits; timestamps; depth); totals too.
__device__ __forceinline__ void cta_scan3(uint32_t c, TsM t, DM d, uint32_t &c_ex, TsM &t_ex, DM &d_ex, uint32_t &c_tot,
                                          TsM &t_tot, DM &d_tot, ScanSmem &ss) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  uint32_t ci = c;
  TsM ti = t;
  DM di = d;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    uint32_t uc = __shfl_up_sync(0xffffffffu, ci, o);
    uint32_t uh = __shfl_up_sync(0xffffffffu, ti.has, o);
    uint64_t uv = __shfl_up_sync(0xffffffffu, ti.v, o);
    int us = __shfl_up_sync(0xffffffffu, di.s, o);
    int um = __shfl_up_sync(0xffffffffu, di.m, o);
    if (lane >= o) {
      ci += uc;
      ti = ts_op(TsM{uh, uv}, ti);
      di = d_op(DM{us, um}, di);
    }
  }
  if (lane == 31) {
    ss.c[warp] = ci;
    ss.t[warp] = ti;
    ss.d[warp] = di;
  }
  uint32_t ce = __shfl_up_sync(0xffffffffu, ci, 1);
  uint32_t he = __shfl_up_sync(0xffffffffu, ti.has, 1);
  uint64_t ve = __shfl_up_sync(0xffffffffu, ti.v, 1);
  int se = __shfl_up_sync(0xffffffffu, di.s, 1);
  int me = __shfl_up_sync(0xffffffffu, di.m, 1);
  if (lane == 0) {
    ce = 0;
    he = 0;
    ve = 0;
    se = 0;
    me = 0;
  }
  __syncthreads();
  uint32_t cw = 0;
  TsM tw{0, 0};
  DM dw{0, 0};
  c_tot = 0;
  t_tot = TsM{0, 0};
  d_tot = DM{0, 0};
#pragma unroll
  for (int w = 0; w < kWarps; ++w) {
    if (w < warp) {
      cw += ss.c[w];
      tw = ts_op(tw, ss.t[w]);
      dw = d_op(dw, ss.d[w]);
    }
    c_tot += ss.c[w];
    t_tot = ts_op(t_tot, ss.t[w]);
    d_tot = d_op(d_tot, ss.d[w]);
  }
  c_ex = cw + ce;
  t_ex = ts_op(tw, TsM{he, ve});
  d_ex = d_op(dw, DM{se, me});
}

// ---------------------------------------------------------- smem layout
enum Misc { kErrKey = 0, kFbLo, kFbHi, kValid, kNextStream, kMiscWords = 16 };

struct Layout {
  uint32_t buf_bytes, off_meta, off_buf, off_ts, off_dk, off_fn, off_cls, off_tally, off_thr, total;
};

__host__ __device__ inline Layout make_layout(uint32_t P, uint32_t emax, uint32_t stages, uint32_t n_classes,
                                              uint32_t n_funcs, bool cls_smem, bool tally_smem) {
  Layout L;
  L.buf_bytes = P + 32;  // packet + zeroed tail words
  L.off_meta = 16;
  L.off_buf = 128;
  uint32_t o = L.off_buf + stages * L.buf_bytes;
  o = (o + 15u) & ~15u;
  L.off_ts = o;
  o += emax * 8;
  L.off_dk = o;
  o += emax * 4;
  L.off_fn = o;
  o += emax * 2;
  o = (o + 15u) & ~15u;
  L.off_cls = o;
  if (cls_smem) o += n_classes * 8;
  o = (o + 15u) & ~15u;
  L.off_tally = o;
  if (tally_smem) o += n_funcs * 24 + 16;
  o = (o + 15u) & ~15u;
  L.off_thr = o;
  o += kT * 4 /*sx*/ + 2 * kWarps * 4 /*wx*/ + (kT + 4) * 4 /*tk0*/ + kT * 4 /*segmin*/ + kT * 4 /*sufmin*/ +
       kWarps * 4 /*wmin*/ + kMiscWords * 4 + sizeof(ScanSmem) + 64;
  L.total = (o + 127u) & ~127u;
  return L;
}

// Walks the event chain from o inside the segment [a, b): marks o and every
// offset reached by a full event step; runs of unknown class ids are crossed
// one word at a time (jumping to the next candidate).  Stops when the chain
// leaves the segment or, if `stop` is given, lands on one of its offsets.
template <int BW, bool CLS_SMEM>
__device__ __forceinline__ uint32_t seg_walk(const uint32_t *C, uint32_t o, uint32_t a, uint32_t b,
                                             const Bits<BW> &cand, const Bits<BW> *stop, Bits<BW> &marks,
                                             const uint64_t *cls_s, const uint64_t *cls_g) {
  while (o < b) {
    const uint32_t i = o - a;
    if (stop && stop->test(i)) return o;
    marks.set(i);
    if (!cand.test(i)) {
      const uint32_t nxt = cand.next_after(i);
      if (a + nxt >= b) return b;
      o = a + nxt;
    }
    const uint32_t w0 = C[o], w1 = C[o + 1];
    const uint32_t fw = cls_fixedw(class_row<CLS_SMEM>(cls_s, cls_g, w1 & 0xFFFFu));
    o = o + 2 + ((w0 >> 26) & 2u) + fw + (((w1 >> 16) + 3u) >> 2);
  }
  return o;
}

template <int BW, int STAGES, bool CLS_SMEM, bool TALLY_SMEM>
__global__ void __launch_bounds__(kT) k_analyze(AnalyzeParams p, unsigned int *status) {
  extern __shared__ __align__(128) uint8_t sm[];
  constexpr uint32_t SEGW = 32u * BW;
  const int tid = threadIdx.x;
  const int lane = tid & 31, warp = tid >> 5;
  const uint32_t F = p.n_funcs;
  const Layout L = make_layout(p.P, p.emax, STAGES, p.n_classes, F, CLS_SMEM, TALLY_SMEM);
  uint64_t *bar = reinterpret_cast<uint64_t *>(sm);
  PkDesc *meta = reinterpret_cast<PkDesc *>(sm + L.off_meta);
  uint64_t *s_ts = reinterpret_cast<uint64_t *>(sm + L.off_ts);
  uint32_t *s_dk = reinterpret_cast<uint32_t *>(sm + L.off_dk);
  uint16_t *s_fn = reinterpret_cast<uint16_t *>(sm + L.off_fn);
  uint64_t *s_cls = reinterpret_cast<uint64_t *>(sm + L.off_cls);
  uint32_t *t_cnt = reinterpret_cast<uint32_t *>(sm + L.off_tally);
  uint32_t *t_err = t_cnt + F;
  uint32_t *t_mn = t_err + F;
  uint32_t *t_mx = t_mn + F;
  unsigned long long *t_tot = reinterpret_cast<unsigned long long *>(sm + L.off_tally + ((F * 16u + 15u) & ~15u));
  uint32_t *s_sx = reinterpret_cast<uint32_t *>(sm + L.off_thr);  // speculative exits
  uint32_t *s_wx = s_sx + kT;                                       // warp exits, double-buffered
  uint32_t *s_tk0 = s_wx + 2 * kWarps;                              // first event of each thread
  int *s_segmin = reinterpret_cast<int *>(s_tk0 + kT + 4);           // min post-depth per thread
  int *s_sufmin = s_segmin + kT;                                    // suffix min within the warp
  int *s_wmin = s_sufmin + kT;                                      // min per warp
  uint32_t *s_misc = reinterpret_cast<uint32_t *>(s_wmin + kWarps);
  ScanSmem &ss = *reinterpret_cast<ScanSmem *>(s_misc + kMiscWords);

  const uint64_t w_begin = (uint64_t)blockIdx.x * p.per_cta;
  const uint64_t w_end = (w_begin + p.per_cta < p.n_order) ? w_begin + p.per_cta : p.n_order;
  if (w_begin >= w_end) return;
  auto pos_of = [&](uint64_t w) -> uint64_t { return p.poslist ? p.poslist[w] : w; };

  // ---- one-time setup
  if (CLS_SMEM)
    for (uint32_t c = tid; c < p.n_classes; c += kT) s_cls[c] = p.classes[c];
  if (TALLY_SMEM)
    for (uint32_t f = tid; f < F; f += kT) {
      t_cnt[f] = 0;
      t_err[f] = 0;
      t_mn[f] = 0xFFFFFFFFu;
      t_mx[f] = 0;
      t_tot[f] = 0;
    }
  auto issue = [&](const PkDesc &d, int s) {
    const uint32_t bytes = align16(kPacketHeader + d.content);
    uint8_t *dst = sm + L.off_buf + s * L.buf_bytes;
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    mbar_expect_tx(&bar[s], bytes);
    bulk_copy_g2s(dst, packet_at(p.packets, p.pk_addr, d.pk, p.P), bytes, &bar[s]);
  };
  PkDesc dnext;  // thread 0: descriptor of the packet after the one in flight
  uint64_t fr_base = 0;
  uint32_t fr_left = 0;  // thread 0: current frontier chunk
  if (tid == 0) {
    for (int s = 0; s < STAGES; ++s) mbar_init(&bar[s], 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    const PkDesc d0 = load_desc(p.desc + pos_of(w_begin));
    meta[0] = d0;
    issue(d0, 0);
    if (w_begin + 1 < w_end) dnext = load_desc(p.desc + pos_of(w_begin + 1));
  }
  __syncthreads();

  unsigned long long n_mismatch = 0, n_other = 0, n_pairs = 0;
  unsigned long long n_events = 0, n_disc = 0, n_pk = 0, n_slots = 0;
  unsigned long long n_dev = 0;  // DEV_BEGIN / DEV_END events (device pairing on)
  const bool dev_on = p.cmd.counts != nullptr;  // device-activity records wanted
  uint64_t tmin = ~0ull, tmax = 0;
  uint32_t phase = 0;  // bit s = parity expected next on bar[s]
  uint32_t pending_mask = 1u;
  bool timed_out = false;

  for (uint64_t w = w_begin, it = 0; w < w_end; ++w, ++it) {
    const int stage = STAGES == 2 ? (int)(it & 1) : 0;
    const bool has_next = w + 1 < w_end;
    if (tid == 0) {
      s_misc[kErrKey] = 0xFFFFFFFFu;
      s_misc[kValid] = 0;
      s_misc[kNextStream] = has_next ? dnext.stream : 0xFFFFFFFFu;
      if (STAGES == 2 && has_next) {
        meta[stage ^ 1] = dnext;
        issue(dnext, stage ^ 1);
        if (w + 2 < w_end) dnext = load_desc(p.desc + pos_of(w + 2));
      }
    }
    if (STAGES == 2 && has_next) pending_mask |= 1u << (stage ^ 1);
    const bool ok_wait = mbar_wait_bounded(&bar[stage], (phase >> stage) & 1u);
    if (__syncthreads_or(!ok_wait)) {
      timed_out = true;
      break;
    }
    phase ^= 1u << stage;
    pending_mask &= ~(1u << stage);

    const PkDesc d = meta[stage];
    const uint64_t pos = pos_of(w);
    const bool dense = p.dense_list && d.nev > p.emax;
    if (dense) {
      if (tid == 0) p.dense_list[atomicAdd(p.dense_count, 1ull)] = (uint32_t)pos;
    } else {
      const uint32_t W = d.content >> 2;
      uint32_t *C = reinterpret_cast<uint32_t *>(sm + L.off_buf + stage * L.buf_bytes + kPacketHeader);
      if (tid < 4) C[W + tid] = 0;
      __syncthreads();

      // ---- 1. event boundaries
      const uint32_t a = (uint32_t)tid * SEGW;
      const uint32_t b = min(a + SEGW, W);
      // candidate words: a chain standing on a word whose class id is unknown
      // steps one word at a time, so it can jump straight to the next candidate
      Bits<BW> cand;
      cand.clear();
#pragma unroll 4
      for (uint32_t k = 0; k < SEGW; ++k) {
        const uint32_t i = (k + (uint32_t)lane) & (SEGW - 1);  // rotated: the lanes of a warp hit distinct banks
        const uint32_t o = a + i;
        if (o < b && (C[o + 1] & 0xFFFFu) < p.n_classes) cand.set(i);
      }
      Bits<BW> spec;
      spec.clear();
      const uint32_t spec_x =
          a < b ? seg_walk<BW, CLS_SMEM>(C, a, a, b, cand, nullptr, spec, s_cls, p.classes) : a;
      s_sx[tid] = spec_x;
      __syncthreads();
      Bits<BW> bits;
      // chain entering my segment at y: walk until it meets my speculative
      // chain (from there both are the same chain) or leaves the segment
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
        const uint32_t m = seg_walk<BW, CLS_SMEM>(C, y, a, b, cand, &spec, walked, s_cls, p.classes);
        if (m < b) {
          bits = spec;
          bits.keep_from(m - a);
          bits.merge(walked);
          return spec_x;
        }
        bits = walked;
        return m;
      };
      // warp stitch: one ballot round per lane whose exit breaks its
      // successor's assumed entry
      const bool succ_live = a + SEGW < W;
      uint32_t ent, x;
      auto warp_resolve = [&](uint32_t E) {
        ent = lane == 0 ? E : s_sx[tid - 1];
        x = resolve(ent);
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
      };
      uint32_t E = warp == 0 ? 0u : s_sx[warp * 32 - 1];
      warp_resolve(E);
      // across warps: redo a warp whose guessed entry was wrong (at most kWarps rounds)
      bool stitch_ok = true;
      for (int r = 0;; ++r) {
        if (r > kWarps + 1) {  // unreachable unless the walk is broken; never spin
          stitch_ok = false;
          break;
        }
        const uint32_t xl = __shfl_sync(0xffffffffu, x, 31);
        if (lane == 0) s_wx[(r & 1) * kWarps + warp] = xl;
        __syncthreads();
        const uint32_t want = warp == 0 ? 0u : s_wx[(r & 1) * kWarps + warp - 1];
        const bool redo = warp > 0 && want != E && (uint32_t)warp * 32u * SEGW < W;
        if (redo) {
          E = want;
          warp_resolve(E);
        }
        if (!__syncthreads_or(redo)) break;
      }

      // ---- 2. validation + per-thread summaries
      const uint32_t cnt = bits.count();
      uint32_t n_entry = 0;
      TsM tsum{0, 0};
      DM dsum{0, 0};
      int err_local = -1;
      uint32_t err_code = 0;
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
            } else if ((w0 >> 28) != 0 || c >= p.n_classes || (ext && (w0 & kDeltaMask) != 0)) {
              code = THAPI_E_FORMAT;
            } else {
              cr = class_row<CLS_SMEM>(s_cls, p.classes, c);
              const uint32_t sz = 2 + (ext ? 2 : 0) + cls_fixedw(cr) + (((w1 >> 16) + 3u) >> 2);
              if (oo + sz > W) code = THAPI_E_TRUNCATED;
            }
            if (code) {
              if (err_local < 0) {
                err_local = (int)local;
                err_code = code;
              }
            } else {
              const uint32_t kd = cls_kind(cr);
              const int e = kd == kEntry ? 1 : (kd == kExit ? -1 : 0);
              // interval slot owners: entries, and DEV_BEGINs carrying a command id
              n_entry += (kd == kEntry || (dev_on && kd == kDevBegin && cls_cmdw(cr) >= 0)) ? 1u : 0u;
              dsum.s += e;
              dsum.m = min(dsum.m, dsum.s);
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
      uint32_t c_ex2, c_tot2;
      TsM t_ex, t_tot_m;
      DM d_ex, d_tot;
      cta_scan3(cnt | (n_entry << 16), tsum, dsum, c_ex2, t_ex, d_ex, c_tot2, t_tot_m, d_tot, ss);
      const uint32_t c_ex = c_ex2 & 0xFFFFu, e_ex = c_ex2 >> 16;
      const uint32_t c_tot = c_tot2 & 0xFFFFu, e_tot = c_tot2 >> 16;
      if (err_local >= 0) atomicMin(&s_misc[kErrKey], ((c_ex + (uint32_t)err_local) << 3) | err_code);
      const bool fits = stitch_ok && c_tot == d.nev && c_tot <= p.emax;
      const uint32_t P_p = (uint32_t)(-d_tot.m);
      const uint32_t O_p = (uint32_t)(d_tot.s - d_tot.m);
      if (fits) {
        if (tid == 0) {
          // frontier room from this CTA's chunk (a global atomic only per chunk)
          const uint32_t need = P_p + O_p;
          uint64_t fb = 0;
          if (need) {
            if (need > fr_left) {
              const uint32_t grab = need > kFrontierChunk ? need : kFrontierChunk;
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
          s_misc[kFbLo] = (uint32_t)fb;
          s_misc[kFbHi] = (uint32_t)(fb >> 32);
        }
        // ---- 3. decode into the shared table
        uint64_t t = t_ex.has ? t_ex.v : d.tsb + t_ex.v;
        int depth = d_ex.s;
        int segmin = 0x7FFFFFFF;
        uint32_t k = c_ex;
        uint32_t orank = e_ex;  // slot of the next slot owner
#pragma unroll
        for (int kk = 0; kk < BW; ++kk) {
          uint32_t m = bits.w[kk];
          while (m) {
            const uint32_t oo = a + kk * 32 + (__ffs(m) - 1);
            m &= m - 1;
            const uint32_t w0 = C[oo], w1 = C[oo + 1];
            const bool ext = (w0 & kExtBit) != 0;
            const uint32_t c = w1 & 0xFFFFu;
            const uint64_t cr = c < p.n_classes ? class_row<CLS_SMEM>(s_cls, p.classes, c) : 0ull;
            const uint32_t kd = cls_kind(cr);
            const uint32_t base = oo + 2 + (ext ? 2 : 0);
            t = ext ? ((uint64_t)C[oo + 2] | ((uint64_t)C[oo + 3] << 32)) : t + (w0 & kDeltaMask);
            depth += kd == kEntry ? 1 : (kd == kExit ? -1 : 0);
            uint32_t err = 0;
            const int32_t rw = cls_resw(cr);
            if (kd == kExit && rw >= 0 && base + (uint32_t)rw < W) err = C[base + rw] != 0 ? 1u : 0u;
            // device-activity record of an event carrying a command id
            uint32_t dev_slot = 0;
            if (dev_on && cls_cmdw(cr) >= 0 && (kd == kEntry || kd == kDevBegin || kd == kDevEnd)) {
              const uint32_t q = min(base + (uint32_t)cls_cmdw(cr), W);
              const uint64_t id = (uint64_t)C[q] | ((uint64_t)C[min(q + 1u, W)] << 32);
              atomicAdd(&p.cmd.hist[((kd == kDevBegin ? 0u : kd == kDevEnd ? 1u : 2u) << p.cmd.part_bits) +
                                    cmd_part(id, p.cmd.part_bits)],
                        1u);
              if (kd == kDevBegin) {
                const unsigned long long at = atomicAdd(&p.cmd.counts[0], 1ull);
                if (at < p.cmd.cap_b) p.cmd.b[at] = CmdBegin{id, t, d.evbase + orank, d.group, (uint32_t)pos};
                if (p.slots) {  // invalid until the device join fills it
                  thapi_interval iv{};
                  iv.start_ns = t;
                  iv.stream_id = 0xFFFFFFFFu;
                  p.slots[d.evbase + orank] = iv;
                }
                dev_slot = 1;
              } else if (kd == kDevEnd) {
                const unsigned long long at = atomicAdd(&p.cmd.counts[1], 1ull);
                if (at < p.cmd.cap_e) p.cmd.e[at] = CmdEnd{id, t};
              } else {
                const unsigned long long at = atomicAdd(&p.cmd.counts[2], 1ull);
                if (at < p.cmd.cap_h) p.cmd.h[at] = CmdHost{id, cls_func(cr), 0u};
              }
            }
            if (dev_on && (kd == kDevBegin || kd == kDevEnd)) ++n_dev;
            if (kd == kEntry || dev_slot) ++orank;
            s_ts[k] = t;
            s_dk[k] = ((uint32_t)depth & 0xFFFFu) | (kd << 16) | (err << 19) | (dev_slot << 20);
            s_fn[k] = (uint16_t)cls_func(cr);
            segmin = min(segmin, depth);
            tmin = min(tmin, t);
            tmax = max(tmax, t);
            ++k;
          }
        }
        s_tk0[tid] = c_ex;
        if (tid == 0) s_tk0[kT] = c_tot;
        segmin = cnt ? segmin : 0x7FFFFFFF;
        s_segmin[tid] = segmin;
        int suf = segmin;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
          const int u = __shfl_down_sync(0xffffffffu, suf, o);
          if (lane + o < 32) suf = min(suf, u);
        }
        s_sufmin[tid] = suf;
        if (lane == 0) s_wmin[warp] = suf;
      }
      __syncthreads();
      const uint32_t ekey = s_misc[kErrKey];
      const bool pk_ok = fits && ekey == 0xFFFFFFFFu;
      if (!pk_ok) {
        if (tid == 0) {
          if (!stitch_ok)
            atomicExch(status, (unsigned)THAPI_E_TIMEOUT);
          else if (ekey != 0xFFFFFFFFu)
            atomicMin(p.content_err, err_key(d.pk, ekey >> 3, ekey & 7u));
          else
            atomicMin(p.content_err, err_key(d.pk, c_tot, THAPI_E_FORMAT));
        }
      } else {
        // ---- 4. match, tally, frontier, interval slots
        const uint64_t fbase = (uint64_t)s_misc[kFbLo] | ((uint64_t)s_misc[kFbHi] << 32);
        const uint32_t k0 = c_ex, k1 = c_ex + cnt;
        const uint32_t wlast = (uint32_t)warp * 32 + 31;
        int mrun = d_ex.m;  // running minimum of the post-depth before event i (<= 0)
        uint32_t rank = e_ex;
        uint32_t valid = 0;
        for (uint32_t i = k0; i < k1; ++i) {
          const uint32_t dk = s_dk[i];
          const uint32_t kd = (dk >> 16) & 7u;
          const int post = post_of(dk);
          if (kd == kEntry) {
            const int r = post - 1;
            // the exit: first later event with post-depth <= r
            int j = -1;
            for (uint32_t q = i + 1; q < k1; ++q)
              if (post_of(s_dk[q]) <= r) {
                j = (int)q;
                break;
              }
            if (j < 0 && (uint32_t)tid < wlast && s_sufmin[tid + 1] <= r) {
              for (uint32_t t2 = tid + 1; t2 <= wlast; ++t2)
                if (s_segmin[t2] <= r) {
                  const uint32_t e2 = s_tk0[t2 + 1];
                  for (uint32_t q = s_tk0[t2]; q < e2; ++q)
                    if (post_of(s_dk[q]) <= r) {
                      j = (int)q;
                      break;
                    }
                  break;
                }
            }
            if (j < 0)
              for (int w2 = warp + 1; w2 < kWarps; ++w2)
                if (s_wmin[w2] <= r) {
                  for (uint32_t t2 = (uint32_t)w2 * 32; t2 < (uint32_t)w2 * 32 + 32; ++t2)
                    if (s_segmin[t2] <= r) {
                      const uint32_t e2 = s_tk0[t2 + 1];
                      for (uint32_t q = s_tk0[t2]; q < e2; ++q)
                        if (post_of(s_dk[q]) <= r) {
                          j = (int)q;
                          break;
                        }
                      break;
                    }
                  break;
                }
            thapi_interval iv;
            iv.start_ns = s_ts[i];
            iv.stream_id = (uint32_t)(-mrun);  // pending exits before this entry (the level is finished later)
            iv.func_id = s_fn[i];
            iv.level = (uint8_t)min(r - mrun, 255);
            if (j < 0) {
              iv.end_ns = 0;
              iv.flags = kIvOpen;
              if (fbase != ~0ull) {
                Frontier fr;
                fr.ts = s_ts[i];
                fr.aux = p.slots ? rank : 0xFFFFFFFFu;
                fr.func = s_fn[i];
                fr.flags = 0;
                p.frontier[fbase + P_p + (uint32_t)(r - d_tot.m)] = fr;
              }
            } else if (s_fn[j] == s_fn[i]) {
              ++valid;
              if (p.side) {  // self time: the exit's position and the entry's exact packet-relative depth
                SelfSlot &ss = p.side[d.evbase + rank];
                ss.exit_pos = d.evbase + (uint32_t)j;
                ss.level = (uint32_t)(r - mrun);
              }
              const uint64_t dur = s_ts[j] - s_ts[i];
              const uint32_t err = (s_dk[j] >> 19) & 1u;
              const uint32_t f = s_fn[i];
              iv.end_ns = s_ts[j];
              iv.flags = (uint8_t)(kIvValid | err);
              if (TALLY_SMEM && dur < (1ull << 32)) {
                atomicAdd(&t_cnt[f], 1u);
                atomicAdd(&t_tot[f], (unsigned long long)dur);
                atomicMin(&t_mn[f], (uint32_t)dur);
                atomicMax(&t_mx[f], (uint32_t)dur);
                if (err) atomicAdd(&t_err[f], 1u);
              } else {
                Cell &cell = p.tally[(uint64_t)d.group * F + f];
                atomicAdd(&cell.count, 1ull);
                atomicAdd(&cell.total, (unsigned long long)dur);
                atomicMin(&cell.mn, (unsigned long long)dur);
                atomicMax(&cell.mx, (unsigned long long)dur);
                if (err) atomicAdd(&cell.err, 1ull);
              }
            } else {
              iv.end_ns = s_ts[j];
              iv.flags = 0;  // mismatched pair: no interval
              ++n_mismatch;
            }
            if (p.slots) p.slots[d.evbase + rank] = iv;
            if (p.side) p.side[d.evbase + rank].entry_pos = d.evbase + i;
            ++rank;
          } else if (kd == kExit) {
            if (post < mrun && fbase != ~0ull) {
              Frontier fr;
              fr.ts = s_ts[i];
              fr.aux = i;
              fr.func = s_fn[i];
              fr.flags = (uint16_t)((dk >> 19) & 1u);
              p.frontier[fbase + (uint32_t)(-post - 1)] = fr;
            }
          } else {
            ++n_other;
            if (dk & (1u << 20)) ++rank;  // a DEV_BEGIN's slot, written above
          }
          mrun = min(mrun, post);
        }
        n_pairs += valid;
        if (valid) atomicAdd(&s_misc[kValid], valid);
      }
      __syncthreads();
      if (pk_ok && tid == 0) {
        p.sum_pend[pos] = P_p;
        p.sum_open[pos] = O_p;
        p.sum_fbase[pos] = (uint64_t)s_misc[kFbLo] | ((uint64_t)s_misc[kFbHi] << 32);
        p.sum_nslot[pos] = e_tot;
        p.sum_nvalid[pos] = s_misc[kValid];
        n_events += c_tot;
        if (p.slots) n_slots += e_tot;
        n_disc += d.disc;
        n_pk += 1;
      }
    }

    // ---- 5. flush the shared tally when the stream changes
    if (TALLY_SMEM) {
      if (s_misc[kNextStream] != d.stream) {
        for (uint32_t f = tid; f < F; f += kT) {
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
    }
    __syncthreads();  // buffers, table and misc words free for the next packet
    if (STAGES == 1 && has_next) {
      if (tid == 0) {
        meta[0] = dnext;
        issue(dnext, 0);
        if (w + 2 < w_end) dnext = load_desc(p.desc + pos_of(w + 2));
      }
      pending_mask |= 1u;
    }
  }

  if (timed_out) {
    // wait (bounded) for copies still in flight into this CTA's buffers, then leave
    for (int s = 0; s < STAGES; ++s)
      if (pending_mask & (1u << s)) (void)mbar_wait_bounded(&bar[s], (phase >> s) & 1u);
    if (tid == 0) atomicExch(status, (unsigned)THAPI_E_TIMEOUT);
  }

  // ---- CTA-level diagnostics
  for (int off = 16; off > 0; off >>= 1) {
    n_mismatch += __shfl_down_sync(0xffffffffu, n_mismatch, off);
    n_other += __shfl_down_sync(0xffffffffu, n_other, off);
    n_pairs += __shfl_down_sync(0xffffffffu, n_pairs, off);
    n_dev += __shfl_down_sync(0xffffffffu, n_dev, off);
    tmin = min(tmin, __shfl_down_sync(0xffffffffu, tmin, off));
    tmax = max(tmax, __shfl_down_sync(0xffffffffu, tmax, off));
  }
  if (lane == 0) {
    if (n_mismatch) atomicAdd(&p.diag[dMismatch], n_mismatch);
    if (n_other) atomicAdd(&p.diag[dOther], n_other);
    if (n_pairs) atomicAdd(&p.diag[dPairs], n_pairs);
    if (n_dev) atomicAdd(&p.diag[dDevEvents], n_dev);
    if (tmin != ~0ull) atomicMin(&p.tminmax[0], (unsigned long long)tmin);
    if (tmax) atomicMax(&p.tminmax[1], (unsigned long long)tmax);
  }
  if (tid == 0) {
    atomicAdd(&p.diag[dEvents], n_events);
    atomicAdd(&p.diag[dDiscarded], n_disc);
    atomicAdd(&p.diag[dPackets], n_pk);
    if (n_slots && p.slots_written) atomicAdd(p.slots_written, n_slots);
  }
}

template <int BW, int STAGES, bool CS, bool TS>
cudaError_t launch_one(const AnalyzeParams &p, uint32_t grid, uint32_t smem, cudaStream_t s, unsigned *status) {
  auto fn = k_analyze<BW, STAGES, CS, TS>;
  cudaError_t e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  fn<<<grid, kT, smem, s>>>(p, status);
  count_launches(1);
  return cudaGetLastError();
}

template <int BW, int STAGES>
cudaError_t launch_bw(const AnalyzeParams &p, bool cs, bool ts, uint32_t grid, uint32_t smem, cudaStream_t s,
                      unsigned *status) {
  if (cs && ts) return launch_one<BW, STAGES, true, true>(p, grid, smem, s, status);
  if (cs) return launch_one<BW, STAGES, true, false>(p, grid, smem, s, status);
  if (ts) return launch_one<BW, STAGES, false, true>(p, grid, smem, s, status);
  return launch_one<BW, STAGES, false, false>(p, grid, smem, s, status);
}

}  // namespace

// Shared-memory bytes of one CTA (host side, for occupancy and admission).
uint32_t analyze_smem_bytes(uint32_t P, uint32_t emax, int stages, uint32_t n_classes, uint32_t n_funcs) {
  Layout L = make_layout(P, emax, (uint32_t)stages, n_classes, n_funcs, n_classes <= kClsSmemMax,
                         n_funcs <= kTallySmemMax);
  return L.total;
}

// Frontier items a launch may leave unused at the end of its CTAs' chunks.
uint64_t analyze_frontier_slack(uint32_t grid) { return (uint64_t)grid * kFrontierChunk; }

// Launches the analysis over p.n_order work items with `grid` CTAs.
cudaError_t launch_analyze(const AnalyzeParams &p, int stages, uint32_t grid, cudaStream_t s, unsigned *status) {
  bool cs = p.n_classes <= kClsSmemMax;
  bool ts = p.n_funcs <= kTallySmemMax;
  uint32_t smem = analyze_smem_bytes(p.P, p.emax, stages, p.n_classes, p.n_funcs);
  uint32_t wmax = (p.P - kPacketHeader) / 4;
  int bw = (int)((wmax + 32u * kT - 1) / (32u * kT));
  if (bw <= 1) bw = 1;
  if (stages == 2) {
    if (bw == 1) return launch_bw<1, 2>(p, cs, ts, grid, smem, s, status);
    if (bw == 2) return launch_bw<2, 2>(p, cs, ts, grid, smem, s, status);
    return launch_bw<4, 2>(p, cs, ts, grid, smem, s, status);
  }
  if (bw == 1) return launch_bw<1, 1>(p, cs, ts, grid, smem, s, status);
  if (bw == 2) return launch_bw<2, 1>(p, cs, ts, grid, smem, s, status);
  return launch_bw<4, 1>(p, cs, ts, grid, smem, s, status);
}

}  // namespace thapi

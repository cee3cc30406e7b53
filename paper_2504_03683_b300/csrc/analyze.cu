// analyze.cu — fused decode + in-packet pairing + tally: one CTA per packet.
//
// Each persistent CTA (128 threads) walks a contiguous run of the
// stream-ordered packet list.  Packets are staged into shared memory with
// cp.async.bulk (TMA bulk copy, mbarrier completion), double-buffered so the
// next packet is in flight while the current one is analysed:
//
//  1. boundaries: event sizes depend on the class and var_len, so finding
//     where events start is a serial chain.  Every thread walks its own
//     32-word segment speculatively from the segment start, marking the
//     offsets it visits in a bitmap; then segments are stitched: a thread
//     whose true entry offset (the previous segment's exit) lies on its chain
//     keeps the chain from there, otherwise it re-walks until the chains
//     merge.  Iterated until no exit changes, the bitmap holds exactly the
//     true event starts (the chain from offset 0).
//  2. validation of every true event in the documented check order.
//  3. decode: timestamps by a CTA-wide scan of (has-absolute, sum) over the
//     deltas seeded with ts_begin (EXT events reset it), depth by a scan of
//     the (sum, min-prefix) monoid over +1 entry / -1 exit; events go to a
//     shared-memory table {ts, post-depth|kind|err, func}.
//  4. in-packet matching: an entry at depth r pairs with the first later event
//     whose post-depth is <= r (necessarily its exit); entries with none are
//     "open", exits that reach a new minimum are "pending" — both go to a
//     per-packet frontier that frontier.cu resolves across packets.  Matched
//     pairs are tallied per function in shared memory (the CTA's packets
//     belong to one stream at a time) and flushed to the global
//     (group, function) table when the stream changes.
//  5. optional interval slots (timeline), dense per packet in entry order.
#include "internal.cuh"

namespace thapi {

namespace {

constexpr int kT = 128;
constexpr int kWarps = kT / 32;
constexpr int kClsSmemMax = 1024;
constexpr int kTallySmemMax = 512;
constexpr uint32_t kWaitLimit = 1u << 22;

__device__ __forceinline__ uint32_t smem_addr(const void *p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void mbar_init(uint64_t *bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_addr(bar)), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_expect_tx(uint64_t *bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_addr(bar)), "r"(bytes)
               : "memory");
}
__device__ __forceinline__ void bulk_copy_g2s(void *dst, const void *src, uint32_t bytes, uint64_t *bar) {
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
          smem_addr(dst)),
      "l"(src), "r"(bytes), "r"(smem_addr(bar))
      : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(uint64_t *bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\tselp.u32 %0, 1, 0, p;\n\t}"
      : "=r"(ok)
      : "r"(smem_addr(bar)), "r"(parity)
      : "memory");
  return ok != 0;
}
__device__ __forceinline__ bool mbar_wait_bounded(uint64_t *bar, uint32_t parity) {
  for (uint32_t it = 0; it < kWaitLimit; ++it)
    if (mbar_try_wait(bar, parity)) return true;
  return false;
}

__device__ __forceinline__ uint32_t align16(uint32_t v) { return (v + 15u) & ~15u; }

// ---------------------------------------------------------------- monoids
struct TsM {
  uint32_t has;
  uint64_t v;
};
__device__ __forceinline__ TsM ts_op(TsM a, TsM b) { return b.has ? b : TsM{a.has, a.v + b.v}; }
struct DM {
  int s, m;  // sum, minimum prefix (including the empty prefix, so m <= 0)
};
__device__ __forceinline__ DM d_op(DM a, DM b) { return DM{a.s + b.s, min(a.m, a.s + b.m)}; }

struct ScanSmem {
  uint32_t c[kWarps];
  TsM t[kWarps];
  DM d[kWarps];
  uint32_t c2[kWarps];
};

// CTA-wide exclusive scans of the three per-thread summaries; totals returned.
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
  // exclusive within the warp
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
  for (int w = 0; w < warp; ++w) {
    cw += ss.c[w];
    tw = ts_op(tw, ss.t[w]);
    dw = d_op(dw, ss.d[w]);
  }
  c_ex = cw + ce;
  t_ex = ts_op(tw, TsM{he, ve});
  d_ex = d_op(dw, DM{se, me});
  c_tot = 0;
  t_tot = TsM{0, 0};
  d_tot = DM{0, 0};
  for (int w = 0; w < kWarps; ++w) {
    c_tot += ss.c[w];
    t_tot = ts_op(t_tot, ss.t[w]);
    d_tot = d_op(d_tot, ss.d[w]);
  }
  __syncthreads();
}

__device__ __forceinline__ uint32_t cta_scan_u32(uint32_t v, uint32_t &tot, ScanSmem &ss) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  uint32_t inc = v;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    uint32_t u = __shfl_up_sync(0xffffffffu, inc, o);
    if (lane >= o) inc += u;
  }
  if (lane == 31) ss.c2[warp] = inc;
  __syncthreads();
  uint32_t base = 0;
  tot = 0;
  for (int w = 0; w < kWarps; ++w) {
    if (w < warp) base += ss.c2[w];
    tot += ss.c2[w];
  }
  __syncthreads();
  return base + inc - v;
}

// ---------------------------------------------------------- smem layout
struct Layout {
  uint32_t buf_bytes, off_buf, off_ts, off_dk, off_fn, off_mt, off_cls, off_tally, off_thr, total;
};

__host__ __device__ inline Layout make_layout(uint32_t P, uint32_t emax, uint32_t stages, uint32_t n_classes,
                                              uint32_t n_funcs, bool cls_smem, bool tally_smem) {
  Layout L;
  L.buf_bytes = P + 32;  // packet + zeroed tail words
  L.off_buf = 64;
  uint32_t o = L.off_buf + stages * L.buf_bytes;
  o = (o + 15u) & ~15u;
  L.off_ts = o;
  o += emax * 8;
  L.off_dk = o;
  o += emax * 4;
  L.off_fn = o;
  o += emax * 2;
  L.off_mt = o;
  o += emax * 2;
  o = (o + 15u) & ~15u;
  L.off_cls = o;
  if (cls_smem) o += n_classes * 8;
  o = (o + 15u) & ~15u;
  L.off_tally = o;
  if (tally_smem) o += n_funcs * 32 + 16;
  o = (o + 15u) & ~15u;
  L.off_thr = o;
  o += kT * 4 /*ex*/ + (kT + 4) * 4 /*tk0*/ + kT * 4 /*segmin*/ + 64 /*misc*/ + sizeof(ScanSmem) + 64;
  L.total = (o + 127u) & ~127u;
  return L;
}

__device__ __forceinline__ int post_of(uint32_t dk) { return (int)(int16_t)(dk & 0xFFFFu); }

template <int BW>
struct Bits {
  uint32_t w[BW];
  __device__ __forceinline__ void clear() {
#pragma unroll
    for (int i = 0; i < BW; ++i) w[i] = 0;
  }
  __device__ __forceinline__ void set(uint32_t i) {
#pragma unroll
    for (int k = 0; k < BW; ++k)
      if ((i >> 5) == (uint32_t)k) w[k] |= 1u << (i & 31);
  }
  __device__ __forceinline__ bool test(uint32_t i) const {
    bool r = false;
#pragma unroll
    for (int k = 0; k < BW; ++k)
      if ((i >> 5) == (uint32_t)k) r = (w[k] >> (i & 31)) & 1u;
    return r;
  }
  // keep bits with index >= i
  __device__ __forceinline__ void keep_from(uint32_t i) {
#pragma unroll
    for (int k = 0; k < BW; ++k) {
      uint32_t lo = (uint32_t)k * 32;
      if (i >= lo + 32)
        w[k] = 0;
      else if (i > lo)
        w[k] &= ~((1u << (i - lo)) - 1u);
    }
  }
  __device__ __forceinline__ uint32_t count() const {
    uint32_t c = 0;
#pragma unroll
    for (int k = 0; k < BW; ++k) c += __popc(w[k]);
    return c;
  }
};

template <bool CLS_SMEM>
__device__ __forceinline__ uint64_t class_row(const uint64_t *cls_s, const uint64_t *cls_g, uint32_t c) {
  if (CLS_SMEM) return cls_s[c];
  return __ldg(cls_g + c);
}

// Next offset of the event chain (same function for speculative and true walks).
template <bool CLS_SMEM>
__device__ __forceinline__ uint32_t chain_next(const uint32_t *C, uint32_t o, const uint64_t *cls_s,
                                               const uint64_t *cls_g, uint32_t n_classes) {
  uint32_t w0 = C[o], w1 = C[o + 1];
  uint32_t c = w1 & 0xFFFFu;
  if (c >= n_classes) return o + 1;
  uint32_t fw = cls_fixedw(class_row<CLS_SMEM>(cls_s, cls_g, c));
  return o + 2 + ((w0 >> 26) & 2u) + fw + (((w1 >> 16) + 3u) >> 2);
}

template <int BW, int STAGES, bool CLS_SMEM, bool TALLY_SMEM>
__global__ void __launch_bounds__(kT) k_analyze(AnalyzeParams p, unsigned int *status) {
  extern __shared__ __align__(128) uint8_t sm[];
  constexpr uint32_t SEGW = 32u * BW;
  const int tid = threadIdx.x;
  const uint32_t F = p.n_funcs;
  const Layout L = make_layout(p.P, p.emax, STAGES, p.n_classes, F, CLS_SMEM, TALLY_SMEM);
  uint64_t *bar = reinterpret_cast<uint64_t *>(sm);
  uint64_t *s_ts = reinterpret_cast<uint64_t *>(sm + L.off_ts);
  uint32_t *s_dk = reinterpret_cast<uint32_t *>(sm + L.off_dk);
  uint16_t *s_fn = reinterpret_cast<uint16_t *>(sm + L.off_fn);
  int16_t *s_mt = reinterpret_cast<int16_t *>(sm + L.off_mt);
  uint64_t *s_cls = reinterpret_cast<uint64_t *>(sm + L.off_cls);
  uint32_t *t_cnt = reinterpret_cast<uint32_t *>(sm + L.off_tally);
  uint32_t *t_err = t_cnt + F;
  unsigned long long *t_tot = reinterpret_cast<unsigned long long *>(sm + L.off_tally + ((F * 8u + 15u) & ~15u));
  unsigned long long *t_mn = t_tot + F;
  unsigned long long *t_mx = t_mn + F;
  uint32_t *s_ex = reinterpret_cast<uint32_t *>(sm + L.off_thr);
  uint32_t *s_tk0 = s_ex + kT;
  int *s_segmin = reinterpret_cast<int *>(s_tk0 + kT + 4);
  uint32_t *s_misc = reinterpret_cast<uint32_t *>(s_segmin + kT);  // [0] ok, [1] err key lo, [2] fbase lo, [3] fbase hi
  ScanSmem &ss = *reinterpret_cast<ScanSmem *>(s_misc + 16);

  const uint64_t w_begin = (uint64_t)blockIdx.x * p.per_cta;
  const uint64_t w_end = (w_begin + p.per_cta < p.n_order) ? w_begin + p.per_cta : p.n_order;
  if (w_begin >= w_end) return;

  // ---- one-time setup
  if (CLS_SMEM)
    for (uint32_t c = tid; c < p.n_classes; c += kT) s_cls[c] = p.classes[c];
  if (TALLY_SMEM)
    for (uint32_t f = tid; f < F; f += kT) {
      t_cnt[f] = 0;
      t_err[f] = 0;
      t_tot[f] = 0;
      t_mn[f] = ~0ull;
      t_mx[f] = 0;
    }
  if (tid == 0) {
    for (int s = 0; s < STAGES; ++s) mbar_init(&bar[s], 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  // dense packets (more events than the SoA holds) go to a second launch
  if (p.dense_list)
    for (uint64_t w = w_begin + tid; w < w_end; w += kT) {
      uint32_t pk = p.order[w];
      if (p.pk_nev[pk] > p.emax) {
        unsigned long long k = atomicAdd(p.dense_count, 1ull);
        p.dense_list[k] = (uint32_t)w;
      }
    }
  __syncthreads();

  auto pos_of = [&](uint64_t w) -> uint64_t { return p.poslist ? p.poslist[w] : w; };
  auto skip = [&](uint64_t w) -> bool { return p.dense_list && p.pk_nev[p.order[w]] > p.emax; };
  auto next_work = [&](uint64_t w) -> uint64_t {
    while (w < w_end && skip(w)) ++w;
    return w;
  };
  auto issue = [&](uint64_t w, int s) {
    uint64_t pos = pos_of(w);
    uint32_t pk = p.order[pos];
    uint32_t bytes = align16(kPacketHeader + p.pk_content[pk]);
    uint8_t *dst = sm + L.off_buf + s * L.buf_bytes;
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    mbar_expect_tx(&bar[s], bytes);
    bulk_copy_g2s(dst, p.packets + (uint64_t)pk * p.P, bytes, &bar[s]);
  };

  // thread-local diagnostics
  unsigned long long n_mismatch = 0, n_other = 0, n_pairs = 0;
  unsigned long long n_events = 0, n_disc = 0, n_pk = 0, n_slots = 0;
  uint64_t tmin = ~0ull, tmax = 0;
  uint32_t phase = 0;  // bit s = parity expected next on bar[s]
  bool timed_out = false;
  int stage = 0;
  uint32_t pending_mask = 0;  // stages with a copy in flight (tracked by every thread identically)

  uint64_t w = next_work(w_begin);
  if (w < w_end) {
    if (tid == 0) issue(w, 0);
    pending_mask |= 1u;
  }
  while (w < w_end) {
    const uint64_t wn = next_work(w + 1);
    if (STAGES == 2 && wn < w_end) {
      if (tid == 0) issue(wn, stage ^ 1);
      pending_mask |= 1u << (stage ^ 1);
    }
    bool ok_wait = mbar_wait_bounded(&bar[stage], (phase >> stage) & 1u);
    if (__syncthreads_or(!ok_wait)) {
      timed_out = true;
      break;
    }
    phase ^= 1u << stage;
    pending_mask &= ~(1u << stage);

    const uint64_t pos = pos_of(w);
    const uint32_t pk = p.order[pos];
    const uint32_t content = p.pk_content[pk];
    const uint32_t nev = p.pk_nev[pk];
    const uint32_t W = content >> 2;
    const uint32_t stream = p.pk_stream[pk];
    const uint32_t group = p.stream_group[stream];
    uint32_t *C = reinterpret_cast<uint32_t *>(sm + L.off_buf + stage * L.buf_bytes + kPacketHeader);
    if (tid < 4) C[W + tid] = 0;
    __syncthreads();

    // ---- 1. speculative segment walks
    const uint32_t a = (uint32_t)tid * SEGW;
    const uint32_t b = min(a + SEGW, W);
    Bits<BW> bits;
    bits.clear();
    uint32_t o = a;
    while (o < b) {
      bits.set(o - a);
      o = chain_next<CLS_SMEM>(C, o, s_cls, p.classes, p.n_classes);
    }
    uint32_t x = max(o, a);
    uint32_t entry = a;
    s_ex[tid] = x;
    // ---- stitch segments until no exit changes (converges in at most kT rounds:
    // after round r the first r segments are final)
    bool stitch_ok = true;
    for (int round = 0;; ++round) {
      if (round > 2 * kT + 2) {  // unreachable unless the walk is broken; never spin
        stitch_ok = false;
        break;
      }
      __syncthreads();
      uint32_t y = tid == 0 ? 0u : s_ex[tid - 1];
      bool changed = false;
      if (y != entry) {
        entry = y;
        uint32_t nx = x;
        if (y >= b) {
          bits.clear();
          nx = y;
        } else if (bits.test(y - a)) {
          bits.keep_from(y - a);
        } else {
          uint32_t m = y;
          while (m < b && !bits.test(m - a)) m = chain_next<CLS_SMEM>(C, m, s_cls, p.classes, p.n_classes);
          if (m < b) {
            bits.keep_from(m - a);
          } else {
            bits.clear();
            nx = m;
          }
          uint32_t q = y;
          while (q < m && q < b) {
            bits.set(q - a);
            q = chain_next<CLS_SMEM>(C, q, s_cls, p.classes, p.n_classes);
          }
        }
        if (nx != x) {
          x = nx;
          changed = true;
        }
      }
      __syncthreads();
      s_ex[tid] = x;
      if (!__syncthreads_or(changed)) break;
    }

    // ---- 2. validation + per-thread summaries
    uint32_t cnt = bits.count();
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
          uint32_t oo = a + k * 32 + (__ffs(m) - 1);
          m &= m - 1;
          uint32_t code = 0;
          uint32_t w0 = C[oo], w1 = C[oo + 1];
          uint32_t c = w1 & 0xFFFFu;
          uint64_t cr = 0;
          bool ext = (w0 & kExtBit) != 0;
          if (oo + 2 > W) {
            code = THAPI_E_TRUNCATED;
          } else if ((w0 >> 28) != 0 || c >= p.n_classes || (ext && (w0 & kDeltaMask) != 0)) {
            code = THAPI_E_FORMAT;
          } else {
            cr = class_row<CLS_SMEM>(s_cls, p.classes, c);
            uint32_t sz = 2 + (ext ? 2 : 0) + cls_fixedw(cr) + (((w1 >> 16) + 3u) >> 2);
            if (oo + sz > W) code = THAPI_E_TRUNCATED;
          }
          if (code) {
            if (err_local < 0) {
              err_local = (int)local;
              err_code = code;
            }
          } else {
            uint32_t kd = cls_kind(cr);
            int e = kd == kEntry ? 1 : (kd == kExit ? -1 : 0);
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
    uint32_t c_ex, c_tot;
    TsM t_ex, t_tot_m;
    DM d_ex, d_tot;
    if (tid == 0) s_misc[1] = 0xFFFFFFFFu;
    cta_scan3(cnt, tsum, dsum, c_ex, t_ex, d_ex, c_tot, t_tot_m, d_tot, ss);
    if (err_local >= 0) atomicMin(&s_misc[1], ((c_ex + (uint32_t)err_local) << 3) | err_code);
    __syncthreads();
    const uint32_t ekey = s_misc[1];
    const bool pk_ok = stitch_ok && ekey == 0xFFFFFFFFu && c_tot == nev && c_tot <= p.emax;
    if (!stitch_ok) {
      if (tid == 0) atomicExch(status, (unsigned)THAPI_E_TIMEOUT);
    } else if (!pk_ok) {
      if (tid == 0) {
        if (ekey != 0xFFFFFFFFu)
          atomicMin(p.content_err, err_key(pk, ekey >> 3, ekey & 7u));
        else
          atomicMin(p.content_err, err_key(pk, c_tot, THAPI_E_FORMAT));
      }
    } else {
      // ---- 3. decode into the shared table
      const uint64_t tsb = p.pk_tsb[pk];
      uint64_t t = t_ex.has ? t_ex.v : tsb + t_ex.v;
      int depth = d_ex.s;
      int segmin = 0x7FFFFFFF;
      uint32_t k = c_ex;
#pragma unroll
      for (int kk = 0; kk < BW; ++kk) {
        uint32_t m = bits.w[kk];
        while (m) {
          uint32_t oo = a + kk * 32 + (__ffs(m) - 1);
          m &= m - 1;
          uint32_t w0 = C[oo], w1 = C[oo + 1];
          bool ext = (w0 & kExtBit) != 0;
          uint64_t cr = class_row<CLS_SMEM>(s_cls, p.classes, w1 & 0xFFFFu);
          uint32_t kd = cls_kind(cr);
          uint32_t base = oo + 2 + (ext ? 2 : 0);
          t = ext ? ((uint64_t)C[oo + 2] | ((uint64_t)C[oo + 3] << 32)) : t + (w0 & kDeltaMask);
          int e = kd == kEntry ? 1 : (kd == kExit ? -1 : 0);
          depth += e;
          uint32_t err = 0;
          int32_t rw = cls_resw(cr);
          if (kd == kExit && rw >= 0) err = C[base + rw] != 0 ? 1u : 0u;
          s_ts[k] = t;
          s_dk[k] = ((uint32_t)depth & 0xFFFFu) | (kd << 16) | (err << 19);
          s_fn[k] = (uint16_t)cls_func(cr);
          segmin = min(segmin, depth);
          tmin = min(tmin, t);
          tmax = max(tmax, t);
          ++k;
        }
      }
      s_tk0[tid] = c_ex;
      if (tid == 0) s_tk0[kT] = c_tot;
      s_segmin[tid] = cnt ? segmin : 0x7FFFFFFF;
      __syncthreads();

      // ---- 4a. in-packet matching and tally
      uint32_t nslot = 0;
      {
        const uint32_t k0 = c_ex, k1 = c_ex + cnt;
        for (uint32_t i = k0; i < k1; ++i) {
          uint32_t dk = s_dk[i];
          uint32_t kd = (dk >> 16) & 7u;
          if (kd == kEntry) {
            int r = post_of(dk) - 1;
            int j = -1;
            for (uint32_t q = i + 1; q < k1; ++q)
              if (post_of(s_dk[q]) <= r) {
                j = (int)q;
                break;
              }
            if (j < 0)
              for (int t2 = tid + 1; t2 < kT && j < 0; ++t2)
                if (s_segmin[t2] <= r) {
                  uint32_t e2 = s_tk0[t2 + 1];
                  for (uint32_t q = s_tk0[t2]; q < e2; ++q)
                    if (post_of(s_dk[q]) <= r) {
                      j = (int)q;
                      break;
                    }
                }
            if (j < 0) {
              s_mt[i] = -1;
              ++nslot;
            } else if (s_fn[j] == s_fn[i]) {
              s_mt[i] = (int16_t)j;
              ++nslot;
              ++n_pairs;
              uint64_t dur = s_ts[j] - s_ts[i];
              uint32_t err = (s_dk[j] >> 19) & 1u;
              uint32_t f = s_fn[i];
              if (TALLY_SMEM) {
                atomicAdd(&t_cnt[f], 1u);
                atomicAdd(&t_tot[f], (unsigned long long)dur);
                atomicMin(&t_mn[f], (unsigned long long)dur);
                atomicMax(&t_mx[f], (unsigned long long)dur);
                if (err) atomicAdd(&t_err[f], 1u);
              } else {
                Cell &cell = p.tally[(uint64_t)group * F + f];
                atomicAdd(&cell.count, 1ull);
                atomicAdd(&cell.total, (unsigned long long)dur);
                atomicMin(&cell.mn, (unsigned long long)dur);
                atomicMax(&cell.mx, (unsigned long long)dur);
                if (err) atomicAdd(&cell.err, 1ull);
              }
            } else {
              s_mt[i] = -2;
              ++n_mismatch;
            }
          } else if (kd != kExit) {
            ++n_other;
          }
        }
      }
      uint32_t slot_tot;
      uint32_t slot_ex = cta_scan_u32(nslot, slot_tot, ss);
      const uint32_t P_p = (uint32_t)(-d_tot.m);
      const uint32_t O_p = (uint32_t)(d_tot.s - d_tot.m);
      if (tid == 0) {
        uint64_t fb = 0;
        if (P_p + O_p) {
          fb = atomicAdd(p.frontier_top, (unsigned long long)(P_p + O_p));
          if (fb + P_p + O_p > p.frontier_cap) fb = ~0ull;  // overflow: host retries with more room
        }
        s_misc[2] = (uint32_t)fb;
        s_misc[3] = (uint32_t)(fb >> 32);
        p.sum_pend[pos] = P_p;
        p.sum_open[pos] = O_p;
        p.sum_fbase[pos] = fb;
        p.sum_nslot[pos] = slot_tot;
        p.sum_nvalid[pos] = slot_tot - O_p;
        n_events += c_tot;
        if (p.slots) n_slots += slot_tot;
        n_disc += p.pk_disc[pk];
        n_pk += 1;
      }
      __syncthreads();
      const uint64_t fbase = (uint64_t)s_misc[2] | ((uint64_t)s_misc[3] << 32);

      // ---- 4b. frontier items and interval slots
      {
        const uint32_t k0 = c_ex, k1 = c_ex + cnt;
        int mrun = d_ex.m;  // running minimum of post-depth before event i (<= 0)
        uint32_t rank = slot_ex;
        const uint64_t sbase = p.evbase[pos];
        for (uint32_t i = k0; i < k1; ++i) {
          uint32_t dk = s_dk[i];
          uint32_t kd = (dk >> 16) & 7u;
          int post = post_of(dk);
          if (kd == kEntry) {
            int mt = s_mt[i];
            if (mt >= -1) {
              int pre = post - 1;
              if (p.slots) {
                thapi_interval iv;
                iv.start_ns = s_ts[i];
                iv.end_ns = mt >= 0 ? s_ts[mt] : 0;
                iv.stream_id = (uint32_t)(-mrun);
                iv.func_id = s_fn[i];
                iv.level = (uint8_t)min(pre - mrun, 255);
                iv.flags = mt >= 0 ? (uint8_t)(kIvValid | ((s_dk[mt] >> 19) & 1u)) : kIvOpen;
                p.slots[sbase + rank] = iv;
              }
              if (mt == -1 && fbase != ~0ull) {
                Frontier fr;
                fr.ts = s_ts[i];
                fr.aux = p.slots ? rank : 0xFFFFFFFFu;
                fr.func = s_fn[i];
                fr.flags = 0;
                p.frontier[fbase + P_p + (uint32_t)(pre - d_tot.m)] = fr;
              }
              ++rank;
            }
          } else if (kd == kExit && post < mrun && fbase != ~0ull) {
            Frontier fr;
            fr.ts = s_ts[i];
            fr.aux = (dk >> 19) & 1u;
            fr.func = s_fn[i];
            fr.flags = 0;
            p.frontier[fbase + (uint32_t)(-post - 1)] = fr;
          }
          mrun = min(mrun, post);
        }
      }
    }
    __syncthreads();

    // ---- 5. flush the shared tally when the stream changes
    if (TALLY_SMEM) {
      bool flush = wn >= w_end || p.pk_stream[p.order[pos_of(wn)]] != stream;
      if (flush) {
        for (uint32_t f = tid; f < F; f += kT) {
          uint32_t c = t_cnt[f];
          if (c) {
            Cell &cell = p.tally[(uint64_t)group * F + f];
            atomicAdd(&cell.count, (unsigned long long)c);
            atomicAdd(&cell.total, t_tot[f]);
            atomicMin(&cell.mn, t_mn[f]);
            atomicMax(&cell.mx, t_mx[f]);
            if (t_err[f]) atomicAdd(&cell.err, (unsigned long long)t_err[f]);
            t_cnt[f] = 0;
            t_err[f] = 0;
            t_tot[f] = 0;
            t_mn[f] = ~0ull;
            t_mx[f] = 0;
          }
        }
        __syncthreads();
      }
    }
    if (STAGES == 1 && wn < w_end) {
      if (tid == 0) issue(wn, 0);
      pending_mask |= 1u;
    }
    if (STAGES == 2) stage ^= 1;
    w = wn;
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
    tmin = min(tmin, __shfl_down_sync(0xffffffffu, tmin, off));
    tmax = max(tmax, __shfl_down_sync(0xffffffffu, tmax, off));
  }
  if ((tid & 31) == 0) {
    if (n_mismatch) atomicAdd(&p.diag[dMismatch], n_mismatch);
    if (n_other) atomicAdd(&p.diag[dOther], n_other);
    if (n_pairs) atomicAdd(&p.diag[dPairs], n_pairs);
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

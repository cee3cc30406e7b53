// device_util.cuh — device helpers shared by the analysis kernels: TMA bulk
// copies with mbarrier completion (bounded waits), the scan monoids, a small
// register bitmap, class-row and packet-descriptor loads.
#pragma once

#include "internal.cuh"

namespace thapi {
namespace dev {

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
__device__ __forceinline__ bool mbar_wait_limit(uint64_t *bar, uint32_t parity, uint32_t limit) {
  for (uint32_t it = 0; it < limit; ++it)
    if (mbar_try_wait(bar, parity)) return true;
  return false;
}
__device__ __forceinline__ bool mbar_wait_bounded(uint64_t *bar, uint32_t parity) {
  return mbar_wait_limit(bar, parity, kWaitLimit);
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

__device__ __forceinline__ int post_of(uint32_t dk) { return (int)(int16_t)(dk & 0xFFFFu); }

template <int BW>
struct Bits {
  uint32_t w[BW];
  __device__ __forceinline__ void clear() {
#pragma unroll
    for (int i = 0; i < BW; ++i) w[i] = 0;
  }
  // set/test take a word-relative offset per word (no index select), so that
  // the words stay in registers
  __device__ __forceinline__ void set(uint32_t i) {
#pragma unroll
    for (int k = 0; k < BW; ++k) {
      const uint32_t d = i - 32u * k;
      w[k] |= d < 32u ? 1u << d : 0u;
    }
  }
  __device__ __forceinline__ bool test(uint32_t i) const {
    uint32_t r = 0;
#pragma unroll
    for (int k = 0; k < BW; ++k) {
      const uint32_t d = i - 32u * k;
      r |= d < 32u ? (w[k] >> d) & 1u : 0u;
    }
    return r != 0;
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
  // smallest set index greater than i, or 32 * BW
  __device__ __forceinline__ uint32_t next_after(uint32_t i) const {
#pragma unroll
    for (int k = 0; k < BW; ++k) {
      const uint32_t lo = (uint32_t)k * 32;
      if (i + 1 >= lo + 32) continue;
      uint32_t m = w[k];
      if (i + 1 > lo) m &= ~((1u << (i + 1 - lo)) - 1u);
      if (m) return lo + (uint32_t)(__ffs(m) - 1);
    }
    return 32u * BW;
  }
  __device__ __forceinline__ void merge(const Bits &o) {
#pragma unroll
    for (int k = 0; k < BW; ++k) w[k] |= o.w[k];
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

__device__ __forceinline__ PkDesc load_desc(const PkDesc *d) {
  PkDesc r;
  const uint4 *s = reinterpret_cast<const uint4 *>(d);
  const uint4 a = __ldg(s), b = __ldg(s + 1), c = __ldg(s + 2);
  r.pk = a.x;
  r.content = a.y;
  r.nev = a.z;
  r.stream = a.w;
  r.group = b.x;
  r.disc = b.y;
  r.pad0 = b.z;
  r.pad1 = b.w;
  r.tsb = (uint64_t)c.x | ((uint64_t)c.y << 32);
  r.evbase = (uint64_t)c.z | ((uint64_t)c.w << 32);
  return r;
}


}  // namespace dev
}  // namespace thapi

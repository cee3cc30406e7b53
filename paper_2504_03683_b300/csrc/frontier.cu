// frontier.cu — entry/exit pairing across packets of one stream.
//
// Each packet leaves P pending exits (exits that pop below its starting
// depth, in order) and O open entries (bottom to top).  Per stream, a warp
// scans the packets with the bracket-matching monoid
//   (p1, o1) . (p2, o2) = (p1 + max(p2 - o1, 0), o2 + max(o1 - p2, 0))
// which gives A = entries open before each packet (the clamped depth carried
// across packets) and, for the whole stream, the unmatched exits (p) and the
// unmatched entries (o).  Then the k-th pending exit of packet i pops level
// L = A_i - 1 - k (k < A_i), whose open entry lives in the latest earlier
// packet q of the stream with base_q = max(A_q - P_q, 0) <= L, at index
// L - base_q of q's opens.  This is the (stream, level) match of the paper's
// interval pairing restated for packets.
#include "internal.cuh"

namespace thapi {

namespace {

__device__ __forceinline__ void mono(uint32_t &p1, uint32_t &o1, uint32_t p2, uint32_t o2) {
  uint32_t np = p1 + (p2 > o1 ? p2 - o1 : 0u);
  uint32_t no = o2 + (o1 > p2 ? o1 - p2 : 0u);
  p1 = np;
  o1 = no;
}

}  // namespace

__global__ void k_frontier_scan(FrontierParams p) {
  const int lane = threadIdx.x & 31;
  const uint64_t warp_global = ((uint64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const uint64_t n_warps = ((uint64_t)gridDim.x * blockDim.x) >> 5;
  for (uint64_t s = warp_global; s < p.n_streams; s += n_warps) {
    const uint32_t first = p.stream_first[s], cnt = p.stream_count[s];
    uint32_t cp = 0, co = 0;  // carry
    for (uint32_t base = 0; base < cnt; base += 32) {
      uint32_t i = first + base + lane;
      bool in = base + lane < cnt;
      uint32_t Pp = in ? p.sum_pend[i] : 0u, Op = in ? p.sum_open[i] : 0u;
      uint32_t ip = Pp, io = Op;  // inclusive within the warp
#pragma unroll
      for (int o = 1; o < 32; o <<= 1) {
        uint32_t up = __shfl_up_sync(0xffffffffu, ip, o);
        uint32_t uo = __shfl_up_sync(0xffffffffu, io, o);
        if (lane >= o) {
          uint32_t tp = up, to = uo;
          mono(tp, to, ip, io);
          ip = tp;
          io = to;
        }
      }
      uint32_t ep = __shfl_up_sync(0xffffffffu, ip, 1), eo = __shfl_up_sync(0xffffffffu, io, 1);
      if (lane == 0) ep = eo = 0;
      uint32_t xp = cp, xo = co;
      mono(xp, xo, ep, eo);  // exclusive prefix including the carry
      if (in) {
        p.A[i] = xo;
        p.base[i] = xo > Pp ? xo - Pp : 0u;
      }
      uint32_t tp = __shfl_sync(0xffffffffu, ip, 31), to = __shfl_sync(0xffffffffu, io, 31);
      mono(cp, co, tp, to);
    }
    if (lane == 0) {
      if (cp) atomicAdd(&p.diag[dUnExit], (unsigned long long)cp);
      if (co) atomicAdd(&p.diag[dUnEntry], (unsigned long long)co);
    }
  }
}

__global__ void k_frontier_match(FrontierParams p) {
  uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
  unsigned long long pairs = 0, mism = 0;
  if (i < p.n_order) {
    const uint32_t P = p.sum_pend[i];
    const uint32_t A = p.A[i];
    const uint32_t m = P < A ? P : A;
    if (m) {
      const uint32_t pk = p.order[i];
      const uint32_t stream = p.pk_stream[pk];
      const uint32_t first = p.stream_first[stream];
      const uint32_t group = p.stream_group[stream];
      const uint64_t fb_i = p.sum_fbase[i];
      uint64_t q = i;
      for (uint32_t k = 0; k < m; ++k) {
        const uint32_t L = A - 1 - k;
        // levels only decrease with k, so the search resumes from the last hit
        if (q == i) q = i - 1;
        while (q > first && p.base[q] > L) --q;
        const uint32_t idx = L - p.base[q];
        const Frontier en = p.frontier[p.sum_fbase[q] + p.sum_pend[q] + idx];
        const Frontier ex = p.frontier[fb_i + k];
        if (en.func == ex.func) {
          ++pairs;
          const uint64_t dur = ex.ts - en.ts;
          Cell &cell = p.tally[(uint64_t)group * p.n_funcs + en.func];
          atomicAdd(&cell.count, 1ull);
          atomicAdd(&cell.total, (unsigned long long)dur);
          atomicMin(&cell.mn, (unsigned long long)dur);
          atomicMax(&cell.mx, (unsigned long long)dur);
          if (ex.flags) atomicAdd(&cell.err, 1ull);
          if (p.slots && en.aux != 0xFFFFFFFFu) {
            thapi_interval &iv = p.slots[p.evbase[q] + en.aux];
            iv.end_ns = ex.ts;
            iv.flags = (uint8_t)(kIvValid | (ex.flags ? kIvErr : 0u));
            atomicAdd(&p.sum_nvalid[q], 1u);
            if (p.side) {  // self time: the exit's position and the absolute level
              SelfSlot &ss = p.side[p.evbase[q] + en.aux];
              ss.exit_pos = p.evbase[i] + ex.aux;
              ss.level = L | kSelfAbs;
            }
          }
        } else {
          ++mism;
        }
      }
    }
  }
  for (int off = 16; off > 0; off >>= 1) {
    pairs += __shfl_down_sync(0xffffffffu, pairs, off);
    mism += __shfl_down_sync(0xffffffffu, mism, off);
  }
  if ((threadIdx.x & 31) == 0) {
    if (pairs) atomicAdd(&p.diag[dPairs], pairs);
    if (mism) atomicAdd(&p.diag[dMismatch], mism);
  }
}

}  // namespace thapi

namespace thapi {

void launch_frontier(const FrontierParams &p, cudaStream_t s) {
  if (p.n_streams) {
    uint64_t threads = (uint64_t)p.n_streams * 32;
    unsigned grid = (unsigned)((threads + 255) / 256);
    k_frontier_scan<<<grid, 256, 0, s>>>(p);
    count_launches(1);
  }
  if (p.n_order) {
    k_frontier_match<<<(unsigned)((p.n_order + 255) / 256), 256, 0, s>>>(p);
    count_launches(1);
  }
}

}  // namespace thapi

// index.cu — packet index and header validation.
//
// One thread per packet reads the 32-byte header (two 16-byte loads), checks
// it and records stream, event count, content size, seq, ts_begin and the
// discarded counter.  Packets are then grouped by stream with the stable
// radix sort (file order is kept inside a stream), seq monotonicity is checked
// between neighbours of one stream, and an exclusive scan of the event counts
// in stream order gives every packet its first event slot.
#include <algorithm>

#include "internal.cuh"

namespace thapi {

__global__ void k_packet_headers(IndexParams p) {
  uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
  unsigned long long rb = 0;
  if (i < p.n_packets) {
  const uint4 *h = reinterpret_cast<const uint4 *>(packet_at(p.packets, p.pk_addr, i, p.P));
  uint4 a = __ldg(h);
  uint4 b = __ldg(h + 1);
  uint32_t magic = a.x, stream = a.y, content = b.x, nev = b.y, seq = b.z, disc = b.w;
  uint64_t tsb = (uint64_t)a.z | ((uint64_t)a.w << 32);
  uint32_t ns = p.n_streams, soff = 0;
  if (p.pk_trace) {  // a batch: the packet names a stream of its own trace
    const uint32_t t = p.pk_trace[i];
    ns = p.t_nstreams[t];
    soff = p.t_soff[t];
  }
  bool bad = magic != kPacketMagic || stream >= ns || (content & 3u) != 0 ||
             content > p.P - kPacketHeader || nev > content / 8u;
  stream += soff;
  if (bad) {
    atomicMin(p.hdr_err, (unsigned long long)i);
    stream = p.n_streams;  // sentinel group, sorted last
    content = 0;
    nev = 0;
  }
  p.pk_stream[i] = stream;
  p.pk_nev[i] = nev;
  p.pk_content[i] = content;
  p.pk_seq[i] = seq;
  p.pk_disc[i] = disc;
  p.pk_tsb[i] = tsb;
  if (!bad) rb = kPacketHeader + content;
  }
  for (int o = 16; o > 0; o >>= 1) rb += __shfl_down_sync(0xffffffffu, rb, o);
  if ((threadIdx.x & 31) == 0 && rb) atomicAdd(p.read_bytes, rb);
}

// Byte ranges gathered into one buffer, a block per source: 16-byte copies
// while source and destination are both 16-byte aligned, bytes for the rest.
__global__ void k_gather_bytes(const uint8_t *const *src, const uint64_t *len, const uint64_t *off, uint32_t n,
                               uint8_t *dst) {
  for (uint32_t i = blockIdx.x; i < n; i += gridDim.x) {
    const uint8_t *s = src[i];
    uint8_t *d = dst + off[i];
    const uint64_t l = len[i];
    const bool vec = ((reinterpret_cast<uintptr_t>(s) | reinterpret_cast<uintptr_t>(d)) & 15u) == 0;
    const uint64_t l16 = vec ? l / 16 : 0;
    for (uint64_t k = threadIdx.x; k < l16; k += blockDim.x)
      reinterpret_cast<uint4 *>(d)[k] = reinterpret_cast<const uint4 *>(s)[k];
    for (uint64_t k = l16 * 16 + threadIdx.x; k < l; k += blockDim.x) d[k] = s[k];
  }
}

// The trace of each packet of a batch: the last trace whose first packet is
// at or before it (binary search of the traces' first packets).
__global__ void k_packet_traces(const uint64_t *first, uint32_t nt, uint64_t n, uint32_t *pk_trace) {
  const uint64_t q = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (q >= n) return;
  uint32_t lo = 0, hi = nt;  // first[lo] <= q < first[hi] (first[nt] taken as n)
  while (hi - lo > 1) {
    const uint32_t mid = lo + (hi - lo) / 2;
    if (first[mid] <= q)
      lo = mid;
    else
      hi = mid;
  }
  pk_trace[q] = lo;
}

// The address of each packet of a batch read in place: src[t] is trace t's
// first packet, first[t] its first packet in the batch.
__global__ void k_packet_addrs(const uint8_t *const *src, const uint64_t *first, const uint32_t *pk_trace, uint64_t n,
                               uint32_t P, uint64_t *addr) {
  const uint64_t q = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (q >= n) return;
  const uint32_t t = pk_trace[q];
  addr[q] = reinterpret_cast<uint64_t>(src[t] + (q - first[t]) * P);
}

// Sort keys/values for grouping by stream.
__global__ void k_stream_keys(const uint32_t *pk_stream, uint64_t n, uint64_t *keys, uint32_t *vals) {
  uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  keys[i] = pk_stream[i];
  vals[i] = (uint32_t)i;
}

// Stream bounds and seq check over the stream-ordered list; also gathers the
// per-packet event counts in stream order for the scan.
__global__ void k_stream_bounds(const uint64_t *skey, const uint32_t *order, const uint32_t *pk_seq,
                                const uint32_t *pk_nev, uint64_t n, uint32_t n_streams, uint32_t *stream_first,
                                uint64_t *ev, unsigned long long *hdr_err) {
  uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  uint32_t s = (uint32_t)skey[i];
  uint32_t pk = order[i];
  ev[i] = pk_nev[pk];
  if (s >= n_streams) return;
  bool first = i == 0 || (uint32_t)skey[i - 1] != s;
  if (first) stream_first[s] = (uint32_t)i;
  if (!first && pk_seq[pk] <= pk_seq[order[i - 1]]) atomicMin(hdr_err, (unsigned long long)pk);
}

// count = last + 1 - first (second pass, after stream_first is known)
__global__ void k_stream_counts(const uint64_t *skey, uint64_t n, uint32_t n_streams, const uint32_t *stream_first,
                                uint32_t *stream_count) {
  uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  uint32_t s = (uint32_t)skey[i];
  if (s >= n_streams) return;
  bool last = i + 1 == n || (uint32_t)skey[i + 1] != s;
  if (last) stream_count[s] = (uint32_t)(i + 1 - stream_first[s]);
}

}  // namespace thapi

namespace thapi {

static unsigned grid_for(uint64_t n, unsigned t) { return (unsigned)((n + t - 1) / t); }

void launch_packet_headers(const IndexParams &p, cudaStream_t s) {
  if (p.n_packets) {
    k_packet_headers<<<grid_for(p.n_packets, 256), 256, 0, s>>>(p);
    count_launches(1);
  }
}
void launch_packet_traces(const uint64_t *first, uint32_t nt, uint64_t n, uint32_t *pk_trace, cudaStream_t s) {
  if (n && nt) {
    k_packet_traces<<<grid_for(n, 256), 256, 0, s>>>(first, nt, n, pk_trace);
    count_launches(1);
  }
}
void launch_packet_addrs(const uint8_t *const *src, const uint64_t *first, const uint32_t *pk_trace, uint64_t n,
                         uint32_t P, uint64_t *addr, cudaStream_t s) {
  if (n) {
    k_packet_addrs<<<grid_for(n, 256), 256, 0, s>>>(src, first, pk_trace, n, P, addr);
    count_launches(1);
  }
}

void launch_gather_bytes(const uint8_t *const *src, const uint64_t *len, const uint64_t *off, uint32_t n,
                         uint8_t *dst, cudaStream_t s) {
  if (n) {
    k_gather_bytes<<<n < 4096u ? n : 4096u, 256, 0, s>>>(src, len, off, n, dst);
    count_launches(1);
  }
}

void launch_stream_keys(const uint32_t *pk_stream, uint64_t n, uint64_t *keys, uint32_t *vals, cudaStream_t s) {
  if (n) {
    k_stream_keys<<<grid_for(n, 256), 256, 0, s>>>(pk_stream, n, keys, vals);
    count_launches(1);
  }
}
void launch_stream_bounds(const uint64_t *skey, const uint32_t *order, const uint32_t *pk_seq, const uint32_t *pk_nev,
                          uint64_t n, uint32_t n_streams, uint32_t *stream_first, uint32_t *stream_count,
                          uint64_t *ev, unsigned long long *hdr_err, cudaStream_t s) {
  if (!n) return;
  k_stream_bounds<<<grid_for(n, 256), 256, 0, s>>>(skey, order, pk_seq, pk_nev, n, n_streams, stream_first, ev,
                                                    hdr_err);
  k_stream_counts<<<grid_for(n, 256), 256, 0, s>>>(skey, n, n_streams, stream_first, stream_count);
  count_launches(2);
}

}  // namespace thapi

namespace thapi {

__global__ void k_widen_u32(const uint32_t *in, uint64_t *out, uint64_t n) {
  uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) out[i] = in[i];
}

void launch_widen_u32(const uint32_t *in, uint64_t *out, uint64_t n, cudaStream_t s) {
  if (n) {
    k_widen_u32<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(in, out, n);
    count_launches(1);
  }
}

}  // namespace thapi

namespace thapi {

// One descriptor per order position, so the analysis reads a packet's facts
// with three 16-byte loads instead of a chain of dependent ones.
__global__ void k_build_desc(const uint32_t *order, const uint32_t *pk_stream, const uint32_t *pk_nev,
                             const uint32_t *pk_content, const uint32_t *pk_disc, const uint64_t *pk_tsb,
                             const uint32_t *stream_group, const uint64_t *evbase, uint64_t n, PkDesc *desc) {
  uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const uint32_t pk = order[i];
  PkDesc d;
  d.pk = pk;
  d.content = pk_content[pk];
  d.nev = pk_nev[pk];
  d.stream = pk_stream[pk];
  d.group = stream_group[d.stream];
  d.disc = pk_disc[pk];
  d.pad0 = d.pad1 = 0;
  d.tsb = pk_tsb[pk];
  d.evbase = evbase[i];
  desc[i] = d;
}

void launch_build_desc(const uint32_t *order, const uint32_t *pk_stream, const uint32_t *pk_nev,
                       const uint32_t *pk_content, const uint32_t *pk_disc, const uint64_t *pk_tsb,
                       const uint32_t *stream_group, const uint64_t *evbase, uint64_t n, PkDesc *desc, cudaStream_t s) {
  if (!n) return;
  k_build_desc<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(order, pk_stream, pk_nev, pk_content, pk_disc, pk_tsb,
                                                           stream_group, evbase, n, desc);
  count_launches(1);
}

}  // namespace thapi

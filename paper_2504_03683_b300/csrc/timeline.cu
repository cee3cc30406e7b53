// timeline.cu — global interval timeline.
//
// Interval slots are written per packet in entry order and packets are laid
// out in stream order, so the slot array is already ordered by
// (stream, entry position).  A warp per packet compacts the valid slots
// (finishing their absolute level with the depth carried into the packet);
// ordering them by start time (relative to the trace's first timestamp) is
// done by bucket.cu, or by a stable LSD radix sort over only as many bits as
// the span needs when the buckets do not fit shared memory.  Either way the
// timeline order is (start, stream, entry position).  Window queries [t0, t1)
// over the ordered timeline are in window.cu.
#include <algorithm>

#include "internal.cuh"

namespace thapi {

__global__ void k_timeline_compact(const thapi_interval *slots, const uint64_t *evbase, const uint32_t *nslot,
                                   const uint64_t *out_base, const uint32_t *A, const uint32_t *order,
                                   const uint32_t *pk_stream, uint64_t n_order, uint64_t t_min,
                                   thapi_interval *rec, void *keys, bool key32, uint32_t *vals, BucketCells bc) {
  const int lane = threadIdx.x & 31;
  const uint64_t wg = ((uint64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const uint64_t nw = ((uint64_t)gridDim.x * blockDim.x) >> 5;
  // one chunk of slots and the next packet's fields are loaded ahead
  uint64_t n_sb = 0, n_ob = 0;
  uint32_t n_n = 0, n_a = 0, n_stream = 0;
  auto fields = [&](uint64_t i) {
    if (i >= n_order) return;
    n_sb = evbase[i];
    n_n = nslot[i];
    n_a = A[i];
    n_stream = pk_stream[order[i]];
    n_ob = out_base[i];
  };
  fields(wg);
  for (uint64_t i = wg; i < n_order; i += nw) {
    const uint64_t sb = n_sb;
    const uint32_t n = n_n;
    const uint32_t a = n_a;
    const uint32_t stream = n_stream;
    uint64_t ob = n_ob;
    fields(i + nw);
    thapi_interval nxt;
    bool n_in = (uint32_t)lane < n;
    if (n_in) nxt = slots[sb + lane];
    for (uint32_t c = 0; c < n; c += 32) {
      const bool in = n_in;
      thapi_interval iv = nxt;
      n_in = c + 32 + lane < n;
      if (n_in) nxt = slots[sb + c + 32 + lane];
      bool valid = false;
      if (in) valid = (iv.flags & kIvValid) != 0;
      uint32_t bal = __ballot_sync(0xffffffffu, valid);
      const uint64_t at = ob + __popc(bal & ((1u << lane) - 1u));
      uint64_t key = 0;
      if (valid) {
        uint32_t npend = iv.stream_id;
        uint32_t above = a > npend ? a - npend : 0u;
        uint32_t lvl = above + iv.level;
        iv.level = (uint8_t)(lvl > 255u ? 255u : lvl);
        iv.stream_id = stream;
        iv.flags &= (uint8_t)(kIvErr | kIvDevice);
        rec[at] = iv;
        key = iv.start_ns - t_min;
        if (!keys) {  // the bucket path takes its keys from the records
        } else if (key32) {
          static_cast<uint32_t *>(keys)[at] = (uint32_t)key;
        } else {
          static_cast<uint64_t *>(keys)[at] = key;
        }
        if (vals) vals[at] = (uint32_t)at;
      }
      if (bc.cnt) {  // (bucket, stream) cells: records and first record, one atomic pair per run of a cell
        const uint64_t b = key >> bc.shift;
        const uint32_t cell = valid ? (b < bc.nb ? (uint32_t)b : bc.nb - 1) * bc.S + stream : 0xFFFFFFFFu;
        // valid lanes are consecutive records; a run head differs from the previous valid lane's cell
        const uint32_t prev_lane = 31 - __clz((bal & ((1u << lane) - 1u)) | 1u);
        const uint32_t prev_cell = __shfl_sync(0xffffffffu, cell, prev_lane);
        const bool head = valid && (lane == (uint32_t)(__ffs(bal) - 1) || prev_cell != cell);
        const uint32_t heads = __ballot_sync(0xffffffffu, head);
        if (head) {
          const uint32_t after = heads & ~((2u << lane) - 1u);  // later heads
          const uint32_t end = after ? (uint32_t)(__ffs(after) - 1) : 32u;
          const uint32_t upto = end >= 32 ? bal : (bal & ((1u << end) - 1u));
          atomicAdd(&bc.cnt[cell], (uint32_t)__popc(upto & ~((1u << lane) - 1u)));
          atomicMin(&bc.first[cell], (uint32_t)at);
        }
      }
      ob += __popc(bal);
    }
  }
}

// keys[i] = start of rec[i] - t_min (the radix sort's keys when the
// compaction left them out for the bucket path and that path gave up)
__global__ void k_rec_keys(const thapi_interval *rec, uint64_t n, uint64_t t_min, void *keys, bool key32) {
  const uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const uint64_t key = rec[i].start_ns - t_min;
  if (key32)
    static_cast<uint32_t *>(keys)[i] = (uint32_t)key;
  else
    static_cast<uint64_t *>(keys)[i] = key;
}

__global__ void k_iota_u32(uint32_t *v, uint64_t n) {
  const uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) v[i] = (uint32_t)i;
}

// out[i] = rec[vals[i]], four records in flight per thread.
__global__ void k_timeline_gather(const thapi_interval *__restrict__ rec, const uint32_t *__restrict__ vals,
                                  uint64_t n, thapi_interval *__restrict__ out) {
  const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
  for (uint64_t i0 = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i0 < n; i0 += 4 * stride) {
    uint32_t v[4];
    thapi_interval g[4];
#pragma unroll
    for (int u = 0; u < 4; ++u) {
      const uint64_t i = i0 + u * stride;
      v[u] = i < n ? vals[i] : 0u;
    }
#pragma unroll
    for (int u = 0; u < 4; ++u)
      if (i0 + u * stride < n) g[u] = rec[v[u]];
#pragma unroll
    for (int u = 0; u < 4; ++u)
      if (i0 + u * stride < n) out[i0 + u * stride] = g[u];
  }
}

}  // namespace thapi

namespace thapi {

void launch_timeline_compact(const thapi_interval *slots, const uint64_t *evbase, const uint32_t *nslot,
                             const uint64_t *out_base, const uint32_t *A, const uint32_t *order,
                             const uint32_t *pk_stream, uint64_t n_order, uint64_t t_min, thapi_interval *rec,
                             void *keys, bool key32, uint32_t *vals, const BucketCells *cells, int num_sms,
                             cudaStream_t s) {
  if (!n_order) return;
  uint64_t warps = n_order;
  uint64_t cap = (uint64_t)num_sms * 64;  // 64 warps per SM worth of CTAs
  if (warps > cap) warps = cap;
  unsigned grid = (unsigned)((warps * 32 + 255) / 256);
  k_timeline_compact<<<grid, 256, 0, s>>>(slots, evbase, nslot, out_base, A, order, pk_stream, n_order, t_min, rec,
                                          keys, key32, vals, cells ? *cells : BucketCells{});
  count_launches(1);
}

void launch_timeline_gather(const thapi_interval *rec, const uint32_t *vals, uint64_t n, thapi_interval *out,
                            cudaStream_t s) {
  if (n) {
    int dev = 0, sms = 148;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    const uint64_t blocks = std::min<uint64_t>((n + 1023) / 1024, (uint64_t)sms * 8);
    k_timeline_gather<<<(unsigned)std::max<uint64_t>(blocks, 1), 256, 0, s>>>(rec, vals, n, out);
    count_launches(1);
  }
}

void launch_rec_keys(const thapi_interval *rec, uint64_t n, uint64_t t_min, void *keys, bool key32, cudaStream_t s) {
  if (n) {
    k_rec_keys<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(rec, n, t_min, keys, key32);
    count_launches(1);
  }
}

void launch_iota_u32(uint32_t *v, uint64_t n, cudaStream_t s) {
  if (n) {
    k_iota_u32<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(v, n);
    count_launches(1);
  }
}

}  // namespace thapi

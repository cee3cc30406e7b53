// merge.cu — merge of tally rows (across traces and ranks).
//
// The paper's tools gather per-node results into one global result (the
// local -> global aggregation of its analysis, Sec. 3.4).  Tally rows are
// exact integer aggregates, so rows with the same key (host_id, pid, tid,
// func_id) combine exactly: counts, totals and error counts add (totals in
// u64, as in the tally itself), minima and maxima take the min and the max.
//
// Device steps: keys split in two u64 halves, a stable LSD radix sort on the
// low half then the high half gives the key order; key boundaries, an
// exclusive scan of them and reductions into the output rows (one row per
// distinct key, already in key order).
#include "internal.cuh"

namespace thapi {

namespace {

__device__ __forceinline__ uint64_t key_lo(const thapi_tally_row &r) { return ((uint64_t)r.tid << 32) | r.func_id; }
__device__ __forceinline__ uint64_t key_hi(const thapi_tally_row &r) { return ((uint64_t)r.host_id << 32) | r.pid; }

__global__ void k_merge_keys(const thapi_tally_row *rows, uint64_t n, uint64_t *lo, uint32_t *idx) {
  const uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  lo[i] = key_lo(rows[i]);
  idx[i] = (uint32_t)i;
}

__global__ void k_merge_hi(const thapi_tally_row *rows, const uint32_t *perm, uint64_t n, uint64_t *hi) {
  const uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) hi[i] = key_hi(rows[perm[i]]);
}

// flag[i] = 1 where the i-th row in key order starts a new key
__global__ void k_merge_flags(const thapi_tally_row *rows, const uint32_t *perm, uint64_t n, uint64_t *flag) {
  const uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  bool head = i == 0;
  if (!head) {
    const thapi_tally_row &a = rows[perm[i - 1]], &b = rows[perm[i]];
    head = key_hi(a) != key_hi(b) || key_lo(a) != key_lo(b);
  }
  flag[i] = head ? 1u : 0u;
}

__global__ void k_merge_init(thapi_tally_row *out, uint64_t m) {
  const uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= m) return;
  thapi_tally_row r{};
  r.min_ns = ~0ull;
  out[i] = r;
}

// excl: exclusive scan of the head flags; the row's output index is
// excl + head - 1.
__global__ void k_merge_reduce(const thapi_tally_row *rows, const uint32_t *perm, const uint64_t *excl, uint64_t n,
                               thapi_tally_row *out) {
  const uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const thapi_tally_row r = rows[perm[i]];
  bool head = i == 0;
  if (!head) {
    const thapi_tally_row &a = rows[perm[i - 1]];
    head = key_hi(a) != key_hi(r) || key_lo(a) != key_lo(r);
  }
  thapi_tally_row &o = out[excl[i] + (head ? 1u : 0u) - 1u];
  if (head) {
    o.host_id = r.host_id;
    o.pid = r.pid;
    o.tid = r.tid;
    o.func_id = r.func_id;
  }
  atomicAdd(reinterpret_cast<unsigned long long *>(&o.count), (unsigned long long)r.count);
  atomicAdd(reinterpret_cast<unsigned long long *>(&o.total_ns), (unsigned long long)r.total_ns);
  atomicMin(reinterpret_cast<unsigned long long *>(&o.min_ns), (unsigned long long)r.min_ns);
  atomicMax(reinterpret_cast<unsigned long long *>(&o.max_ns), (unsigned long long)r.max_ns);
  atomicAdd(reinterpret_cast<unsigned long long *>(&o.err_count), (unsigned long long)r.err_count);
}

unsigned blocks(uint64_t n) { return (unsigned)((n + 255) / 256); }

}  // namespace

// rows: n rows in device memory (any order).  out: at least n rows of device
// memory.  *m_dev receives the number of distinct keys.
bool tally_merge_device(const thapi_tally_row *rows, uint64_t n, thapi_tally_row *out, uint64_t *m_dev, Scratch &sc,
                        cudaStream_t s) {
  if (n == 0) return cudaMemsetAsync(m_dev, 0, sizeof(uint64_t), s) == cudaSuccess;
  uint64_t *k1 = static_cast<uint64_t *>(sc.get(n * sizeof(uint64_t)));
  uint64_t *k2 = static_cast<uint64_t *>(sc.get(n * sizeof(uint64_t)));
  uint32_t *v1 = static_cast<uint32_t *>(sc.get(n * sizeof(uint32_t)));
  uint32_t *v2 = static_cast<uint32_t *>(sc.get(n * sizeof(uint32_t)));
  uint64_t *flag = static_cast<uint64_t *>(sc.get(n * sizeof(uint64_t)));
  if (sc.failed) return false;
  k_merge_keys<<<blocks(n), 256, 0, s>>>(rows, n, k1, v1);
  bool alt = false;
  radix_sort_pairs(k1, v1, k2, v2, n, 64, &alt, sc, s);  // by (tid, func)
  if (sc.failed) return false;
  uint32_t *perm = alt ? v2 : v1;
  uint32_t *perm_alt = alt ? v1 : v2;
  uint64_t *hi = alt ? k1 : k2, *hi_alt = alt ? k2 : k1;
  k_merge_hi<<<blocks(n), 256, 0, s>>>(rows, perm, n, hi);
  bool alt2 = false;
  radix_sort_pairs(hi, perm, hi_alt, perm_alt, n, 64, &alt2, sc, s);  // then stably by (host, pid)
  if (sc.failed) return false;
  const uint32_t *order = alt2 ? perm_alt : perm;
  k_merge_flags<<<blocks(n), 256, 0, s>>>(rows, order, n, flag);
  scan_exclusive_u64(flag, n, m_dev, sc, s);
  if (sc.failed) return false;
  k_merge_init<<<blocks(n), 256, 0, s>>>(out, n);
  k_merge_reduce<<<blocks(n), 256, 0, s>>>(rows, order, flag, n, out);
  count_launches(5);
  return cudaGetLastError() == cudaSuccess;
}

}  // namespace thapi

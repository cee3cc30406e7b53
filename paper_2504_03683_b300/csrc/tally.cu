// tally.cu — the global (group, function) tally table: initialisation and
// compaction of non-empty cells into rows ordered by (host_id, pid, tid,
// func_id).  Groups are numbered in (host_id, pid, tid) order by the host, so
// cell order is row order.
#include "internal.cuh"

namespace thapi {

__global__ void k_tally_init(Cell *cells, uint64_t n) {
  uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  cells[i] = Cell{0ull, 0ull, ~0ull, 0ull, 0ull};
}

__global__ void k_tally_flags(const Cell *cells, uint64_t n, uint64_t *flags) {
  uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  flags[i] = cells[i].count ? 1u : 0u;
}

__global__ void k_tally_rows(const Cell *cells, uint64_t n, const uint64_t *pos, const uint32_t *group_keys,
                             uint32_t n_funcs, thapi_tally_row *rows) {
  uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const Cell c = cells[i];
  if (!c.count) return;
  uint64_t g = i / n_funcs;
  thapi_tally_row r;
  r.host_id = group_keys[3 * g];
  r.pid = group_keys[3 * g + 1];
  r.tid = group_keys[3 * g + 2];
  r.func_id = (uint32_t)(i - g * n_funcs);
  r.count = c.count;
  r.total_ns = c.total;
  r.min_ns = c.mn;
  r.max_ns = c.mx;
  r.err_count = c.err;
  rows[pos[i]] = r;
}

}  // namespace thapi

namespace thapi {

void launch_tally_init(Cell *cells, uint64_t n, cudaStream_t s) {
  if (n) {
    k_tally_init<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(cells, n);
    count_launches(1);
  }
}

// Writes the non-empty cells as rows; *n_rows_dev receives the row count.
// `rows` must hold up to n rows; `flags` is scratch of n u64.
void launch_tally_compact(const Cell *cells, uint64_t n, const uint32_t *group_keys, uint32_t n_funcs,
                          uint64_t *flags, thapi_tally_row *rows, uint64_t *n_rows_dev, Scratch &sc,
                          cudaStream_t s) {
  if (!n) {
    cudaMemsetAsync(n_rows_dev, 0, sizeof(uint64_t), s);
    return;
  }
  unsigned g = (unsigned)((n + 255) / 256);
  k_tally_flags<<<g, 256, 0, s>>>(cells, n, flags);
  scan_exclusive_u64(flags, n, n_rows_dev, sc, s);
  k_tally_rows<<<g, 256, 0, s>>>(cells, n, flags, group_keys, n_funcs, rows);
  count_launches(2);
}

}  // namespace thapi

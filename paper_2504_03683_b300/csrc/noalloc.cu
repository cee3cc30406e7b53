// noalloc.cu — a tally entry point that makes no device allocation.
//
// Who needs it: a profiling agent that tallies a trace on the node while the
// traced application keeps running in the same CUDA context (the on-node
// aggregation a tracing tool performs between application phases).  Such
// applications, or the caching allocators of their frameworks, usually hold
// nearly all device memory; an allocation made by the agent can then fail,
// or make the application's next allocation fail, or change the
// application's memory behaviour that the tool is supposed to observe, not
// disturb.  This entry point therefore takes every byte of working memory
// from one fixed array in device global memory that is part of the loaded
// library, and the caller passes the trace and the output rows in memory it
// already owns.  No cudaMalloc / cudaFree / pool or torch allocation is made.
//
// The array is a file-scope __device__ variable: every GPU that loads the
// library holds it until the process exits.  Its device address is looked up
// once per device (cudaGetSymbolAddress, with that device current) by the
// first call on that device.  Every call uses the whole array and leaves its
// contents behind; the calls reinitialise everything they read.  Calls whose
// work overlaps on the GPU (other streams, other host threads) race on the
// array; host calls are serialised by a lock, and each call waits for its own
// GPU work before returning.
#include <algorithm>
#include <mutex>

#include "internal.cuh"

namespace thapi {

namespace {

constexpr uint64_t kStaticScratchBytes = 32ull << 20;  // per device
constexpr uint64_t kStaticMaxPackets = 4096;
constexpr uint64_t kStaticMaxEvents = 1ull << 20;
constexpr uint64_t kStaticMaxCells = 1ull << 16;  // (host, pid, tid) groups x functions

static __device__ __align__(256) uint8_t g_static_scratch[kStaticScratchBytes];

struct Arena {
  uint8_t *base;
  uint64_t cap;
  uint64_t off;
};

void *arena_alloc(uint64_t bytes, void * /*stream*/, void *user) {
  Arena *a = static_cast<Arena *>(user);
  const uint64_t at = (a->off + 255u) & ~255ull;
  if (at > a->cap || bytes > a->cap - at) return nullptr;
  a->off = at + bytes;
  return a->base + at;
}

void arena_free(void *, uint64_t, void *, void *) {}

struct DeviceSetup {
  bool done = false;
  uint8_t *scratch = nullptr;
  int num_sms = 0, smem_per_sm = 0, smem_per_block = 0;
  thapi_ctx *ctx = nullptr;
};

std::mutex g_mu;
DeviceSetup g_setup[64];

enum Words { wHdrErr = 0, wContentErr, wDiag0, wTmin = wDiag0 + dCount, wTmax, wFrontTop, wDense, wEvents, wStatus,
             wRows, wReadBytes, wSlots, wCount };

int stages_for(const DeviceSetup &d, uint32_t P, uint32_t emax, uint32_t ncls, uint32_t nf) {
  for (int st = 2; st >= 1; --st)
    if ((int)analyze_smem_bytes(P, emax, st, ncls, nf) <= d.smem_per_block) return st;
  return 0;
}

int tally_static(const uint8_t *dev, uint64_t nbytes, thapi_tally_row *rows, uint64_t cap, uint64_t *n_rows,
                 thapi_diag *diag, cudaStream_t s) {
  int device = 0;
  if (cudaGetDevice(&device) != cudaSuccess || device < 0 || device >= 64) return THAPI_E_CUDA;
  DeviceSetup &ds = g_setup[device];
  if (!ds.done) {
    void *ptr = nullptr;
    if (cudaGetSymbolAddress(&ptr, g_static_scratch) != cudaSuccess) {
      cudaGetLastError();
      return THAPI_E_CUDA;
    }
    if (cudaDeviceGetAttribute(&ds.num_sms, cudaDevAttrMultiProcessorCount, device) != cudaSuccess ||
        cudaDeviceGetAttribute(&ds.smem_per_sm, cudaDevAttrMaxSharedMemoryPerMultiprocessor, device) !=
            cudaSuccess ||
        cudaDeviceGetAttribute(&ds.smem_per_block, cudaDevAttrMaxSharedMemoryPerBlockOptin, device) !=
            cudaSuccess)
      return THAPI_E_CUDA;
    // a bare context whose allocations all come from the array (no pool, no
    // driver allocation): it only carries the allocator hooks set per call
    ds.ctx = hooked_ctx_create(device, arena_alloc, arena_free, nullptr);
    if (!ds.ctx) return THAPI_E_CUDA;
    ds.scratch = static_cast<uint8_t *>(ptr);
    ds.done = true;
  }

  TraceDescription td;
  int rc = describe_device_trace(dev, nbytes, s, td);
  if (rc != THAPI_OK) return rc;
  const uint64_t n = td.n_packets;
  const uint32_t P = td.P, S = td.n_streams, F = td.n_funcs;
  const uint64_t cells = (uint64_t)td.groups * F;
  if (n > kStaticMaxPackets || cells > kStaticMaxCells) return THAPI_E_UNSUPPORTED;
  const uint8_t *packets = dev + td.packets_off;
  if (reinterpret_cast<uintptr_t>(packets) % 16 != 0) return THAPI_E_INVALID;

  Arena arena{ds.scratch, kStaticScratchBytes, 0};
  rc = thapi_ctx_set_allocator(ds.ctx, arena_alloc, arena_free, &arena);
  if (rc != THAPI_OK) return rc;
  Scratch sc;
  sc.ctx = ds.ctx;
  sc.stream = s;
  auto get = [&](uint64_t bytes) { return sc.get(bytes ? bytes : 16); };
#define SGET(ptr, T, count) T *ptr = static_cast<T *>(get((uint64_t)(count) * sizeof(T)))

  unsigned long long w[wCount];
  for (int i = 0; i < wCount; ++i) w[i] = 0;
  w[wHdrErr] = w[wContentErr] = w[wTmin] = ~0ull;
  SGET(words, uint64_t, wCount);
  SGET(d_cls, uint64_t, td.n_classes);
  SGET(d_group, uint32_t, td.stream_group.size());
  SGET(d_gkeys, uint32_t, td.group_keys.size());
  SGET(pk_stream, uint32_t, n + 1);
  SGET(pk_nev, uint32_t, n + 1);
  SGET(pk_content, uint32_t, n + 1);
  SGET(pk_seq, uint32_t, n + 1);
  SGET(pk_disc, uint32_t, n + 1);
  SGET(pk_tsb, uint64_t, n + 1);
  SGET(keys, uint64_t, n + 1);
  SGET(keys_alt, uint64_t, n + 1);
  SGET(vals, uint32_t, n + 1);
  SGET(vals_alt, uint32_t, n + 1);
  SGET(evbase, uint64_t, n + 1);
  SGET(stream_first, uint32_t, S + 1);
  SGET(stream_count, uint32_t, S + 1);
  if (sc.failed) return THAPI_E_UNSUPPORTED;
  auto ck = [](cudaError_t e) {
    if (e != cudaSuccess) cudaGetLastError();
    return e == cudaSuccess;
  };
  auto sync_words = [&]() {
    return ck(cudaMemcpyAsync(w, words, sizeof(w), cudaMemcpyDeviceToHost, s)) && ck(cudaStreamSynchronize(s));
  };
  if (!ck(cudaMemcpyAsync(words, w, sizeof(w), cudaMemcpyHostToDevice, s)) ||
      (td.n_classes && !ck(cudaMemcpyAsync(d_cls, td.cls.data(), 8ull * td.n_classes, cudaMemcpyHostToDevice, s))) ||
      !ck(cudaMemcpyAsync(d_group, td.stream_group.data(), 4ull * td.stream_group.size(), cudaMemcpyHostToDevice,
                          s)) ||
      (td.groups && !ck(cudaMemcpyAsync(d_gkeys, td.group_keys.data(), 4ull * td.group_keys.size(),
                                        cudaMemcpyHostToDevice, s))) ||
      !ck(cudaMemsetAsync(stream_first, 0, 4ull * (S + 1), s)) || !ck(cudaMemsetAsync(stream_count, 0, 4ull * (S + 1), s)))
    return THAPI_E_CUDA;

  // ---- index: headers, group by stream, seq check, event offsets
  unsigned long long *hdr_err = reinterpret_cast<unsigned long long *>(words + wHdrErr);
  launch_packet_headers(IndexParams{packets, nullptr, reinterpret_cast<unsigned long long *>(words + wReadBytes), P, n, S,
                                    pk_stream, pk_nev, pk_content, pk_seq, pk_disc, pk_tsb, hdr_err},
                        s);
  launch_stream_keys(pk_stream, n, keys, vals, s);
  bool in_alt = false;
  int sbits = 1;
  while ((1ull << sbits) <= (uint64_t)S) ++sbits;
  radix_sort_pairs(keys, vals, keys_alt, vals_alt, n, sbits, &in_alt, sc, s);
  if (sc.failed) return THAPI_E_UNSUPPORTED;
  const uint64_t *skey = in_alt ? keys_alt : keys;
  const uint32_t *order = in_alt ? vals_alt : vals;
  launch_stream_bounds(skey, order, pk_seq, pk_nev, n, S, stream_first, stream_count, evbase, hdr_err, s);
  scan_exclusive_u64(evbase, n, words + wEvents, sc, s);
  if (sc.failed) return THAPI_E_UNSUPPORTED;
  if (!ck(cudaGetLastError()) || !sync_words()) return THAPI_E_CUDA;
  if (w[wHdrErr] != ~0ull) return THAPI_E_FORMAT;
  const uint64_t total_events = n ? w[wEvents] : 0;
  if (total_events > kStaticMaxEvents) return THAPI_E_UNSUPPORTED;

  // ---- analysis buffers; the frontier takes what is left of the array
  SGET(desc, PkDesc, n + 1);
  SGET(tally, Cell, cells + 1);
  SGET(sum_pend, uint32_t, n + 1);
  SGET(sum_open, uint32_t, n + 1);
  SGET(sum_nslot, uint32_t, n + 1);
  SGET(sum_nvalid, uint32_t, n + 1);
  SGET(dense_list, uint32_t, n + 1);
  SGET(A, uint32_t, n + 1);
  SGET(base, uint32_t, n + 1);
  SGET(sum_fbase, uint64_t, n + 1);
  SGET(flags, uint64_t, cells + 1);
  SGET(rows_tmp, thapi_tally_row, cells + 1);
  if (sc.failed) return THAPI_E_UNSUPPORTED;
  // scan temporaries of the compaction below come from the same array
  const uint64_t reserve = 4096 + ((cells + 4095) / 2048 + 64) * 8 * 4;
  const uint64_t left = arena.cap > arena.off + reserve + 256 ? arena.cap - arena.off - reserve - 256 : 0;
  const uint64_t fcap = left / sizeof(Frontier);
  Frontier *frontier = static_cast<Frontier *>(get(fcap * sizeof(Frontier)));
  if (sc.failed || !frontier) return THAPI_E_UNSUPPORTED;
  launch_build_desc(order, pk_stream, pk_nev, pk_content, pk_disc, pk_tsb, d_group, evbase, n, desc, s);
  launch_tally_init(tally, cells, s);
  unsigned *status = reinterpret_cast<unsigned *>(words + wStatus);
  AnalyzeParams ap{};
  ap.packets = packets;
  ap.P = P;
  ap.emax = ((P - kPacketHeader) / 4) / 4;
  ap.n_order = n;
  ap.poslist = nullptr;
  ap.desc = desc;
  ap.classes = d_cls;
  ap.n_classes = td.n_classes;
  ap.n_funcs = F;
  ap.tally = tally;
  ap.sum_pend = sum_pend;
  ap.sum_open = sum_open;
  ap.sum_nslot = sum_nslot;
  ap.sum_nvalid = sum_nvalid;
  ap.sum_fbase = sum_fbase;
  ap.frontier = frontier;
  ap.frontier_top = reinterpret_cast<unsigned long long *>(words + wFrontTop);
  ap.frontier_cap = fcap;
  ap.slots = nullptr;  // tally only
  ap.content_err = reinterpret_cast<unsigned long long *>(words + wContentErr);
  ap.diag = reinterpret_cast<unsigned long long *>(words + wDiag0);
  ap.tminmax = reinterpret_cast<unsigned long long *>(words + wTmin);
  ap.slots_written = nullptr;
  ap.dense_list = dense_list;
  ap.dense_count = reinterpret_cast<unsigned long long *>(words + wDense);
  if (n) {
    // at most one CTA per SM, so the per-CTA frontier chunks stay within the array
    const int st = stages_for(ds, P, ap.emax, td.n_classes, F);
    if (!st) return THAPI_E_UNSUPPORTED;
    uint64_t grid = std::min<uint64_t>(n, (uint64_t)ds.num_sms);
    const uint64_t per = (n + grid - 1) / grid;
    grid = (n + per - 1) / per;
    ap.per_cta = (uint32_t)per;
    if (!ck(launch_analyze(ap, st, (uint32_t)grid, s, status)) || !sync_words()) return THAPI_E_CUDA;
    if (w[wDense]) {
      AnalyzeParams dp = ap;
      dp.emax = ((P - kPacketHeader) / 4) / 2 + 1;
      dp.n_order = w[wDense];
      dp.poslist = dense_list;
      dp.dense_list = nullptr;
      dp.dense_count = nullptr;
      const int dst = stages_for(ds, P, dp.emax, td.n_classes, F);
      if (!dst) return THAPI_E_UNSUPPORTED;
      uint64_t dgrid = std::min<uint64_t>(dp.n_order, (uint64_t)ds.num_sms);
      const uint64_t dper = (dp.n_order + dgrid - 1) / dgrid;
      dgrid = (dp.n_order + dper - 1) / dper;
      dp.per_cta = (uint32_t)dper;
      if (!ck(launch_analyze(dp, dst, (uint32_t)dgrid, s, status)) || !sync_words()) return THAPI_E_CUDA;
    }
  }
  if (w[wStatus] == THAPI_E_TIMEOUT) return THAPI_E_TIMEOUT;
  if (w[wContentErr] != ~0ull) return (int)(w[wContentErr] & 7u);
  if (w[wFrontTop] > fcap) return THAPI_E_UNSUPPORTED;

  // ---- pairing across packets, then rows
  FrontierParams fp{};
  fp.n_order = n;
  fp.n_streams = S;
  fp.order = order;
  fp.pk_stream = pk_stream;
  fp.stream_first = stream_first;
  fp.stream_count = stream_count;
  fp.sum_pend = sum_pend;
  fp.sum_open = sum_open;
  fp.sum_fbase = sum_fbase;
  fp.A = A;
  fp.base = base;
  fp.evbase = evbase;
  fp.frontier = frontier;
  fp.stream_group = d_group;
  fp.n_funcs = F;
  fp.tally = tally;
  fp.slots = nullptr;
  fp.sum_nvalid = sum_nvalid;
  fp.diag = reinterpret_cast<unsigned long long *>(words + wDiag0);
  launch_frontier(fp, s);
  launch_tally_compact(tally, cells, d_gkeys, F, flags, rows_tmp, words + wRows, sc, s);
  if (sc.failed) return THAPI_E_UNSUPPORTED;
  if (!ck(cudaGetLastError()) || !sync_words()) return THAPI_E_CUDA;
#undef SGET
  const uint64_t nr = cells ? w[wRows] : 0;
  *n_rows = nr;
  if (diag) {
    diag->events = w[wDiag0 + dEvents];
    diag->pairs = w[wDiag0 + dPairs];
    diag->unmatched_entries = w[wDiag0 + dUnEntry];
    diag->unmatched_exits = w[wDiag0 + dUnExit];
    diag->mismatched_pairs = w[wDiag0 + dMismatch];
    diag->other_events = w[wDiag0 + dOther];
    diag->discarded = w[wDiag0 + dDiscarded];
    diag->packets = w[wDiag0 + dPackets];
  }
  if (cap == 0) return THAPI_OK;
  if (cap < nr) return THAPI_E_RANGE;
  if (nr && (!ck(cudaMemcpyAsync(rows, rows_tmp, nr * sizeof(thapi_tally_row), cudaMemcpyDeviceToDevice, s)) ||
             !ck(cudaStreamSynchronize(s))))
    return THAPI_E_CUDA;
  return THAPI_OK;
}

}  // namespace

}  // namespace thapi

extern "C" int thapi_tally_static(const void *dev_bytes, uint64_t nbytes, thapi_tally_row *rows, uint64_t cap,
                                  uint64_t *n_rows, thapi_diag *diag, void *cuda_stream) {
  if (!dev_bytes || !n_rows || (cap && !rows)) return THAPI_E_INVALID;
  if (reinterpret_cast<uintptr_t>(dev_bytes) % 16 != 0) return THAPI_E_INVALID;
  std::lock_guard<std::mutex> lock(thapi::g_mu);
  return thapi::tally_static(static_cast<const uint8_t *>(dev_bytes), nbytes, rows, cap, n_rows, diag,
                             static_cast<cudaStream_t>(cuda_stream));
}

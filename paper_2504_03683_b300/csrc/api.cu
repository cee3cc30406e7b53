// api.cu — the C ABI: contexts, trace loading (validate, index, decode, pair,
// tally, timeline) and queries over the resident results.
//
// Host code here checks the small file header and tables (the packet area is
// validated on the device), numbers the (host, pid, tid) groups in order,
// stages the packets in device memory and drives the kernels of index.cu,
// analyze.cu, frontier.cu, tally.cu and timeline.cu on the caller's stream.
// No step of the analysis runs on the CPU.
#include <algorithm>
#include <atomic>
#include <chrono>
#include <cstring>
#include <map>
#include <mutex>
#include <new>
#include <thread>
#include <tuple>
#include <vector>

#include "internal.cuh"

namespace thapi {
// Load configuration the autotuner chooses: analysis packet runs per resident
// CTA (more runs: shorter runs, finer load balance) and the device join's
// partition size (records aimed at per partition: 1536 << shift, 1536 >> -shift).
struct Tuning {
  uint32_t grid_mult = 2;  // two runs per resident CTA: a second wave balances uneven packets
  int32_t part_shift = 0;
};
}  // namespace thapi

// the ABI's struct layouts (include/thapi.h), as the binding reads them
static_assert(sizeof(thapi_tally_row) == 56, "tally row");
static_assert(sizeof(thapi_interval) == 24, "interval");
static_assert(sizeof(thapi_event) == 40, "event");
static_assert(sizeof(thapi_trace_info) == 104, "trace info");
static_assert(sizeof(thapi_load_timing) == 112, "load timing");

struct TraceRec {
  cudaStream_t stream = nullptr;
  thapi_trace_info info{};
  thapi_diag diag{};
  thapi_tally_row *rows = nullptr;
  uint64_t rows_bytes = 0;
  thapi_interval *tl = nullptr;
  uint64_t tl_bytes = 0;
  thapi_tally_row *dev_rows = nullptr;
  uint64_t dev_rows_bytes = 0;
  thapi_device_diag dev_diag{};
  thapi_tally_row *self_rows = nullptr;  // self-time rows (loaded with self time on)
  uint64_t self_rows_bytes = 0, n_self_rows = 0;
  std::vector<char> strings;
  std::vector<uint32_t> host_name, func_name;
  std::vector<uint16_t> func_layer;
  thapi_load_timing timing{};
  // window index (prefix maxima of interval ends per block), built by the first window query
  std::mutex win_mu;
  uint64_t *win_bmax = nullptr;
  uint64_t win_bytes = 0;
};

struct thapi_ctx {
  int device = 0;
  uint64_t cap = 0;
  uint64_t used = 0;
  thapi_alloc_fn alloc_fn = nullptr;
  thapi_free_fn free_fn = nullptr;
  void *user = nullptr;
  cudaMemPool_t pool = nullptr;  // without allocator hooks: a stream-ordered pool that keeps freed memory
  int num_sms = 0;
  int smem_per_sm = 0;
  int smem_per_block = 0;
  std::map<uint64_t, TraceRec *> traces;
  uint64_t next_id = 1;
  int err_level = 0;
  uint64_t err_packet = 0, err_event = 0;
  int timing = 0;
  int self_time = 0;
  int autotune = 0;
  std::map<uint64_t, thapi::Tuning> tuned;  // per load shape (tune_key): the configuration kept
  // guards traces, next_id, used, tuned and the error location, so that loads
  // and queries of the serving loop may run from several host threads
  std::mutex mu;
  // pinned host memory the file heads of a batch's device traces are read
  // into (kept between batches: pinning is slow, pageable copies slower)
  std::mutex heads_mu;
  uint8_t *heads = nullptr;
  uint64_t heads_cap = 0;
};

namespace thapi {

static std::atomic<uint64_t> g_launches{0};
void count_launches(uint64_t k) { g_launches.fetch_add(k, std::memory_order_relaxed); }
uint64_t launches_total() { return g_launches.load(std::memory_order_relaxed); }

// CUDA events bracketing the phases of one load (only when timing is on).
struct PhaseClock {
  enum { kIdx0 = 0, kIdx1, kAn0, kAn1, kDn0, kDn1, kFr0, kFr1, kJo0, kJo1, kTa1, kSe0, kSe1, kPc0, kPc1, kPd0, kPd1, kCo0, kCo1, kSo1, kGa1, kN };
  cudaEvent_t ev[kN] = {};
  bool on = false, dense = false;
  void init(bool enable) {
    on = enable;
    if (!on) return;
    for (auto &e : ev)
      if (cudaEventCreate(&e) != cudaSuccess) {
        on = false;
        cudaGetLastError();
        return;
      }
  }
  void rec(int i, cudaStream_t s) {
    if (on) cudaEventRecord(ev[i], s);
  }
  float ms(int a, int b) {
    float t = 0.f;
    if (on && cudaEventElapsedTime(&t, ev[a], ev[b]) != cudaSuccess) {
      cudaGetLastError();
      t = 0.f;
    }
    return t;
  }
  ~PhaseClock() {
    for (auto &e : ev)
      if (e) cudaEventDestroy(e);
  }
};

// Where a load failed (thapi_last_error_location).
static void set_err(thapi_ctx *c, int level, uint64_t packet, uint64_t event) {
  std::lock_guard<std::mutex> g(c->mu);
  c->err_level = level;
  c->err_packet = packet;
  c->err_event = event;
}

static void *dev_alloc(thapi_ctx *c, uint64_t bytes, cudaStream_t s) {
  if (bytes == 0) bytes = 256;
  bytes = (bytes + 255u) & ~255ull;
  if (c->alloc_fn) return c->alloc_fn(bytes, (void *)s, c->user);
  void *p = nullptr;
  const cudaError_t e = c->pool ? cudaMallocFromPoolAsync(&p, bytes, c->pool, s) : cudaMallocAsync(&p, bytes, s);
  if (e != cudaSuccess) {
    cudaGetLastError();
    return nullptr;
  }
  return p;
}

static void dev_free(thapi_ctx *c, void *p, uint64_t bytes, cudaStream_t s) {
  if (!p) return;
  if (bytes == 0) bytes = 256;
  bytes = (bytes + 255u) & ~255ull;
  if (c->free_fn)
    c->free_fn(p, bytes, (void *)s, c->user);
  else
    cudaFreeAsync(p, s);
}

void *Scratch::get(uint64_t bytes) {
  void *p = dev_alloc(ctx, bytes, stream);
  if (!p) {
    failed = 1;
    return nullptr;
  }
  bufs.push_back({p, bytes});
  return p;
}

void Scratch::adopt(void *p, uint64_t bytes) {
  if (p) bufs.push_back({p, bytes});
}

void Scratch::release_all() {
  for (auto &b : bufs) dev_free(ctx, b.first, b.second, stream);
  bufs.clear();
}

// ------------------------------------------------------------ host parse
struct Reader {
  const uint8_t *host;
  const uint8_t *dev;
  uint64_t n;
  cudaStream_t s;
  const uint8_t *pre = nullptr;  // a host copy of the first pre_n bytes of a device trace
  uint64_t pre_n = 0;
  bool get(uint64_t off, uint64_t len, std::vector<uint8_t> &out) const {
    out.resize(len);
    if (!len) return true;
    if (pre && off + len <= pre_n) {
      std::memcpy(out.data(), pre + off, len);
      return true;
    }
    if (host) {
      std::memcpy(out.data(), host + off, len);
      return true;
    }
    if (cudaMemcpyAsync(out.data(), dev + off, len, cudaMemcpyDeviceToHost, s) != cudaSuccess) return false;
    return cudaStreamSynchronize(s) == cudaSuccess;
  }
};

template <class T>
static T rd(const uint8_t *p) {
  T v;
  std::memcpy(&v, p, sizeof(T));
  return v;
}

static bool in_file(uint64_t off, uint64_t count, uint64_t size, uint64_t n) {
  if (off > n) return false;
  if (size && count > (n - off) / size) return false;
  return true;
}

static bool name_ok(const std::vector<uint8_t> &strs, uint32_t off) {
  if (off >= strs.size()) return false;
  return std::memchr(strs.data() + off, 0, strs.size() - off) != nullptr;
}

struct HostLayout {
  uint32_t P = 0, n_streams = 0, n_classes = 0, n_funcs = 0, n_hosts = 0;
  uint64_t n_packets = 0, packets_off = 0;
  std::vector<uint64_t> cls;
  std::vector<uint32_t> srow;  // 4 words per stream
  std::vector<uint32_t> host_name, func_name;
  std::vector<uint16_t> func_layer;
  std::vector<uint8_t> strings;
};

// Table offsets of a file header: streams, classes, functions, hosts,
// strings (and the string block's size).
struct TableAt {
  uint64_t st = 0, cl = 0, fn = 0, ho = 0, so = 0, sb = 0;
};

// The 128-byte file header b of a trace of n bytes, in the documented check
// order (the table rows are checked by the callers).
static int parse_head(const uint8_t *b, uint64_t n, HostLayout &L, TableAt &o) {
  if (rd<uint32_t>(b) != kTraceMagic || rd<uint16_t>(b + 4) != 1 || rd<uint16_t>(b + 6) != kHeaderBytes)
    return THAPI_E_FORMAT;
  L.P = rd<uint32_t>(b + 8);
  L.n_streams = rd<uint32_t>(b + 12);
  L.n_classes = rd<uint32_t>(b + 16);
  L.n_funcs = rd<uint32_t>(b + 20);
  L.n_hosts = rd<uint32_t>(b + 24);
  L.n_packets = rd<uint64_t>(b + 32);
  o.st = rd<uint64_t>(b + 40);
  o.cl = rd<uint64_t>(b + 48);
  o.fn = rd<uint64_t>(b + 56);
  o.ho = rd<uint64_t>(b + 64);
  o.so = rd<uint64_t>(b + 72);
  o.sb = rd<uint64_t>(b + 80);
  L.packets_off = rd<uint64_t>(b + 88);
  if (L.P < 256 || L.P > kMaxPacket || (L.P & (L.P - 1))) return THAPI_E_FORMAT;
  if (L.n_classes > 65536 || L.n_funcs > 65536) return THAPI_E_FORMAT;
  if (!in_file(o.st, L.n_streams, 16, n) || !in_file(o.cl, L.n_classes, 16, n) || !in_file(o.fn, L.n_funcs, 8, n) ||
      !in_file(o.ho, L.n_hosts, 8, n) || !in_file(o.so, o.sb, 1, n))
    return THAPI_E_TRUNCATED;
  if (L.packets_off % 256 != 0) return THAPI_E_FORMAT;
  if (!in_file(L.packets_off, L.n_packets, L.P, n)) return THAPI_E_TRUNCATED;
  return THAPI_OK;
}

// Stream rows: 4 words each, the host inside the trace.
static bool parse_streams(const uint8_t *ss, HostLayout &L) {
  L.srow.resize(4ull * L.n_streams);
  for (uint32_t s = 0; s < L.n_streams; ++s) {
    for (int j = 0; j < 4; ++j) L.srow[4ull * s + j] = rd<uint32_t>(ss + 16ull * s + 4 * j);
    if (L.srow[4ull * s] >= L.n_hosts) return false;
  }
  return true;
}

// File header and tables, in the documented check order.
static int parse_layout(const Reader &r, HostLayout &L) {
  if (r.n < kHeaderBytes) return THAPI_E_TRUNCATED;
  std::vector<uint8_t> h;
  if (!r.get(0, kHeaderBytes, h)) return THAPI_E_CUDA;
  TableAt o;
  const int rc = parse_head(h.data(), r.n, L, o);
  if (rc != THAPI_OK) return rc;
  const uint64_t st = o.st, cl = o.cl, fn = o.fn, ho = o.ho, so = o.so, sb = o.sb;
  std::vector<uint8_t> hs, fs, cs, ss;
  if (!r.get(so, sb, L.strings) || !r.get(ho, 8ull * L.n_hosts, hs) || !r.get(fn, 8ull * L.n_funcs, fs) ||
      !r.get(cl, 16ull * L.n_classes, cs) || !r.get(st, 16ull * L.n_streams, ss))
    return THAPI_E_CUDA;
  L.host_name.resize(L.n_hosts);
  for (uint32_t i = 0; i < L.n_hosts; ++i) {
    L.host_name[i] = rd<uint32_t>(hs.data() + 8ull * i);
    if (!name_ok(L.strings, L.host_name[i])) return THAPI_E_FORMAT;
  }
  L.func_name.resize(L.n_funcs);
  L.func_layer.resize(L.n_funcs);
  for (uint32_t i = 0; i < L.n_funcs; ++i) {
    L.func_name[i] = rd<uint32_t>(fs.data() + 8ull * i);
    L.func_layer[i] = rd<uint16_t>(fs.data() + 8ull * i + 4);
    if (!name_ok(L.strings, L.func_name[i])) return THAPI_E_FORMAT;
  }
  L.cls.resize(L.n_classes);
  for (uint32_t k = 0; k < L.n_classes; ++k) {
    const uint8_t *row = cs.data() + 16ull * k;
    uint32_t func = rd<uint16_t>(row);
    uint32_t kind = row[2];
    uint32_t fixed = rd<uint16_t>(row + 4);
    int32_t roff = rd<int16_t>(row + 6), coff = rd<int16_t>(row + 8);
    if (func >= L.n_funcs || kind > kSample || (fixed & 3u)) return THAPI_E_FORMAT;
    if (roff != -1 && (roff < 0 || (roff & 3) || (uint32_t)roff + 4 > fixed)) return THAPI_E_FORMAT;
    if (coff != -1 && (coff < 0 || (coff & 3) || (uint32_t)coff + 8 > fixed)) return THAPI_E_FORMAT;
    L.cls[k] = (uint64_t)(fixed >> 2) | ((uint64_t)kind << 14) | ((uint64_t)func << 17) |
               ((uint64_t)(roff >= 0 ? (roff >> 2) + 1 : 0) << 33) |
               ((uint64_t)(coff >= 0 ? (coff >> 2) + 1 : 0) << 48);
  }
  return parse_streams(ss.data(), L) ? THAPI_OK : THAPI_E_FORMAT;
}

// A trace of a batch whose class table, function table and function-name
// bytes [nlo, nhi) of its string block equal those of the batch's first trace
// (which parse_layout checked): raw holds its first raw_n bytes in host
// memory, first / o0 the first trace's.  Returns the check result of the
// header, host names and stream rows, in parse_layout's order (the equal
// tables pass as the first trace's did), and sets *same; with *same false
// (a table differs or lies past raw_n) nothing but the header is read and the
// caller parses the trace in full (so too with first null).  Host names are
// offsets into the trace's own string block, which stays in raw (nothing is
// copied).
static int parse_like_first(const uint8_t *raw, uint64_t raw_n, uint64_t n, const uint8_t *first, const TableAt &o0,
                            const HostLayout &a, uint64_t nlo, uint64_t nhi, HostLayout &L, bool *same) {
  *same = false;
  if (n < kHeaderBytes) return THAPI_E_TRUNCATED;
  if (!first || raw_n < kHeaderBytes) return THAPI_OK;
  TableAt o;
  const int rc = parse_head(raw, n, L, o);
  if (rc != THAPI_OK) return rc;
  auto within = [&](uint64_t off, uint64_t len) { return off <= raw_n && len <= raw_n - off; };
  const uint64_t ncl = 16ull * L.n_classes, nfn = 8ull * L.n_funcs;
  if (L.P != a.P || L.n_classes != a.n_classes || L.n_funcs != a.n_funcs || !within(o.cl, ncl) ||
      !within(o.fn, nfn) || !within(o.so, o.sb) || !within(o.ho, 8ull * L.n_hosts) ||
      !within(o.st, 16ull * L.n_streams) || std::memcmp(raw + o.cl, first + o0.cl, ncl) != 0 ||
      std::memcmp(raw + o.fn, first + o0.fn, nfn) != 0 ||
      (a.n_funcs && (o.sb < nhi || std::memcmp(raw + o.so + nlo, first + o0.so + nlo, nhi - nlo) != 0)))
    return THAPI_OK;
  *same = true;
  const uint8_t *strs = raw + o.so;
  L.host_name.resize(L.n_hosts);
  for (uint32_t i = 0; i < L.n_hosts; ++i) {
    const uint32_t off = rd<uint32_t>(raw + o.ho + 8ull * i);
    if (off >= o.sb || !std::memchr(strs + off, 0, o.sb - off)) return THAPI_E_FORMAT;
    L.host_name[i] = off;
  }
  return parse_streams(raw + o.st, L) ? THAPI_OK : THAPI_E_FORMAT;
}

// A context whose every device allocation goes through the given hooks, for
// callers that bring their own device memory (the static-scratch tally): the
// device's attributes are read, and nothing is created on the device (no
// memory pool, unlike thapi_ctx_create).
thapi_ctx *hooked_ctx_create(int device, thapi_alloc_fn alloc, thapi_free_fn free_fn, void *user) {
  thapi_ctx *c = new (std::nothrow) thapi_ctx();
  if (!c) return nullptr;
  c->device = device;
  c->alloc_fn = alloc;
  c->free_fn = free_fn;
  c->user = user;
  if (cudaDeviceGetAttribute(&c->num_sms, cudaDevAttrMultiProcessorCount, device) != cudaSuccess ||
      cudaDeviceGetAttribute(&c->smem_per_sm, cudaDevAttrMaxSharedMemoryPerMultiprocessor, device) != cudaSuccess ||
      cudaDeviceGetAttribute(&c->smem_per_block, cudaDevAttrMaxSharedMemoryPerBlockOptin, device) != cudaSuccess) {
    cudaGetLastError();
    delete c;
    return nullptr;
  }
  return c;
}

// Header, tables and (host, pid, tid) group numbering of a trace in device
// memory, for callers outside the loader (the static-scratch tally).
int describe_device_trace(const uint8_t *dev, uint64_t nbytes, cudaStream_t s, TraceDescription &td) {
  HostLayout L;
  const Reader r{nullptr, dev, nbytes, s};
  const int rc = parse_layout(r, L);
  if (rc != THAPI_OK) return rc;
  for (uint32_t i = 0; i < L.n_streams; ++i)  // per-CPU buffers need the allocating path
    if (L.srow[4ull * i + 3] & kStreamPerCpu) return THAPI_E_UNSUPPORTED;
  td.P = L.P;
  td.n_streams = L.n_streams;
  td.n_classes = L.n_classes;
  td.n_funcs = L.n_funcs;
  td.n_hosts = L.n_hosts;
  td.n_packets = L.n_packets;
  td.packets_off = L.packets_off;
  td.cls = L.cls;
  std::vector<std::tuple<uint32_t, uint32_t, uint32_t, uint32_t>> keyed(L.n_streams);
  for (uint32_t i = 0; i < L.n_streams; ++i)
    keyed[i] = std::make_tuple(L.srow[4ull * i], L.srow[4ull * i + 1], L.srow[4ull * i + 2], i);
  std::sort(keyed.begin(), keyed.end());
  td.stream_group.assign(L.n_streams ? L.n_streams : 1, 0);
  td.group_keys.clear();
  td.groups = 0;
  for (uint32_t i = 0; i < L.n_streams; ++i) {
    if (i == 0 || std::get<0>(keyed[i]) != std::get<0>(keyed[i - 1]) ||
        std::get<1>(keyed[i]) != std::get<1>(keyed[i - 1]) || std::get<2>(keyed[i]) != std::get<2>(keyed[i - 1])) {
      td.group_keys.push_back(std::get<0>(keyed[i]));
      td.group_keys.push_back(std::get<1>(keyed[i]));
      td.group_keys.push_back(std::get<2>(keyed[i]));
      ++td.groups;
    }
    td.stream_group[std::get<3>(keyed[i])] = td.groups - 1;
  }
  return THAPI_OK;
}

// Misc device words of one load.
enum Misc {
  mHdrErr = 0,
  mContentErr,
  mDiag0,
  mTmin = mDiag0 + dCount,
  mTmax,
  mFrontTop,
  mDense,
  mEvents,
  mStatus,
  mRows,
  mIv,
  mReadBytes,
  mSlots,
  mCmdCount0,                 // device-activity records: begin, end, host
  mJoin0 = mCmdCount0 + 3,    // join results: pairs, intervals, unjoined, ambiguous, host entries of pairs, overflow
  mDevRows = mJoin0 + 6,
  mPartMax,                   // records of the largest command-id partition
  mPcCount,                   // per-CPU records
  mPcAll,                     // per-CPU buffers: events
  mPcRead,                    // per-CPU buffers: packet bytes (32 + content)
  mPcEntries,                 // per-CPU buffers: ENTRY events (interval slots)
  mPcRows,                    // per-CPU thread tally rows
  mMerged,                    // tally rows after merging the thread rows
  mSelfWord,                  // self time: largest level
  mSelfRows,                  // self-time rows of per-thread streams
  mSelfPcRows,                // self-time rows of per-CPU threads
  mSelfMerged,                // self-time rows after merging
  mCount
};

// Coarse peak device memory of one load (packets when copied, index, tally
// cells, interval slots, the timeline's sort; device-activity records and
// self-time records when the trace has them): what admission against the
// context's cap charges up front.  G = (host, pid, tid) groups.
static uint64_t load_estimate(const HostLayout &L, uint64_t G, bool copies_packets, bool self_on) {
  const uint64_t n = L.n_packets, P = L.P, cells = G * (uint64_t)L.n_funcs;
  const uint64_t est_events = n * (uint64_t)((P - kPacketHeader) / 8);
  bool dev_on = false;
  for (uint64_t c : L.cls) {
    const uint32_t k = cls_kind(c);
    dev_on = dev_on || k == kDevBegin || k == kDevEnd || (k == kEntry && cls_cmdw(c) >= 0);
  }
  return (copies_packets ? n * P : 0) + n * 128 + cells * 80 + est_events * 24 +
         (dev_on ? est_events * 48 + cells * 80 : 0) + (self_on ? est_events * 96 + cells * 120 : 0);
}

// Number of (host, pid, tid) groups of the per-thread streams.
static uint64_t group_count(const HostLayout &L) {
  std::vector<std::tuple<uint32_t, uint32_t, uint32_t>> k;
  for (uint32_t i = 0; i < L.n_streams; ++i)
    if (!(L.srow[4ull * i + 3] & kStreamPerCpu))
      k.push_back(std::make_tuple(L.srow[4ull * i], L.srow[4ull * i + 1], L.srow[4ull * i + 2]));
  std::sort(k.begin(), k.end());
  return (uint64_t)(std::unique(k.begin(), k.end()) - k.begin());
}

#define CK(x)                                   \
  do {                                          \
    if ((x) != cudaSuccess) {                   \
      cudaGetLastError();                       \
      return THAPI_E_CUDA;                      \
    }                                           \
  } while (0)

class Loader {
 public:
  Loader(thapi_ctx *c, const uint8_t *host, const uint8_t *dev, uint64_t nbytes, cudaStream_t s)
      : c_(c), host_(host), dev_(dev), nbytes_(nbytes), s_(s) {
    sc_.ctx = c;
    sc_.stream = s;
  }
  ~Loader() {
    sc_.release_all();
    if (tr_) {
      dev_free(c_, tr_->rows, tr_->rows_bytes, s_);
      dev_free(c_, tr_->tl, tr_->tl_bytes, s_);
      dev_free(c_, tr_->dev_rows, tr_->dev_rows_bytes, s_);
      dev_free(c_, tr_->self_rows, tr_->self_rows_bytes, s_);
      delete tr_;
    }
    cudaStreamSynchronize(s_);
  }
  int run();
  // decode only: every event to HOST `out` (capacity cap), *n = events; no trace is kept
  void set_decode(thapi_event *out, uint64_t cap, uint64_t *n) {
    dec_out_ = out;
    dec_cap_ = cap;
    dec_n_ = n;
  }
  TraceRec *take() {
    TraceRec *t = tr_;
    tr_ = nullptr;
    return t;
  }
  // the load's status with a scratch failure that was a timed-out wait reported as such
  int status(int rc) const { return rc == THAPI_E_NOMEM && sc_.failed == 2 ? THAPI_E_TIMEOUT : rc; }
  void set_tuning(const Tuning &t) { tune_ = t; }
  // the serving loop charged this load against the cap already
  void set_admitted() { admitted_ = true; }
  void set_input(const uint8_t *host, const uint8_t *dev, uint64_t nbytes) {
    host_ = host;
    dev_ = dev;
    nbytes_ = nbytes;
  }
  // a batch: n traces (host or device bytes) loaded as one trace
  void set_batch(const void *const *bytes, const uint64_t *nbytes, uint32_t n, bool on_device) {
    bptr_.assign(bytes, bytes + n);
    bn_.assign(nbytes, nbytes + n);
    bdev_ = on_device;
    nbytes_ = 0;
    for (uint32_t t = 0; t < n; ++t) nbytes_ += nbytes[t];
  }

 private:
  int parse_batch(HostLayout &L);
  Tuning tune_;
  bool admitted_ = false;
  std::vector<const void *> bptr_;
  std::vector<uint64_t> bn_;
  std::vector<HostLayout> blay_;
  bool bdev_ = false;

  template <class T>
  T *alloc(uint64_t count) {
    return static_cast<T *>(sc_.get((count ? count : 1) * sizeof(T)));
  }
  int sync_misc() {
    CK(cudaMemcpyAsync(misc_h_, misc_, sizeof(misc_h_), cudaMemcpyDeviceToHost, s_));
    CK(cudaStreamSynchronize(s_));
    return THAPI_OK;
  }

  thapi_ctx *c_;
  const uint8_t *host_, *dev_;
  uint64_t nbytes_;
  cudaStream_t s_;
  Scratch sc_;
  TraceRec *tr_ = nullptr;
  uint64_t *misc_ = nullptr;
  unsigned long long misc_h_[mCount];
  PhaseClock clk_;
  thapi_event *dec_out_ = nullptr;
  uint64_t dec_cap_ = 0, *dec_n_ = nullptr;
  int decode(const HostLayout &L, uint64_t n, uint64_t total_events, const uint8_t *packets, const uint32_t *order,
             const uint32_t *pk_stream, const uint32_t *pk_nev, const uint32_t *pk_content, const uint32_t *pk_disc,
             const uint64_t *pk_tsb, const uint32_t *d_group, const uint64_t *evbase, const uint64_t *d_cls,
             const uint32_t *d_gkeys);
};

// Decode-only tail of a load: descriptors, the decode kernel, the records to the host.
int Loader::decode(const HostLayout &L, uint64_t n, uint64_t total_events, const uint8_t *packets,
                   const uint32_t *order, const uint32_t *pk_stream, const uint32_t *pk_nev, const uint32_t *pk_content,
                   const uint32_t *pk_disc, const uint64_t *pk_tsb, const uint32_t *d_group, const uint64_t *evbase,
                   const uint64_t *d_cls, const uint32_t *d_gkeys) {
  *dec_n_ = total_events;
  if (dec_cap_ == 0) return THAPI_OK;
  if (dec_cap_ < total_events) return THAPI_E_RANGE;
  if (!total_events) return THAPI_OK;
  const uint32_t nw = decode_warps(L.P, L.n_classes, c_->smem_per_block);
  if (!nw) return THAPI_E_UNSUPPORTED;
  int rc;
  thapi_event *d_ev = alloc<thapi_event>(total_events);
  PkDesc *desc = alloc<PkDesc>(n);
  if (sc_.failed) return THAPI_E_NOMEM;
  launch_build_desc(order, pk_stream, pk_nev, pk_content, pk_disc, pk_tsb, d_group, evbase, n, desc, s_);
  misc_h_[mContentErr] = ~0ull;
  CK(cudaMemcpyAsync(misc_ + mContentErr, misc_h_ + mContentErr, sizeof(uint64_t), cudaMemcpyHostToDevice, s_));
  DecodeParams dp{};
  dp.packets = packets;
  dp.P = L.P;
  dp.n_classes = L.n_classes;
  dp.n_order = n;
  dp.desc = desc;
  dp.classes = d_cls;
  dp.out = d_ev;
  dp.content_err = reinterpret_cast<unsigned long long *>(misc_ + mContentErr);
  dp.group_keys = d_gkeys;
  const uint64_t grid = std::min<uint64_t>((n + nw - 1) / nw, (uint64_t)c_->num_sms * 4);
  CK(launch_decode_warp(dp, nw, (uint32_t)std::max<uint64_t>(grid, 1), s_));
  if ((rc = sync_misc()) != THAPI_OK) return rc;
  if (misc_h_[mContentErr] != ~0ull) {
    const unsigned long long k = misc_h_[mContentErr];
    set_err(c_, 2, k >> 20, (k >> 3) & 0x1FFFFu);
    return (int)(k & 7u);
  }
  CK(cudaMemcpyAsync(dec_out_, d_ev, total_events * sizeof(thapi_event), cudaMemcpyDeviceToHost, s_));
  CK(cudaStreamSynchronize(s_));
  return THAPI_OK;
}

// Double-buffered packets when they fit the per-CTA shared memory, else single.
static int pick_stages(thapi_ctx *c, uint32_t P, uint32_t emax, uint32_t n_classes, uint32_t n_funcs) {
  for (int st = 2; st >= 1; --st)
    if ((int)analyze_smem_bytes(P, emax, st, n_classes, n_funcs) <= c->smem_per_block) return st;
  return 0;
}

static int blocks_per_sm(thapi_ctx *c, uint32_t smem) {
  int b = std::min(16, c->smem_per_sm / (int)(smem + 1024));
  return b < 1 ? 1 : b;
}

// A batch's tables: every trace parsed and checked (same packet size, class
// table, function names and layers), then one layout whose streams and hosts
// are the traces' in order (host ids and stream ids offset by the earlier
// traces' counts) and whose strings are the traces' string tables one after
// the other.  A trace that fails its own checks reports level 0, packet =
// its index in the batch.
int Loader::parse_batch(HostLayout &L) {
  const uint32_t nt = (uint32_t)bptr_.size();
  blay_.assign(nt, HostLayout{});
  // device traces: every trace's head (file header and tables, up to its
  // packets) gathered by one kernel and read back at once, in two rounds
  std::unique_lock<std::mutex> heads_lock(c_->heads_mu, std::defer_lock);
  uint8_t *heads = nullptr;
  std::vector<uint64_t> head_off(nt + 1, 0), head_len(nt, 0);
  if (bdev_) {
    heads_lock.lock();
    const void **d_src = static_cast<const void **>(sc_.get(nt * sizeof(void *)));
    uint64_t *d_len = static_cast<uint64_t *>(sc_.get(nt * sizeof(uint64_t)));
    uint64_t *d_off = static_cast<uint64_t *>(sc_.get(nt * sizeof(uint64_t)));
    if (sc_.failed) return THAPI_E_NOMEM;
    CK(cudaMemcpyAsync(d_src, bptr_.data(), nt * sizeof(void *), cudaMemcpyHostToDevice, s_));
    for (int round = 0; round < 2; ++round) {
      std::vector<uint64_t> len(nt);
      for (uint32_t t = 0; t < nt; ++t) {
        len[t] = std::min<uint64_t>(bn_[t], kHeaderBytes);
        if (round == 1 && head_len[t] >= 96)  // up to the packets (at most 16 MB), from the header read before
          len[t] = std::max<uint64_t>(
              len[t], std::min<uint64_t>(std::min<uint64_t>(bn_[t], rd<uint64_t>(heads + head_off[t] + 88)),
                                         16ull << 20));
      }
      for (uint32_t t = 0; t < nt; ++t) {  // each head at a 16-byte boundary (16-byte copies)
        head_len[t] = len[t];
        head_off[t + 1] = head_off[t] + (len[t] + 15) / 16 * 16;
      }
      uint8_t *d_dst = static_cast<uint8_t *>(sc_.get(std::max<uint64_t>(head_off[nt], 1)));
      if (sc_.failed) return THAPI_E_NOMEM;
      CK(cudaMemcpyAsync(d_len, head_len.data(), nt * sizeof(uint64_t), cudaMemcpyHostToDevice, s_));
      CK(cudaMemcpyAsync(d_off, head_off.data(), nt * sizeof(uint64_t), cudaMemcpyHostToDevice, s_));
      launch_gather_bytes(reinterpret_cast<const uint8_t *const *>(d_src), d_len, d_off, nt, d_dst, s_);
      if (c_->heads_cap < head_off[nt]) {
        if (c_->heads) cudaFreeHost(c_->heads);
        c_->heads = nullptr;
        c_->heads_cap = 0;
        const uint64_t want = std::max<uint64_t>(head_off[nt], 1) * 5 / 4;
        if (cudaHostAlloc(reinterpret_cast<void **>(&c_->heads), want, cudaHostAllocDefault) != cudaSuccess) {
          cudaGetLastError();
          c_->heads = nullptr;
          return THAPI_E_NOMEM;
        }
        c_->heads_cap = want;
      }
      heads = c_->heads;
      CK(cudaMemcpyAsync(heads, d_dst, head_off[nt], cudaMemcpyDeviceToHost, s_));
      CK(cudaStreamSynchronize(s_));
    }
  }
  // the traces' tables parsed on host threads (each trace on its own), trace 0
  // first: every other trace is checked against it as it is parsed.  The
  // first failing trace in batch order is the one reported, file errors
  // before disagreements.
  std::vector<int> rcs(nt, THAPI_OK);
  std::vector<char> agree(nt, 1);
  auto reader = [&](uint32_t t) {
    const uint8_t *p = static_cast<const uint8_t *>(bptr_[t]);
    Reader r{bdev_ ? nullptr : p, bdev_ ? p : nullptr, bn_[t], s_};
    if (bdev_) {
      r.pre = heads + head_off[t];
      r.pre_n = head_len[t];
    }
    return r;
  };
  rcs[0] = parse_layout(reader(0), blay_[0]);
  if (rcs[0] != THAPI_OK) {
    set_err(c_, 0, 0, 0);
    return rcs[0];
  }
  const HostLayout &a = blay_[0];
  auto fname = [](const HostLayout &x, uint32_t f) { return reinterpret_cast<const char *>(x.strings.data()) + x.func_name[f]; };
  // the bytes of trace 0's function names (from the lowest name offset to the
  // end of the highest name): traces whose names sit at the same offsets and
  // whose bytes there are equal have the same names (one comparison instead
  // of one per name; the traces' host names usually differ, so whole string
  // tables rarely match)
  uint64_t nlo = ~0ull, nhi = 0;
  for (uint32_t f = 0; f < a.n_funcs; ++f) {
    nlo = std::min<uint64_t>(nlo, a.func_name[f]);
    nhi = std::max<uint64_t>(nhi, a.func_name[f] + std::strlen(fname(a, f)) + 1);
  }
  auto same_as_first = [&](const HostLayout &x) {
    if (x.P != a.P || x.cls != a.cls || x.n_funcs != a.n_funcs || x.func_layer != a.func_layer) return false;
    if (x.func_name == a.func_name &&
        (x.strings == a.strings ||
         (a.n_funcs && x.strings.size() >= nhi && std::memcmp(a.strings.data() + nlo, x.strings.data() + nlo, nhi - nlo) == 0)))
      return true;
    for (uint32_t f = 0; f < a.n_funcs; ++f)
      if (std::strcmp(fname(a, f), fname(x, f)) != 0) return false;
    return true;
  };
  // a trace's bytes in host memory: its gathered head, or the trace itself
  auto raw_of = [&](uint32_t t, uint64_t *raw_n) -> const uint8_t * {
    *raw_n = bdev_ ? head_len[t] : bn_[t];
    return bdev_ ? heads + head_off[t] : static_cast<const uint8_t *>(bptr_[t]);
  };
  uint64_t first_n = 0;
  const uint8_t *first = raw_of(0, &first_n);
  TableAt o0;
  {
    HostLayout tmp;
    if (parse_head(first, bn_[0], tmp, o0) != THAPI_OK) return THAPI_E_FORMAT;  // not reached: checked above
    auto within = [&](uint64_t off, uint64_t len) { return off <= first_n && len <= first_n - off; };
    if (!within(o0.cl, 16ull * a.n_classes) || !within(o0.fn, 8ull * a.n_funcs) || !within(o0.so, o0.sb))
      first = nullptr;  // trace 0's tables are not all in host memory: every trace is parsed in full
  }
  // per trace its string block (host names are offsets into it)
  std::vector<const uint8_t *> t_str(nt, nullptr);
  std::vector<uint64_t> t_strn(nt, 0);
  t_str[0] = a.strings.data();
  t_strn[0] = a.strings.size();
  const uint32_t hw = std::max(1u, std::thread::hardware_concurrency());
  const uint32_t nthreads = nt < 64 ? 1u : std::min<uint32_t>(std::min(32u, hw), nt);
  auto run_pool = [&](auto body) {
    std::vector<std::thread> pool;
    for (uint32_t k = 1; k < nthreads; ++k) pool.emplace_back(body, k);
    body(0u);
    for (auto &th : pool) th.join();
  };
  // a trace whose tables equal trace 0's only has its header, host names and
  // stream rows read; any other is parsed in full and compared
  run_pool([&](uint32_t first_t) {
    for (uint32_t t = 1 + first_t; t < nt; t += nthreads) {
      uint64_t raw_n = 0;
      const uint8_t *raw = raw_of(t, &raw_n);
      bool same = false;
      rcs[t] = parse_like_first(raw, raw_n, bn_[t], first, o0, a, nlo, nhi, blay_[t], &same);
      if (rcs[t] != THAPI_OK) continue;
      if (same) {
        const uint64_t so = rd<uint64_t>(raw + 72), sb = rd<uint64_t>(raw + 80);
        t_str[t] = raw + so;
        t_strn[t] = sb;
        continue;
      }
      blay_[t] = HostLayout{};
      rcs[t] = parse_layout(reader(t), blay_[t]);
      if (rcs[t] == THAPI_OK) {
        agree[t] = same_as_first(blay_[t]) ? 1 : 0;
        t_str[t] = blay_[t].strings.data();
        t_strn[t] = blay_[t].strings.size();
      }
    }
  });
  for (uint32_t t = 0; t < nt; ++t)
    if (rcs[t] != THAPI_OK) {
      set_err(c_, 0, t, 0);
      return rcs[t];
    }
  for (uint32_t t = 0; t < nt; ++t)
    if (!agree[t]) return THAPI_E_UNSUPPORTED;
  L.P = a.P;
  L.n_classes = a.n_classes;
  L.n_funcs = a.n_funcs;
  L.cls = a.cls;
  L.func_name = a.func_name;
  L.func_layer = a.func_layer;
  L.packets_off = 0;
  // the combined tables: trace 0's string block (its function and host
  // names), then the host names of the other traces; stream rows with their
  // hosts renumbered from prefix sums
  std::vector<uint64_t> host_at(nt + 1, 0), stream_at(nt + 1, 0);
  uint64_t packets = 0;
  for (uint32_t t = 0; t < nt; ++t) {
    const HostLayout &b = blay_[t];
    host_at[t + 1] = host_at[t] + b.n_hosts;
    stream_at[t + 1] = stream_at[t] + b.n_streams;
    packets += b.n_packets;
  }
  const uint64_t streams = stream_at[nt], hosts = host_at[nt];
  if (streams >= 0xFFFFFFFFull || hosts >= 0xFFFFFFFFull) return THAPI_E_UNSUPPORTED;
  L.strings = a.strings;
  L.host_name.resize(hosts);
  for (uint32_t h = 0; h < a.n_hosts; ++h) L.host_name[h] = a.host_name[h];
  for (uint32_t t = 1; t < nt; ++t) {
    const HostLayout &b = blay_[t];
    for (uint32_t h = 0; h < b.n_hosts; ++h) {
      const char *nm = reinterpret_cast<const char *>(t_str[t] + b.host_name[h]);
      const size_t len = std::strlen(nm) + 1;  // NUL-terminated inside the block (checked)
      if (L.strings.size() + len >= 0xFFFFFFFFull) return THAPI_E_UNSUPPORTED;
      L.host_name[host_at[t] + h] = (uint32_t)L.strings.size();
      L.strings.insert(L.strings.end(), nm, nm + len);
    }
  }
  L.srow.resize(4 * streams);
  for (uint32_t t = 0; t < nt; ++t) {
    const HostLayout &b = blay_[t];
    for (uint32_t s = 0; s < b.n_streams; ++s) {
      uint32_t *row = L.srow.data() + 4 * (stream_at[t] + s);
      row[0] = b.srow[4ull * s] + (uint32_t)host_at[t];
      for (int j = 1; j < 4; ++j) row[j] = b.srow[4ull * s + j];
    }
  }
  L.n_streams = (uint32_t)streams;
  L.n_hosts = (uint32_t)hosts;
  L.n_packets = packets;
  return THAPI_OK;
}

int Loader::run() {
  const auto host_t0 = std::chrono::steady_clock::now();
  HostLayout L;
  int rc;
  if (!bptr_.empty()) {
    rc = parse_batch(L);
  } else {
    const Reader r{host_, dev_, nbytes_, s_};
    rc = parse_layout(r, L);
  }
  if (rc != THAPI_OK) return rc;
  const uint64_t n = L.n_packets;
  const uint32_t P = L.P, S = L.n_streams, F = L.n_funcs;

  // (host, pid, tid) groups numbered in order
  // per-thread streams numbered in (host, pid, tid) order; per-CPU buffers
  // (stream flags bit 1) form no group: their events name their threads
  std::vector<std::tuple<uint32_t, uint32_t, uint32_t, uint32_t>> keyed;
  bool has_pc = false;
  std::vector<uint32_t> stream_host(S ? S : 1, 0);
  for (uint32_t i = 0; i < S; ++i) {
    stream_host[i] = L.srow[4ull * i];
    if (L.srow[4ull * i + 3] & kStreamPerCpu)
      has_pc = true;
    else
      keyed.push_back(std::make_tuple(L.srow[4ull * i], L.srow[4ull * i + 1], L.srow[4ull * i + 2], i));
  }
  std::sort(keyed.begin(), keyed.end());
  std::vector<uint32_t> stream_group(S ? S : 1, kPerCpuGroup), group_keys;
  uint32_t G = 0;
  for (size_t i = 0; i < keyed.size(); ++i) {
    if (i == 0 || std::get<0>(keyed[i]) != std::get<0>(keyed[i - 1]) ||
        std::get<1>(keyed[i]) != std::get<1>(keyed[i - 1]) || std::get<2>(keyed[i]) != std::get<2>(keyed[i - 1])) {
      group_keys.push_back(std::get<0>(keyed[i]));
      group_keys.push_back(std::get<1>(keyed[i]));
      group_keys.push_back(std::get<2>(keyed[i]));
      ++G;
    }
    stream_group[std::get<3>(keyed[i])] = G - 1;
  }
  const uint64_t cells = (uint64_t)G * F;
  if (cells > (1ull << 28) || n >= 0xFFFFFFFFull) return THAPI_E_UNSUPPORTED;

  // device-activity pairing: records of events carrying a command id, their table, a device tally
  bool dev_on = false;
  for (uint64_t c : L.cls) {
    const uint32_t k = cls_kind(c);
    dev_on = dev_on || k == kDevBegin || k == kDevEnd || (k == kEntry && cls_cmdw(c) >= 0);
  }
  // self time: a side record per slot, then per interval its record, sort keys and children's sum
  const bool self_on = c_->self_time != 0;
  // admission: coarse peak of this load (unless the serving loop admitted it already)
  if (!admitted_) {
    const uint64_t est = load_estimate(L, G, host_ || (!bptr_.empty() && !bdev_), self_on);
    std::lock_guard<std::mutex> g(c_->mu);
    if (c_->cap && c_->used + est > c_->cap) return THAPI_E_NOMEM;
  }

  tr_ = new (std::nothrow) TraceRec();
  if (!tr_) return THAPI_E_NOMEM;
  tr_->stream = s_;
  clk_.init(c_->timing != 0);
  tr_->timing.parse_ms =
      std::chrono::duration<float, std::milli>(std::chrono::steady_clock::now() - host_t0).count();
  const uint64_t launches0 = launches_total();
  uint64_t analyze_launches = 0;

  // ---- the packet area on the device
  const uint8_t *packets = nullptr;
  uint64_t *pk_addr = nullptr;  // a batch of device traces: every packet read where it is
  uint32_t *d_pk_trace = nullptr, *d_t_soff = nullptr, *d_t_ns = nullptr;
  if (!bptr_.empty()) {  // a batch: host traces' packets copied into one area in batch order;
                         // device traces' packets read in place through an address per packet
    const uint32_t nt = (uint32_t)bptr_.size();
    uint8_t *pk = bdev_ ? nullptr : alloc<uint8_t>(n * (uint64_t)P);
    if (bdev_) pk_addr = alloc<uint64_t>(n);
    d_pk_trace = alloc<uint32_t>(n);
    d_t_soff = alloc<uint32_t>(nt);
    d_t_ns = alloc<uint32_t>(nt);
    if (sc_.failed) return THAPI_E_NOMEM;
    std::vector<uint32_t> t_soff(nt), t_ns(nt);
    std::vector<const uint8_t *> t_src(nt);
    std::vector<uint64_t> t_first(nt);
    uint64_t at = 0;
    uint32_t soff = 0;
    for (uint32_t t = 0; t < nt; ++t) {
      const HostLayout &b = blay_[t];
      const uint8_t *src = static_cast<const uint8_t *>(bptr_[t]) + b.packets_off;
      if (!bdev_ && b.n_packets)
        CK(cudaMemcpyAsync(pk + at * P, src, b.n_packets * (uint64_t)P, cudaMemcpyHostToDevice, s_));
      if (bdev_ && b.n_packets && reinterpret_cast<uintptr_t>(src) % 16 != 0) return THAPI_E_INVALID;
      t_src[t] = src;
      t_first[t] = at;
      t_soff[t] = soff;
      t_ns[t] = b.n_streams;
      at += b.n_packets;
      soff += b.n_streams;
    }
    {  // per packet its trace (from the traces' first packets), and with device
       // traces the address of every packet, no copy
      uint64_t *d_first = static_cast<uint64_t *>(sc_.get(nt * sizeof(uint64_t)));
      const uint8_t **d_src = bdev_ ? static_cast<const uint8_t **>(sc_.get(nt * sizeof(void *))) : nullptr;
      if (sc_.failed) return THAPI_E_NOMEM;
      CK(cudaMemcpyAsync(d_first, t_first.data(), nt * sizeof(uint64_t), cudaMemcpyHostToDevice, s_));
      launch_packet_traces(d_first, nt, n, d_pk_trace, s_);
      if (bdev_ && n) {
        CK(cudaMemcpyAsync(d_src, t_src.data(), nt * sizeof(void *), cudaMemcpyHostToDevice, s_));
        launch_packet_addrs(d_src, d_first, d_pk_trace, n, P, pk_addr, s_);
      }
      CK(cudaGetLastError());
    }
    CK(cudaMemcpyAsync(d_t_soff, t_soff.data(), 4ull * nt, cudaMemcpyHostToDevice, s_));
    CK(cudaMemcpyAsync(d_t_ns, t_ns.data(), 4ull * nt, cudaMemcpyHostToDevice, s_));
    CK(cudaStreamSynchronize(s_));  // the host tables above go out of scope
    packets = pk;
  } else if (host_) {
    uint8_t *pk = alloc<uint8_t>(n * (uint64_t)P);
    if (!pk) return THAPI_E_NOMEM;
    if (n) CK(cudaMemcpyAsync(pk, host_ + L.packets_off, n * (uint64_t)P, cudaMemcpyHostToDevice, s_));
    packets = pk;
  } else {
    packets = dev_ + L.packets_off;
    if (reinterpret_cast<uintptr_t>(packets) % 16 != 0) return THAPI_E_INVALID;
  }

  // ---- small tables and counters
  misc_ = alloc<uint64_t>(mCount);
  uint64_t *d_cls = alloc<uint64_t>(L.n_classes);
  uint32_t *d_group = alloc<uint32_t>(S);
  uint32_t *d_gkeys = alloc<uint32_t>(group_keys.size());
  if (!misc_ || !d_cls || !d_group || !d_gkeys) return THAPI_E_NOMEM;
  for (int i = 0; i < mCount; ++i) misc_h_[i] = 0;
  misc_h_[mHdrErr] = misc_h_[mContentErr] = misc_h_[mTmin] = ~0ull;
  CK(cudaMemcpyAsync(misc_, misc_h_, sizeof(misc_h_), cudaMemcpyHostToDevice, s_));
  if (L.n_classes) CK(cudaMemcpyAsync(d_cls, L.cls.data(), 8ull * L.n_classes, cudaMemcpyHostToDevice, s_));
  if (S) CK(cudaMemcpyAsync(d_group, stream_group.data(), 4ull * S, cudaMemcpyHostToDevice, s_));
  if (G) CK(cudaMemcpyAsync(d_gkeys, group_keys.data(), 4ull * group_keys.size(), cudaMemcpyHostToDevice, s_));

  // ---- index: headers, group by stream (stable), seq check, event offsets
  uint32_t *pk_stream = alloc<uint32_t>(n), *pk_nev = alloc<uint32_t>(n), *pk_content = alloc<uint32_t>(n);
  uint32_t *pk_seq = alloc<uint32_t>(n), *pk_disc = alloc<uint32_t>(n);
  uint64_t *pk_tsb = alloc<uint64_t>(n), *keys = alloc<uint64_t>(n), *keys_alt = alloc<uint64_t>(n);
  uint32_t *vals = alloc<uint32_t>(n), *vals_alt = alloc<uint32_t>(n);
  uint64_t *evbase = alloc<uint64_t>(n);
  uint32_t *stream_first = alloc<uint32_t>(S), *stream_count = alloc<uint32_t>(S);
  if (sc_.failed) return THAPI_E_NOMEM;
  CK(cudaMemsetAsync(stream_first, 0, 4ull * (S ? S : 1), s_));
  CK(cudaMemsetAsync(stream_count, 0, 4ull * (S ? S : 1), s_));
  unsigned long long *hdr_err = reinterpret_cast<unsigned long long *>(misc_ + mHdrErr);
  clk_.rec(PhaseClock::kIdx0, s_);
  launch_packet_headers(IndexParams{packets, pk_addr, reinterpret_cast<unsigned long long *>(misc_ + mReadBytes), P,
                                    n, S, pk_stream, pk_nev, pk_content, pk_seq, pk_disc, pk_tsb, hdr_err, d_pk_trace,
                                    d_t_soff, d_t_ns},
                        s_);
  launch_stream_keys(pk_stream, n, keys, vals, s_);
  bool in_alt = false;
  int sbits = 1;
  while ((1ull << sbits) <= (uint64_t)S) ++sbits;  // the invalid-stream sentinel S must fit
  radix_sort_pairs(keys, vals, keys_alt, vals_alt, n, sbits, &in_alt, sc_, s_);
  if (sc_.failed) return THAPI_E_NOMEM;
  const uint64_t *skey = in_alt ? keys_alt : keys;
  const uint32_t *order = in_alt ? vals_alt : vals;
  launch_stream_bounds(skey, order, pk_seq, pk_nev, n, S, stream_first, stream_count, evbase, hdr_err, s_);
  scan_exclusive_u64(evbase, n, misc_ + mEvents, sc_, s_);
  if (sc_.failed) return THAPI_E_NOMEM;
  clk_.rec(PhaseClock::kIdx1, s_);
  CK(cudaGetLastError());
  if ((rc = sync_misc()) != THAPI_OK) return rc;
  if (misc_h_[mHdrErr] != ~0ull) {
    set_err(c_, 1, misc_h_[mHdrErr], 0);
    return THAPI_E_FORMAT;
  }
  const uint64_t total_events = n ? misc_h_[mEvents] : 0;
  if (dec_n_)
    return decode(L, n, total_events, packets, order, pk_stream, pk_nev, pk_content, pk_disc, pk_tsb, d_group, evbase,
                  d_cls, d_gkeys);

  // ---- decode + pair + tally per packet
  Cell *tally = alloc<Cell>(cells);
  uint32_t *sum_pend = alloc<uint32_t>(n), *sum_open = alloc<uint32_t>(n), *sum_nslot = alloc<uint32_t>(n);
  uint32_t *sum_nvalid = alloc<uint32_t>(n), *dense_list = alloc<uint32_t>(n);
  uint32_t *A = alloc<uint32_t>(n), *base = alloc<uint32_t>(n);
  uint64_t *sum_fbase = alloc<uint64_t>(n);
  thapi_interval *slots = alloc<thapi_interval>(total_events);
  if (self_on && total_events >= 0x80000000ull) return THAPI_E_UNSUPPORTED;  // levels below the kSelfAbs bit
  SelfSlot *side = self_on ? alloc<SelfSlot>(total_events) : nullptr;
  if (sc_.failed) return THAPI_E_NOMEM;
  PkDesc *desc = alloc<PkDesc>(n);
  if (!desc) return THAPI_E_NOMEM;
  launch_build_desc(order, pk_stream, pk_nev, pk_content, pk_disc, pk_tsb, d_group, evbase, n, desc, s_);
  const uint32_t emax_main = ((P - kPacketHeader) / 4) / 4;
  const int stages = n ? pick_stages(c_, P, emax_main, L.n_classes, F) : 1;
  if (!stages) return THAPI_E_UNSUPPORTED;
  // warp-per-packet kernel for packets up to 32 KB, the CTA kernel otherwise
  WarpPlan wplan;
  const bool warp_path = plan_analyze_warp(P, L.n_classes, c_->smem_per_block, c_->smem_per_sm, &wplan);
  // per-CPU buffers: packets up to 32 KB (the warp kernels), 32-bit event indexes
  if (has_pc && (!warp_path || total_events >= 0xFFFFFFFFull || !decode_warps(P, L.n_classes, c_->smem_per_block)))
    return THAPI_E_UNSUPPORTED;
  uint64_t grid = 1, per = 1;
  if (n) {
    if (warp_path) {
      grid = (uint64_t)c_->num_sms * wplan.ctas_per_sm * std::max<uint32_t>(1, tune_.grid_mult);
    } else {
      const uint32_t smem = analyze_smem_bytes(P, emax_main, stages, L.n_classes, F);
      grid = (uint64_t)c_->num_sms * blocks_per_sm(c_, smem);
    }
    per = (n + grid - 1) / grid;
    grid = (n + per - 1) / per;
  }
  uint64_t fcap = total_events / 16 + 4096 +
                  (warp_path ? analyze_warp_frontier_slack(grid * wplan.nw) : analyze_frontier_slack((uint32_t)grid)) +
                  analyze_frontier_slack((uint32_t)c_->num_sms * 16);
  Frontier *frontier = nullptr;
  unsigned *status = reinterpret_cast<unsigned *>(misc_ + mStatus);
  uint32_t *run_start = alloc<uint32_t>(grid + 1);
  if (!run_start) return THAPI_E_NOMEM;
  CmdOut cmd;
  if (dev_on && total_events >= 0xFFFFFFFFull) return THAPI_E_UNSUPPORTED;  // 32-bit record indexes
  uint64_t cap_b = dev_on ? total_events / 2 + 1024 : 0, cap_e = cap_b, cap_h = cap_b;
  // command-id partitions: about 1.5k records each at most (the records are at most the events)
  int part_bits = 1;
  const uint64_t part_target =
      tune_.part_shift >= 0 ? 1536ull << tune_.part_shift : 1536ull >> (uint32_t)(-tune_.part_shift);
  while (part_bits < 18 && (total_events >> part_bits) > part_target) ++part_bits;
  const uint64_t n_part = 1ull << part_bits;
  uint32_t *part_hist = dev_on ? alloc<uint32_t>(3 * n_part) : nullptr;
  if (dev_on && !part_hist) return THAPI_E_NOMEM;
  for (int attempt = 0;; ++attempt) {
    if (dev_on) {  // (re)sized per attempt: a second attempt knows the exact counts
      cmd.b = alloc<CmdBegin>(cap_b);
      cmd.e = alloc<CmdEnd>(cap_e);
      cmd.h = alloc<CmdHost>(cap_h);
      if (sc_.failed) return THAPI_E_NOMEM;
      cmd.cap_b = cap_b;
      cmd.cap_e = cap_e;
      cmd.cap_h = cap_h;
      cmd.counts = reinterpret_cast<unsigned long long *>(misc_ + mCmdCount0);
      cmd.hist = part_hist;
      cmd.part_bits = part_bits;
      CK(cudaMemsetAsync(misc_ + mCmdCount0, 0, 3 * sizeof(uint64_t), s_));
      CK(cudaMemsetAsync(part_hist, 0, 3 * n_part * sizeof(uint32_t), s_));
    }
    frontier = static_cast<Frontier *>(dev_alloc(c_, fcap * sizeof(Frontier), s_));
    if (!frontier) return THAPI_E_NOMEM;
    sc_.adopt(frontier, fcap * sizeof(Frontier));
    launch_tally_init(tally, cells, s_);
    misc_h_[mContentErr] = ~0ull;
    for (int d = 0; d < dCount; ++d) misc_h_[mDiag0 + d] = 0;
    misc_h_[mTmin] = ~0ull;
    misc_h_[mTmax] = misc_h_[mFrontTop] = misc_h_[mDense] = misc_h_[mStatus] = 0;
    CK(cudaMemcpyAsync(misc_ + mContentErr, misc_h_ + mContentErr, sizeof(uint64_t) * (mStatus - mContentErr + 1),
                       cudaMemcpyHostToDevice, s_));
    misc_h_[mSlots] = 0;
    CK(cudaMemcpyAsync(misc_ + mSlots, misc_h_ + mSlots, sizeof(uint64_t), cudaMemcpyHostToDevice, s_));
    AnalyzeParams ap{};
    ap.packets = packets;
    ap.pk_addr = pk_addr;
    ap.P = P;
    ap.emax = emax_main;
    ap.n_order = n;
    ap.poslist = nullptr;
    ap.desc = desc;
    ap.classes = d_cls;
    ap.n_classes = L.n_classes;
    ap.n_funcs = F;
    ap.tally = tally;
    ap.sum_pend = sum_pend;
    ap.sum_open = sum_open;
    ap.sum_nslot = sum_nslot;
    ap.sum_nvalid = sum_nvalid;
    ap.sum_fbase = sum_fbase;
    ap.frontier = frontier;
    ap.frontier_top = reinterpret_cast<unsigned long long *>(misc_ + mFrontTop);
    ap.frontier_cap = fcap;
    ap.slots = slots;
    ap.content_err = reinterpret_cast<unsigned long long *>(misc_ + mContentErr);
    ap.diag = reinterpret_cast<unsigned long long *>(misc_ + mDiag0);
    ap.tminmax = reinterpret_cast<unsigned long long *>(misc_ + mTmin);
    ap.dense_list = dense_list;
    ap.dense_count = reinterpret_cast<unsigned long long *>(misc_ + mDense);
    ap.slots_written = reinterpret_cast<unsigned long long *>(misc_ + mSlots);
    ap.cmd = cmd;
    ap.side = side;
    ap.run_start = nullptr;
    if (n && warp_path) {
      ap.run_start = run_start;
      launch_cost_split(evbase, n, total_events, (uint32_t)grid, run_start, s_);
    }
    if (n) {
      ap.per_cta = (uint32_t)per;
      clk_.rec(PhaseClock::kAn0, s_);
      if (warp_path)
        CK(launch_analyze_warp(ap, wplan, (uint32_t)grid, s_, status));
      else
        CK(launch_analyze(ap, stages, (uint32_t)grid, s_, status));
      clk_.rec(PhaseClock::kAn1, s_);
      analyze_launches = 1;
      if ((rc = sync_misc()) != THAPI_OK) return rc;
      if (misc_h_[mDense]) {
        AnalyzeParams dp = ap;
        dp.run_start = nullptr;
        dp.emax = ((P - kPacketHeader) / 4) / 2 + 1;
        dp.n_order = misc_h_[mDense];
        dp.poslist = dense_list;
        dp.dense_list = nullptr;
        dp.dense_count = nullptr;
        const int dstages = pick_stages(c_, P, dp.emax, L.n_classes, F);
        if (!dstages) return THAPI_E_UNSUPPORTED;
        uint32_t dsmem = analyze_smem_bytes(P, dp.emax, dstages, L.n_classes, F);
        uint64_t dgrid = std::min<uint64_t>(dp.n_order, (uint64_t)c_->num_sms * blocks_per_sm(c_, dsmem));
        uint64_t dper = (dp.n_order + dgrid - 1) / dgrid;
        dp.per_cta = (uint32_t)dper;
        dgrid = (dp.n_order + dper - 1) / dper;
        clk_.rec(PhaseClock::kDn0, s_);
        CK(launch_analyze(dp, dstages, (uint32_t)dgrid, s_, status));
        clk_.rec(PhaseClock::kDn1, s_);
        clk_.dense = true;
        analyze_launches = 2;
        if ((rc = sync_misc()) != THAPI_OK) return rc;
      }
    }
    if (misc_h_[mStatus] == THAPI_E_TIMEOUT) return THAPI_E_TIMEOUT;
    if (misc_h_[mContentErr] != ~0ull) {
      const unsigned long long k = misc_h_[mContentErr];
      set_err(c_, 2, k >> 20, (k >> 3) & 0x1FFFFu);
      return (int)(k & 7u);
    }
    const uint64_t nb = misc_h_[mCmdCount0], ne = misc_h_[mCmdCount0 + 1], nh = misc_h_[mCmdCount0 + 2];
    const bool cmd_over = dev_on && (nb > cap_b || ne > cap_e || nh > cap_h);
    if ((misc_h_[mFrontTop] <= fcap && !cmd_over) || attempt >= 1) break;
    // retry once with the exact frontier size and record counts
    fcap = std::max(fcap, (uint64_t)misc_h_[mFrontTop]);
    cap_b = std::max(cap_b, nb);
    cap_e = std::max(cap_e, ne);
    cap_h = std::max(cap_h, nh);
  }
  if (misc_h_[mFrontTop] > fcap) return THAPI_E_NOMEM;
  if (dev_on && (misc_h_[mCmdCount0] > cap_b || misc_h_[mCmdCount0 + 1] > cap_e || misc_h_[mCmdCount0 + 2] > cap_h))
    return THAPI_E_NOMEM;

  // ---- pairing across packets
  {
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
    fp.slots = slots;
    fp.sum_nvalid = sum_nvalid;
    fp.diag = reinterpret_cast<unsigned long long *>(misc_ + mDiag0);
    fp.side = side;
    clk_.rec(PhaseClock::kFr0, s_);
    launch_frontier(fp, s_);
    clk_.rec(PhaseClock::kFr1, s_);
  }

  // ---- per-CPU buffers: their events' records, then their threads paired
  PcPairOut pco;
  if (has_pc) {
    clk_.rec(PhaseClock::kPc0, s_);
    uint32_t *d_shost = alloc<uint32_t>(S);
    PcRec *pcrec = alloc<PcRec>(total_events);
    uint64_t *pc_base = alloc<uint64_t>(n);
    if (sc_.failed) return THAPI_E_NOMEM;
    launch_pc_count(desc, n, pc_base, s_);
    scan_exclusive_u64(pc_base, n, misc_ + mPcAll, sc_, s_);
    if (sc_.failed) return THAPI_E_NOMEM;
    CK(cudaMemcpyAsync(d_shost, stream_host.data(), 4ull * S, cudaMemcpyHostToDevice, s_));
    CK(cudaMemsetAsync(misc_ + mPcCount, 0, sizeof(uint64_t), s_));
    PcParams pp{};
    pp.packets = packets;
    pp.pk_addr = pk_addr;
    pp.P = P;
    pp.n_classes = L.n_classes;
    pp.n_order = n;
    pp.desc = desc;
    pp.classes = d_cls;
    pp.stream_host = d_shost;
    pp.rec = pcrec;
    pp.pc_base = pc_base;
    pp.cap = total_events;
    pp.count = reinterpret_cast<unsigned long long *>(misc_ + mPcCount);
    pp.slots = slots;
    pp.sum_nslot = sum_nslot;
    pp.content_err = reinterpret_cast<unsigned long long *>(misc_ + mContentErr);
    pp.diag = reinterpret_cast<unsigned long long *>(misc_ + mDiag0);
    pp.tminmax = reinterpret_cast<unsigned long long *>(misc_ + mTmin);
    const uint32_t nw = decode_warps(P, L.n_classes, c_->smem_per_block);
    const uint64_t g = std::min<uint64_t>((n + nw - 1) / nw, (uint64_t)c_->num_sms * 4);
    clk_.rec(PhaseClock::kPd0, s_);
    CK(launch_percpu_decode(pp, nw, (uint32_t)std::max<uint64_t>(g, 1), s_));
    clk_.rec(PhaseClock::kPd1, s_);
    launch_pc_bytes(desc, sum_nslot, n, reinterpret_cast<unsigned long long *>(misc_ + mPcRead), s_);
    if ((rc = sync_misc()) != THAPI_OK) return rc;
    if (misc_h_[mContentErr] != ~0ull) {
      const unsigned long long k = misc_h_[mContentErr];
      set_err(c_, 2, k >> 20, (k >> 3) & 0x1FFFFu);
      return (int)(k & 7u);
    }
    const uint64_t m = misc_h_[mPcCount];
    const uint64_t t0 = misc_h_[mTmin], t1 = misc_h_[mTmax];
    int tb = 1;
    while (tb < 64 && t1 > t0 && ((t1 - t0) >> tb)) ++tb;
    rc = percpu_pair(pcrec, misc_h_[mPcAll], m, m ? t0 : 0, tb, F, slots, sum_nvalid,
                     reinterpret_cast<unsigned long long *>(misc_ + mDiag0), self_on, c_->num_sms, sc_, s_, &pco);
    if (rc != THAPI_OK) return rc;
    clk_.rec(PhaseClock::kPc1, s_);
  }

  // ---- device-activity pairing: command table, then device intervals and tally
  Cell *dcells = nullptr;
  if (dev_on) {
    const uint64_t nb = misc_h_[mCmdCount0], ne = misc_h_[mCmdCount0 + 1], nh = misc_h_[mCmdCount0 + 2];
    if (nb + ne + nh >= 0xFFFFFFFFull) return THAPI_E_UNSUPPORTED;  // 32-bit counts per table entry
    dcells = alloc<Cell>(cells);
    if (!dcells) return THAPI_E_NOMEM;
    launch_tally_init(dcells, cells, s_);
    CK(cudaMemsetAsync(misc_ + mJoin0, 0, 6 * sizeof(uint64_t), s_));
    JoinParams jp{};
    jp.b = cmd.b;
    jp.e = cmd.e;
    jp.h = cmd.h;
    jp.nb = nb;
    jp.ne = ne;
    jp.nh = nh;
    jp.slots = slots;
    jp.sum_nvalid = sum_nvalid;
    jp.dcells = dcells;
    jp.n_funcs = F;
    jp.out = reinterpret_cast<unsigned long long *>(misc_ + mJoin0);
    clk_.rec(PhaseClock::kJo0, s_);
    // partitioned join when every partition fits a shared-memory table
    PartPlan pp{};
    pp.part_bits = part_bits;
    pp.hist = part_hist;
    pp.base = alloc<uint64_t>(3 * n_part + 1);
    pp.cursor = reinterpret_cast<unsigned long long *>(alloc<uint64_t>(3 * n_part));
    pp.max_records = reinterpret_cast<unsigned long long *>(misc_ + mPartMax);
    if (sc_.failed) return THAPI_E_NOMEM;
    CK(cudaMemsetAsync(misc_ + mPartMax, 0, sizeof(uint64_t), s_));
    launch_part_prep(pp, s_);
    scan_exclusive_u64(pp.base, 3 * n_part, pp.base + 3 * n_part, sc_, s_);
    if (sc_.failed) return THAPI_E_NOMEM;
    CK(cudaGetLastError());
    if ((rc = sync_misc()) != THAPI_OK) return rc;
    if (misc_h_[mPartMax] <= kPartMaxRecords) {
      pp.pb = alloc<CmdBegin>(nb);
      pp.pe = alloc<CmdEnd>(ne);
      pp.ph = alloc<CmdHost>(nh);
      if (sc_.failed) return THAPI_E_NOMEM;
      launch_part_scatter(jp, pp, c_->num_sms, s_);
      launch_part_join(jp, pp, misc_h_[mPartMax], s_);
    } else {
      // one global table: room for twice the largest record kind, short probes;
      // if an insert runs out of probes, a table with room for twice every record
      for (int attempt = 0; attempt < 2; ++attempt) {
        const uint64_t want = attempt == 0 ? 2 * std::max(nb, std::max(ne, nh)) : 2 * (nb + ne + nh);
        uint64_t cap = 1024;
        while (cap < want) cap <<= 1;
        jp.tab = alloc<CmdEntry>(cap + 1);
        if (!jp.tab) return THAPI_E_NOMEM;
        jp.mask = cap - 1;
        jp.probe_limit = attempt == 0 ? 4096 : cap;
        CK(cudaMemsetAsync(jp.tab, 0, (cap + 1) * sizeof(CmdEntry), s_));
        launch_cmd_insert(jp, c_->num_sms, s_);
        if (attempt == 1) break;
        CK(cudaGetLastError());
        if ((rc = sync_misc()) != THAPI_OK) return rc;
        if (!misc_h_[mJoin0 + 5]) break;
        CK(cudaMemsetAsync(misc_ + mJoin0 + 5, 0, sizeof(uint64_t), s_));
      }
      launch_cmd_emit(jp, c_->num_sms, s_);
    }
    clk_.rec(PhaseClock::kJo1, s_);
  }

  // ---- tally rows (host calls; device intervals apart) and interval offsets
  uint64_t *flags = alloc<uint64_t>(cells);
  thapi_tally_row *rows_tmp = alloc<thapi_tally_row>(cells);
  thapi_tally_row *drows_tmp = dev_on ? alloc<thapi_tally_row>(cells) : nullptr;
  uint64_t *obase = alloc<uint64_t>(n);
  if (sc_.failed) return THAPI_E_NOMEM;
  launch_tally_compact(tally, cells, d_gkeys, F, flags, rows_tmp, misc_ + mRows, sc_, s_);
  if (dev_on) launch_tally_compact(dcells, cells, d_gkeys, F, flags, drows_tmp, misc_ + mDevRows, sc_, s_);
  const uint64_t pc_cells = pco.threads * F;
  thapi_tally_row *pcrows = nullptr;
  if (pc_cells) {  // the threads of the per-CPU buffers, compacted like the per-thread rows
    uint64_t *pcflags = alloc<uint64_t>(pc_cells);
    pcrows = alloc<thapi_tally_row>(pc_cells);
    if (sc_.failed) return THAPI_E_NOMEM;
    launch_tally_compact(pco.cells, pc_cells, pco.keys, F, pcflags, pcrows, misc_ + mPcRows, sc_, s_);
  }
  launch_widen_u32(sum_nvalid, obase, n, s_);
  scan_exclusive_u64(obase, n, misc_ + mIv, sc_, s_);
  if (sc_.failed) return THAPI_E_NOMEM;
  clk_.rec(PhaseClock::kTa1, s_);
  CK(cudaGetLastError());
  if ((rc = sync_misc()) != THAPI_OK) return rc;
  uint64_t n_rows = cells ? misc_h_[mRows] : 0;
  const uint64_t n_dev_rows = dev_on && cells ? misc_h_[mDevRows] : 0;
  if (pc_cells && misc_h_[mPcRows]) {  // merge them into the per-thread rows (equal keys combine)
    const uint64_t n_pc = misc_h_[mPcRows];
    thapi_tally_row *both = alloc<thapi_tally_row>(n_rows + n_pc);
    thapi_tally_row *merged = alloc<thapi_tally_row>(n_rows + n_pc);
    if (sc_.failed) return THAPI_E_NOMEM;
    if (n_rows)
      CK(cudaMemcpyAsync(both, rows_tmp, n_rows * sizeof(thapi_tally_row), cudaMemcpyDeviceToDevice, s_));
    CK(cudaMemcpyAsync(both + n_rows, pcrows, n_pc * sizeof(thapi_tally_row), cudaMemcpyDeviceToDevice, s_));
    if (!tally_merge_device(both, n_rows + n_pc, merged, misc_ + mMerged, sc_, s_))
      return sc_.failed ? THAPI_E_NOMEM : THAPI_E_CUDA;
    if ((rc = sync_misc()) != THAPI_OK) return rc;
    n_rows = misc_h_[mMerged];
    rows_tmp = merged;
  }
  const uint64_t n_iv = n ? misc_h_[mIv] : 0;
  if (n_iv >= 0xFFFFFFFFull) return THAPI_E_UNSUPPORTED;

  // ---- self time (when asked for): per-thread streams here (when the trace has any), per-CPU
  //      threads from their pairing
  if (self_on) {
    clk_.rec(PhaseClock::kSe0, s_);
    Cell *scells = alloc<Cell>(cells);
    uint64_t *sflags = alloc<uint64_t>(cells);
    thapi_tally_row *srows = alloc<thapi_tally_row>(cells);
    if (sc_.failed) return THAPI_E_NOMEM;
    launch_tally_init(scells, cells, s_);
    SelfIn si{};
    si.slots = slots;
    si.side = side;
    si.evbase = evbase;
    si.obase = obase;
    si.nslot = sum_nslot;
    si.A = A;
    si.order = order;
    si.pk_stream = pk_stream;
    si.stream_group = d_group;
    si.n_funcs = F;
    si.n_streams = S;
    si.n_order = n;
    si.n_iv = n_iv;
    si.num_sms = c_->num_sms;
    if (G && (rc = self_time(si, scells, misc_ + mSelfWord, sc_, s_)) != THAPI_OK) return rc;
    launch_tally_compact(scells, cells, d_gkeys, F, sflags, srows, misc_ + mSelfRows, sc_, s_);
    thapi_tally_row *spcrows = nullptr;
    if (pco.self_cells && pc_cells) {
      uint64_t *pflags = alloc<uint64_t>(pc_cells);
      spcrows = alloc<thapi_tally_row>(pc_cells);
      if (sc_.failed) return THAPI_E_NOMEM;
      launch_tally_compact(pco.self_cells, pc_cells, pco.keys, F, pflags, spcrows, misc_ + mSelfPcRows, sc_, s_);
    }
    if (sc_.failed) return THAPI_E_NOMEM;
    CK(cudaGetLastError());
    if ((rc = sync_misc()) != THAPI_OK) return rc;
    uint64_t ns = cells ? misc_h_[mSelfRows] : 0;
    if (spcrows && misc_h_[mSelfPcRows]) {  // per-CPU threads' rows merge into the per-thread rows
      const uint64_t n_pc = misc_h_[mSelfPcRows];
      thapi_tally_row *both = alloc<thapi_tally_row>(ns + n_pc);
      thapi_tally_row *merged = alloc<thapi_tally_row>(ns + n_pc);
      if (sc_.failed) return THAPI_E_NOMEM;
      if (ns) CK(cudaMemcpyAsync(both, srows, ns * sizeof(thapi_tally_row), cudaMemcpyDeviceToDevice, s_));
      CK(cudaMemcpyAsync(both + ns, spcrows, n_pc * sizeof(thapi_tally_row), cudaMemcpyDeviceToDevice, s_));
      if (!tally_merge_device(both, ns + n_pc, merged, misc_ + mSelfMerged, sc_, s_))
        return sc_.failed ? THAPI_E_NOMEM : THAPI_E_CUDA;
      if ((rc = sync_misc()) != THAPI_OK) return rc;
      ns = misc_h_[mSelfMerged];
      srows = merged;
    }
    tr_->n_self_rows = ns;
    tr_->self_rows_bytes = std::max<uint64_t>(ns, 1) * sizeof(thapi_tally_row);
    tr_->self_rows = static_cast<thapi_tally_row *>(dev_alloc(c_, tr_->self_rows_bytes, s_));
    if (!tr_->self_rows) return THAPI_E_NOMEM;
    if (ns) CK(cudaMemcpyAsync(tr_->self_rows, srows, ns * sizeof(thapi_tally_row), cudaMemcpyDeviceToDevice, s_));
    clk_.rec(PhaseClock::kSe1, s_);
  }
  if (dev_on && misc_h_[mJoin0 + 5]) return THAPI_E_CUDA;  // a join table without room: not reached
  tr_->rows_bytes = std::max<uint64_t>(n_rows, 1) * sizeof(thapi_tally_row);
  tr_->rows = static_cast<thapi_tally_row *>(dev_alloc(c_, tr_->rows_bytes, s_));
  if (!tr_->rows) return THAPI_E_NOMEM;
  if (n_rows)
    CK(cudaMemcpyAsync(tr_->rows, rows_tmp, n_rows * sizeof(thapi_tally_row), cudaMemcpyDeviceToDevice, s_));
  if (dev_on) {
    tr_->dev_rows_bytes = std::max<uint64_t>(n_dev_rows, 1) * sizeof(thapi_tally_row);
    tr_->dev_rows = static_cast<thapi_tally_row *>(dev_alloc(c_, tr_->dev_rows_bytes, s_));
    if (!tr_->dev_rows) return THAPI_E_NOMEM;
    if (n_dev_rows)
      CK(cudaMemcpyAsync(tr_->dev_rows, drows_tmp, n_dev_rows * sizeof(thapi_tally_row), cudaMemcpyDeviceToDevice,
                         s_));
  }

  // ---- timeline: compact valid slots, sort by start, gather
  thapi_interval *rec = alloc<thapi_interval>(n_iv);
  uint64_t *k1 = alloc<uint64_t>(n_iv);
  if (sc_.failed) return THAPI_E_NOMEM;
  const uint64_t tmin = misc_h_[mTmin], tmax = misc_h_[mTmax];
  int bits = 0;
  if (n_iv && tmax > tmin) {
    const uint64_t span = tmax - tmin;
    while (bits < 64 && (span >> bits)) ++bits;
  }
  BucketCells bcells;
  const bool bucket_on = bucket_plan(n_iv, bits, S, sc_, s_, &bcells);
  if (sc_.failed) return THAPI_E_NOMEM;
  clk_.rec(PhaseClock::kCo0, s_);
  launch_timeline_compact(slots, evbase, sum_nslot, obase, A, order, pk_stream, n, n_iv ? tmin : 0, rec,
                          bucket_on ? nullptr : k1, bits <= 32, nullptr, bucket_on ? &bcells : nullptr, c_->num_sms,
                          s_);
  clk_.rec(PhaseClock::kCo1, s_);
  tr_->tl_bytes = std::max<uint64_t>(n_iv, 1) * sizeof(thapi_interval);
  tr_->tl = static_cast<thapi_interval *>(dev_alloc(c_, tr_->tl_bytes, s_));
  if (!tr_->tl) return THAPI_E_NOMEM;
  if (!bucket_on || !bucket_run(bcells, tmin, n_iv, rec, tr_->tl, sc_, s_, c_->num_sms)) {
    if (sc_.failed) return THAPI_E_NOMEM;
    CK(cudaGetLastError());
    uint64_t *k2 = alloc<uint64_t>(n_iv);
    uint32_t *v1 = alloc<uint32_t>(n_iv), *v2 = alloc<uint32_t>(n_iv);
    if (sc_.failed) return THAPI_E_NOMEM;
    if (bucket_on) launch_rec_keys(rec, n_iv, n_iv ? tmin : 0, k1, bits <= 32, s_);
    radix_sort_gather(k1, v1, k2, v2, n_iv, bits, rec, tr_->tl, sc_, s_);
  }
  if (sc_.failed) return THAPI_E_NOMEM;
  clk_.rec(PhaseClock::kSo1, s_);
  clk_.rec(PhaseClock::kGa1, s_);
  CK(cudaGetLastError());
  if ((rc = sync_misc()) != THAPI_OK) return rc;
  {
    thapi_load_timing &t = tr_->timing;
    t.launches = launches_total() - launches0;
    t.analyze_launches = analyze_launches;
    t.analyze_read_bytes = misc_h_[mReadBytes] - misc_h_[mPcRead];
    t.percpu_read_bytes = misc_h_[mPcRead];
    t.percpu_write_bytes = 32ull * misc_h_[mPcAll] + sizeof(thapi_interval) * misc_h_[mPcEntries];
    t.analyze_write_bytes = misc_h_[mSlots] * sizeof(thapi_interval) +
                            (dev_on ? misc_h_[mCmdCount0] * sizeof(CmdBegin) + misc_h_[mCmdCount0 + 1] * sizeof(CmdEnd) +
                                          misc_h_[mCmdCount0 + 2] * sizeof(CmdHost)
                                    : 0);
    t.grid_mult = std::max<uint32_t>(1, tune_.grid_mult);
    t.call_ms = std::chrono::duration<float, std::milli>(std::chrono::steady_clock::now() - host_t0).count();
    t.part_shift = tune_.part_shift;
    if (clk_.on && n) {
      t.index_ms = clk_.ms(PhaseClock::kIdx0, PhaseClock::kIdx1);
      t.analyze_ms = clk_.ms(PhaseClock::kAn0, PhaseClock::kAn1) +
                     (clk_.dense ? clk_.ms(PhaseClock::kDn0, PhaseClock::kDn1) : 0.f);
      t.frontier_ms = clk_.ms(PhaseClock::kFr0, PhaseClock::kFr1);
      t.join_ms = dev_on ? clk_.ms(PhaseClock::kJo0, PhaseClock::kJo1) : 0.f;
      t.self_ms = self_on ? clk_.ms(PhaseClock::kSe0, PhaseClock::kSe1) : 0.f;
      t.percpu_ms = has_pc ? clk_.ms(PhaseClock::kPc0, PhaseClock::kPc1) : 0.f;
      t.percpu_decode_ms = has_pc ? clk_.ms(PhaseClock::kPd0, PhaseClock::kPd1) : 0.f;
      t.tally_ms = clk_.ms(dev_on ? PhaseClock::kJo1 : PhaseClock::kFr1, PhaseClock::kTa1);
      t.compact_ms = clk_.ms(PhaseClock::kCo0, PhaseClock::kCo1);
      t.sort_ms = clk_.ms(PhaseClock::kCo1, PhaseClock::kSo1);
      t.gather_ms = clk_.ms(PhaseClock::kSo1, PhaseClock::kGa1);
      t.total_ms = clk_.ms(PhaseClock::kIdx0, PhaseClock::kGa1);
    }
  }

  // ---- record
  thapi_diag &d = tr_->diag;
  d.events = misc_h_[mDiag0 + dEvents];
  d.pairs = misc_h_[mDiag0 + dPairs];
  d.unmatched_entries = misc_h_[mDiag0 + dUnEntry];
  d.unmatched_exits = misc_h_[mDiag0 + dUnExit];
  d.mismatched_pairs = misc_h_[mDiag0 + dMismatch];
  d.other_events = misc_h_[mDiag0 + dOther];
  d.discarded = misc_h_[mDiag0 + dDiscarded];
  d.packets = misc_h_[mDiag0 + dPackets];
  thapi_device_diag &dd = tr_->dev_diag;
  dd.dev_events = misc_h_[mDiag0 + dDevEvents];
  if (dev_on) {
    dd.dev_pairs = misc_h_[mJoin0];
    dd.dev_intervals = misc_h_[mJoin0 + 1];
    dd.dev_unjoined = misc_h_[mJoin0 + 2];
    dd.dev_ambiguous = misc_h_[mJoin0 + 3];
    dd.host_cmd_entries = misc_h_[mCmdCount0 + 2];
    dd.host_unjoined = dd.host_cmd_entries - misc_h_[mJoin0 + 4];
  }
  dd.dev_unpaired = dd.dev_events - 2 * dd.dev_pairs;
  thapi_trace_info &inf = tr_->info;
  inf.nbytes = nbytes_;
  inf.n_packets = n;
  inf.events = d.events;
  inf.intervals = n_iv;
  inf.tally_rows = n_rows;
  inf.n_streams = S;
  inf.n_classes = L.n_classes;
  inf.n_funcs = F;
  inf.n_hosts = L.n_hosts;
  inf.packet_bytes = P;
  inf.t_min = tmin == ~0ull ? 0 : tmin;
  inf.t_max = tmax;
  inf.device_bytes = tr_->rows_bytes + tr_->tl_bytes + tr_->dev_rows_bytes + tr_->self_rows_bytes;
  inf.self_time = self_on ? 1u : 0u;
  inf.device_rows = n_dev_rows;
  inf.device_intervals = dd.dev_intervals;
  tr_->strings.assign(L.strings.begin(), L.strings.end());
  tr_->host_name = L.host_name;
  tr_->func_name = L.func_name;
  tr_->func_layer = L.func_layer;
  return THAPI_OK;
}

// Releases the device results of a load that is not kept.
static void drop_trace(thapi_ctx *c, TraceRec *t) {
  dev_free(c, t->win_bmax, t->win_bytes, t->stream);
  dev_free(c, t->rows, t->rows_bytes, t->stream);
  dev_free(c, t->tl, t->tl_bytes, t->stream);
  dev_free(c, t->dev_rows, t->dev_rows_bytes, t->stream);
  dev_free(c, t->self_rows, t->self_rows_bytes, t->stream);
  cudaStreamSynchronize(t->stream);
  delete t;
}

// A load's shape for the autotuner: packet size, device pairing on, batch,
// and the size class (log2 of the packet count).
static uint64_t tune_key(const HostLayout &L, bool batch, uint64_t bytes) {
  bool dev_on = false;
  for (uint64_t cl : L.cls) {
    const uint32_t k = cls_kind(cl);
    dev_on = dev_on || k == kDevBegin || k == kDevEnd || (k == kEntry && cls_cmdw(cl) >= 0);
  }
  int sz = 0;
  while (((bytes / L.P) >> sz) > 1) ++sz;
  return (uint64_t)L.P | ((uint64_t)dev_on << 32) | ((uint64_t)batch << 33) | ((uint64_t)sz << 40);
}

// One load (configure sets the loader's input), with the context's tuned
// configuration for its shape; with autotuning on and the shape not tuned
// yet, every candidate configuration is loaded once and dropped (the results
// are the same), each knob takes the value whose best trial was fastest in
// the phase it acts on (runs per CTA: the analysis; partition size: the device
// join), and the trace is loaded with that configuration, which is
// remembered for the shape.
template <class Configure>
static int load_tuned(thapi_ctx *c, cudaStream_t s, const Reader &head, bool batch, uint64_t bytes,
                      Configure configure, thapi_trace_id *out, bool admitted = false) {
  auto once = [&](const Tuning &t, TraceRec **tr) {
    Loader ld(c, nullptr, nullptr, 0, s);
    configure(ld);
    ld.set_tuning(t);
    if (admitted) ld.set_admitted();
    const int rc = ld.status(ld.run());
    if (rc == THAPI_OK) *tr = ld.take();
    return rc;
  };
  TraceRec *tr = nullptr;
  int rc = THAPI_OK;
  uint64_t key = 0;
  bool tuned = false;
  if (c->autotune) {
    HostLayout L;
    if (parse_layout(head, L) == THAPI_OK) {
      key = tune_key(L, batch, bytes);
      {
        std::lock_guard<std::mutex> g(c->mu);
        tuned = c->tuned.count(key) != 0;
      }
      if (!tuned) {  // try every candidate; each knob is chosen by the phase it acts on
        const bool dev_on = (key >> 32) & 1;
        const uint32_t grids[3] = {1u, 2u, 4u};
        const int32_t parts[3] = {-1, 0, 1};
        float an_best[3] = {1e30f, 1e30f, 1e30f}, jo_best[3] = {1e30f, 1e30f, 1e30f};
        const int timing = c->timing;
        c->timing = 1;
        for (int g = 0; g < 3 && rc == THAPI_OK; ++g)
          for (int q = 0; q < 3 && rc == THAPI_OK; ++q) {
            if (!dev_on && parts[q] != 0) continue;
            TraceRec *cand = nullptr;
            rc = once(Tuning{grids[g], parts[q]}, &cand);
            if (rc != THAPI_OK) break;
            an_best[g] = std::min(an_best[g], cand->timing.analyze_ms);   // the grid acts on the analysis
            jo_best[q] = std::min(jo_best[q], cand->timing.join_ms);      // the partition size on the join
            drop_trace(c, cand);
          }
        c->timing = timing;
        if (rc != THAPI_OK) return rc;
        // a knob leaves its default only for a clear gain (3 %): single trials are noisy
        int bg = 1, bq = 1;  // the defaults: 2 runs per CTA, 1536-record partitions
        for (int g = 0; g < 3; ++g)
          if (g != 1 && an_best[g] < 0.97f * an_best[1] && an_best[g] < an_best[bg]) bg = g;
        for (int q = 0; q < 3 && dev_on; ++q)
          if (q != 1 && jo_best[q] < 0.97f * jo_best[1] && jo_best[q] < jo_best[bq]) bq = q;
        std::lock_guard<std::mutex> g(c->mu);
        c->tuned[key] = Tuning{grids[bg], parts[bq]};  // the load below runs with it
      }
    }
  }
  if (!tr) {
    Tuning t{};
    {
      std::lock_guard<std::mutex> g(c->mu);
      const auto it = c->tuned.find(key);
      if (c->autotune && it != c->tuned.end()) t = it->second;
    }
    rc = once(t, &tr);
    if (rc != THAPI_OK) return rc;
  }
  std::lock_guard<std::mutex> g(c->mu);
  const uint64_t id = c->next_id++;
  c->traces[id] = tr;
  c->used += tr->info.device_bytes;
  *out = id;
  return THAPI_OK;
}

static int load_common(thapi_ctx *c, const uint8_t *host, const uint8_t *dev, uint64_t nbytes, void *stream,
                       thapi_trace_id *out) {
  if (!c || !out || (!host && !dev)) return THAPI_E_INVALID;
  if (cudaSetDevice(c->device) != cudaSuccess) return THAPI_E_CUDA;
  set_err(c, 0, 0, 0);
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  const Reader head{host, dev, nbytes, s};
  return load_tuned(
      c, s, head, false, nbytes, [&](Loader &ld) { ld.set_input(host, dev, nbytes); }, out);
}

static int load_batch(thapi_ctx *c, const void *const *bytes, const uint64_t *nbytes, uint32_t n, int on_device,
                      void *stream, thapi_trace_id *out) {
  if (!c || !out || !bytes || !nbytes || n == 0) return THAPI_E_INVALID;
  for (uint32_t t = 0; t < n; ++t)
    if (!bytes[t]) return THAPI_E_INVALID;
  if (cudaSetDevice(c->device) != cudaSuccess) return THAPI_E_CUDA;
  set_err(c, 0, 0, 0);
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  const uint8_t *b0 = static_cast<const uint8_t *>(bytes[0]);
  const Reader head{on_device ? nullptr : b0, on_device ? b0 : nullptr, nbytes[0], s};  // the shape from trace 0
  uint64_t total = 0;
  for (uint32_t t = 0; t < n; ++t) total += nbytes[t];
  return load_tuned(
      c, s, head, true, total, [&](Loader &ld) { ld.set_batch(bytes, nbytes, n, on_device != 0); }, out);
}

static int decode_common(thapi_ctx *c, const uint8_t *host, uint64_t nbytes, thapi_event *out, uint64_t cap,
                         uint64_t *n_out, void *stream) {
  if (!c || !host || !n_out || (cap && !out)) return THAPI_E_INVALID;
  if (cudaSetDevice(c->device) != cudaSuccess) return THAPI_E_CUDA;
  set_err(c, 0, 0, 0);
  Loader ld(c, host, nullptr, nbytes, static_cast<cudaStream_t>(stream));
  ld.set_decode(out, cap, n_out);
  return ld.status(ld.run());
}

static TraceRec *find(thapi_ctx *c, thapi_trace_id id) {
  if (!c) return nullptr;
  std::lock_guard<std::mutex> g(c->mu);
  auto it = c->traces.find(id);
  return it == c->traces.end() ? nullptr : it->second;
}

// Releases a trace's device results in stream order on `s` and forgets it;
// the memory counts as used until the frees have completed.
int free_trace_on(thapi_ctx *c, thapi_trace_id id, cudaStream_t s) {
  TraceRec *t = nullptr;
  {
    std::lock_guard<std::mutex> g(c->mu);
    auto it = c->traces.find(id);
    if (it == c->traces.end()) return THAPI_E_INVALID;
    t = it->second;
    c->traces.erase(it);
  }
  cudaSetDevice(c->device);
  dev_free(c, t->rows, t->rows_bytes, s);
  dev_free(c, t->tl, t->tl_bytes, s);
  dev_free(c, t->dev_rows, t->dev_rows_bytes, s);
  dev_free(c, t->self_rows, t->self_rows_bytes, s);
  dev_free(c, t->win_bmax, t->win_bytes, s);
  const bool ok = cudaStreamSynchronize(s) == cudaSuccess;
  {
    std::lock_guard<std::mutex> g(c->mu);
    c->used -= std::min(c->used, t->info.device_bytes + t->win_bytes);
  }
  delete t;
  return ok ? THAPI_OK : THAPI_E_CUDA;
}

// Device-visible address of a destination buffer: device or managed memory
// as it is, pinned host memory through its device mapping; null for pageable
// host memory (whose copies are staged).
void *device_view(void *p) {
  cudaPointerAttributes a{};
  if (!p || cudaPointerGetAttributes(&a, p) != cudaSuccess) {
    cudaGetLastError();
    return nullptr;
  }
  if (a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged) return p;
  if (a.type == cudaMemoryTypeHost) return a.devicePointer;
  return nullptr;
}

// Builds a trace's window index (per block of interval slots in timeline
// order, the running maximum of their ends) the first time a window of it is
// asked for; queries on any stream find it complete afterwards.
static int ensure_win_index(thapi_ctx *c, TraceRec *tr, cudaStream_t s) {
  std::lock_guard<std::mutex> g(tr->win_mu);
  if (tr->win_bmax || tr->info.intervals == 0) return THAPI_OK;
  const uint64_t nb = (tr->info.intervals + kWinBlock - 1) / kWinBlock;
  const uint64_t bytes = nb * sizeof(uint64_t);
  uint64_t *b = static_cast<uint64_t *>(dev_alloc(c, bytes, s));
  if (!b) return THAPI_E_NOMEM;
  launch_win_index(tr->tl, tr->info.intervals, b, s);
  if (cudaGetLastError() != cudaSuccess || cudaStreamSynchronize(s) != cudaSuccess) {
    cudaGetLastError();
    dev_free(c, b, bytes, s);
    return THAPI_E_CUDA;
  }
  std::lock_guard<std::mutex> gc(c->mu);
  tr->win_bytes = bytes;
  tr->win_bmax = b;
  c->used += bytes;
  return THAPI_OK;
}

// The window [t0, t1) of a resident timeline: its intervals in timeline order
// to dst (device-visible; null: count only) when they fit cap, and their
// number to *total (device-visible).  Enqueued on s; w: a WinWork in device
// memory, used by one query at a time.
int window_enqueue(thapi_ctx *c, TraceRec *tr, uint64_t t0, uint64_t t1, thapi_interval *dst, uint64_t cap,
                   WinWork *w, unsigned long long *total, cudaStream_t s) {
  const int rc = ensure_win_index(c, tr, s);
  if (rc != THAPI_OK) return rc;
  launch_win_query(tr->tl, tr->info.intervals, tr->win_bmax, t0, t1, w, 2u * (uint32_t)c->num_sms, dst, cap, total,
                   s);
  return cudaGetLastError() == cudaSuccess ? THAPI_OK : THAPI_E_CUDA;
}

// The window's matches into HOST memory `out` once their number n is known:
// small results through the memory's device mapping when it is pinned, the
// others staged in device memory (`stage`, room for n intervals; null: taken
// from the context here) and copied by the copy engine, which moves large
// blocks over the host link faster than stores from the SMs.  Synchronises s.
constexpr uint64_t kMappedMax = 1ull << 20;
static int window_to_host(thapi_ctx *c, TraceRec *tr, uint64_t t0, uint64_t t1, void *out, uint64_t n,
                          thapi_interval *stage, WinWork *w, unsigned long long *total, cudaStream_t s) {
  if (!n) return THAPI_OK;
  const uint64_t bytes = n * sizeof(thapi_interval);
  thapi_interval *mapped = bytes <= kMappedMax ? static_cast<thapi_interval *>(device_view(out)) : nullptr;
  if (mapped) {
    int rc = window_enqueue(c, tr, t0, t1, mapped, n, w, total, s);
    if (rc == THAPI_OK && cudaStreamSynchronize(s) != cudaSuccess) rc = THAPI_E_CUDA;
    return rc;
  }
  Scratch sc;
  sc.ctx = c;
  sc.stream = s;
  if (!stage) stage = static_cast<thapi_interval *>(sc.get(bytes));
  int rc = stage ? window_enqueue(c, tr, t0, t1, stage, n, w, total, s) : THAPI_E_NOMEM;
  if (rc == THAPI_OK && (cudaMemcpyAsync(out, stage, bytes, cudaMemcpyDeviceToHost, s) != cudaSuccess ||
                         cudaStreamSynchronize(s) != cudaSuccess))
    rc = THAPI_E_CUDA;
  sc.release_all();
  cudaStreamSynchronize(s);
  return rc;
}

int timeline_copy_id(thapi_ctx *c, thapi_trace_id id, void *out, uint64_t n, bool device_out, cudaStream_t s) {
  TraceRec *tr = find(c, id);
  if (!tr || n != tr->info.intervals) return THAPI_E_INVALID;
  if (!n) return THAPI_OK;
  return cudaMemcpyAsync(out, tr->tl, n * sizeof(thapi_interval),
                         device_out ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost, s) == cudaSuccess
             ? THAPI_OK
             : THAPI_E_CUDA;
}

int window_to_host_id(thapi_ctx *c, thapi_trace_id id, uint64_t t0, uint64_t t1, void *out, uint64_t n,
                      thapi_interval *stage, WinWork *w, unsigned long long *total, cudaStream_t s) {
  TraceRec *tr = find(c, id);
  if (!tr) return THAPI_E_INVALID;
  return window_to_host(c, tr, t0, t1, out, n, stage, w, total, s);
}

static int timeline_impl(thapi_ctx *c, thapi_trace_id id, uint64_t t0, uint64_t t1, thapi_interval *out,
                         uint64_t cap, uint64_t *n_out, bool device_out, cudaStream_t s) {
  TraceRec *tr = find(c, id);
  if (!tr || !n_out || (cap && !out)) return THAPI_E_INVALID;
  if (cudaSetDevice(c->device) != cudaSuccess) return THAPI_E_CUDA;
  const uint64_t total = tr->info.intervals;
  const bool full = t0 == 0 && t1 == ~0ull;
  if (full || total == 0) {  // the whole timeline (or nothing): one copy
    const uint64_t cnt = full ? total : 0;
    *n_out = cnt;
    if (cap == 0) return THAPI_OK;
    if (cap < cnt) return THAPI_E_RANGE;
    if (cnt == 0) return THAPI_OK;
    cudaError_t e = cudaMemcpyAsync(out, tr->tl, cnt * sizeof(thapi_interval),
                                    device_out ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost, s);
    if (e != cudaSuccess) return THAPI_E_CUDA;
    if (!device_out && cudaStreamSynchronize(s) != cudaSuccess) return THAPI_E_CUDA;
    return THAPI_OK;
  }
  Scratch sc;
  sc.ctx = c;
  sc.stream = s;
  WinWork *w = static_cast<WinWork *>(sc.get(sizeof(WinWork)));
  unsigned long long *tot = static_cast<unsigned long long *>(sc.get(sizeof(unsigned long long)));
  if (!w || !tot) {
    sc.release_all();
    return THAPI_E_NOMEM;
  }
  // device destinations take the matches in the counting pass; host ones
  // are written once the count is known
  thapi_interval *dst = cap && device_out ? out : nullptr;
  int rc = window_enqueue(c, tr, t0, t1, dst, dst ? cap : 0, w, tot, s);
  unsigned long long cnt = 0;
  if (rc == THAPI_OK && (cudaMemcpyAsync(&cnt, tot, sizeof(cnt), cudaMemcpyDeviceToHost, s) != cudaSuccess ||
                         cudaStreamSynchronize(s) != cudaSuccess))
    rc = THAPI_E_CUDA;
  if (rc == THAPI_OK) {
    *n_out = cnt;
    if (cap && cap < cnt)
      rc = THAPI_E_RANGE;
    else if (cap && !device_out)
      rc = window_to_host(c, tr, t0, t1, out, cnt, nullptr, w, tot, s);
  }
  sc.release_all();
  cudaStreamSynchronize(s);
  return rc;
}

// ---------------------------------------------------------------- serving-loop hooks (server.cu)
int ctx_device(const thapi_ctx *c) { return c->device; }
int ctx_num_sms(const thapi_ctx *c) { return c->num_sms; }
void ctx_memory(thapi_ctx *c, uint64_t *cap, uint64_t *used) {
  std::lock_guard<std::mutex> g(c->mu);
  *cap = c->cap;
  *used = c->used;
}
void *ctx_alloc(thapi_ctx *c, uint64_t bytes, cudaStream_t s) { return dev_alloc(c, bytes, s); }
void ctx_free(thapi_ctx *c, void *p, uint64_t bytes, cudaStream_t s) { dev_free(c, p, bytes, s); }

// What admission charges for loading this trace (the load's coarse peak).
int load_charge(thapi_ctx *c, const uint8_t *host, const uint8_t *dev, uint64_t nbytes, cudaStream_t s,
                uint64_t *est) {
  HostLayout L;
  const Reader r{host, dev, nbytes, s};
  const int rc = parse_layout(r, L);
  if (rc != THAPI_OK) return rc;
  *est = load_estimate(L, group_count(L), host != nullptr, c->self_time != 0);
  return THAPI_OK;
}

// A load the serving loop admitted (no cap check here).  The trace is left
// bound to no stream: later frees outside the loop use the default stream.
int load_admitted(thapi_ctx *c, const uint8_t *host, const uint8_t *dev, uint64_t nbytes, cudaStream_t s,
                  thapi_trace_id *out) {
  if (!c || !out || (!host && !dev)) return THAPI_E_INVALID;
  if (cudaSetDevice(c->device) != cudaSuccess) return THAPI_E_CUDA;
  const Reader head{host, dev, nbytes, s};
  const int rc = load_tuned(
      c, s, head, false, nbytes, [&](Loader &ld) { ld.set_input(host, dev, nbytes); }, out, true);
  if (rc == THAPI_OK) {
    std::lock_guard<std::mutex> g(c->mu);
    c->traces[*out]->stream = nullptr;
  }
  return rc;
}

int trace_sizes(thapi_ctx *c, thapi_trace_id id, uint64_t *rows, uint64_t *intervals, uint64_t *events) {
  TraceRec *t = find(c, id);
  if (!t) return THAPI_E_INVALID;
  *rows = t->info.tally_rows;
  *intervals = t->info.intervals;
  *events = t->info.events;
  return THAPI_OK;
}

// Tally rows to dst (host or device memory; the copy is enqueued on s).
int tally_enqueue(thapi_ctx *c, thapi_trace_id id, thapi_tally_row *dst, uint64_t cap, uint64_t *n, cudaStream_t s) {
  TraceRec *t = find(c, id);
  if (!t) return THAPI_E_INVALID;
  *n = t->info.tally_rows;
  if (cap < *n) return THAPI_E_RANGE;
  if (*n && cudaMemcpyAsync(dst, t->rows, *n * sizeof(thapi_tally_row), cudaMemcpyDefault, s) != cudaSuccess)
    return THAPI_E_CUDA;
  return THAPI_OK;
}

int window_enqueue_id(thapi_ctx *c, thapi_trace_id id, uint64_t t0, uint64_t t1, thapi_interval *dst, uint64_t cap,
                      WinWork *w, unsigned long long *total, cudaStream_t s) {
  TraceRec *t = find(c, id);
  if (!t) return THAPI_E_INVALID;
  return window_enqueue(c, t, t0, t1, dst, cap, w, total, s);
}

static int tally_impl(thapi_ctx *c, thapi_trace_id id, thapi_tally_row *rows, uint64_t cap, uint64_t *n_rows,
                      thapi_diag *diag, bool device_out, cudaStream_t s) {
  TraceRec *tr = find(c, id);
  if (!tr || !n_rows || (cap && !rows)) return THAPI_E_INVALID;
  if (cudaSetDevice(c->device) != cudaSuccess) return THAPI_E_CUDA;
  const uint64_t n = tr->info.tally_rows;
  *n_rows = n;
  if (diag) *diag = tr->diag;
  if (cap == 0) return THAPI_OK;
  if (cap < n) return THAPI_E_RANGE;
  if (!n) return THAPI_OK;
  if (cudaMemcpyAsync(rows, tr->rows, n * sizeof(thapi_tally_row),
                      device_out ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost, s) != cudaSuccess)
    return THAPI_E_CUDA;
  if (!device_out && cudaStreamSynchronize(s) != cudaSuccess) return THAPI_E_CUDA;
  return THAPI_OK;
}

static int device_tally_impl(thapi_ctx *c, thapi_trace_id id, thapi_tally_row *rows, uint64_t cap, uint64_t *n_rows,
                             thapi_device_diag *diag) {
  TraceRec *tr = find(c, id);
  if (!tr || !n_rows || (cap && !rows)) return THAPI_E_INVALID;
  if (cudaSetDevice(c->device) != cudaSuccess) return THAPI_E_CUDA;
  const uint64_t n = tr->info.device_rows;
  *n_rows = n;
  if (diag) *diag = tr->dev_diag;
  if (cap == 0) return THAPI_OK;
  if (cap < n) return THAPI_E_RANGE;
  if (!n) return THAPI_OK;
  if (cudaMemcpyAsync(rows, tr->dev_rows, n * sizeof(thapi_tally_row), cudaMemcpyDeviceToHost, tr->stream) !=
      cudaSuccess)
    return THAPI_E_CUDA;
  if (cudaStreamSynchronize(tr->stream) != cudaSuccess) return THAPI_E_CUDA;
  return THAPI_OK;
}

}  // namespace thapi

using namespace thapi;

extern "C" {

int thapi_ctx_create(thapi_ctx **out, int device, uint64_t hbm_cap_bytes) {
  if (!out) return THAPI_E_INVALID;
  *out = nullptr;
  int ndev = 0;
  if (cudaGetDeviceCount(&ndev) != cudaSuccess || device < 0 || device >= ndev) {
    cudaGetLastError();
    return device < 0 || (ndev > 0 && device >= ndev) ? THAPI_E_INVALID : THAPI_E_CUDA;
  }
  if (cudaSetDevice(device) != cudaSuccess) return THAPI_E_CUDA;
  thapi_ctx *c = new (std::nothrow) thapi_ctx();
  if (!c) return THAPI_E_NOMEM;
  c->device = device;
  c->cap = hbm_cap_bytes;
  if (cudaDeviceGetAttribute(&c->num_sms, cudaDevAttrMultiProcessorCount, device) != cudaSuccess ||
      cudaDeviceGetAttribute(&c->smem_per_sm, cudaDevAttrMaxSharedMemoryPerMultiprocessor, device) != cudaSuccess ||
      cudaDeviceGetAttribute(&c->smem_per_block, cudaDevAttrMaxSharedMemoryPerBlockOptin, device) != cudaSuccess) {
    delete c;
    return THAPI_E_CUDA;
  }
  // the context's own pool: memory freed by one load is reused by the next
  // without going back to the driver at each synchronisation
  cudaMemPoolProps props{};
  props.allocType = cudaMemAllocationTypePinned;
  props.location.type = cudaMemLocationTypeDevice;
  props.location.id = device;
  if (cudaMemPoolCreate(&c->pool, &props) == cudaSuccess) {
    uint64_t keep = ~0ull;
    cudaMemPoolSetAttribute(c->pool, cudaMemPoolAttrReleaseThreshold, &keep);
    // memory freed on one stream is reused by another only once the free has
    // completed: no waits between the streams of concurrent loads and queries
    int no = 0;
    cudaMemPoolSetAttribute(c->pool, cudaMemPoolReuseAllowInternalDependencies, &no);
  } else {
    cudaGetLastError();
    c->pool = nullptr;  // the device's default pool then
  }
  *out = c;
  return THAPI_OK;
}

int thapi_ctx_set_allocator(thapi_ctx *ctx, thapi_alloc_fn alloc, thapi_free_fn free_fn, void *user) {
  if (!ctx || (!alloc) != (!free_fn)) return THAPI_E_INVALID;
  if (!ctx->traces.empty()) return THAPI_E_INVALID;
  ctx->alloc_fn = alloc;
  ctx->free_fn = free_fn;
  ctx->user = user;
  return THAPI_OK;
}

int thapi_ctx_destroy(thapi_ctx *ctx) {
  if (!ctx) return THAPI_E_INVALID;
  cudaSetDevice(ctx->device);
  for (auto &kv : ctx->traces) {
    TraceRec *t = kv.second;
    dev_free(ctx, t->rows, t->rows_bytes, t->stream);
    dev_free(ctx, t->tl, t->tl_bytes, t->stream);
    dev_free(ctx, t->dev_rows, t->dev_rows_bytes, t->stream);
    dev_free(ctx, t->self_rows, t->self_rows_bytes, t->stream);
    dev_free(ctx, t->win_bmax, t->win_bytes, t->stream);
    cudaStreamSynchronize(t->stream);
    delete t;
  }
  ctx->traces.clear();
  if (ctx->heads) cudaFreeHost(ctx->heads);
  if (ctx->pool) {
    cudaDeviceSynchronize();  // every stream-ordered free has completed
    cudaMemPoolDestroy(ctx->pool);
  }
  delete ctx;
  return THAPI_OK;
}

int thapi_trace_load(thapi_ctx *ctx, const void *bytes, uint64_t nbytes, void *cuda_stream, thapi_trace_id *out) {
  if (!bytes) return THAPI_E_INVALID;
  return load_common(ctx, static_cast<const uint8_t *>(bytes), nullptr, nbytes, cuda_stream, out);
}

int thapi_trace_load_device(thapi_ctx *ctx, const void *dev_bytes, uint64_t nbytes, void *cuda_stream,
                            thapi_trace_id *out) {
  if (!dev_bytes) return THAPI_E_INVALID;
  if (reinterpret_cast<uintptr_t>(dev_bytes) % 16 != 0) return THAPI_E_INVALID;
  return load_common(ctx, nullptr, static_cast<const uint8_t *>(dev_bytes), nbytes, cuda_stream, out);
}

int thapi_decode(thapi_ctx *ctx, const void *bytes, uint64_t nbytes, thapi_event *out, uint64_t cap, uint64_t *n_out,
                 void *cuda_stream) {
  return decode_common(ctx, static_cast<const uint8_t *>(bytes), nbytes, out, cap, n_out, cuda_stream);
}

int thapi_trace_load_batch(thapi_ctx *ctx, const void *const *bytes, const uint64_t *nbytes, uint32_t n,
                           int on_device, void *cuda_stream, thapi_trace_id *out) {
  return load_batch(ctx, bytes, nbytes, n, on_device, cuda_stream, out);
}

int thapi_trace_free(thapi_ctx *ctx, thapi_trace_id id) {
  TraceRec *t = find(ctx, id);
  if (!t) return THAPI_E_INVALID;
  return free_trace_on(ctx, id, t->stream);
}

int thapi_tally(thapi_ctx *ctx, thapi_trace_id id, thapi_tally_row *rows, uint64_t cap, uint64_t *n_rows,
                thapi_diag *diag) {
  TraceRec *t = find(ctx, id);
  return tally_impl(ctx, id, rows, cap, n_rows, diag, false, t ? t->stream : nullptr);
}

int thapi_tally_device(thapi_ctx *ctx, thapi_trace_id id, thapi_tally_row *rows, uint64_t cap, uint64_t *n_rows,
                       thapi_diag *diag, void *cuda_stream) {
  return tally_impl(ctx, id, rows, cap, n_rows, diag, true, static_cast<cudaStream_t>(cuda_stream));
}

int thapi_device_tally(thapi_ctx *ctx, thapi_trace_id id, thapi_tally_row *rows, uint64_t cap, uint64_t *n_rows,
                       thapi_device_diag *diag) {
  return device_tally_impl(ctx, id, rows, cap, n_rows, diag);
}

int thapi_tally_merge(thapi_ctx *ctx, const thapi_tally_row *rows, uint64_t n, thapi_tally_row *out, uint64_t cap,
                      uint64_t *n_out, void *cuda_stream) {
  if (!ctx || !n_out || (n && !rows) || (cap && !out)) return THAPI_E_INVALID;
  if (n >= 0xFFFFFFFFull) return THAPI_E_UNSUPPORTED;
  if (cudaSetDevice(ctx->device) != cudaSuccess) return THAPI_E_CUDA;
  cudaStream_t s = static_cast<cudaStream_t>(cuda_stream);
  Scratch sc;
  sc.ctx = ctx;
  sc.stream = s;
  int rc = THAPI_OK;
  uint64_t m = 0;
  do {
    thapi_tally_row *d_in = static_cast<thapi_tally_row *>(sc.get(std::max<uint64_t>(n, 1) * sizeof(thapi_tally_row)));
    thapi_tally_row *d_out = static_cast<thapi_tally_row *>(sc.get(std::max<uint64_t>(n, 1) * sizeof(thapi_tally_row)));
    uint64_t *d_m = static_cast<uint64_t *>(sc.get(sizeof(uint64_t)));
    if (sc.failed) {
      rc = THAPI_E_NOMEM;
      break;
    }
    if (n && cudaMemcpyAsync(d_in, rows, n * sizeof(thapi_tally_row), cudaMemcpyHostToDevice, s) != cudaSuccess) {
      rc = THAPI_E_CUDA;
      break;
    }
    if (!tally_merge_device(d_in, n, d_out, d_m, sc, s)) {
      rc = sc.failed == 2 ? THAPI_E_TIMEOUT : sc.failed ? THAPI_E_NOMEM : THAPI_E_CUDA;
      break;
    }
    if (cudaMemcpyAsync(&m, d_m, sizeof(m), cudaMemcpyDeviceToHost, s) != cudaSuccess ||
        cudaStreamSynchronize(s) != cudaSuccess) {
      rc = THAPI_E_CUDA;
      break;
    }
    *n_out = m;
    if (cap == 0) break;
    if (cap < m) {
      rc = THAPI_E_RANGE;
      break;
    }
    if (m && (cudaMemcpyAsync(out, d_out, m * sizeof(thapi_tally_row), cudaMemcpyDeviceToHost, s) != cudaSuccess ||
              cudaStreamSynchronize(s) != cudaSuccess))
      rc = THAPI_E_CUDA;
  } while (false);
  sc.release_all();
  cudaStreamSynchronize(s);
  return rc;
}

int thapi_timeline(thapi_ctx *ctx, thapi_trace_id id, uint64_t t0, uint64_t t1, thapi_interval *out, uint64_t cap,
                   uint64_t *n_out) {
  TraceRec *t = find(ctx, id);
  return timeline_impl(ctx, id, t0, t1, out, cap, n_out, false, t ? t->stream : nullptr);
}

int thapi_timeline_device(thapi_ctx *ctx, thapi_trace_id id, uint64_t t0, uint64_t t1, thapi_interval *out,
                          uint64_t cap, uint64_t *n_out, void *cuda_stream) {
  return timeline_impl(ctx, id, t0, t1, out, cap, n_out, true, static_cast<cudaStream_t>(cuda_stream));
}

int thapi_trace_info_get(thapi_ctx *ctx, thapi_trace_id id, thapi_trace_info *info) {
  TraceRec *t = find(ctx, id);
  if (!t || !info) return THAPI_E_INVALID;
  *info = t->info;
  return THAPI_OK;
}

int thapi_trace_strings(thapi_ctx *ctx, thapi_trace_id id, int kind, uint32_t index, char *buf, uint64_t cap,
                        uint64_t *len) {
  TraceRec *t = find(ctx, id);
  if (!t || !len) return THAPI_E_INVALID;
  const std::vector<uint32_t> &tab = kind == 0 ? t->host_name : t->func_name;
  if ((kind != 0 && kind != 1) || index >= tab.size()) return THAPI_E_INVALID;
  const char *s = t->strings.data() + tab[index];
  uint64_t l = std::strlen(s);
  *len = l;
  if (!buf || cap < l + 1) return THAPI_E_RANGE;
  std::memcpy(buf, s, l + 1);
  return THAPI_OK;
}

int thapi_trace_func_layer(thapi_ctx *ctx, thapi_trace_id id, uint32_t func_id, uint32_t *layer) {
  TraceRec *t = find(ctx, id);
  if (!t || !layer || func_id >= t->func_layer.size()) return THAPI_E_INVALID;
  *layer = t->func_layer[func_id];
  return THAPI_OK;
}

int thapi_check_device_wait(thapi_ctx *ctx, uint32_t limit, void *cuda_stream) {
  if (!ctx || limit == 0) return THAPI_E_INVALID;
  if (cudaSetDevice(ctx->device) != cudaSuccess) return THAPI_E_CUDA;
  cudaStream_t s = static_cast<cudaStream_t>(cuda_stream);
  Scratch sc;
  sc.ctx = ctx;
  sc.stream = s;
  unsigned *d_status = static_cast<unsigned *>(sc.get(sizeof(unsigned)));
  if (sc.failed) return THAPI_E_NOMEM;
  unsigned status = THAPI_E_CUDA;
  int rc = THAPI_OK;
  if (cudaMemsetAsync(d_status, 0, sizeof(unsigned), s) != cudaSuccess || launch_wait_check(limit, d_status, s) != cudaSuccess ||
      cudaMemcpyAsync(&status, d_status, sizeof(unsigned), cudaMemcpyDeviceToHost, s) != cudaSuccess ||
      cudaStreamSynchronize(s) != cudaSuccess)
    rc = THAPI_E_CUDA;
  sc.release_all();
  cudaStreamSynchronize(s);
  return rc != THAPI_OK ? rc : (int)status;
}

int thapi_ctx_set_autotune(thapi_ctx *ctx, int enable) {
  if (!ctx) return THAPI_E_INVALID;
  ctx->autotune = enable ? 1 : 0;
  return THAPI_OK;
}

int thapi_ctx_set_timing(thapi_ctx *ctx, int enable) {
  if (!ctx) return THAPI_E_INVALID;
  ctx->timing = enable ? 1 : 0;
  return THAPI_OK;
}

int thapi_ctx_set_self_time(thapi_ctx *ctx, int enable) {
  if (!ctx) return THAPI_E_INVALID;
  ctx->self_time = enable ? 1 : 0;
  return THAPI_OK;
}

int thapi_self_tally(thapi_ctx *ctx, thapi_trace_id id, thapi_tally_row *rows, uint64_t cap, uint64_t *n_rows) {
  TraceRec *t = find(ctx, id);
  if (!t || !n_rows || (cap && !rows) || !t->self_rows) return THAPI_E_INVALID;
  if (cudaSetDevice(ctx->device) != cudaSuccess) return THAPI_E_CUDA;
  const uint64_t n = t->n_self_rows;
  *n_rows = n;
  if (cap == 0) return THAPI_OK;
  if (cap < n) return THAPI_E_RANGE;
  if (!n) return THAPI_OK;
  if (cudaMemcpyAsync(rows, t->self_rows, n * sizeof(thapi_tally_row), cudaMemcpyDeviceToHost, t->stream) !=
      cudaSuccess)
    return THAPI_E_CUDA;
  return cudaStreamSynchronize(t->stream) == cudaSuccess ? THAPI_OK : THAPI_E_CUDA;
}

int thapi_trace_timing(thapi_ctx *ctx, thapi_trace_id id, thapi_load_timing *out) {
  TraceRec *t = find(ctx, id);
  if (!t || !out) return THAPI_E_INVALID;
  *out = t->timing;
  return THAPI_OK;
}

uint64_t thapi_kernel_launches(void) { return launches_total(); }

int thapi_last_error_location(thapi_ctx *ctx, int *level, uint64_t *packet, uint64_t *event) {
  if (!ctx || !level || !packet || !event) return THAPI_E_INVALID;
  *level = ctx->err_level;
  *packet = ctx->err_packet;
  *event = ctx->err_event;
  return THAPI_OK;
}

const char *thapi_strerror(int code) {
  switch (code) {
    case THAPI_OK: return "ok";
    case THAPI_E_INVALID: return "invalid argument";
    case THAPI_E_FORMAT: return "trace breaks a layout rule";
    case THAPI_E_TRUNCATED: return "trace is truncated";
    case THAPI_E_NOMEM: return "out of device memory or over the context's HBM cap";
    case THAPI_E_TIMEOUT: return "a bounded device wait gave up";
    case THAPI_E_CUDA: return "CUDA runtime error";
    case THAPI_E_RANGE: return "output capacity too small";
    case THAPI_E_UNSUPPORTED: return "trace outside this build's limits";
    case THAPI_PENDING: return "request not completed yet";
    default: return "unknown status";
  }
}

}  // extern "C"

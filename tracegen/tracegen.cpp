// tracegen — seeded synthetic trace writer for the THPT trace layout.
//
// This module only WRITES inputs.  It holds none of the analysis arithmetic
// (no decoding, pairing, tallying or sorting of what it wrote); both the CPU
// oracle and the CUDA library are checked against traces it produces, and the
// per-call ground truth it records while writing is what the pin tests compare
// the oracle's tallies with.
//
// Layout written (little-endian; every offset in bytes):
//   file header (128 B), stream table (16 B rows), class table (16 B rows),
//   function table (8 B rows), host table (8 B rows), string table,
//   then n_packets fixed-size packets starting at a 256-aligned offset.
//   Packet = 32 B header {magic, stream_id, ts_begin, content_bytes,
//   n_events, seq, discarded} + events + zero padding.
//   Event  = u32 tsw (bits 26:0 delta ns from the previous event of the
//   packet, or from ts_begin for the first; bit 27 EXT: a u64 absolute
//   timestamp follows the 8-byte header and the delta bits are 0),
//   u16 class_id, u16 var_len, [u64 ts if EXT], fixed part, payload,
//   zero padding to 4 bytes.
//
// Workload models (the paper's analysis inputs are traces of intercepted API
// entry/exit calls, Sec. 3.2; layered portable-over-vendor APIs nest on one
// thread, Sec. 4.3; events may be dropped by the ring buffers, Sec. 3.1):
//   FLAT     one API of n_flat functions, calls nest up to max_depth.
//   LAYERED  portable layer calls contain 1-3 vendor calls, vendor calls may
//            nest vendor calls, message-passing calls are leaves at depth 0.
//   DEVICE   launch/memcpy host calls carrying unique 64-bit command ids;
//            device streams carry DEV_BEGIN/DEV_END events for each command.
//
// Random numbers: SplitMix64 seeds one xoshiro256** state per stream and role
// (structure vs payload bytes), both from Blackman & Vigna's published
// definitions, so a stream's bytes do not depend on thread scheduling.

#include <algorithm>
#include <array>
#include <atomic>
#include <cmath>
#include <cstdint>
#include <cstdlib>
#include <cstring>
#include <functional>
#include <new>
#include <string>
#include <thread>
#include <vector>

namespace {

constexpr uint32_t kTraceMagic = 0x54504854u;   // bytes "THPT"
constexpr uint32_t kPacketMagic = 0x31544B50u;  // bytes "PKT1"
constexpr uint32_t kExtBit = 1u << 27;
constexpr uint64_t kDeltaLimit = 1ull << 27;

enum : uint8_t { K_ENTRY = 0, K_EXIT = 1, K_DEV_BEGIN = 2, K_DEV_END = 3, K_SAMPLE = 4 };
enum : uint32_t { MODEL_FLAT = 1, MODEL_LAYERED = 2, MODEL_DEVICE = 4 };

// ---------------------------------------------------------------- PRNG
struct SplitMix64 {
  uint64_t s;
  uint64_t next() {
    uint64_t z = (s += 0x9E3779B97F4A7C15ull);
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
  }
};

struct Xoshiro256ss {
  uint64_t s[4];
  static uint64_t rotl(uint64_t x, int k) { return (x << k) | (x >> (64 - k)); }
  void seed(uint64_t v) {
    SplitMix64 sm{v};
    for (auto &w : s) w = sm.next();
  }
  uint64_t next() {
    const uint64_t result = rotl(s[1] * 5, 7) * 9;
    const uint64_t t = s[1] << 17;
    s[2] ^= s[0];
    s[3] ^= s[1];
    s[1] ^= s[2];
    s[0] ^= s[3];
    s[2] ^= t;
    s[3] = rotl(s[3], 45);
    return result;
  }
  double uniform() { return (double)(next() >> 11) * (1.0 / 9007199254740992.0); }  // [0,1)
  uint32_t below(uint32_t n) { return (uint32_t)(((next() >> 32) * (uint64_t)n) >> 32); }
  double normal() {  // Box-Muller, one value per call
    double u1 = uniform();
    double u2 = uniform();
    if (u1 < 1e-300) u1 = 1e-300;
    return std::sqrt(-2.0 * std::log(u1)) * std::cos(6.283185307179586 * u2);
  }
  double expo(double mean) { return -mean * std::log(1.0 - uniform()); }
};

}  // namespace

extern "C" {

typedef struct tg_config {
  uint64_t seed;
  uint64_t total_calls;     // API calls (entry+exit pairs) over all host streams
  uint32_t n_hosts;
  uint32_t pids_per_host;
  uint32_t tids_per_pid;
  uint32_t packet_bytes;    // power of two, 256..65536
  uint32_t model;           // 1 flat, 2 layered, 4 device
  uint32_t max_depth;       // nesting levels 0..max_depth-1
  uint32_t n_flat;          // flat model: functions of the single API
  uint32_t n_portable;      // layered model
  uint32_t n_vendor;
  uint32_t n_mpi;
  uint32_t var_min;         // payload bytes, uniform in [var_min, var_max]
  uint32_t var_max;
  uint32_t n_threads;       // 0 = hardware concurrency
  uint32_t n_device_streams;  // device model
  double dur_median_ns;     // log-normal self time median
  double dur_sigma;         // log-normal sigma
  double gap_mean_ns;       // exponential gap between calls
  double p_err;             // probability an EXIT carries a nonzero result
  double p_drop;            // probability an event is dropped (not written)
  double p_long_gap;        // probability a top-level gap is long (forces EXT)
  double long_gap_ns;       // long gap length scale
  double p_ext;             // probability an event uses EXT although its delta fits
  double p_nest;            // probability that a nestable call has children
  double p_sample;          // probability of an extra SAMPLE event after a call
  double dev_dur_median_ns; // device model: log-normal median of a command's device time (0 = dur_median_ns)
  uint32_t n_cpus;          // > 0: per-CPU buffers, n_cpus per host (flat and layered models)
  uint32_t reserved;
  double slice_ns;          // per-CPU buffers: scheduling time slice
} tg_config;

// Ground-truth record of one generated call (entry and exit as written, before drops).
typedef struct tg_call {
  uint64_t start_ns;
  uint64_t end_ns;
  uint32_t stream_id;
  uint16_t func_id;
  uint8_t level;
  // bit0 err result, bit1 entry (or DEV_BEGIN) dropped, bit2 exit (or DEV_END) dropped,
  // bit3 device interval (func = the issuing host call's function), bit4 that host call's ENTRY dropped
  uint8_t flags;
} tg_call;

// Ground-truth record of one written (not dropped) event, in stream order.
typedef struct tg_event {
  uint64_t ts;
  uint64_t cmd;
  uint32_t stream_id;
  uint16_t class_id;
  uint16_t var_len;
  int32_t result;
  uint8_t ext;
  uint8_t kind;
  uint16_t func_id;
} tg_event;

}  // extern "C"

namespace {

struct ClassInfo {
  uint16_t func;
  uint8_t kind;
  uint16_t fixed;
  int16_t result_off;
  int16_t cmd_off;
};

struct Ev {
  uint64_t ts;
  uint64_t cmd;
  int32_t result;
  uint16_t cls;
  uint16_t var_len;
  bool dropped;
  bool force_ext;
  uint32_t vpid, vtid;  // the thread, written into per-CPU buffer events
};

struct StreamDesc {
  uint32_t host, pid, tid, flags;
};

struct Model {
  std::vector<ClassInfo> classes;
  std::vector<std::string> func_names;
  std::vector<uint16_t> func_layer;
  std::vector<std::string> host_names;
  std::vector<StreamDesc> streams;
  uint32_t n_host_streams = 0;
  // layered model function ranges
  uint32_t portable0 = 0, vendor0 = 0, mpi0 = 0;
  // device model
  uint32_t dev_begin_cls = 0, dev_end_cls = 0;
  uint32_t sample_cls = 0xffffffffu;
};

uint32_t align4(uint32_t v) { return (v + 3u) & ~3u; }

Model build_model(const tg_config &c) {
  Model m;
  auto add_func = [&](const std::string &name, uint16_t layer) {
    m.func_names.push_back(name);
    m.func_layer.push_back(layer);
    return (uint32_t)m.func_names.size() - 1;
  };
  auto add_call_classes = [&](uint32_t f, bool carries_cmd) {
    ClassInfo e{};
    e.func = (uint16_t)f;
    e.kind = K_ENTRY;
    e.fixed = (uint16_t)(8u * (f % 3u));
    e.result_off = -1;
    e.cmd_off = -1;
    if (carries_cmd) {
      e.fixed = 16;
      e.cmd_off = 8;
    }
    ClassInfo x{};
    x.func = (uint16_t)f;
    x.kind = K_EXIT;
    x.fixed = (uint16_t)(4u + 4u * (f % 2u));
    x.result_off = 0;
    x.cmd_off = -1;
    m.classes.push_back(e);
    m.classes.push_back(x);
  };
  if (c.model == MODEL_FLAT) {
    for (uint32_t i = 0; i < c.n_flat; ++i) add_call_classes(add_func("apiFunc" + std::to_string(i), 0), false);
  } else if (c.model == MODEL_LAYERED) {
    m.portable0 = 0;
    for (uint32_t i = 0; i < c.n_portable; ++i) add_call_classes(add_func("portFunc" + std::to_string(i), 0), false);
    m.vendor0 = (uint32_t)m.func_names.size();
    for (uint32_t i = 0; i < c.n_vendor; ++i) add_call_classes(add_func("vendFunc" + std::to_string(i), 1), false);
    m.mpi0 = (uint32_t)m.func_names.size();
    for (uint32_t i = 0; i < c.n_mpi; ++i) add_call_classes(add_func("MPI_Func" + std::to_string(i), 2), false);
  } else {  // device model: launch-like and copy-like calls carry a command id
    for (uint32_t i = 0; i < c.n_flat; ++i) add_call_classes(add_func("devCmd" + std::to_string(i), 0), true);
    uint32_t fk = add_func("deviceKernel", 3);
    ClassInfo b{};
    b.func = (uint16_t)fk;
    b.kind = K_DEV_BEGIN;
    b.fixed = 8;
    b.result_off = -1;
    b.cmd_off = 0;
    ClassInfo e = b;
    e.kind = K_DEV_END;
    m.dev_begin_cls = (uint32_t)m.classes.size();
    m.classes.push_back(b);
    m.dev_end_cls = (uint32_t)m.classes.size();
    m.classes.push_back(e);
  }
  if (c.p_sample > 0) {
    uint32_t fs = add_func("telemetrySample", 4);
    ClassInfo s{};
    s.func = (uint16_t)fs;
    s.kind = K_SAMPLE;
    s.fixed = 8;
    s.result_off = -1;
    s.cmd_off = -1;
    m.sample_cls = (uint32_t)m.classes.size();
    m.classes.push_back(s);
  }
  for (uint32_t h = 0; h < c.n_hosts; ++h) m.host_names.push_back("x4204c0s" + std::to_string(h) + "b0n0");
  for (uint32_t h = 0; h < c.n_hosts; ++h)
    for (uint32_t p = 0; p < c.pids_per_host; ++p)
      for (uint32_t t = 0; t < c.tids_per_pid; ++t) {
        uint32_t pid = 124000u + h * 1000u + p * 16u;
        m.streams.push_back({h, pid, pid + t, 0});
      }
  m.n_host_streams = (uint32_t)m.streams.size();
  if (c.model == MODEL_DEVICE) {
    for (uint32_t d = 0; d < c.n_device_streams; ++d) {
      uint32_t h = d % (c.n_hosts ? c.n_hosts : 1);
      m.streams.push_back({h, 900000u + d, 990000u + d, 1});
    }
  }
  return m;
}

// ------------------------------------------------------- packet writer
// A command issued by a host call (device model): id, submit time (the call's
// exit), the call's function and whether its ENTRY event was dropped.
struct IssuedCmd {
  uint64_t cmd, submit;
  uint32_t func;
  bool entry_dropped;
};

struct PacketSink {
  // Pass 1 (bytes == nullptr): records ts_begin per packet.
  // Pass 2: writes packets at bytes + packets_off + file_index[seq] * P.
  uint32_t P = 0;
  uint32_t stream = 0;
  uint8_t *bytes = nullptr;
  uint64_t packets_off = 0;
  const uint64_t *file_index = nullptr;
  const std::vector<ClassInfo> *classes = nullptr;
  Xoshiro256ss *rng_bytes = nullptr;
  std::vector<uint64_t> ts_begins;  // pass 1 output
  std::vector<tg_event> *events = nullptr;
  uint32_t hdr = 8;                 // event header bytes: 16 in a per-CPU buffer (+ u32 vpid, u32 vtid)
  std::vector<Ev> *capture = nullptr;  // non-null: keep the events (a thread's, before CPU scheduling)

  uint32_t seq = 0;
  uint32_t used = 0, n = 0, discarded = 0;
  uint64_t ts_begin = 0, prev_ts = 0;
  bool open = false;
  uint8_t *cur = nullptr;

  void start(uint64_t t0) {
    prev_ts = t0;
    open_packet(t0);
  }
  void open_packet(uint64_t tb) {
    ts_begin = tb;
    used = 0;
    n = 0;
    discarded = 0;
    open = true;
    if (bytes) {
      cur = bytes + packets_off + file_index[seq] * (uint64_t)P;
      std::memset(cur, 0, P);
    } else {
      ts_begins.push_back(tb);
    }
  }
  void close_packet() {
    if (!open) return;
    if (bytes) {
      uint32_t hdr[8];
      hdr[0] = kPacketMagic;
      hdr[1] = stream;
      std::memcpy(&hdr[2], &ts_begin, 8);
      hdr[4] = used;
      hdr[5] = n;
      hdr[6] = seq;
      hdr[7] = discarded;
      std::memcpy(cur, hdr, 32);
    }
    ++seq;
    open = false;
  }
  void put(const Ev &ev) {
    if (capture) {
      capture->push_back(ev);
      return;
    }
    if (ev.dropped) {
      ++discarded;
      return;
    }
    const ClassInfo &ci = (*classes)[ev.cls];
    uint64_t delta = ev.ts - prev_ts;
    bool ext = ev.force_ext || ev.ts < prev_ts || delta >= kDeltaLimit;
    uint32_t size = hdr + (ext ? 8u : 0u) + ci.fixed + align4(ev.var_len);
    if (used + size > P - 32u) {
      close_packet();
      open_packet(prev_ts);
      delta = ev.ts - prev_ts;
      ext = ev.force_ext || ev.ts < prev_ts || delta >= kDeltaLimit;
      size = hdr + (ext ? 8u : 0u) + ci.fixed + align4(ev.var_len);
    }
    if (bytes) {
      uint8_t *p = cur + 32 + used;
      uint32_t tsw = ext ? kExtBit : (uint32_t)delta;
      std::memcpy(p, &tsw, 4);
      std::memcpy(p + 4, &ev.cls, 2);
      std::memcpy(p + 6, &ev.var_len, 2);
      uint32_t o = hdr;
      if (hdr == 16) {
        std::memcpy(p + 8, &ev.vpid, 4);
        std::memcpy(p + 12, &ev.vtid, 4);
      }
      if (ext) {
        std::memcpy(p + hdr, &ev.ts, 8);
        o = hdr + 8;
      }
      // fixed part: filler handles, then the typed fields
      for (uint32_t k = 0; k < ci.fixed; k += 8) {
        uint64_t h = 0x00007fff00000000ull | (rng_bytes->next() & 0xfffffff8ull);
        uint32_t take = std::min<uint32_t>(8u, ci.fixed - k);
        std::memcpy(p + o + k, &h, take);
      }
      if (ci.result_off >= 0) std::memcpy(p + o + ci.result_off, &ev.result, 4);
      if (ci.cmd_off >= 0) std::memcpy(p + o + ci.cmd_off, &ev.cmd, 8);
      o += ci.fixed;
      for (uint32_t k = 0; k < ev.var_len; k += 8) {
        uint64_t r = rng_bytes->next();
        uint32_t take = std::min<uint32_t>(8u, ev.var_len - k);
        std::memcpy(p + o + k, &r, take);
      }
      if (events) {
        tg_event te{};
        te.ts = ev.ts;
        te.cmd = ci.cmd_off >= 0 ? ev.cmd : 0;
        te.stream_id = stream;
        te.class_id = ev.cls;
        te.var_len = ev.var_len;
        te.result = ci.result_off >= 0 ? ev.result : 0;
        te.ext = ext ? 1 : 0;
        te.kind = ci.kind;
        te.func_id = ci.func;
        events->push_back(te);
      }
    }
    used += size;
    ++n;
    prev_ts = ev.ts;
  }
  void finish() {
    if (open && (n > 0 || discarded > 0)) close_packet();
    open = false;
  }
};

// ------------------------------------------------------ call generators
struct HostStreamGen {
  const tg_config &c;
  const Model &m;
  Xoshiro256ss rng;
  PacketSink &sink;
  std::vector<tg_call> *truth;
  uint32_t stream;
  uint64_t budget;  // calls left
  uint64_t t;
  // device model: commands issued by this stream
  std::vector<IssuedCmd> *cmds = nullptr;
  uint64_t cmd_counter = 0;

  HostStreamGen(const tg_config &c_, const Model &m_, PacketSink &s, std::vector<tg_call> *tr, uint32_t st, uint64_t b)
      : c(c_), m(m_), sink(s), truth(tr), stream(st), budget(b), t(0) {}

  uint64_t lognormal_ns() {
    double v = c.dur_median_ns * std::exp(c.dur_sigma * rng.normal());
    if (!(v >= 0)) v = 0;
    if (v > 1e15) v = 1e15;
    return (uint64_t)std::llround(v);
  }
  uint64_t gap_ns(double mean) {
    double v = rng.expo(mean);
    if (!(v >= 0)) v = 0;
    return (uint64_t)std::llround(v);
  }
  uint16_t var_len() {
    uint32_t span = c.var_max - c.var_min + 1;
    return (uint16_t)(c.var_min + rng.below(span));
  }
  uint32_t skewed(uint32_t n) {  // low ids are hotter
    double u = rng.uniform();
    uint32_t k = (uint32_t)(u * u * n);
    return k < n ? k : n - 1;
  }
  Ev make(uint32_t cls) {
    Ev e{};
    e.cls = (uint16_t)cls;
    e.var_len = var_len();
    e.dropped = rng.uniform() < c.p_drop;
    e.force_ext = c.p_ext > 0 && rng.uniform() < c.p_ext;
    return e;
  }
  void maybe_sample() {
    if (m.sample_cls != 0xffffffffu && rng.uniform() < c.p_sample) {
      t += gap_ns(c.gap_mean_ns * 0.25);
      Ev s = make(m.sample_cls);
      s.ts = t;
      sink.put(s);
    }
  }

  // Emits one call (and its children) at nesting level d; returns nothing,
  // advances t.  kind: 0 flat, 1 portable, 2 vendor, 3 mpi, 4 device cmd.
  void call(uint32_t d, int kind) {
    if (budget == 0) return;
    --budget;
    uint32_t f;
    switch (kind) {
      case 0: f = skewed(c.n_flat); break;
      case 1: f = m.portable0 + skewed(c.n_portable); break;
      case 2: f = m.vendor0 + skewed(c.n_vendor); break;
      case 3: f = m.mpi0 + skewed(c.n_mpi); break;
      default: f = skewed(c.n_flat); break;
    }
    uint64_t self = lognormal_ns();
    uint64_t pre = (uint64_t)(self * rng.uniform());
    uint64_t post = self - pre;
    Ev en = make(2 * f);
    en.ts = t;
    uint64_t cmd = 0;
    if (kind == 4) {
      cmd = rng.next();
      en.cmd = cmd;
    }
    size_t truth_idx = 0;
    if (truth) {
      truth_idx = truth->size();
      tg_call tc{};
      tc.start_ns = t;
      tc.stream_id = stream;
      tc.func_id = (uint16_t)f;
      tc.level = (uint8_t)std::min<uint32_t>(d, 255);
      tc.flags = en.dropped ? 2 : 0;
      truth->push_back(tc);
    }
    sink.put(en);
    t += pre;
    // children
    uint32_t nchild = 0;
    int child_kind = kind;
    if (d + 1 < c.max_depth) {
      if (kind == 1) {
        nchild = 1 + rng.below(3);
        child_kind = 2;
      } else if ((kind == 0 || kind == 2) && rng.uniform() < c.p_nest) {
        nchild = 1 + rng.below(2);
      }
    }
    for (uint32_t k = 0; k < nchild && budget > 0; ++k) {
      t += gap_ns(c.gap_mean_ns * 0.25);
      call(d + 1, child_kind);
      t += gap_ns(c.gap_mean_ns * 0.25);
    }
    t += post;
    Ev ex = make(2 * f + 1);
    ex.ts = t;
    bool err = rng.uniform() < c.p_err;
    ex.result = err ? (int32_t)(1 + rng.below(70)) * (rng.below(2) ? 1 : -1) : 0;
    if (truth) {
      tg_call &tc = (*truth)[truth_idx];
      tc.end_ns = t;
      if (err) tc.flags |= 1;
      if (ex.dropped) tc.flags |= 4;
    }
    sink.put(ex);
    if (kind == 4 && cmds) cmds->push_back({cmd, t, f, en.dropped});
  }

  void run(uint64_t t0) {
    t = t0;
    sink.start(t0);
    while (budget > 0) {
      uint64_t g = gap_ns(c.gap_mean_ns);
      if (c.p_long_gap > 0 && rng.uniform() < c.p_long_gap)
        g += (uint64_t)(c.long_gap_ns * (0.5 + 0.5 * rng.uniform()));
      t += g;
      int kind;
      if (c.model == MODEL_FLAT) {
        kind = 0;
      } else if (c.model == MODEL_LAYERED) {
        double u = rng.uniform();
        kind = u < 0.5 ? 1 : (u < 0.8 ? 2 : 3);
      } else {
        kind = 4;
      }
      call(0, kind);
      maybe_sample();
    }
    sink.finish();
  }
};

struct Plan {
  tg_config c;
  Model m;
  uint64_t stream_table_off = 0, class_table_off = 0, func_table_off = 0, host_table_off = 0;
  uint64_t strings_off = 0, strings_bytes = 0, packets_off = 0, total_bytes = 0;
  std::vector<std::string> strings;  // concatenated later
  std::vector<uint32_t> func_name_off, host_name_off;
  std::vector<uint64_t> calls_per_stream;
  std::vector<uint64_t> t0;
  std::vector<std::vector<uint64_t>> file_index;  // [stream][seq]
  uint64_t n_packets = 0;
  // device model: per device stream, its commands in time order
  struct DevWork {
    uint64_t cmd, begin, end;
    uint32_t func;
    bool host_dropped;
  };
  std::vector<std::vector<DevWork>> dev_work;
  // per-CPU buffers: every thread's events (host stream order), and per
  // buffer (host * n_cpus + cpu) references to them in (ts, thread, index) order
  struct EvRef {
    uint64_t ts;
    uint32_t thread, idx;
  };
  bool per_cpu = false;
  std::vector<std::vector<Ev>> th_events;
  std::vector<std::vector<EvRef>> cpu_refs;
  std::vector<StreamDesc> out_streams;  // the file's stream table
  std::vector<uint64_t> out_t0;
};

void for_streams(uint32_t n, uint32_t threads, const std::function<void(uint32_t)> &fn) {
  if (threads == 0) threads = std::max(1u, std::thread::hardware_concurrency());
  threads = std::min<uint32_t>(threads, std::max<uint32_t>(n, 1));
  std::atomic<uint32_t> next{0};
  auto worker = [&]() {
    for (;;) {
      uint32_t s = next.fetch_add(1);
      if (s >= n) break;
      fn(s);
    }
  };
  std::vector<std::thread> pool;
  for (uint32_t i = 1; i < threads; ++i) pool.emplace_back(worker);
  worker();
  for (auto &th : pool) th.join();
}

uint64_t stream_seed(uint64_t seed, uint32_t stream, uint32_t role) {
  SplitMix64 sm{seed ^ (0xA5A5A5A5ull * (stream + 1)) ^ ((uint64_t)role << 56)};
  sm.next();
  return sm.next() ^ ((uint64_t)stream << 20);
}

// Device model: the host streams' command lists are turned into device work.
// Each command goes to device stream (cmd mod D) and starts after its submit
// time and after the previous command of that device stream ends.
void plan_device_work(Plan &pl, const std::vector<std::vector<IssuedCmd>> &cmds) {
  const tg_config &c = pl.c;
  uint32_t D = c.n_device_streams;
  pl.dev_work.assign(D, {});
  std::vector<std::vector<std::pair<uint64_t, const IssuedCmd *>>> per_dev(D);  // (submit, command)
  for (auto &lst : cmds)
    for (auto &ic : lst) per_dev[(uint32_t)(ic.cmd % D)].push_back({ic.submit, &ic});
  for (uint32_t d = 0; d < D; ++d) {
    auto &v = per_dev[d];
    std::sort(v.begin(), v.end(), [](const std::pair<uint64_t, const IssuedCmd *> &a,
                                     const std::pair<uint64_t, const IssuedCmd *> &b) {
      if (a.first != b.first) return a.first < b.first;
      return a.second->cmd < b.second->cmd;
    });
    Xoshiro256ss r;
    r.seed(stream_seed(c.seed, 0x40000000u + d, 2));
    uint64_t free_at = 0;
    for (auto &sc : v) {
      uint64_t begin = std::max(free_at, sc.first + (uint64_t)std::llround(r.expo(c.gap_mean_ns)));
      const double med = c.dev_dur_median_ns > 0 ? c.dev_dur_median_ns : c.dur_median_ns;
      double dv = med * std::exp(c.dur_sigma * r.normal());
      uint64_t dur = (uint64_t)std::llround(dv > 1e12 ? 1e12 : (dv < 0 ? 0 : dv));
      pl.dev_work[d].push_back({sc.second->cmd, begin, begin + dur, sc.second->func, sc.second->entry_dropped});
      free_at = begin + dur;
    }
  }
}

struct DeviceStreamGen {
  const tg_config &c;
  const Model &m;
  PacketSink &sink;
  std::vector<tg_call> *truth;
  uint32_t stream;
  const std::vector<Plan::DevWork> &work;
  Xoshiro256ss rng;
  void run(uint64_t t0) {
    sink.start(t0);
    for (auto &w : work) {
      Ev b{};
      b.cls = (uint16_t)m.dev_begin_cls;
      b.var_len = 0;
      b.cmd = w.cmd;
      b.ts = w.begin;
      b.dropped = rng.uniform() < c.p_drop;
      Ev e = b;
      e.cls = (uint16_t)m.dev_end_cls;
      e.ts = w.end;
      e.dropped = rng.uniform() < c.p_drop;
      if (truth) {  // the device interval, labelled with the issuing host call's function
        tg_call tc{};
        tc.start_ns = w.begin;
        tc.end_ns = w.end;
        tc.stream_id = stream;
        tc.func_id = (uint16_t)w.func;
        tc.level = 0;
        tc.flags = (uint8_t)(8 | (b.dropped ? 2 : 0) | (e.dropped ? 4 : 0) | (w.host_dropped ? 16 : 0));
        truth->push_back(tc);
      }
      sink.put(b);
      sink.put(e);
    }
    sink.finish();
  }
};

void run_stream(Plan &pl, uint32_t s, PacketSink &sink, std::vector<tg_call> *truth, std::vector<IssuedCmd> *cmds) {
  const tg_config &c = pl.c;
  sink.P = c.packet_bytes;
  sink.stream = s;
  sink.classes = &pl.m.classes;
  if (s < pl.m.n_host_streams) {
    HostStreamGen g(c, pl.m, sink, truth, s, pl.calls_per_stream[s]);
    g.rng.seed(stream_seed(c.seed, s, 0));
    g.cmds = cmds;
    g.run(pl.t0[s]);
  } else {
    uint32_t d = s - pl.m.n_host_streams;
    DeviceStreamGen g{c, pl.m, sink, truth, s, pl.dev_work[d], {}};
    g.rng.seed(stream_seed(c.seed, s, 0));
    g.run(pl.t0[s]);
  }
}

// A per-CPU buffer: the events its CPU ran, each naming its thread.
void run_cpu_stream(Plan &pl, uint32_t o, PacketSink &sink) {
  sink.P = pl.c.packet_bytes;
  sink.stream = o;
  sink.classes = &pl.m.classes;
  sink.hdr = 16;
  sink.start(pl.out_t0[o]);
  for (const Plan::EvRef &r : pl.cpu_refs[o]) {
    Ev ev = pl.th_events[r.thread][r.idx];
    ev.vpid = pl.m.streams[r.thread].pid;
    ev.vtid = pl.m.streams[r.thread].tid;
    sink.put(ev);
  }
  sink.finish();
}

// Per-CPU scheduling: time is cut into slices of slice_ns; in slice j the
// k-th thread of a host runs on CPU (k + j) mod n_cpus, so threads migrate at
// slice boundaries and a CPU interleaves the threads it runs in one slice.
void schedule_cpus(Plan &pl) {
  const tg_config &c = pl.c;
  const uint32_t C = c.n_cpus, T = c.pids_per_host * c.tids_per_pid;
  const uint64_t slice = std::max<uint64_t>(1, (uint64_t)std::llround(c.slice_ns));
  pl.cpu_refs.assign((size_t)c.n_hosts * C, {});
  pl.out_streams.clear();
  for (uint32_t h = 0; h < c.n_hosts; ++h)
    for (uint32_t q = 0; q < C; ++q) pl.out_streams.push_back({h, 0, q, 2});
  for_streams(c.n_hosts, c.n_threads, [&](uint32_t h) {
    for (uint32_t k = 0; k < T; ++k) {
      const uint32_t th = h * T + k;
      const std::vector<Ev> &ev = pl.th_events[th];
      for (uint32_t i = 0; i < ev.size(); ++i) {
        const uint32_t cpu = (uint32_t)((k + ev[i].ts / slice) % C);
        pl.cpu_refs[(size_t)h * C + cpu].push_back({ev[i].ts, th, i});
      }
    }
    for (uint32_t q = 0; q < C; ++q) {
      auto &v = pl.cpu_refs[(size_t)h * C + q];
      std::sort(v.begin(), v.end(), [](const Plan::EvRef &a, const Plan::EvRef &b) {
        if (a.ts != b.ts) return a.ts < b.ts;
        if (a.thread != b.thread) return a.thread < b.thread;
        return a.idx < b.idx;
      });
    }
  });
  pl.out_t0.assign(pl.out_streams.size(), 0);
  for (size_t o = 0; o < pl.out_streams.size(); ++o)
    pl.out_t0[o] = pl.cpu_refs[o].empty() ? pl.t0[0] : pl.cpu_refs[o][0].ts;
}

void put32(std::vector<uint8_t> &b, uint64_t off, uint32_t v) { std::memcpy(&b[off], &v, 4); }

}  // namespace

extern "C" {

typedef struct tg_plan tg_plan;

void tg_default_config(tg_config *c) {
  std::memset(c, 0, sizeof(*c));
  c->seed = 0;
  c->total_calls = 100000;
  c->n_hosts = 1;
  c->pids_per_host = 1;
  c->tids_per_pid = 4;
  c->packet_bytes = 4096;
  c->model = MODEL_FLAT;
  c->max_depth = 3;
  c->n_flat = 40;
  c->n_portable = 60;
  c->n_vendor = 120;
  c->n_mpi = 30;
  c->var_min = 0;
  c->var_max = 48;
  c->n_threads = 0;
  c->n_device_streams = 64;
  c->dur_median_ns = 2000.0;
  c->dur_sigma = 1.0;
  c->gap_mean_ns = 1000.0;
  c->p_err = 0.0;
  c->p_drop = 0.0;
  c->p_long_gap = 0.0;
  c->long_gap_ns = 3e8;
  c->p_ext = 0.0;
  c->p_nest = 0.3;
  c->p_sample = 0.0;
  c->dev_dur_median_ns = 0.0;
  c->n_cpus = 0;
  c->slice_ns = 200000.0;
}

// Validates the config and runs the sizing pass.  Returns nullptr on a bad config.
tg_plan *tg_plan_create(const tg_config *cfg) {
  const tg_config &c = *cfg;
  uint32_t P = c.packet_bytes;
  if (P < 256 || P > 65536 || (P & (P - 1))) return nullptr;
  if (c.n_hosts == 0 || c.pids_per_host == 0 || c.tids_per_pid == 0) return nullptr;
  if (c.var_max < c.var_min || c.var_max > 4096) return nullptr;
  if (c.max_depth == 0) return nullptr;
  if (c.model != MODEL_FLAT && c.model != MODEL_LAYERED && c.model != MODEL_DEVICE) return nullptr;
  if ((c.model == MODEL_FLAT || c.model == MODEL_DEVICE) && c.n_flat == 0) return nullptr;
  if (c.model == MODEL_LAYERED && (c.n_portable == 0 || c.n_vendor == 0 || c.n_mpi == 0)) return nullptr;
  if (c.model == MODEL_DEVICE && c.n_device_streams == 0) return nullptr;
  if (c.n_cpus && (c.model == MODEL_DEVICE || c.n_cpus > 4096 || !(c.slice_ns >= 1.0))) return nullptr;
  // largest event must fit a packet
  uint32_t max_ev = (c.n_cpus ? 16 : 8) + 8 + 16 + align4(c.var_max);
  if (max_ev > P - 32) return nullptr;

  Plan *pl = new (std::nothrow) Plan();
  if (!pl) return nullptr;
  pl->c = c;
  pl->m = build_model(c);
  Model &m = pl->m;
  uint32_t S = (uint32_t)m.streams.size();
  uint32_t HS = m.n_host_streams;
  pl->calls_per_stream.assign(S, 0);
  for (uint32_t s = 0; s < HS; ++s)
    pl->calls_per_stream[s] = c.total_calls / HS + (s < c.total_calls % HS ? 1 : 0);
  pl->t0.resize(S);
  {
    Xoshiro256ss r;
    r.seed(stream_seed(c.seed, 0xffffffu, 3));
    for (uint32_t s = 0; s < S; ++s) pl->t0[s] = 1700000000000000000ull + (r.next() % 1000000ull);
  }
  // sizing pass
  std::vector<std::vector<uint64_t>> ts_begins(S);
  std::vector<std::vector<IssuedCmd>> cmds(HS);
  if (c.n_cpus) {  // per-CPU buffers: threads' events kept, scheduled onto CPUs, then sized per buffer
    pl->per_cpu = true;
    pl->th_events.assign(HS, {});
    for_streams(HS, c.n_threads, [&](uint32_t s) {
      PacketSink sink;
      sink.capture = &pl->th_events[s];
      run_stream(*pl, s, sink, nullptr, nullptr);
    });
    schedule_cpus(*pl);
    S = (uint32_t)pl->out_streams.size();
    ts_begins.assign(S, {});
    for_streams(S, c.n_threads, [&](uint32_t o) {
      PacketSink sink;
      run_cpu_stream(*pl, o, sink);
      ts_begins[o] = std::move(sink.ts_begins);
    });
  } else {
    for_streams(HS, c.n_threads, [&](uint32_t s) {
      PacketSink sink;
      run_stream(*pl, s, sink, nullptr, c.model == MODEL_DEVICE ? &cmds[s] : nullptr);
      ts_begins[s] = std::move(sink.ts_begins);
    });
  }
  if (c.model == MODEL_DEVICE) {
    plan_device_work(*pl, cmds);
    // a device stream's first packet starts no later than its first event, so
    // its packets' ts_begin (and with it the file order) follow its seq order
    for (uint32_t d = 0; d < S - HS; ++d)
      if (!pl->dev_work[d].empty()) pl->t0[HS + d] = std::min(pl->t0[HS + d], pl->dev_work[d][0].begin);
    for_streams(S - HS, c.n_threads, [&](uint32_t d) {
      PacketSink sink;
      run_stream(*pl, HS + d, sink, nullptr, nullptr);
      ts_begins[HS + d] = std::move(sink.ts_begins);
    });
  }
  // file order: packets sorted by (ts_begin, stream, seq), as a flush-order muxed file
  struct PK {
    uint64_t tb;
    uint32_t s, q;
  };
  std::vector<PK> all;
  for (uint32_t s = 0; s < S; ++s)
    for (uint32_t q = 0; q < ts_begins[s].size(); ++q) all.push_back({ts_begins[s][q], s, q});
  std::sort(all.begin(), all.end(), [](const PK &a, const PK &b) {
    if (a.tb != b.tb) return a.tb < b.tb;
    if (a.s != b.s) return a.s < b.s;
    return a.q < b.q;
  });
  pl->file_index.assign(S, {});
  for (uint32_t s = 0; s < S; ++s) pl->file_index[s].assign(ts_begins[s].size(), 0);
  for (uint64_t i = 0; i < all.size(); ++i) pl->file_index[all[i].s][all[i].q] = i;
  pl->n_packets = all.size();

  // table layout
  std::vector<uint8_t> strings;
  auto add_str = [&](const std::string &s) {
    uint32_t off = (uint32_t)strings.size();
    strings.insert(strings.end(), s.begin(), s.end());
    strings.push_back(0);
    return off;
  };
  for (auto &f : m.func_names) pl->func_name_off.push_back(add_str(f));
  for (auto &h : m.host_names) pl->host_name_off.push_back(add_str(h));
  pl->strings.assign(1, std::string(strings.begin(), strings.end()));
  uint64_t off = 128;
  pl->stream_table_off = off;
  off += 16ull * S;
  pl->class_table_off = off;
  off += 16ull * m.classes.size();
  pl->func_table_off = off;
  off += 8ull * m.func_names.size();
  pl->host_table_off = off;
  off += 8ull * m.host_names.size();
  pl->strings_off = off;
  pl->strings_bytes = strings.size();
  off += strings.size();
  off = (off + 255) & ~255ull;
  pl->packets_off = off;
  pl->total_bytes = off + pl->n_packets * (uint64_t)P;
  return reinterpret_cast<tg_plan *>(pl);
}

uint64_t tg_plan_bytes(const tg_plan *p) { return reinterpret_cast<const Plan *>(p)->total_bytes; }
uint64_t tg_plan_packets(const tg_plan *p) { return reinterpret_cast<const Plan *>(p)->n_packets; }
uint32_t tg_plan_streams(const tg_plan *p) {
  const Plan *pl = reinterpret_cast<const Plan *>(p);
  return (uint32_t)(pl->per_cpu ? pl->out_streams.size() : pl->m.streams.size());
}

// Writes the trace into out[0 .. tg_plan_bytes).  Optional ground truth:
// calls (one tg_call per generated call, stream-major, entry order) and
// events (one tg_event per written event, stream-major, stream order).
// Pass a null pointer to skip either; *n_calls / *n_events receive counts
// (the caller sizes the arrays with a first call where both are null and the
// counts are read back through tg_plan_truth_sizes).
int tg_plan_write(tg_plan *p, void *out, tg_call *calls, uint64_t calls_cap, uint64_t *n_calls,
                  tg_event *events, uint64_t events_cap, uint64_t *n_events) {
  Plan &pl = *reinterpret_cast<Plan *>(p);
  const tg_config &c = pl.c;
  Model &m = pl.m;
  const std::vector<StreamDesc> &file_streams = pl.per_cpu ? pl.out_streams : m.streams;
  uint32_t S = (uint32_t)file_streams.size();
  std::vector<uint8_t> head(pl.packets_off, 0);
  put32(head, 0, kTraceMagic);
  uint16_t ver = 1, hb = 128;
  std::memcpy(&head[4], &ver, 2);
  std::memcpy(&head[6], &hb, 2);
  put32(head, 8, c.packet_bytes);
  put32(head, 12, S);
  put32(head, 16, (uint32_t)m.classes.size());
  put32(head, 20, (uint32_t)m.func_names.size());
  put32(head, 24, (uint32_t)m.host_names.size());
  std::memcpy(&head[32], &pl.n_packets, 8);
  std::memcpy(&head[40], &pl.stream_table_off, 8);
  std::memcpy(&head[48], &pl.class_table_off, 8);
  std::memcpy(&head[56], &pl.func_table_off, 8);
  std::memcpy(&head[64], &pl.host_table_off, 8);
  std::memcpy(&head[72], &pl.strings_off, 8);
  std::memcpy(&head[80], &pl.strings_bytes, 8);
  std::memcpy(&head[88], &pl.packets_off, 8);
  for (uint32_t s = 0; s < S; ++s) {
    uint64_t o = pl.stream_table_off + 16ull * s;
    put32(head, o, file_streams[s].host);
    put32(head, o + 4, file_streams[s].pid);
    put32(head, o + 8, file_streams[s].tid);
    put32(head, o + 12, file_streams[s].flags);
  }
  for (uint32_t k = 0; k < m.classes.size(); ++k) {
    uint64_t o = pl.class_table_off + 16ull * k;
    const ClassInfo &ci = m.classes[k];
    std::memcpy(&head[o], &ci.func, 2);
    head[o + 2] = ci.kind;
    head[o + 3] = 0;
    std::memcpy(&head[o + 4], &ci.fixed, 2);
    std::memcpy(&head[o + 6], &ci.result_off, 2);
    std::memcpy(&head[o + 8], &ci.cmd_off, 2);
  }
  for (uint32_t f = 0; f < m.func_names.size(); ++f) {
    uint64_t o = pl.func_table_off + 8ull * f;
    put32(head, o, pl.func_name_off[f]);
    std::memcpy(&head[o + 4], &m.func_layer[f], 2);
  }
  for (uint32_t h = 0; h < m.host_names.size(); ++h) put32(head, pl.host_table_off + 8ull * h, pl.host_name_off[h]);
  std::memcpy(&head[pl.strings_off], pl.strings[0].data(), pl.strings_bytes);
  uint8_t *bytes = static_cast<uint8_t *>(out);
  std::memcpy(bytes, head.data(), head.size());

  bool want_truth = calls != nullptr || events != nullptr || n_calls != nullptr || n_events != nullptr;
  if (want_truth && pl.per_cpu) return 2;  // no ground truth for per-CPU buffers
  std::vector<std::vector<tg_call>> tcalls(want_truth ? S : 0);
  std::vector<std::vector<tg_event>> tevents(want_truth ? S : 0);
  auto body = [&](uint32_t s) {
    PacketSink sink;
    sink.bytes = bytes;
    sink.packets_off = pl.packets_off;
    sink.file_index = pl.file_index[s].data();
    Xoshiro256ss rb;
    rb.seed(stream_seed(c.seed, s, 1));
    sink.rng_bytes = &rb;
    sink.events = want_truth ? &tevents[s] : nullptr;
    if (pl.per_cpu) {
      run_cpu_stream(pl, s, sink);
      return;
    }
    std::vector<IssuedCmd> cmds;
    run_stream(pl, s, sink, want_truth ? &tcalls[s] : nullptr, c.model == MODEL_DEVICE ? &cmds : nullptr);
  };
  for_streams(S, c.n_threads, body);
  if (want_truth) {
    uint64_t nc = 0, ne = 0;
    for (uint32_t s = 0; s < S; ++s) {
      for (auto &x : tcalls[s]) {
        if (calls && nc < calls_cap) calls[nc] = x;
        ++nc;
      }
      for (auto &x : tevents[s]) {
        if (events && ne < events_cap) events[ne] = x;
        ++ne;
      }
    }
    if (n_calls) *n_calls = nc;
    if (n_events) *n_events = ne;
    if ((calls && nc > calls_cap) || (events && ne > events_cap)) return 1;
  }
  return 0;
}

void tg_plan_destroy(tg_plan *p) { delete reinterpret_cast<Plan *>(p); }

}  // extern "C"

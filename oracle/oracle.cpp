// THPT trace-analysis ORACLE — test infrastructure only.
//
// A plain, sequential, obviously-correct CPU statement of what the CUDA
// library computes: validate the trace, decode every event, rebuild its
// timestamp, pair entry and exit events with a per-thread call stack, tally
// per (hostname, pid, tid, function) in an ordered map, and order the
// intervals by start time.  Only tests/, the smoke check and the benchmark's
// CPU-baseline leg may load this library; the product path never does.  It
// shares no code, header or table with the CUDA library.
//
// What the paper fixes, and where:
//  * every intercepted API call leaves an entry and an exit event, the exit
//    carrying the call's result (Sec. 3.2);
//  * interval plugins time calls from the start and end of these events
//    (Sec. 3.3); layered APIs nest on one thread, so a call's time includes
//    the calls it makes (Sec. 4.3, the HIP-over-Level-Zero tally where
//    hipDeviceSynchronize contains the zeEventHostSynchronize spin);
//  * the tally reports per function Time, Calls, Min and Max grouped by
//    hostname / process / thread (Sec. 3.4 and the Sec. 4.3 table);
//  * events may be dropped rather than block the application (Sec. 3.1), so
//    unmatched entries and exits occur and are counted, not paired;
//  * messages are serialised by time before the plugins see them (Sec. 3.4),
//    which is the timeline order.
// The paper fixes no binary layout (it only names CTF, Sec. 3.1); the layout
// read here is the project's own THPT layout, restated below independently of
// the CUDA library's reader.
//
// Readings where the paper is silent (each also listed in the design notes):
//  * a stream is one (host, pid, tid) thread of execution;
//  * duration = exit ts - entry ts in u64 arithmetic (inclusive time);
//  * error <=> the exit's i32 result is nonzero (0 when the class has none);
//  * an exit on an empty stack is an unmatched exit; an exit whose popped
//    entry has another function is a mismatched pair; both are excluded from
//    tally and timeline, as are entries still open at the end of the stream;
//  * interval level = stack depth of the entry (0 = outermost), saturated
//    at 255;
//  * timeline order = (start ts, stream id, entry position in the stream);
//    window [t0, t1) keeps intervals with start < t1 and end >= t0.
//
// Device activity (the paper's GPU profiling code records device start and
// end times of the commands a host API call submits, Sec. 3.3, and the
// timeline shows device rows beside the host rows, Sec. 3.6).  Readings:
//  * a command is named by a u64 command id carried by DEV_BEGIN / DEV_END
//    events and by the ENTRY of the host call that submitted it (classes
//    with a command offset);
//  * per command id c, let B, E, H count its DEV_BEGIN, DEV_END and host
//    ENTRY events.  c is a device pair when B = E = 1 and the end ts is not
//    below the begin ts; a device pair with H = 1 is joined and becomes a
//    device interval [begin ts, end ts] on the begin's stream, labelled with
//    the host call's function, level 0, flags bit 2; H = 0 leaves the pair
//    unjoined and H > 1 ambiguous (both excluded);
//  * device intervals are tallied apart from the host calls, per (host, pid,
//    tid of the device stream, function of the host call); they have no
//    result, so their error count is 0;
//  * in the timeline a device interval sits at the position of its DEV_BEGIN
//    in its stream;
//  * the same ns clock for host and device events.
//
// Per-CPU buffers (LTTng keeps one ring buffer per CPU, Sec. 3.1, so one
// buffer interleaves the events of many threads, each event carrying the
// thread's vpid / vtid context, Sec. 3.2).  Readings:
//  * a stream whose flags have bit 1 set is a per-CPU buffer; each of its
//    events has a 16-byte header: tsw, class, var_len, then u32 vpid, u32 vtid
//    (before the EXT timestamp);
//  * a thread is (host of the buffer, vpid, vtid); its events from all the
//    per-CPU buffers are ordered by (ts, stream id, position in the stream)
//    and paired with one call stack, as a per-thread stream would be; tally
//    rows are keyed by (host, vpid, vtid, function) and merge with rows of
//    per-thread streams of the same key; an interval belongs to its entry's
//    stream and takes the entry's position in the timeline order;
//  * device activity is paired over per-thread and device streams only.
//
// Self (exclusive) time, for the layering analysis of Sec. 4.3 (how much of
// hipDeviceSynchronize is its own time and how much the nested
// zeEventHostSynchronize calls).  Readings:
//  * a call's self time = its duration minus the durations of the calls that
//    are paired directly inside it (the entries pushed right above its entry
//    on the same stack and closed by an exit of the same function), in u64
//    arithmetic; calls deeper down count only toward their own parent;
//  * a mismatched or unmatched call has no duration: it takes nothing off
//    its parent's self time, and the paired calls directly inside it take
//    nothing off any call's self time;
//  * self rows have the tally's keys, counts and error counts; total / min /
//    max are over self times.

#include <algorithm>
#include <cstdint>
#include <cstring>
#include <map>
#include <new>
#include <thread>
#include <tuple>
#include <vector>

namespace {

enum {
  ORC_OK = 0,
  ORC_E_INVALID = 1,
  ORC_E_FORMAT = 2,
  ORC_E_TRUNCATED = 3,
};

enum { KIND_ENTRY = 0, KIND_EXIT = 1, KIND_DEV_BEGIN = 2, KIND_DEV_END = 3, KIND_SAMPLE = 4 };
const uint32_t STREAM_PER_CPU = 2u;  // stream flags bit 1: a per-CPU buffer

const uint32_t TRACE_MAGIC = 0x54504854u;   // "THPT"
const uint32_t PACKET_MAGIC = 0x31544B50u;  // "PKT1"
const uint32_t EXT = 1u << 27;
const uint32_t DELTA_MASK = (1u << 27) - 1u;

uint16_t rd16(const uint8_t *p) {
  uint16_t v;
  std::memcpy(&v, p, 2);
  return v;
}
int16_t rd16s(const uint8_t *p) {
  int16_t v;
  std::memcpy(&v, p, 2);
  return v;
}
uint32_t rd32(const uint8_t *p) {
  uint32_t v;
  std::memcpy(&v, p, 4);
  return v;
}
int32_t rd32s(const uint8_t *p) {
  int32_t v;
  std::memcpy(&v, p, 4);
  return v;
}
uint64_t rd64(const uint8_t *p) {
  uint64_t v;
  std::memcpy(&v, p, 8);
  return v;
}

struct Class {
  uint16_t func;
  uint8_t kind;
  uint16_t fixed;
  int16_t result_off;
  int16_t cmd_off;
};

struct Stream {
  uint32_t host, pid, tid, flags;
};

struct Trace {
  const uint8_t *b;
  uint64_t n;
  uint32_t P;
  uint32_t n_streams, n_classes, n_funcs, n_hosts;
  uint64_t n_packets, packets_off;
  std::vector<Class> classes;
  std::vector<Stream> streams;
};

// ``off + count * size <= n`` without overflow.
bool fits(uint64_t off, uint64_t count, uint64_t size, uint64_t n) {
  if (off > n) return false;
  if (size != 0 && count > (n - off) / size) return false;
  return true;
}

bool name_ok(const uint8_t *strings, uint64_t strings_bytes, uint32_t off) {
  if (off >= strings_bytes) return false;
  for (uint64_t i = off; i < strings_bytes; ++i)
    if (strings[i] == 0) return true;
  return false;
}

struct Loc {
  int level = 0;  // 0 file/tables, 1 packet header, 2 packet content
  uint64_t packet = 0;
  uint64_t event = 0;
};

// File header and tables, in the documented check order.
int parse_file(const uint8_t *b, uint64_t n, Trace &t) {
  if (n < 128) return ORC_E_TRUNCATED;
  if (rd32(b) != TRACE_MAGIC) return ORC_E_FORMAT;
  if (rd16(b + 4) != 1) return ORC_E_FORMAT;
  if (rd16(b + 6) != 128) return ORC_E_FORMAT;
  t.b = b;
  t.n = n;
  t.P = rd32(b + 8);
  t.n_streams = rd32(b + 12);
  t.n_classes = rd32(b + 16);
  t.n_funcs = rd32(b + 20);
  t.n_hosts = rd32(b + 24);
  t.n_packets = rd64(b + 32);
  uint64_t st_off = rd64(b + 40), cl_off = rd64(b + 48), fn_off = rd64(b + 56), ho_off = rd64(b + 64);
  uint64_t str_off = rd64(b + 72), str_bytes = rd64(b + 80);
  t.packets_off = rd64(b + 88);
  if (t.P < 256 || t.P > 65536 || (t.P & (t.P - 1)) != 0) return ORC_E_FORMAT;
  if (t.n_classes > 65536 || t.n_funcs > 65536) return ORC_E_FORMAT;
  if (!fits(st_off, t.n_streams, 16, n)) return ORC_E_TRUNCATED;
  if (!fits(cl_off, t.n_classes, 16, n)) return ORC_E_TRUNCATED;
  if (!fits(fn_off, t.n_funcs, 8, n)) return ORC_E_TRUNCATED;
  if (!fits(ho_off, t.n_hosts, 8, n)) return ORC_E_TRUNCATED;
  if (!fits(str_off, str_bytes, 1, n)) return ORC_E_TRUNCATED;
  if (t.packets_off % 256 != 0) return ORC_E_FORMAT;
  if (!fits(t.packets_off, t.n_packets, t.P, n)) return ORC_E_TRUNCATED;
  const uint8_t *strings = b + str_off;
  for (uint32_t h = 0; h < t.n_hosts; ++h)
    if (!name_ok(strings, str_bytes, rd32(b + ho_off + 8ull * h))) return ORC_E_FORMAT;
  for (uint32_t f = 0; f < t.n_funcs; ++f)
    if (!name_ok(strings, str_bytes, rd32(b + fn_off + 8ull * f))) return ORC_E_FORMAT;
  t.classes.resize(t.n_classes);
  for (uint32_t k = 0; k < t.n_classes; ++k) {
    const uint8_t *r = b + cl_off + 16ull * k;
    Class c;
    c.func = rd16(r);
    c.kind = r[2];
    c.fixed = rd16(r + 4);
    c.result_off = rd16s(r + 6);
    c.cmd_off = rd16s(r + 8);
    if (c.func >= t.n_funcs) return ORC_E_FORMAT;
    if (c.kind > KIND_SAMPLE) return ORC_E_FORMAT;
    if (c.fixed % 4 != 0) return ORC_E_FORMAT;
    if (c.result_off != -1 && (c.result_off < 0 || c.result_off % 4 != 0 || c.result_off + 4 > c.fixed))
      return ORC_E_FORMAT;
    if (c.cmd_off != -1 && (c.cmd_off < 0 || c.cmd_off % 4 != 0 || c.cmd_off + 8 > c.fixed)) return ORC_E_FORMAT;
    t.classes[k] = c;
  }
  t.streams.resize(t.n_streams);
  for (uint32_t s = 0; s < t.n_streams; ++s) {
    const uint8_t *r = b + st_off + 16ull * s;
    Stream st{rd32(r), rd32(r + 4), rd32(r + 8), rd32(r + 12)};
    if (st.host >= t.n_hosts) return ORC_E_FORMAT;
    t.streams[s] = st;
  }
  return ORC_OK;
}

const uint8_t *packet_at(const Trace &t, uint64_t i) { return t.b + t.packets_off + i * (uint64_t)t.P; }

// Walks one packet's events, checking each in the documented order.
// Returns the code and sets *bad_event to the failing event's index.
int check_content(const Trace &t, const uint8_t *pk, uint64_t *bad_event) {
  uint32_t content = rd32(pk + 16);
  uint32_t n_events = rd32(pk + 20);
  const uint32_t sid = rd32(pk + 4);
  const uint32_t hdr = (t.streams[sid].flags & STREAM_PER_CPU) ? 16 : 8;  // per-CPU: + vpid, vtid
  const uint8_t *c = pk + 32;
  uint64_t off = 0;
  uint64_t k = 0;
  while (off < content) {
    *bad_event = k;
    if (off + hdr > content) return ORC_E_TRUNCATED;
    uint32_t tsw = rd32(c + off);
    uint16_t cls = rd16(c + off + 4);
    uint16_t var_len = rd16(c + off + 6);
    if ((tsw >> 28) != 0) return ORC_E_FORMAT;
    if (cls >= t.n_classes) return ORC_E_FORMAT;
    bool ext = (tsw & EXT) != 0;
    if (ext && (tsw & DELTA_MASK) != 0) return ORC_E_FORMAT;
    uint64_t size = hdr + (ext ? 8 : 0) + t.classes[cls].fixed + ((var_len + 3u) & ~3u);
    if (off + size > content) return ORC_E_TRUNCATED;
    off += size;
    ++k;
  }
  *bad_event = k;
  if (k != n_events) return ORC_E_FORMAT;
  return ORC_OK;
}

}  // namespace

extern "C" {

typedef struct orc_row {
  uint32_t host_id, pid, tid, func_id;
  uint64_t count, total_ns, min_ns, max_ns, err_count;
} orc_row;

typedef struct orc_interval {
  uint64_t start_ns, end_ns;
  uint32_t stream_id;
  uint16_t func_id;
  uint8_t level;
  uint8_t flags;  // bit0 err, bit2 device interval
} orc_interval;

typedef struct orc_diag {
  uint64_t events, pairs, unmatched_entries, unmatched_exits, mismatched_pairs, other_events, discarded, packets;
} orc_diag;

typedef struct orc_dev_diag {
  uint64_t dev_events;       // DEV_BEGIN and DEV_END events
  uint64_t dev_pairs;        // commands with one begin and one end, end >= begin
  uint64_t dev_intervals;    // device pairs joined to exactly one host entry
  uint64_t dev_unpaired;     // device events not in a device pair
  uint64_t dev_unjoined;     // device pairs with no host entry
  uint64_t dev_ambiguous;    // device pairs with several host entries
  uint64_t host_cmd_entries; // host entries carrying a command id
  uint64_t host_unjoined;    // of those, entries whose command is no device pair
} orc_dev_diag;

typedef struct orc_event {
  uint64_t ts;
  uint64_t cmd;
  uint32_t stream_id;
  uint16_t class_id;
  uint16_t var_len;
  int32_t result;
  uint8_t ext;
  uint8_t kind;
  uint16_t func_id;
  uint32_t vpid, vtid;  // the event's context in a per-CPU buffer, else the stream's pid / tid
} orc_event;

typedef struct orc_opts {
  const uint32_t *streams;  // optional subset of stream ids to analyse (null = all)
  uint32_t n_subset;
  uint32_t want_intervals;  // build the timeline
  uint64_t t0, t1;          // timeline window [t0, t1)
} orc_opts;

}  // extern "C"

namespace {

struct Result {
  int code = ORC_OK;
  Loc loc;
  std::vector<orc_row> rows;
  std::vector<orc_interval> intervals;
  orc_diag diag{};
  std::vector<orc_event> events;
  std::vector<orc_row> dev_rows;
  orc_dev_diag dev{};
  std::vector<orc_row> self_rows;
};

// Everything one command id gathered over the trace.
struct DevBegin {
  uint64_t ts;
  uint32_t stream;
  uint64_t seq;
};
struct Command {
  std::vector<DevBegin> begins;
  std::vector<uint64_t> ends;
  std::vector<uint16_t> host_funcs;
};

struct Open {
  uint16_t func;
  uint64_t ts;
  uint64_t seq;     // entry position in its stream
  uint32_t stream;  // entry's stream
  uint64_t child;   // sum of the durations of the calls paired directly inside
};

// One ENTRY / EXIT event of a per-CPU buffer, kept until its thread is paired.
struct ThreadEvent {
  uint64_t ts;
  uint32_t stream;
  uint64_t seq;
  uint8_t kind;
  uint16_t func;
  int32_t result;
};


struct Keyed {
  uint64_t start;
  uint32_t stream;
  uint64_t seq;
  orc_interval iv;
};

// Validates everything (file, then every packet header in file order, then
// every packet's content in file order).  With a subset, only the subset's
// packets are checked.
int validate(const uint8_t *b, uint64_t n, Trace &t, Loc &loc, const std::vector<char> *keep) {
  int rc = parse_file(b, n, t);
  if (rc != ORC_OK) {
    loc.level = 0;
    return rc;
  }
  std::vector<int64_t> last_seq(t.n_streams, -1);
  for (uint64_t i = 0; i < t.n_packets; ++i) {
    const uint8_t *pk = packet_at(t, i);
    uint32_t sid = rd32(pk + 4);
    if (keep && (sid >= t.n_streams || !(*keep)[sid])) continue;
    loc.level = 1;
    loc.packet = i;
    if (rd32(pk) != PACKET_MAGIC) return ORC_E_FORMAT;
    if (sid >= t.n_streams) return ORC_E_FORMAT;
    uint32_t content = rd32(pk + 16);
    if (content % 4 != 0 || content > t.P - 32) return ORC_E_FORMAT;
    if (rd32(pk + 20) > content / 8) return ORC_E_FORMAT;
    uint32_t seq = rd32(pk + 24);
    if (last_seq[sid] >= 0 && (int64_t)seq <= last_seq[sid]) return ORC_E_FORMAT;
    last_seq[sid] = seq;
  }
  for (uint64_t i = 0; i < t.n_packets; ++i) {
    const uint8_t *pk = packet_at(t, i);
    uint32_t sid = rd32(pk + 4);
    if (keep && (sid >= t.n_streams || !(*keep)[sid])) continue;
    uint64_t ev = 0;
    rc = check_content(t, pk, &ev);
    if (rc != ORC_OK) {
      loc.level = 2;
      loc.packet = i;
      loc.event = ev;
      return rc;
    }
  }
  return ORC_OK;
}

// Groups packet indices by stream, keeping file order inside each stream.
std::vector<std::vector<uint64_t>> packets_by_stream(const Trace &t, const std::vector<char> *keep) {
  std::vector<std::vector<uint64_t>> by(t.n_streams);
  for (uint64_t i = 0; i < t.n_packets; ++i) {
    uint32_t sid = rd32(packet_at(t, i) + 4);
    if (sid >= t.n_streams || (keep && !(*keep)[sid])) continue;
    by[sid].push_back(i);
  }
  return by;
}

void analyse(const Trace &t, const orc_opts &o, const std::vector<char> *keep, Result &r, bool collect_events) {
  auto by = packets_by_stream(t, keep);
  std::map<std::tuple<uint32_t, uint32_t, uint32_t, uint32_t>, orc_row> tally, self_tally;
  std::map<uint64_t, Command> commands;
  std::map<std::tuple<uint32_t, uint32_t, uint32_t>, std::vector<ThreadEvent>> threads;  // per-CPU buffers
  std::vector<Keyed> ivs;
  orc_diag &d = r.diag;
  // One ENTRY or EXIT of the thread (host, pid, tid) whose call stack is `stack`.
  auto pair = [&](std::vector<Open> &stack, uint32_t host, uint32_t pid, uint32_t tid, uint8_t kind, uint16_t func,
                  uint64_t ts, int32_t result, uint32_t stream, uint64_t seq) {
    if (kind == KIND_ENTRY) {
      stack.push_back({func, ts, seq, stream, 0});
      return;
    }
    if (stack.empty()) {
      d.unmatched_exits += 1;
      return;
    }
    Open en = stack.back();
    stack.pop_back();
    if (en.func != func) {
      d.mismatched_pairs += 1;
      return;
    }
    uint64_t dur = ts - en.ts;
    bool err = result != 0;
    d.pairs += 1;
    auto key = std::make_tuple(host, pid, tid, (uint32_t)func);
    auto it = tally.find(key);
    if (it == tally.end()) {
      orc_row row{host, pid, tid, func, 0, 0, UINT64_MAX, 0, 0};
      it = tally.emplace(key, row).first;
    }
    orc_row &row = it->second;
    row.count += 1;
    row.total_ns += dur;
    row.min_ns = std::min(row.min_ns, dur);
    row.max_ns = std::max(row.max_ns, dur);
    row.err_count += err ? 1 : 0;
    // self time: this call's duration less its direct children's; then its own
    // duration goes to its parent, the entry now on top of the stack
    const uint64_t self = dur - en.child;
    auto st = self_tally.find(key);
    if (st == self_tally.end()) st = self_tally.emplace(key, orc_row{host, pid, tid, func, 0, 0, UINT64_MAX, 0, 0}).first;
    orc_row &srow = st->second;
    srow.count += 1;
    srow.total_ns += self;
    srow.min_ns = std::min(srow.min_ns, self);
    srow.max_ns = std::max(srow.max_ns, self);
    srow.err_count += err ? 1 : 0;
    if (!stack.empty()) stack.back().child += dur;
    if (o.want_intervals && en.ts < o.t1 && ts >= o.t0) {
      orc_interval iv{};
      iv.start_ns = en.ts;
      iv.end_ns = ts;
      iv.stream_id = en.stream;
      iv.func_id = func;
      iv.level = (uint8_t)std::min<size_t>(stack.size(), 255);
      iv.flags = err ? 1 : 0;
      ivs.push_back({en.ts, en.stream, en.seq, iv});
    }
  };
  for (uint32_t s = 0; s < t.n_streams; ++s) {
    if (keep && !(*keep)[s]) continue;
    const Stream &st = t.streams[s];
    const bool per_cpu = (st.flags & STREAM_PER_CPU) != 0;
    const uint32_t hdr = per_cpu ? 16 : 8;
    std::vector<Open> stack;
    uint64_t seq_in_stream = 0;
    for (uint64_t pi : by[s]) {
      const uint8_t *pk = packet_at(t, pi);
      uint64_t ts_prev = rd64(pk + 8);
      uint32_t n_events = rd32(pk + 20);
      d.discarded += rd32(pk + 28);
      d.packets += 1;
      const uint8_t *c = pk + 32;
      uint64_t off = 0;
      for (uint32_t k = 0; k < n_events; ++k) {
        uint32_t tsw = rd32(c + off);
        uint16_t cls = rd16(c + off + 4);
        uint16_t var_len = rd16(c + off + 6);
        const uint32_t vpid = per_cpu ? rd32(c + off + 8) : st.pid, vtid = per_cpu ? rd32(c + off + 12) : st.tid;
        bool ext = (tsw & EXT) != 0;
        uint64_t ts = ext ? rd64(c + off + hdr) : ts_prev + (uint64_t)(tsw & DELTA_MASK);
        ts_prev = ts;
        const Class &ci = t.classes[cls];
        const uint8_t *fixed = c + off + hdr + (ext ? 8 : 0);
        int32_t result = ci.result_off >= 0 ? rd32s(fixed + ci.result_off) : 0;
        uint64_t cmd = ci.cmd_off >= 0 ? rd64(fixed + ci.cmd_off) : 0;
        off += hdr + (ext ? 8 : 0) + ci.fixed + ((var_len + 3u) & ~3u);
        d.events += 1;
        if (collect_events) {
          orc_event e{};
          e.ts = ts;
          e.cmd = cmd;
          e.stream_id = s;
          e.class_id = cls;
          e.var_len = var_len;
          e.result = result;
          e.ext = ext ? 1 : 0;
          e.kind = ci.kind;
          e.func_id = ci.func;
          e.vpid = vpid;
          e.vtid = vtid;
          r.events.push_back(e);
        }
        if (!per_cpu && ci.kind == KIND_ENTRY && ci.cmd_off >= 0) {
          r.dev.host_cmd_entries += 1;
          commands[cmd].host_funcs.push_back(ci.func);
        }
        if (ci.kind == KIND_DEV_BEGIN || ci.kind == KIND_DEV_END) {
          r.dev.dev_events += 1;
          if (!per_cpu && ci.cmd_off >= 0) {
            if (ci.kind == KIND_DEV_BEGIN)
              commands[cmd].begins.push_back({ts, s, seq_in_stream});
            else
              commands[cmd].ends.push_back(ts);
          }
        }
        if (ci.kind == KIND_ENTRY || ci.kind == KIND_EXIT) {
          if (per_cpu)
            threads[std::make_tuple(st.host, vpid, vtid)].push_back(
                {ts, s, seq_in_stream, ci.kind, ci.func, result});
          else
            pair(stack, st.host, st.pid, st.tid, ci.kind, ci.func, ts, result, s, seq_in_stream);
        } else {
          d.other_events += 1;
        }
        ++seq_in_stream;
      }
    }
    d.unmatched_entries += stack.size();
  }
  // threads of the per-CPU buffers: their events in (ts, stream, position) order, one stack each
  for (auto &kv : threads) {
    std::vector<ThreadEvent> &ev = kv.second;
    std::stable_sort(ev.begin(), ev.end(), [](const ThreadEvent &a, const ThreadEvent &b) {
      if (a.ts != b.ts) return a.ts < b.ts;
      if (a.stream != b.stream) return a.stream < b.stream;
      return a.seq < b.seq;
    });
    std::vector<Open> stack;
    const uint32_t host = std::get<0>(kv.first), pid = std::get<1>(kv.first), tid = std::get<2>(kv.first);
    for (const ThreadEvent &e : ev) pair(stack, host, pid, tid, e.kind, e.func, e.ts, e.result, e.stream, e.seq);
    d.unmatched_entries += stack.size();
  }
  for (auto &kv : tally) r.rows.push_back(kv.second);
  for (auto &kv : self_tally) r.self_rows.push_back(kv.second);

  // device activity: one pass over the commands, in command-id order
  std::map<std::tuple<uint32_t, uint32_t, uint32_t, uint32_t>, orc_row> dev_tally;
  for (auto &kv : commands) {
    const Command &c = kv.second;
    const bool pair = c.begins.size() == 1 && c.ends.size() == 1 && c.ends[0] >= c.begins[0].ts;
    if (!pair) {
      r.dev.host_unjoined += c.host_funcs.size();
      continue;
    }
    r.dev.dev_pairs += 1;
    if (c.host_funcs.empty()) {
      r.dev.dev_unjoined += 1;
      continue;
    }
    if (c.host_funcs.size() > 1) {
      r.dev.dev_ambiguous += 1;
      continue;
    }
    r.dev.dev_intervals += 1;
    const DevBegin &b = c.begins[0];
    const uint64_t te = c.ends[0];
    const uint16_t f = c.host_funcs[0];
    const Stream &st = t.streams[b.stream];
    const uint64_t dur = te - b.ts;
    auto key = std::make_tuple(st.host, st.pid, st.tid, (uint32_t)f);
    auto it = dev_tally.find(key);
    if (it == dev_tally.end()) it = dev_tally.emplace(key, orc_row{st.host, st.pid, st.tid, f, 0, 0, UINT64_MAX, 0, 0}).first;
    orc_row &row = it->second;
    row.count += 1;
    row.total_ns += dur;
    row.min_ns = std::min(row.min_ns, dur);
    row.max_ns = std::max(row.max_ns, dur);
    if (o.want_intervals && b.ts < o.t1 && te >= o.t0) {
      orc_interval iv{};
      iv.start_ns = b.ts;
      iv.end_ns = te;
      iv.stream_id = b.stream;
      iv.func_id = f;
      iv.level = 0;
      iv.flags = 4;
      ivs.push_back({b.ts, b.stream, b.seq, iv});
    }
  }
  r.dev.dev_unpaired = r.dev.dev_events - 2 * r.dev.dev_pairs;
  for (auto &kv : dev_tally) r.dev_rows.push_back(kv.second);

  std::sort(ivs.begin(), ivs.end(), [](const Keyed &a, const Keyed &b) {
    if (a.start != b.start) return a.start < b.start;
    if (a.stream != b.stream) return a.stream < b.stream;
    return a.seq < b.seq;
  });
  r.intervals.reserve(ivs.size());
  for (auto &k : ivs) r.intervals.push_back(k.iv);
}

}  // namespace

extern "C" {

typedef struct orc_result orc_result;

// Runs validation and analysis.  Returns the status code; *out (always set
// unless allocation fails) carries rows, diag, intervals and the error location.
int orc_run(const void *bytes, uint64_t nbytes, const orc_opts *opts, orc_result **out) {
  Result *r = new (std::nothrow) Result();
  if (!r) return ORC_E_INVALID;
  *out = reinterpret_cast<orc_result *>(r);
  orc_opts o{};
  if (opts) o = *opts;
  if (!opts) {
    o.want_intervals = 1;
    o.t0 = 0;
    o.t1 = UINT64_MAX;
  }
  const uint8_t *b = static_cast<const uint8_t *>(bytes);
  Trace t{};
  std::vector<char> keep;
  const std::vector<char> *keep_p = nullptr;
  if (o.streams) {
    // the subset is applied after the file header is known
    int rc0 = parse_file(b, nbytes, t);
    if (rc0 != ORC_OK) {
      r->code = rc0;
      return rc0;
    }
    keep.assign(t.n_streams, 0);
    for (uint32_t i = 0; i < o.n_subset; ++i)
      if (o.streams[i] < t.n_streams) keep[o.streams[i]] = 1;
    keep_p = &keep;
    t = Trace{};
  }
  int rc = validate(b, nbytes, t, r->loc, keep_p);
  r->code = rc;
  if (rc != ORC_OK) return rc;
  analyse(t, o, keep_p, *r, false);
  return ORC_OK;
}

// The all-cores CPU baseline (a per-stream threaded run of the same
// definition): the selected streams are dealt round robin to `threads`
// std::threads, each of which validates and analyses its subset exactly as
// orc_run does; the partial results are then merged.  Streams pair
// independently only when no stream is a per-CPU buffer and no class carries
// device activity (DEV_BEGIN / DEV_END or a command id), so any other trace,
// or threads <= 1, runs as orc_run.  Merge: rows with one key combine
// (count, total and errors add, min / max), the diagnostics add, and the
// subsets' intervals, each already in (start, stream, entry position) order
// over disjoint streams, merge by (start, stream).  Meant for valid traces:
// an invalid subset returns its own code and location, which need not be the
// whole trace's first failure.
int orc_run_threads(const void *bytes, uint64_t nbytes, const orc_opts *opts, uint32_t threads, orc_result **out) {
  const uint8_t *b = static_cast<const uint8_t *>(bytes);
  Trace t{};
  if (threads <= 1 || parse_file(b, nbytes, t) != ORC_OK) return orc_run(bytes, nbytes, opts, out);
  bool independent = true;
  for (const Stream &st : t.streams) independent = independent && !(st.flags & STREAM_PER_CPU);
  for (const Class &c : t.classes)
    independent = independent && c.kind != KIND_DEV_BEGIN && c.kind != KIND_DEV_END && c.cmd_off < 0;
  if (!independent) return orc_run(bytes, nbytes, opts, out);
  orc_opts o{};
  if (opts) o = *opts;
  if (!opts) {
    o.want_intervals = 1;
    o.t0 = 0;
    o.t1 = UINT64_MAX;
  }
  std::vector<uint32_t> ids;
  if (o.streams) {
    std::vector<char> keep(t.n_streams, 0);
    for (uint32_t i = 0; i < o.n_subset; ++i)
      if (o.streams[i] < t.n_streams) keep[o.streams[i]] = 1;
    for (uint32_t s = 0; s < t.n_streams; ++s)
      if (keep[s]) ids.push_back(s);
  } else {
    for (uint32_t s = 0; s < t.n_streams; ++s) ids.push_back(s);
  }
  const uint32_t k = (uint32_t)std::min<uint64_t>(threads, std::max<uint64_t>(ids.size(), 1));
  std::vector<std::vector<uint32_t>> subset(k);
  for (size_t i = 0; i < ids.size(); ++i) subset[i % k].push_back(ids[i]);
  std::vector<orc_result *> part(k, nullptr);
  std::vector<int> code(k, ORC_OK);
  std::vector<std::thread> pool;
  for (uint32_t j = 0; j < k; ++j)
    pool.emplace_back([&, j]() {
      orc_opts so = o;
      so.streams = subset[j].data();
      so.n_subset = (uint32_t)subset[j].size();
      code[j] = orc_run(bytes, nbytes, &so, &part[j]);
    });
  for (auto &th : pool) th.join();
  Result *r = new (std::nothrow) Result();
  if (!r) {
    for (auto *q : part) delete reinterpret_cast<Result *>(q);
    return ORC_E_INVALID;
  }
  *out = reinterpret_cast<orc_result *>(r);
  for (uint32_t j = 0; j < k; ++j)
    if (code[j] != ORC_OK || !part[j]) {
      if (part[j]) *r = *reinterpret_cast<Result *>(part[j]);
      r->code = part[j] ? code[j] : ORC_E_INVALID;
      for (auto *q : part) delete reinterpret_cast<Result *>(q);
      return r->code;
    }
  std::map<std::tuple<uint32_t, uint32_t, uint32_t, uint32_t>, orc_row> rows;
  auto by_start = [](const orc_interval &x, const orc_interval &y) {
    if (x.start_ns != y.start_ns) return x.start_ns < y.start_ns;
    return x.stream_id < y.stream_id;
  };
  for (uint32_t j = 0; j < k; ++j) {
    Result &q = *reinterpret_cast<Result *>(part[j]);
    for (const orc_row &w : q.rows) {
      auto key = std::make_tuple(w.host_id, w.pid, w.tid, w.func_id);
      auto it = rows.find(key);
      if (it == rows.end()) {
        rows.emplace(key, w);
        continue;
      }
      orc_row &m = it->second;
      m.count += w.count;
      m.total_ns += w.total_ns;
      m.err_count += w.err_count;
      m.min_ns = std::min(m.min_ns, w.min_ns);
      m.max_ns = std::max(m.max_ns, w.max_ns);
    }
    r->diag.events += q.diag.events;
    r->diag.pairs += q.diag.pairs;
    r->diag.unmatched_entries += q.diag.unmatched_entries;
    r->diag.unmatched_exits += q.diag.unmatched_exits;
    r->diag.mismatched_pairs += q.diag.mismatched_pairs;
    r->diag.other_events += q.diag.other_events;
    r->diag.discarded += q.diag.discarded;
    r->diag.packets += q.diag.packets;
    std::vector<orc_interval> both;
    both.reserve(r->intervals.size() + q.intervals.size());
    std::merge(r->intervals.begin(), r->intervals.end(), q.intervals.begin(), q.intervals.end(),
               std::back_inserter(both), by_start);
    r->intervals.swap(both);
    delete reinterpret_cast<Result *>(part[j]);
    part[j] = nullptr;
  }
  for (auto &kv : rows) r->rows.push_back(kv.second);
  return ORC_OK;
}

uint64_t orc_n_rows(const orc_result *r) { return reinterpret_cast<const Result *>(r)->rows.size(); }
const orc_row *orc_rows(const orc_result *r) { return reinterpret_cast<const Result *>(r)->rows.data(); }
uint64_t orc_n_intervals(const orc_result *r) { return reinterpret_cast<const Result *>(r)->intervals.size(); }
const orc_interval *orc_intervals(const orc_result *r) {
  return reinterpret_cast<const Result *>(r)->intervals.data();
}
void orc_get_diag(const orc_result *r, orc_diag *d) { *d = reinterpret_cast<const Result *>(r)->diag; }
uint64_t orc_n_dev_rows(const orc_result *r) { return reinterpret_cast<const Result *>(r)->dev_rows.size(); }
const orc_row *orc_dev_rows(const orc_result *r) { return reinterpret_cast<const Result *>(r)->dev_rows.data(); }
uint64_t orc_n_self_rows(const orc_result *r) { return reinterpret_cast<const Result *>(r)->self_rows.size(); }
const orc_row *orc_self_rows(const orc_result *r) { return reinterpret_cast<const Result *>(r)->self_rows.data(); }
void orc_get_dev_diag(const orc_result *r, orc_dev_diag *d) { *d = reinterpret_cast<const Result *>(r)->dev; }
void orc_error_location(const orc_result *r, int *level, uint64_t *packet, uint64_t *event) {
  const Result *x = reinterpret_cast<const Result *>(r);
  *level = x->loc.level;
  *packet = x->loc.packet;
  *event = x->loc.event;
}
void orc_free(orc_result *r) { delete reinterpret_cast<Result *>(r); }

// Decodes every event (stream order) into out[0..cap); *n = total events.
int orc_decode(const void *bytes, uint64_t nbytes, orc_event *out, uint64_t cap, uint64_t *n) {
  Result r;
  Trace t{};
  int rc = validate(static_cast<const uint8_t *>(bytes), nbytes, t, r.loc, nullptr);
  if (rc != ORC_OK) return rc;
  orc_opts o{};
  analyse(t, o, nullptr, r, true);
  *n = r.events.size();
  for (uint64_t i = 0; i < r.events.size() && i < cap; ++i) out[i] = r.events[i];
  return ORC_OK;
}

}  // extern "C"

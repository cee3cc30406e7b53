// internal.cuh — shared declarations of the CUDA trace-analysis library.
//
// The library reads the THPT layout described in include/thapi.h.  Its own
// restatement of that layout lives here; nothing is shared with the CPU
// oracle used by the tests.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <utility>
#include <vector>

#include "thapi.h"

namespace thapi {

// ------------------------------------------------------------- layout
constexpr uint32_t kTraceMagic = 0x54504854u;   // "THPT"
constexpr uint32_t kPacketMagic = 0x31544B50u;  // "PKT1"
constexpr uint32_t kExtBit = 1u << 27;
constexpr uint32_t kDeltaMask = (1u << 27) - 1u;
constexpr uint32_t kHeaderBytes = 128;
constexpr uint32_t kPacketHeader = 32;
constexpr uint32_t kMaxPacket = 65536;

enum Kind : uint32_t { kEntry = 0, kExit = 1, kDevBegin = 2, kDevEnd = 3, kSample = 4 };

// Packed class row: fixed words (14 bits) | kind << 14 (3) | func << 17 (16)
//   | (result word + 1) << 33 (15, 0 = none) | (cmd word + 1) << 48 (15, 0 = none)
__host__ __device__ inline uint32_t cls_fixedw(uint64_t c) { return (uint32_t)(c & 0x3FFFu); }
__host__ __device__ inline uint32_t cls_kind(uint64_t c) { return (uint32_t)((c >> 14) & 7u); }
__host__ __device__ inline uint32_t cls_func(uint64_t c) { return (uint32_t)((c >> 17) & 0xFFFFu); }
__host__ __device__ inline int32_t cls_resw(uint64_t c) { return (int32_t)((c >> 33) & 0x7FFFu) - 1; }
__host__ __device__ inline int32_t cls_cmdw(uint64_t c) { return (int32_t)((c >> 48) & 0x7FFFu) - 1; }

// Interval slot flags (the output keeps bits 0 and 2).
constexpr uint8_t kIvErr = 1u;
constexpr uint8_t kIvDevice = 1u << 2;  // device interval (device-activity pairing)
constexpr uint8_t kIvOpen = 1u << 6;
constexpr uint8_t kIvValid = 1u << 7;

// Frontier item: an entry still open at the end of its packet, or an exit
// that pops below the packet's starting depth.
struct __align__(16) Frontier {
  uint64_t ts;
  uint32_t aux;   // open: interval slot rank in its packet (or ~0u); pending exit: event index in its packet
  uint16_t func;
  uint16_t flags; // pending exit: error flag
};

// Self-time side record of an interval slot (written only when self time is
// on): event positions (the packet's event base + the event's index in the
// packet) of the entry and of the exit that closes it, and the entry's depth,
// packet-relative clamped (the timeline compaction's level before the depth
// carried into the packet is added) or, with kSelfAbs, absolute (pairs formed
// across packets).
struct SelfSlot {
  uint64_t entry_pos, exit_pos;
  uint32_t level, pad;
};
constexpr uint32_t kSelfAbs = 0x80000000u;

// Tally cell of the global (group, function) table.
struct __align__(8) Cell {
  unsigned long long count, total, mn, mx, err;
};

#ifdef __CUDACC__
// Block b of nb takes chunk spread(b, nb): a bijection of [0, nb) under which
// blocks that run at the same time (consecutive b) take chunks far apart, so
// that their tally atomics spread over many cells instead of the few cells of
// one stretch of the input (the chunks of a group of 1024 consecutive
// blocks lie nb / 1024 apart).
__device__ __forceinline__ uint64_t spread(uint64_t b, uint64_t nb) {
  const uint64_t G = nb < 1024 ? nb : 1024;
  const uint64_t g = b % G, k = b / G, q = nb / G, r = nb % G;
  return g * q + (g < r ? g : r) + k;
}

// One call per active lane tallied into cells[idx], lanes of the warp with
// the same cell combined first so that one lane per distinct cell issues the
// atomics (neighbouring calls often share a cell, and atomics to one address
// serialise).  Every lane of the warp calls it; scr: 32 entries of this warp.
struct CellPart {
  unsigned long long dur;
  unsigned err, pad;
};
__device__ __forceinline__ void warp_tally(Cell *cells, uint64_t idx, bool act, unsigned long long dur, bool err,
                                           CellPart *scr) {
  const uint32_t lane = threadIdx.x & 31;
  const uint32_t peers = __match_any_sync(0xffffffffu, act ? (unsigned long long)idx : ~0ull);
  scr[lane] = CellPart{dur, err ? 1u : 0u, 0u};
  __syncwarp();
  if (act && lane == (uint32_t)(__ffs(peers) - 1)) {
    unsigned long long sum = 0, mn = ~0ull, mx = 0, e = 0;
    for (uint32_t m = peers; m; m &= m - 1) {
      const CellPart c = scr[__ffs(m) - 1];
      sum += c.dur;
      mn = c.dur < mn ? c.dur : mn;
      mx = c.dur > mx ? c.dur : mx;
      e += c.err;
    }
    Cell &c = cells[idx];
    atomicAdd(&c.count, (unsigned long long)__popc(peers));
    atomicAdd(&c.total, sum);
    atomicMin(&c.mn, mn);
    atomicMax(&c.mx, mx);
    if (e) atomicAdd(&c.err, e);
  }
  __syncwarp();
}
#endif

// Device error word: packet file index << 20 | event << 3 | code; ~0 = none.
__host__ __device__ inline unsigned long long err_key(uint64_t packet, uint32_t event, uint32_t code) {
  return ((unsigned long long)packet << 20) | ((unsigned long long)(event & 0x1FFFFu) << 3) | (code & 7u);
}

// Diagnostic counters (device), same order as thapi_diag.
// dDevEvents: DEV_BEGIN / DEV_END events (device-activity diagnostics).
enum Diag { dEvents = 0, dPairs, dUnEntry, dUnExit, dMismatch, dOther, dDiscarded, dPackets, dDevEvents, dCount };

// Device-activity records, one per event that carries a command id, written
// by the analysis kernels in no particular order (join.cu pairs them).
struct __align__(16) CmdBegin {  // DEV_BEGIN
  uint64_t cmd, ts;
  uint64_t slot;                 // its interval slot (global index)
  uint32_t group, pos;           // its stream's (host, pid, tid) group; its packet's order position
};
struct __align__(16) CmdEnd {    // DEV_END
  uint64_t cmd, ts;
};
struct __align__(16) CmdHost {   // ENTRY of the host call that submitted the command
  uint64_t cmd;
  uint32_t func, pad;
};
// Where the analysis writes them: counts[k] grows past cap[k] without writing
// past it (the host then retries with the exact counts).  hist counts the
// records of each kind per hash partition of the command id (join.cu).
struct CmdOut {
  CmdBegin *b = nullptr;
  CmdEnd *e = nullptr;
  CmdHost *h = nullptr;
  uint64_t cap_b = 0, cap_e = 0, cap_h = 0;
  unsigned long long *counts = nullptr;  // [3]: begin, end, host records; null = no device pairing
  uint32_t *hist = nullptr;              // [3][1 << part_bits]
  int part_bits = 1;                     // partition = top part_bits bits of cmd_hash(id), 1..18
};

// Finaliser of SplitMix64 (Steele, Lea & Flood, "Fast splittable
// pseudorandom number generators", OOPSLA 2014): a bijective mix of a
// command id.  Its top bits choose the id's partition, its low bits the
// entry in a partition's table.
__host__ __device__ __forceinline__ uint64_t cmd_hash(uint64_t z) {
  z = (z ^ (z >> 30)) * 0xbf58476d1ce4e5b9ull;
  z = (z ^ (z >> 27)) * 0x94d049bb133111ebull;
  return z ^ (z >> 31);
}
__host__ __device__ __forceinline__ uint32_t cmd_part(uint64_t id, int part_bits) {
  return (uint32_t)(cmd_hash(id) >> (64 - part_bits));
}

// ------------------------------------------------------ kernel params
// Where packet pk (its index in the trace, or in a batch's packet list) is:
// a table of addresses when a batch reads its traces' packets in place,
// else consecutive packets from `packets`.
#ifdef __CUDACC__
__device__ __forceinline__ const uint8_t *packet_at(const uint8_t *packets, const uint64_t *addr, uint64_t pk,
                                                    uint32_t P) {
  return addr ? reinterpret_cast<const uint8_t *>(__ldg(addr + pk)) : packets + pk * (uint64_t)P;
}
#endif

struct IndexParams {
  const uint8_t *packets;  // first packet
  const uint64_t *pk_addr; // per packet its address (a batch read in place), or null
  unsigned long long *read_bytes;  // sum of 32 + content_bytes over valid packets
  uint32_t P;
  uint64_t n_packets;
  uint32_t n_streams;
  uint32_t *pk_stream, *pk_nev, *pk_content, *pk_seq, *pk_disc;
  uint64_t *pk_tsb;
  unsigned long long *hdr_err;  // min packet index with a header error
  // a batch of traces (null: one trace): per packet its trace, per trace its
  // first stream in the batch and its own stream count
  const uint32_t *pk_trace, *t_soff, *t_nstreams;
};

// Stream group of a per-CPU buffer (stream flags bit 1): its events belong to
// the threads named in each event, paired by percpu.cu.
constexpr uint32_t kPerCpuGroup = 0xFFFFFFFFu;
constexpr uint32_t kStreamPerCpu = 2u;

// What the analysis needs of one packet, gathered per order position.
struct __align__(16) PkDesc {
  uint32_t pk, content, nev, stream;  // file index, content bytes, events, stream id
  uint32_t group, disc, pad0, pad1;   // (host, pid, tid) group, discarded counter
  uint64_t tsb, evbase;               // ts_begin, first event slot
};

struct AnalyzeParams {
  const uint8_t *packets;
  const uint64_t *pk_addr;       // per packet its address, or null (see packet_at)
  uint32_t P;
  uint32_t emax;                 // shared-memory event table capacity of this launch
  uint64_t n_order;              // work items of this launch
  const uint32_t *poslist;       // work item -> order position (null: identity)
  const PkDesc *desc;            // per order position
  const uint64_t *classes;       // packed class rows
  uint32_t n_classes, n_funcs;
  Cell *tally;                   // [groups * n_funcs]
  uint32_t *sum_pend, *sum_open, *sum_nslot, *sum_nvalid;  // per order position
  uint64_t *sum_fbase;
  Frontier *frontier;
  unsigned long long *frontier_top;
  uint64_t frontier_cap;
  thapi_interval *slots;         // null: no timeline
  unsigned long long *content_err;
  unsigned long long *diag;      // dCount counters
  unsigned long long *tminmax;   // [0] min ts, [1] max ts
  unsigned long long *slots_written;  // interval slots written (24 B each)
  uint32_t *dense_list;          // packets with more events than emax (order positions)
  unsigned long long *dense_count;
  uint32_t per_cta;              // work items per CTA
  const uint32_t *run_start;     // warp kernel: CTA c takes work items [run_start[c], run_start[c + 1])
  CmdOut cmd;                    // device-activity records (counts null: none)
  SelfSlot *side;                // per interval slot (null: self time off)
};

struct FrontierParams {
  uint64_t n_order;
  uint32_t n_streams;
  const uint32_t *order;
  const uint32_t *pk_stream;
  const uint32_t *stream_first, *stream_count;  // per stream: first order position, packet count
  const uint32_t *sum_pend, *sum_open;
  const uint64_t *sum_fbase;
  uint32_t *A, *base;            // per order position
  const uint64_t *evbase;
  const Frontier *frontier;
  const uint32_t *stream_group;
  uint32_t n_funcs;
  Cell *tally;
  thapi_interval *slots;
  uint32_t *sum_nvalid;
  unsigned long long *diag;
  SelfSlot *side;                // null: self time off
};

// ---------------------------------------------------------- launchers
// Kernels launched by this library since the process started (every launch
// site adds to it; loads report their own delta).
void count_launches(uint64_t k);
uint64_t launches_total();

// Device-wide scans and sorts (scan.cu, radix.cu).  Scratch is allocated by
// the caller through the context allocator.
struct Scratch;
void scan_exclusive_u64(uint64_t *data, uint64_t n, uint64_t *total_dev, Scratch &sc, cudaStream_t s);
void radix_sort_pairs(uint64_t *keys, uint32_t *vals, uint64_t *keys_alt, uint32_t *vals_alt, uint64_t n,
                      int bits, bool *result_in_alt, Scratch &sc, cudaStream_t s);
void radix_sort_pairs32(uint32_t *keys, uint32_t *vals, uint32_t *keys_alt, uint32_t *vals_alt, uint64_t n, int bits,
                        bool *result_in_alt, Scratch &sc, cudaStream_t s);
// bucket.cu: timeline order by start bucket.  bucket_plan sizes the coarse
// buckets and clears the (bucket, stream) cells the compaction counts into;
// bucket_run orders the compacted records (false from either: use
// radix_sort_gather).
struct BucketCells {
  uint32_t *cnt = nullptr, *first = nullptr;  // [nb * S] records and first record index per cell
  int shift = 0;                              // coarse bucket = key >> shift
  uint32_t nb = 0, S = 0;
};
bool bucket_plan(uint64_t n, int bits, uint32_t S, Scratch &sc, cudaStream_t s, BucketCells *bc);
bool bucket_run(const BucketCells &bc, uint64_t t_min, uint64_t n, const thapi_interval *rec, thapi_interval *out,
                Scratch &sc, cudaStream_t s, int num_sms);
// keys hold u32 values when bits <= 32 (u64 otherwise); rec_out[i] = rec[index
// of the i-th smallest key] (stable); vals and vals_alt are work space
void radix_sort_gather(uint64_t *keys, uint32_t *vals, uint64_t *keys_alt, uint32_t *vals_alt, uint64_t n, int bits,
                       const thapi_interval *rec, thapi_interval *rec_out, Scratch &sc, cudaStream_t s);

// File header and tables of a trace, checked, with streams numbered into
// (host, pid, tid) groups in order (api.cu).
struct TraceDescription {
  uint32_t P = 0, n_streams = 0, n_classes = 0, n_funcs = 0, n_hosts = 0, groups = 0;
  uint64_t n_packets = 0, packets_off = 0;
  std::vector<uint64_t> cls;
  std::vector<uint32_t> stream_group, group_keys;
};
int describe_device_trace(const uint8_t *dev, uint64_t nbytes, cudaStream_t s, TraceDescription &td);
// api.cu hooks of the serving loop (server.cu); contexts are thread-safe for these.
int ctx_device(const thapi_ctx *c);
int ctx_num_sms(const thapi_ctx *c);
void ctx_memory(thapi_ctx *c, uint64_t *cap, uint64_t *used);
void *ctx_alloc(thapi_ctx *c, uint64_t bytes, cudaStream_t s);
void ctx_free(thapi_ctx *c, void *p, uint64_t bytes, cudaStream_t s);
int load_charge(thapi_ctx *c, const uint8_t *host, const uint8_t *dev, uint64_t nbytes, cudaStream_t s,
                uint64_t *est);
int load_admitted(thapi_ctx *c, const uint8_t *host, const uint8_t *dev, uint64_t nbytes, cudaStream_t s,
                  thapi_trace_id *out);
int trace_sizes(thapi_ctx *c, thapi_trace_id id, uint64_t *rows, uint64_t *intervals, uint64_t *events);
int tally_enqueue(thapi_ctx *c, thapi_trace_id id, thapi_tally_row *dst, uint64_t cap, uint64_t *n, cudaStream_t s);
struct WinWork;
int window_enqueue_id(thapi_ctx *c, thapi_trace_id id, uint64_t t0, uint64_t t1, thapi_interval *dst, uint64_t cap,
                      WinWork *w, unsigned long long *total, cudaStream_t s);
int free_trace_on(thapi_ctx *c, thapi_trace_id id, cudaStream_t s);
int window_to_host_id(thapi_ctx *c, thapi_trace_id id, uint64_t t0, uint64_t t1, void *out, uint64_t n,
                      thapi_interval *stage, WinWork *w, unsigned long long *total, cudaStream_t s);
// The whole ordered timeline (n intervals, the trace's count) to out, host or
// device memory, enqueued on s (one copy).
int timeline_copy_id(thapi_ctx *c, thapi_trace_id id, void *out, uint64_t n, bool device_out, cudaStream_t s);
void *device_view(void *p);
// A context that allocates only through the given hooks (creates nothing on the device).
thapi_ctx *hooked_ctx_create(int device, thapi_alloc_fn alloc, thapi_free_fn free_fn, void *user);

// Scratch allocator used inside one library call: every buffer it hands out
// is released (in stream order) by release_all.
struct Scratch {
  thapi_ctx *ctx = nullptr;
  cudaStream_t stream = nullptr;
  std::vector<std::pair<void *, uint64_t>> bufs;
  int failed = 0;  // 1: an allocation failed; 2: a bounded device wait ran out (a sort's look-back)
  void *get(uint64_t bytes);
  void adopt(void *p, uint64_t bytes);
  void release_all();
};

}  // namespace thapi

namespace thapi {

// index.cu
void launch_widen_u32(const uint32_t *in, uint64_t *out, uint64_t n, cudaStream_t s);
void launch_build_desc(const uint32_t *order, const uint32_t *pk_stream, const uint32_t *pk_nev,
                       const uint32_t *pk_content, const uint32_t *pk_disc, const uint64_t *pk_tsb,
                       const uint32_t *stream_group, const uint64_t *evbase, uint64_t n, PkDesc *desc, cudaStream_t s);
void launch_packet_headers(const IndexParams &p, cudaStream_t s);
// One warp waits on an mbarrier nothing completes, at most `limit` tries;
// *status (device) = THAPI_E_TIMEOUT when the wait gives up.
cudaError_t launch_wait_check(uint32_t limit, unsigned *status, cudaStream_t s);
// dst + q * P = trace pk_trace[q]'s packet (q - first[t]) at src[t] (16-byte
// aligned), a warp per packet.
// addr[i] = src[t] + (i - first[t]) * P with t = pk_trace[i]: the address of
// each packet of a batch whose traces stay where they are in device memory.
void launch_packet_addrs(const uint8_t *const *src, const uint64_t *first, const uint32_t *pk_trace, uint64_t n,
                         uint32_t P, uint64_t *addr, cudaStream_t s);
// pk_trace[q] = the trace t whose packets [first[t], first[t + 1]) hold q
// (first: nt nondecreasing first-packet indexes, first[0] = 0).
void launch_packet_traces(const uint64_t *first, uint32_t nt, uint64_t n, uint32_t *pk_trace, cudaStream_t s);
// dst[off[i] .. off[i] + len[i]) = src[i][0 .. len[i]) for i < n (a block per source).
void launch_gather_bytes(const uint8_t *const *src, const uint64_t *len, const uint64_t *off, uint32_t n,
                         uint8_t *dst, cudaStream_t s);
void launch_stream_keys(const uint32_t *pk_stream, uint64_t n, uint64_t *keys, uint32_t *vals, cudaStream_t s);
void launch_stream_bounds(const uint64_t *skey, const uint32_t *order, const uint32_t *pk_seq, const uint32_t *pk_nev,
                          uint64_t n, uint32_t n_streams, uint32_t *stream_first, uint32_t *stream_count,
                          uint64_t *ev, unsigned long long *hdr_err, cudaStream_t s);
// analyze.cu
uint32_t analyze_smem_bytes(uint32_t P, uint32_t emax, int stages, uint32_t n_classes, uint32_t n_funcs);
uint64_t analyze_frontier_slack(uint32_t grid);
// analyze_warp.cu: one warp per packet (packets up to 32 KB)
struct WarpPlan {
  uint32_t nw = 0, ctas_per_sm = 0, smem = 0;  // warps per CTA, resident CTAs per SM, dynamic shared memory
};
bool plan_analyze_warp(uint32_t P, uint32_t n_classes, int smem_optin, int smem_per_sm, WarpPlan *out);
cudaError_t launch_analyze_warp(const AnalyzeParams &p, const WarpPlan &wp, uint32_t grid, cudaStream_t s,
                                unsigned *status);
uint64_t analyze_warp_frontier_slack(uint64_t warps);
// Decode of every event (thapi_decode): one warp per packet, packets up to 32 KB.
struct DecodeParams {
  const uint8_t *packets;
  const uint64_t *pk_addr;       // per packet its address, or null (see packet_at)
  uint32_t P, n_classes;
  uint64_t n_order;
  const PkDesc *desc;            // per order position
  const uint64_t *classes;       // packed class rows
  thapi_event *out;              // at desc.evbase + event index
  unsigned long long *content_err;
  const uint32_t *group_keys;    // host, pid, tid per group (per-thread streams' pid / tid)
};
uint32_t decode_warps(uint32_t P, uint32_t n_classes, int smem_optin);  // warps per CTA, 0 = unsupported

// Per-CPU buffers (percpu.cu): one record per ENTRY / EXIT of a per-CPU
// buffer, written by k_percpu_decode (analyze_warp.cu).
constexpr uint8_t kPcNone = 0xFF;  // PcRec.kind of a position that holds no ENTRY / EXIT
struct __align__(8) PcRec {
  uint64_t ts;
  uint64_t thread;     // vpid << 32 | vtid
  uint32_t host;       // the buffer's host
  uint32_t slot;       // ENTRY: its interval slot (global index)
  uint32_t pos;        // order position of its packet
  uint16_t func;
  uint8_t kind, err;   // kEntry / kExit / kPcNone; EXIT result != 0
};
static_assert(sizeof(PcRec) == 32, "per-CPU record");
struct PcParams {
  const uint8_t *packets;
  const uint64_t *pk_addr;       // per packet its address, or null (see packet_at)
  uint32_t P, n_classes;
  uint64_t n_order;
  const PkDesc *desc;
  const uint64_t *classes;
  const uint32_t *stream_host;   // host id per stream
  PcRec *rec;                    // at pc_base[order position] + event index in the packet
  const uint64_t *pc_base;       // per order position: per-CPU events before its packet
  uint64_t cap;
  unsigned long long *count;     // records written (may pass cap: then nothing past it is written)
  thapi_interval *slots;
  uint32_t *sum_nslot;
  unsigned long long *content_err;
  unsigned long long *diag;
  unsigned long long *tminmax;
};
cudaError_t launch_percpu_decode(const PcParams &p, uint32_t nw, uint32_t grid, cudaStream_t s);
// Per order position: the packet's events if it is a per-CPU buffer, else 0
// (their exclusive scan places the records).
void launch_pc_count(const PkDesc *desc, uint64_t n, uint64_t *out, cudaStream_t s);
// Over the per-CPU packets: out[0] += 32 + content bytes, out[1] += their
// interval slots (ENTRY events, from sum_nslot after the decode).
void launch_pc_bytes(const PkDesc *desc, const uint32_t *sum_nslot, uint64_t n, unsigned long long *out,
                     cudaStream_t s);
// Pairs the threads of the per-CPU records (m_all positions in position
// order, m of them ENTRY / EXIT records): thread numbers from a table of
// (host, vpid, vtid) and one stable sort by (thread, ts), or stable sorts by
// ts, thread and host when the table is full or two keys share a
// fingerprint; then the depth monoid scanned per thread and each entry
// matched with its exit by (thread, level).  Tallies into per-thread cells,
// writes the entries' interval slots and raises their packets' interval
// counts; cells / keys are allocated here (sc).
struct PcPairOut {
  Cell *cells = nullptr;           // [threads * n_funcs]
  Cell *self_cells = nullptr;      // [threads * n_funcs], self time (when asked for)
  uint32_t *keys = nullptr;        // [threads * 3] host, vpid, vtid
  uint64_t threads = 0;
};
// Self time of the calls of per-thread streams (self.cu), from the interval
// slots and their SelfSlot records after pairing: cells [groups * n_funcs]
// (initialised by the caller) receive count, total / min / max self time and
// errors.  word: one device word.
struct SelfIn {
  const thapi_interval *slots;
  const SelfSlot *side;
  const uint64_t *evbase, *obase;
  const uint32_t *nslot, *A, *order, *pk_stream, *stream_group;
  uint32_t n_funcs, n_streams;
  uint64_t n_order, n_iv;
  int num_sms;
};
int self_time(const SelfIn &in, Cell *cells, uint64_t *word, Scratch &sc, cudaStream_t s);
// self_on: also the threads' self-time cells (PcPairOut.self_cells).
int percpu_pair(PcRec *rec, uint64_t m_all, uint64_t m, uint64_t t_min, int ts_bits, uint32_t n_funcs,
                thapi_interval *slots, uint32_t *sum_nvalid, unsigned long long *diag, bool self_on, int num_sms,
                Scratch &sc, cudaStream_t s, PcPairOut *out);
cudaError_t launch_decode_warp(const DecodeParams &p, uint32_t nw, uint32_t grid, cudaStream_t s);
// Splits the stream-ordered packets into `grid` contiguous runs of about equal
// cost (events + a per-packet constant): run_start[0..grid].
void launch_cost_split(const uint64_t *evbase, uint64_t n, uint64_t total_events, uint32_t grid, uint32_t *run_start,
                       cudaStream_t s);
cudaError_t launch_analyze(const AnalyzeParams &p, int stages, uint32_t grid, cudaStream_t s, unsigned *status);
// frontier.cu
void launch_frontier(const FrontierParams &p, cudaStream_t s);
// tally.cu
void launch_tally_init(Cell *cells, uint64_t n, cudaStream_t s);
void launch_tally_compact(const Cell *cells, uint64_t n, const uint32_t *group_keys, uint32_t n_funcs,
                          uint64_t *flags, thapi_tally_row *rows, uint64_t *n_rows_dev, Scratch &sc, cudaStream_t s);
// join.cu: device-activity pairing over the command records.  The command
// table has a power-of-two capacity plus one entry (for the zero id) and must
// be zeroed before launch_cmd_insert.
struct __align__(32) CmdEntry {
  unsigned long long key;         // command id (0: free, except in the zero id's own entry)
  unsigned long long nbe;         // begin records | end records << 32
  unsigned long long te;          // sum of its DEV_END timestamps (the timestamp when there is one)
  unsigned long long nhf;         // host records | sum of their functions << 32 (the function when one)
};
struct JoinParams {
  const CmdBegin *b;
  const CmdEnd *e;
  const CmdHost *h;
  uint64_t nb, ne, nh;
  CmdEntry *tab;
  uint64_t mask;                  // capacity - 1
  uint64_t probe_limit;           // entries one insert may probe before it reports overflow
  thapi_interval *slots;
  uint32_t *sum_nvalid;           // per order position
  Cell *dcells;                   // device tally [groups * n_funcs]
  uint32_t n_funcs;
  unsigned long long *out;        // [0..4]: pairs, intervals, unjoined, ambiguous, host entries of pairs; [5]: overflow
};
void launch_cmd_insert(const JoinParams &jp, int num_sms, cudaStream_t s);
void launch_cmd_emit(const JoinParams &jp, int num_sms, cudaStream_t s);
// Partitioned join: records grouped by partition (hist from the analysis),
// then one CTA per partition with its table in shared memory.
constexpr uint32_t kPartMaxRecords = 3072;  // records of one partition the shared-memory table takes
struct PartPlan {
  int part_bits;
  const uint32_t *hist;           // [3][P] records per kind and partition
  uint64_t *base;                 // [3P + 1] exclusive prefix of hist (kind-major), then the total
  unsigned long long *cursor;     // [3P] scatter cursors
  unsigned long long *max_records;  // largest partition (all kinds)
  CmdBegin *pb;                   // partitioned copies
  CmdEnd *pe;
  CmdHost *ph;
};
// Widens hist into base and finds the largest partition (before the scan of base).
void launch_part_prep(const PartPlan &pp, cudaStream_t s);
// Cursors from the scanned base, then every record to its partition.
void launch_part_scatter(const JoinParams &jp, const PartPlan &pp, int num_sms, cudaStream_t s);
// One CTA per partition: pairs, joins, emits (needs max_records <= kPartMaxRecords).
void launch_part_join(const JoinParams &jp, const PartPlan &pp, uint64_t max_records, cudaStream_t s);
// merge.cu: rows (device, any order, n of them) -> out (device, >= n rows):
// one row per distinct (host_id, pid, tid, func_id) in key order, *m_dev = rows.
bool tally_merge_device(const thapi_tally_row *rows, uint64_t n, thapi_tally_row *out, uint64_t *m_dev, Scratch &sc,
                        cudaStream_t s);
// timeline.cu
void launch_timeline_compact(const thapi_interval *slots, const uint64_t *evbase, const uint32_t *nslot,
                             const uint64_t *out_base, const uint32_t *A, const uint32_t *order,
                             const uint32_t *pk_stream, uint64_t n_order, uint64_t t_min, thapi_interval *rec,
                             void *keys, bool key32, uint32_t *vals, const BucketCells *cells, int num_sms,
                             cudaStream_t s);
void launch_timeline_gather(const thapi_interval *rec, const uint32_t *vals, uint64_t n, thapi_interval *out,
                            cudaStream_t s);
void launch_iota_u32(uint32_t *v, uint64_t n, cudaStream_t s);
void launch_rec_keys(const thapi_interval *rec, uint64_t n, uint64_t t_min, void *keys, bool key32, cudaStream_t s);

// window.cu: time-window queries.  A trace's window index holds, per block of
// kWinBlock intervals in timeline order, the running maximum of their ends;
// a query finds its range with it and writes the matches in order.
constexpr uint32_t kWinBlock = 2048;
constexpr uint32_t kWinCtas = 512;  // most CTAs of one query
struct WinWork {                    // device working record of one query in flight
  unsigned long long lo, hi;        // the range searched: [lo, hi)
  unsigned long long cnt[kWinCtas]; // matches per CTA chunk
};
void launch_win_index(const thapi_interval *tl, uint64_t n, uint64_t *bmax, cudaStream_t s);
// matches to out (device-visible; null: count only) only when *total_out <= cap
void launch_win_query(const thapi_interval *tl, uint64_t n, const uint64_t *bmax, uint64_t t0, uint64_t t1,
                      WinWork *w, uint32_t grid, thapi_interval *out, uint64_t cap, unsigned long long *total_out,
                      cudaStream_t s);

}  // namespace thapi

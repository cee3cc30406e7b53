/* thapi.h — C ABI of the B300 trace-analysis library (libthapi.so).
 *
 * The library turns a binary trace of intercepted API entry/exit events into
 * (i) the per-(hostname, pid, tid, function) tally — call count, total / min /
 * max inclusive duration, error-result count — and (ii) the time-ordered
 * interval timeline.  These are the summary ("Tally") and timeline views that
 * THAPI derives from its traces with Babeltrace2 plugins (arxiv 2504.03683,
 * Sec. 3.2: entry and exit points traced with arguments and results;
 * Sec. 3.4: plugins fed messages serialised by time, tally per
 * hostname / process / thread; Sec. 3.6: timeline of host API calls;
 * Sec. 4.3: the worked tally, whose HIP rows include the time of the
 * Level-Zero calls they make).  All arithmetic is on integer nanoseconds; the
 * results are exact.
 *
 * Trace layout ("THPT", little-endian; the paper fixes no layout beyond naming
 * CTF, Sec. 3.1):
 *   header (128 B): u32 magic "THPT", u16 version 1, u16 header_bytes 128,
 *     u32 packet_bytes, u32 n_streams, u32 n_classes, u32 n_funcs,
 *     u32 n_hosts, u32 0, u64 n_packets, u64 stream_table_off,
 *     u64 class_table_off, u64 func_table_off, u64 host_table_off,
 *     u64 strings_off, u64 strings_bytes, u64 packets_off, 32 B reserved;
 *   stream rows {u32 host_id, pid, tid, flags}; class rows {u16 func_id,
 *     u8 kind (0 ENTRY, 1 EXIT, 2 DEV_BEGIN, 3 DEV_END, 4 SAMPLE), u8 0,
 *     u16 fixed_bytes, i16 result_off, i16 cmd_off, 6 B 0}; function rows
 *     {u32 name_off, u16 layer, u16 0}; host rows {u32 name_off, u32 0};
 *     NUL-terminated strings;
 *   n_packets packets of packet_bytes (power of two, 256..65536) from
 *     packets_off (multiple of 256): 32-byte header {u32 magic "PKT1",
 *     u32 stream_id, u64 ts_begin, u32 content_bytes, u32 n_events, u32 seq,
 *     u32 discarded} then 4-byte-aligned events {u32 tsw (bits 26:0 delta ns
 *     from the previous event or ts_begin, bit 27 EXT = a u64 absolute ts
 *     follows and the delta bits are 0, bits 31:28 zero), u16 class_id,
 *     u16 var_len, [u64 ts], fixed part, payload, pad to 4}.
 * Validation order (first failure wins): file header and tables; every packet
 * header in file order; every packet's events in file order.  See
 * thapi_last_error_location.
 *
 * Per-CPU buffers: a stream whose flags have bit 1 set is a per-CPU buffer
 * (one ring buffer per CPU, Sec. 3.1): each of its events has a 16-byte header
 * {u32 tsw, u16 class_id, u16 var_len, u32 vpid, u32 vtid} (then [u64 ts],
 * fixed part, payload).  Its events belong to the thread (host of the
 * buffer, vpid, vtid); a thread's events from all per-CPU buffers are paired
 * like one stream's, in (ts, stream id, position) order; tally rows are keyed
 * by (host, vpid, vtid, function) and combine with per-thread rows of the same
 * key; an interval belongs to its entry's stream.  Per-CPU buffers take no
 * part in device-activity pairing; a trace with them needs packets of at most
 * 32 KB and fewer than 2^32 events (E_UNSUPPORTED otherwise).
 *
 * Semantics: any other stream is one thread.  Per stream, events are paired with a
 * call stack: an EXIT pops the latest open ENTRY; equal functions make an
 * interval [entry ts, exit ts] (level = depth of the entry, 0 outermost,
 * saturated at 255; error flag = the exit's i32 result is nonzero).  An EXIT
 * on an empty stack is an unmatched exit, a pop of another function a
 * mismatched pair, entries still open at the end unmatched entries; all three
 * are counted in thapi_diag and excluded from tally and timeline (events can
 * be dropped by the tracer, Sec. 3.1).  DEV_BEGIN / DEV_END / SAMPLE events are
 * decoded and counted as other events.
 *
 * Device activity (GPU timings of the commands a host call submits, Sec. 3.3;
 * device rows of the timeline, Sec. 3.6): a class with a command offset
 * carries a u64 command id.  Per command id c, with B, E, H the numbers of
 * its DEV_BEGIN, DEV_END and host ENTRY events, c is a device pair when
 * B = E = 1 and end ts >= begin ts.  A device pair with H = 1 is a device
 * interval [begin ts, end ts] on the begin's stream, labelled with the host
 * call's function, level 0, flags THAPI_IV_DEVICE; it joins the timeline at
 * the begin's position in its stream and is tallied apart from the host calls
 * (thapi_device_tally), per (host, pid, tid of its stream, function).  Pairs
 * with H = 0 (unjoined) or H > 1 (ambiguous), and device events outside a
 * pair, are counted in thapi_device_diag.
 *
 * Threading: a context may be used from one host thread at a time, except
 * through a serving loop (thapi_server_*), which drives it from its own
 * worker threads.
 * Errors: every call returns a THAPI_* status; nothing falls back to the CPU.
 */
#ifndef THAPI_H
#define THAPI_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define THAPI_OK 0
#define THAPI_E_INVALID 1     /* bad argument (null pointer, unknown id, misaligned device pointer) */
#define THAPI_E_FORMAT 2      /* the trace breaks a layout rule */
#define THAPI_E_TRUNCATED 3   /* the trace ends inside a table, packet or event */
#define THAPI_E_NOMEM 4       /* device allocation failed, or admission over the context's HBM cap */
#define THAPI_E_TIMEOUT 5     /* a bounded device-side wait gave up */
#define THAPI_E_CUDA 6        /* a CUDA runtime call failed */
#define THAPI_E_RANGE 7       /* output capacity too small; the needed count is returned */
#define THAPI_E_UNSUPPORTED 8 /* valid trace outside this build's limits (see thapi_trace_load) */
/* 9: THAPI_PENDING, a serving-loop request not completed yet (thapi_server_poll) */

typedef struct thapi_ctx thapi_ctx;
typedef uint64_t thapi_trace_id;

/* One tally row (56 B).  Rows are ordered by (host_id, pid, tid, func_id).
 * total_ns / min_ns / max_ns are inclusive call durations (exit ts - entry ts,
 * u64); err_count counts calls whose exit result was nonzero. */
typedef struct thapi_tally_row {
  uint32_t host_id, pid, tid, func_id;
  uint64_t count, total_ns, min_ns, max_ns, err_count;
} thapi_tally_row;

/* One timeline interval (24 B).  Timeline order is (start_ns, stream_id,
 * position of the entry, or of the DEV_BEGIN, in its stream). */
#define THAPI_IV_ERR 1u    /* the call's exit result was nonzero */
#define THAPI_IV_DEVICE 4u /* a device interval (device-activity pairing) */
typedef struct thapi_interval {
  uint64_t start_ns, end_ns;
  uint32_t stream_id;
  uint16_t func_id;
  uint8_t level;
  uint8_t flags;
} thapi_interval;

/* One decoded event (40 B), as thapi_decode returns it. */
typedef struct thapi_event {
  uint64_t ts;        /* rebuilt timestamp (ns) */
  uint64_t cmd;       /* command id (0 if the class has none) */
  uint32_t stream_id;
  uint16_t class_id;
  uint16_t var_len;   /* payload bytes */
  int32_t result;     /* i32 at the class's result offset (0 if none) */
  uint8_t ext;        /* 1: the event carried an absolute timestamp */
  uint8_t kind;       /* class kind (0 ENTRY, 1 EXIT, 2 DEV_BEGIN, 3 DEV_END, 4 SAMPLE) */
  uint16_t func_id;
  uint32_t vpid, vtid; /* the event's thread: its context in a per-CPU buffer, else its stream's pid / tid */
} thapi_event;

/* Diagnostics of one trace (64 B).
 * events = 2*(pairs + mismatched_pairs) + unmatched_entries + unmatched_exits + other_events. */
typedef struct thapi_diag {
  uint64_t events;            /* events decoded */
  uint64_t pairs;             /* matched calls = intervals = sum of tally counts */
  uint64_t unmatched_entries; /* entries still open at the end of their stream */
  uint64_t unmatched_exits;   /* exits met with an empty stack */
  uint64_t mismatched_pairs;  /* pops whose entry had another function */
  uint64_t other_events;      /* DEV_BEGIN, DEV_END and SAMPLE events */
  uint64_t discarded;         /* sum of the packets' discarded counters */
  uint64_t packets;
} thapi_diag;

/* Device-activity diagnostics of one trace (64 B).
 * dev_events = 2*dev_pairs + dev_unpaired;
 * dev_pairs = dev_intervals + dev_unjoined + dev_ambiguous. */
typedef struct thapi_device_diag {
  uint64_t dev_events;        /* DEV_BEGIN and DEV_END events */
  uint64_t dev_pairs;         /* command ids with one begin and one end, end >= begin */
  uint64_t dev_intervals;     /* device pairs joined to exactly one host ENTRY */
  uint64_t dev_unpaired;      /* device events outside a device pair */
  uint64_t dev_unjoined;      /* device pairs with no host ENTRY */
  uint64_t dev_ambiguous;     /* device pairs with several host ENTRY events */
  uint64_t host_cmd_entries;  /* host ENTRY events carrying a command id */
  uint64_t host_unjoined;     /* of those, entries whose command id is no device pair */
} thapi_device_diag;

/* Facts about a loaded trace.  intervals counts host and device intervals. */
typedef struct thapi_trace_info {
  uint64_t nbytes, n_packets, events, intervals, tally_rows, device_bytes;
  uint32_t n_streams, n_classes, n_funcs, n_hosts, packet_bytes;
  uint32_t self_time;         /* 1: loaded with self time on (thapi_self_tally) */
  uint64_t t_min, t_max;      /* smallest / largest event timestamp */
  uint64_t device_rows, device_intervals;  /* device tally rows; device intervals */
} thapi_trace_info;

/* Optional device allocator.  alloc returns device memory of at least `bytes`
 * (aligned to 256 B) usable in stream order on `stream`, or NULL; free
 * releases it in stream order.  Without hooks the library uses
 * cudaMallocAsync / cudaFreeAsync on the call's stream. */
typedef void *(*thapi_alloc_fn)(uint64_t bytes, void *stream, void *user);
typedef void (*thapi_free_fn)(void *ptr, uint64_t bytes, void *stream, void *user);

/* Creates a context on CUDA device `device`: the holder of the decoded traces
 * that stay resident for queries (the paper's analysis runs next to the
 * traced job on its node, Sec. 3.7; it has no API for this, so the context
 * is this library's own).  hbm_cap_bytes caps the device memory held by
 * resident traces (results plus load temporaries); 0 = no cap.  *out receives
 * the context.  Errors: E_INVALID (null out), E_CUDA. */
int thapi_ctx_create(thapi_ctx **out, int device, uint64_t hbm_cap_bytes);

/* Installs allocator hooks (both or neither; NULLs restore the default).
 * Must be called before the first load.  Plumbing with no counterpart in the
 * paper.  Errors: E_INVALID (one hook without the other, or traces loaded). */
int thapi_ctx_set_allocator(thapi_ctx *ctx, thapi_alloc_fn alloc, thapi_free_fn free_fn, void *user);

/* Frees every trace of the context and the context (no paper counterpart).
 * Errors: E_INVALID (null ctx). */
int thapi_ctx_destroy(thapi_ctx *ctx);

/* Loads a trace from HOST memory: copies `bytes` (caller-owned, may be freed on
 * return) to the device on `cuda_stream` (a cudaStream_t, NULL = legacy
 * default stream), validates it, decodes every packet (Sec. 3.1: the tracer's
 * binary trace, with a full timestamp where a delta would not fit), pairs
 * entry/exit events (Sec. 3.2: every call leaves an entry and an exit event,
 * the exit with its result; Sec. 3.3: intervals from the two), builds the
 * tally (Sec. 3.4: per hostname / process / thread and function) and the
 * sorted timeline (Sec. 3.6), and keeps those results resident on the
 * device.  The raw bytes are released before returning.  Blocks until
 * done.  *out receives the trace id.
 * Errors: E_INVALID, E_FORMAT / E_TRUNCATED (see thapi_last_error_location),
 * E_NOMEM (allocation failed or the HBM cap would be exceeded), E_UNSUPPORTED
 * (streams x functions above 2^28 tally cells), E_TIMEOUT, E_CUDA. */
int thapi_trace_load(thapi_ctx *ctx, const void *bytes, uint64_t nbytes, void *cuda_stream, thapi_trace_id *out);

/* As thapi_trace_load (Sec. 3.2-3.6), for a trace already in DEVICE memory
 * (16-byte aligned, caller-owned, read during the call only; not copied).
 * Errors as thapi_trace_load; E_INVALID also for a misaligned pointer. */
int thapi_trace_load_device(thapi_ctx *ctx, const void *dev_bytes, uint64_t nbytes, void *cuda_stream,
                            thapi_trace_id *out);

/* Decodes every event of a trace in HOST memory (caller-owned, copied to the
 * device during the call) and writes one thapi_event per event to HOST
 * memory `out` (capacity `cap`), in stream order (streams by id, packets by
 * seq, events in packet order); *n_out = the trace's event count.  This is
 * the content of the paper's pretty-printed event lines (Sec. 3.2: timestamp,
 * host, vpid, vtid, event name and fields).  The
 * records are the decode step of the analysis (event boundaries, timestamps
 * rebuilt from deltas and absolute values, class, result, command id) made
 * visible, for tools and text output.  cap = 0 is a size query (checks the
 * headers only); 0 < cap < events gives E_RANGE.  Validation as
 * thapi_trace_load (locations through thapi_last_error_location); nothing is
 * kept on the device.  Packets up to 32 KB.
 * Errors: E_INVALID, E_FORMAT / E_TRUNCATED, E_RANGE, E_NOMEM, E_UNSUPPORTED,
 * E_CUDA. */
int thapi_decode(thapi_ctx *ctx, const void *bytes, uint64_t nbytes, thapi_event *out, uint64_t cap, uint64_t *n_out,
                 void *cuda_stream);

/* Loads n traces as one trace (a batch: the per-rank traces of one run, say,
 * analysed together, as the paper's tools read all ranks' traces at once,
 * Sec. 3.4).  bytes[i] / nbytes[i]: trace i in HOST memory, or in device
 * memory with on_device = 1 (16-byte aligned; read during the call only).
 * The result is the trace whose streams are trace 0's, then trace 1's, ...
 * (trace i's stream s becomes stream S_0 + ... + S_{i-1} + s) and whose hosts
 * likewise follow one another (host ids offset the same way, host names from
 * each trace's own string table); function and class ids are the traces'
 * own, which must agree: every trace needs the same packet size, the same
 * class table and the same function names and layers (E_UNSUPPORTED
 * otherwise).  All packets of the batch are indexed, decoded, paired and
 * tallied in one pass (one launch of each kernel over the batch's packet
 * list); tally rows, timeline, device activity and self time are those of
 * the combined trace, so trace i's rows are those whose host_id falls in its
 * range and its intervals those whose stream_id does.  Errors: a trace that
 * fails its file checks gives its code with thapi_last_error_location level
 * 0 and packet = its index in the batch; packet and content errors give the
 * packet's index in the batch (the traces' packets in order). */
int thapi_trace_load_batch(thapi_ctx *ctx, const void *const *bytes, const uint64_t *nbytes, uint32_t n,
                           int on_device, void *cuda_stream, thapi_trace_id *out);

/* Releases a loaded trace's device results (no paper counterpart).
 * Errors: E_INVALID (unknown id). */
int thapi_trace_free(thapi_ctx *ctx, thapi_trace_id id);

/* Copies the tally rows to HOST memory `rows` (capacity `cap` rows) and the
 * diagnostics to `diag` (may be NULL).  The tally is the paper's summary
 * view: per (hostname, process, thread) and API function, the call count and
 * total / min / max inclusive time (Sec. 3.4; the worked HIP-over-Level-Zero
 * table of Sec. 4.3), plus the count of calls whose exit result was nonzero
 * (Sec. 3.2: exits carry the result).  *n_rows = number of rows.  cap = 0 is
 * a size query (returns OK); 0 < cap < rows returns E_RANGE with *n_rows set.
 * Errors: E_INVALID (unknown id, null n_rows), E_RANGE, E_CUDA. */
int thapi_tally(thapi_ctx *ctx, thapi_trace_id id, thapi_tally_row *rows, uint64_t cap, uint64_t *n_rows,
                thapi_diag *diag);

/* Copies the device tally rows (device intervals per (host_id, pid, tid of
 * the device stream, function of the submitting host call), ordered by those
 * keys; err_count is 0) to HOST memory `rows` and the device diagnostics to
 * `diag` (may be NULL): the device-side timings the paper's GPU profiling
 * records for the commands a call submits (Sec. 3.3, Sec. 3.5).  cap
 * semantics and errors as thapi_tally. */
int thapi_device_tally(thapi_ctx *ctx, thapi_trace_id id, thapi_tally_row *rows, uint64_t cap, uint64_t *n_rows,
                       thapi_device_diag *diag);

/* Merges tally rows of several traces or ranks (the paper's local -> global
 * aggregation, Sec. 3.4).  `rows`: n rows in HOST memory, in any order (for
 * example the concatenated results of thapi_tally of several traces, or of
 * several ranks; the 56-byte little-endian row is also the exchange format).
 * Rows with equal (host_id, pid, tid, func_id) combine exactly: count,
 * total_ns and err_count add (total_ns in u64), min_ns / max_ns take the
 * minimum / maximum.  The merged rows go to HOST memory `out` (capacity
 * `cap`), ordered by that key; *n_out = their number (at most n).  cap = 0 is
 * a size query (the merge still runs); 0 < cap < *n_out gives E_RANGE.  Runs
 * on the context's device on `cuda_stream`; blocks until done.
 * Errors: E_INVALID, E_UNSUPPORTED (n >= 2^32), E_NOMEM, E_RANGE, E_CUDA. */
int thapi_tally_merge(thapi_ctx *ctx, const thapi_tally_row *rows, uint64_t n, thapi_tally_row *out, uint64_t cap,
                      uint64_t *n_out, void *cuda_stream);

/* Copies the timeline intervals with start_ns < t1 and end_ns >= t0 (t0 = 0,
 * t1 = UINT64_MAX: all), in timeline order, to HOST memory `out` (capacity
 * `cap`): the paper's timeline view of host API calls and device activity
 * (Sec. 3.6), in the time order its plugins see messages in (Sec. 3.4).
 * *n_out = number selected; cap semantics as thapi_tally.  Errors: E_INVALID,
 * E_RANGE, E_NOMEM (window scratch), E_CUDA. */
int thapi_timeline(thapi_ctx *ctx, thapi_trace_id id, uint64_t t0, uint64_t t1, thapi_interval *out,
                   uint64_t cap, uint64_t *n_out);

/* Device-output form of thapi_tally (Sec. 3.4): `rows` is a DEVICE pointer
 * written in order on `cuda_stream`; the call returns once the copy is
 * enqueued and *n_rows is known.  Errors as thapi_tally. */
int thapi_tally_device(thapi_ctx *ctx, thapi_trace_id id, thapi_tally_row *rows, uint64_t cap, uint64_t *n_rows,
                       thapi_diag *diag, void *cuda_stream);
/* Device-output form of thapi_timeline (Sec. 3.6): `out` is a DEVICE pointer
 * written in order on `cuda_stream`; the call returns once the copy is
 * enqueued and *n_out is known.  Errors as thapi_timeline. */
int thapi_timeline_device(thapi_ctx *ctx, thapi_trace_id id, uint64_t t0, uint64_t t1, thapi_interval *out,
                          uint64_t cap, uint64_t *n_out, void *cuda_stream);

/* Facts about a loaded trace (sizes, counts, time span; no paper counterpart).
 * Errors: E_INVALID (unknown id). */
int thapi_trace_info_get(thapi_ctx *ctx, thapi_trace_id id, thapi_trace_info *info);

/* Copies a NUL-terminated name of a loaded trace into buf (capacity cap):
 * kind 0 = host name of host_id `index`, kind 1 = function name of func_id
 * `index` (the names the tally and timeline show, Sec. 3.4, Sec. 4.3).
 * *len = name length without the NUL.  Errors: E_INVALID (unknown id, kind or
 * index), E_RANGE if it does not fit. */
int thapi_trace_strings(thapi_ctx *ctx, thapi_trace_id id, int kind, uint32_t index, char *buf, uint64_t cap,
                        uint64_t *len);

/* The layer of function func_id (the function row's u16 layer: which API of
 * a layered stack, e.g. HIP over Level Zero, Sec. 4.3) to *layer. */
int thapi_trace_func_layer(thapi_ctx *ctx, thapi_trace_id id, uint32_t func_id, uint32_t *layer);

/* Where the last failed load of this context failed (no paper counterpart;
 * the layout checks are this library's): level 0 = file header or
 * tables, 1 = packet header (packet = file index), 2 = packet content
 * (packet = file index, event = index of the event within the packet, or the
 * event count for a count mismatch). */
int thapi_last_error_location(thapi_ctx *ctx, int *level, uint64_t *packet, uint64_t *event);

/* Per-phase device time of a load, measured with CUDA events on the load
 * stream when timing is enabled on the context (thapi_ctx_set_timing). */
typedef struct thapi_load_timing {
  float index_ms;     /* packet headers, group by stream, seq check, event offsets */
  float analyze_ms;   /* decode + in-packet pairing + tally kernel(s) */
  float frontier_ms;  /* depth carry and pairing across packets */
  float tally_ms;     /* tally rows and interval offsets */
  float compact_ms;   /* timeline slot compaction */
  float sort_ms;      /* timeline radix sort */
  float gather_ms;    /* timeline gather */
  float total_ms;     /* first to last event of the load (includes host waits) */
  uint64_t analyze_read_bytes;   /* sum over packets of 32 + content_bytes (what the analysis must read) */
  uint64_t analyze_write_bytes;  /* written by the analysis: interval slots (24 B each) and
                                    device-activity records (32 B per DEV_BEGIN, 16 B per DEV_END
                                    and per host ENTRY carrying a command id) */
  uint64_t analyze_launches;     /* analysis kernel launches of the load */
  uint64_t launches;             /* all kernel launches of the load */
  float join_ms;                 /* device-activity pairing (includes one host wait) */
  float self_ms;                 /* self time (when on; includes host waits) */
  float percpu_ms;               /* per-CPU buffers: event records, thread order, pairing (includes host waits) */
  float percpu_decode_ms;        /* per-CPU buffers: the record-writing decode kernel alone */
  uint64_t percpu_read_bytes;    /* sum over per-CPU packets of 32 + content_bytes (excluded from
                                    analyze_read_bytes) */
  uint64_t percpu_write_bytes;   /* written by that decode: 32 B per per-CPU event (its record or a
                                    marked hole) and a 24 B interval slot per ENTRY */
  uint32_t grid_mult;            /* configuration used: analysis packet runs per resident CTA */
  int32_t part_shift;            /* configuration used: device-join partition size 1536 << shift records */
  float parse_ms;                /* host: the call's start to the first kernel (file heads and tables read,
                                    checked and combined) */
  float call_ms;                 /* host: wall time of the load call up to its results (scratch release
                                    not included) */
} thapi_load_timing;

/* Copies the per-phase timing of a loaded trace to *out (zeros if timing was
 * off when it was loaded; measurement only, no paper counterpart).
 * Errors: E_INVALID (unknown id, null out). */
int thapi_trace_timing(thapi_ctx *ctx, thapi_trace_id id, thapi_load_timing *out);

/* The failure path of the library's bounded device waits, on purpose (no
 * paper counterpart; failure detection of this library): one
 * warp waits on an mbarrier that nothing completes for at most `limit` tries,
 * gives up, and reports through a status word.  Returns THAPI_E_TIMEOUT (what
 * a load returns when a packet copy never lands), E_INVALID for limit 0;
 * nothing faults and the context stays usable. */
int thapi_check_device_wait(thapi_ctx *ctx, uint32_t limit, void *cuda_stream);

/* Enables (1) or disables (0) the autotuner for subsequent loads (no paper
 * counterpart: the launch configuration is this library's).  Its
 * knobs: the analysis kernel's packet runs per resident CTA (1, 2, 4) and the
 * device join's partition size (records aimed at per partition: 768, 1536,
 * 3072).  The first load of a shape (packet size, device pairing on, batch or
 * not, log2 of the packet count) loads the trace once per candidate — the
 * results are identical — keeps the fastest (device time of the analysis and
 * the device join) and remembers its configuration for later loads of that shape in this
 * context.  Without it a load uses 2 runs per CTA and 1536-record partitions.
 * thapi_trace_timing reports the configuration a load used. */
int thapi_ctx_set_autotune(thapi_ctx *ctx, int enable);

/* Enables (1) or disables (0) per-phase timing of subsequent loads
 * (measurement only, no paper counterpart).  Errors: E_INVALID. */
int thapi_ctx_set_timing(thapi_ctx *ctx, int enable);

/* Enables (1) or disables (0) self time for subsequent loads (off by default).
 *
 * Self (exclusive) time separates what a call spends itself from what the
 * calls it makes take: the layering analysis of the paper (Sec. 4.3), where
 * hipDeviceSynchronize is built on the zeEventHostSynchronize spin.  A call's
 * self time is its duration less the durations of the calls paired directly
 * inside it (the entries pushed right above its entry on its stack and closed
 * with the same function), in u64 arithmetic.  A mismatched or unmatched call
 * has no duration: it takes nothing off its parent, and the calls directly
 * inside it take nothing off any call.  Per-CPU buffers follow their threads'
 * stacks.  Device intervals take no part.  A load with self time on keeps, per
 * event, a 24-byte side record during the load and per interval about 72 bytes
 * more; traces of 2^31 events or more return E_UNSUPPORTED. */
int thapi_ctx_set_self_time(thapi_ctx *ctx, int enable);

/* Copies the self-time rows of a trace loaded with self time on to HOST
 * memory `rows` (the layering analysis of Sec. 4.3: what a call spends
 * itself, apart from the calls it makes): the tally's keys, order, counts and error counts, with
 * total_ns / min_ns / max_ns over the calls' self times.  cap semantics as
 * thapi_tally; E_INVALID if the trace was loaded with self time off. */
int thapi_self_tally(thapi_ctx *ctx, thapi_trace_id id, thapi_tally_row *rows, uint64_t cap, uint64_t *n_rows);

/* Kernels this library has launched in this process (all contexts); a
 * measurement counter with no paper counterpart. */
uint64_t thapi_kernel_launches(void);

/* Tally of a small trace with no device allocation at all (the paper has no
 * counterpart; this is a deployment aid).  For callers that cannot allocate
 * device memory: a tracing agent that tallies on the node while the traced
 * application runs in the same CUDA context, where the application or its
 * framework's caching allocator holds nearly all device memory and an
 * allocation by the agent could fail or disturb the application it observes.
 * `dev_bytes` is the whole trace in DEVICE memory (16-byte aligned, caller-
 * owned); rows are written to DEVICE memory `rows` (capacity `cap`; cap = 0 is
 * a size query, 0 < cap < rows gives E_RANGE) on `cuda_stream`; *n_rows and
 * *diag (may be NULL) are host outputs.  Results equal thapi_trace_load_device
 * followed by thapi_tally.  Working memory is one 32 MiB array in device
 * global memory that belongs to the library (every GPU that loads the library
 * holds it until the process exits).  Limits: at most 4096 packets, 2^20
 * events, 2^16 (host, pid, tid) groups x functions, no per-CPU buffers, and a
 * cross-packet pairing frontier that fits what the array has left; beyond them the call returns
 * E_UNSUPPORTED.  The first call on a device looks up the array's device
 * address, so make that first call before any stream capture.  Calls share
 * the array: host calls are serialised, each returns after its GPU work is
 * done, and work of two calls overlapping on the GPU would race.  Errors:
 * E_INVALID, E_FORMAT / E_TRUNCATED (no location is recorded), E_UNSUPPORTED,
 * E_TIMEOUT, E_RANGE, E_CUDA. */
int thapi_tally_static(const void *dev_bytes, uint64_t nbytes, thapi_tally_row *rows, uint64_t cap,
                       uint64_t *n_rows, thapi_diag *diag, void *cuda_stream);

/* ------------------------------------------------------------------ serving
 * A serving loop over the traces a context keeps resident, with continuous
 * batching.  The paper's analysis runs on the traced job's node and keeps up
 * with it (Sec. 3.7, on-node processing), answering with the tally and
 * timeline views (Sec. 3.4, Sec. 3.6); served, that is a stream of requests:
 * a trace arrives (LOAD: decoded, paired, tallied and ordered as by
 * thapi_trace_load), its tally is asked for (TALLY), the intervals of a time
 * range of its timeline (WINDOW, as thapi_timeline), and it leaves (FREE).
 *
 * Requests that arrive while others are on the GPU do not queue behind them:
 * each starts as soon as a slot of its class is free (load slots and query
 * slots, each a host thread with its own CUDA stream; query streams have the
 * highest priority, load streams the lowest) and, for a load, as soon as the
 * context's HBM cap (thapi_ctx_create) has room for the load's coarse peak
 * next to what is resident and what running loads were charged (admission by
 * HBM footprint; loads are admitted in arrival order; queries and frees pass
 * waiting loads).  A load whose charge exceeds the whole cap is refused
 * (E_NOMEM).  The work of different requests overlaps on the device; every
 * result equals that of the plain entry points.  Per trace, a FREE waits for
 * the queries submitted before it, and queries submitted after it fail with
 * E_INVALID.  While a server runs, its context may be used by other host
 * threads only through thread-safe calls (tally, timeline, info, loads
 * without autotuning). */
#define THAPI_PENDING 9 /* thapi_server_poll: the request has not completed within the wait */

#define THAPI_REQ_LOAD 0u   /* a trace arrives: load it (bytes, nbytes, on_device) */
#define THAPI_REQ_TALLY 1u  /* the tally rows of a trace */
#define THAPI_REQ_WINDOW 2u /* the timeline intervals of a trace with start < t1 and end >= t0 */
#define THAPI_REQ_FREE 3u   /* the trace leaves: its results are released */

typedef struct thapi_server thapi_server;

/* One request (72 B). */
typedef struct thapi_request {
  uint32_t kind;         /* THAPI_REQ_* */
  uint32_t on_device;    /* LOAD: `bytes` is DEVICE memory (16-byte aligned), else HOST memory */
  const void *bytes;     /* LOAD: the trace, caller-owned and unchanged until the request completes */
  uint64_t nbytes;       /* LOAD */
  thapi_trace_id trace;  /* TALLY / WINDOW / FREE: a resident trace (when after = 0) */
  uint64_t after;        /* TALLY / WINDOW / FREE: the ticket of the LOAD that brings the trace in (0: none);
                            the request starts once that load has completed, and fails with its status */
  uint64_t t0, t1;       /* WINDOW: the window [t0, t1) */
  void *out;             /* TALLY / WINDOW: result memory (HOST or DEVICE; pinned host memory is written by
                            the device directly), or NULL: pinned memory the server owns */
  uint64_t cap;          /* capacity of `out` in rows / intervals (E_RANGE with n set when too small) */
} thapi_request;

/* What a request did (64 B).  Times are seconds on the server's clock
 * (thapi_server_now). */
typedef struct thapi_result {
  int32_t status;        /* THAPI_OK or the request's error */
  uint32_t kind;
  thapi_trace_id trace;  /* the trace (LOAD: the new id) */
  uint64_t n;            /* rows / intervals of the result (the count needed on E_RANGE) */
  uint64_t events;       /* events of the trace */
  const void *data;      /* the result: `out`, or server-owned pinned memory valid until thapi_server_release */
  double t_arrival;      /* submission (or, through thapi_server_replay, the scheduled arrival) */
  double t_admit;        /* the request started on its slot */
  double t_done;         /* the result is in place */
} thapi_result;

typedef struct thapi_server_stats {
  uint64_t submitted, completed;
  uint64_t load_waits;      /* loads whose admission waited for device memory */
  uint64_t peak_running;    /* most requests in flight at once */
  uint64_t peak_committed;  /* most device memory resident plus charged to running loads (bytes) */
  uint64_t result_allocs;   /* server-owned results that found no room in the pinned result memory */
} thapi_server_stats;

/* Starts a serving loop on `ctx` with load_slots loads and query_slots
 * queries / frees in flight at most (1..63 together).  The context's cap is
 * the admission cap.  result_bytes (0: 1 GiB) of pinned, device-mapped host
 * memory are set aside once for results the server owns (requests with
 * out = NULL), so that serving pins and unpins nothing; a result that finds
 * no room there gets its own pinned allocation.  Errors: E_INVALID, E_NOMEM,
 * E_CUDA. */
int thapi_server_create(thapi_ctx *ctx, uint32_t load_slots, uint32_t query_slots, uint64_t result_bytes,
                        thapi_server **out);

/* Submits a request; *ticket names it.  The request's own failures (refused
 * load, unknown or departed trace, failed load it waits for, format errors)
 * come back through its result.  Errors: E_INVALID (malformed request, or
 * `after` naming no earlier LOAD), E_NOMEM. */
int thapi_server_submit(thapi_server *s, const thapi_request *req, uint64_t *ticket);

/* Waits up to wait_ms (UINT32_MAX: without limit) for the request to complete
 * and copies its result to *res.  Returns THAPI_PENDING if it has not
 * completed; E_INVALID for an unknown or released ticket. */
int thapi_server_poll(thapi_server *s, uint64_t ticket, uint32_t wait_ms, thapi_result *res);

/* Forgets a completed request and returns its server-owned result memory.
 * Errors: E_INVALID (unknown, released or not completed). */
int thapi_server_release(thapi_server *s, uint64_t ticket);

/* Seconds since the server was created (steady clock). */
double thapi_server_now(thapi_server *s);

/* Replays a schedule: request i is submitted at arrival_s[i] seconds after
 * the call starts (nondecreasing), its `after`, if nonzero, being 1 + the
 * index of an earlier LOAD of the schedule; then every request is waited for
 * and its result copied to results[i] (t_arrival = the scheduled time, so
 * latencies include any delay of the submission).  keep = 0 returns each
 * result's server-owned memory as soon as the request completes
 * (results[i].data is then NULL); keep = 1 keeps it, valid until
 * thapi_server_destroy.  Errors: E_INVALID (a malformed schedule; nothing is
 * submitted). */
int thapi_server_replay(thapi_server *s, const thapi_request *reqs, const double *arrival_s, uint64_t n, int keep,
                        thapi_result *results);

/* Counters of the serving loop so far.  Errors: E_INVALID. */
int thapi_server_stats_get(thapi_server *s, thapi_server_stats *st);

/* Waits for every submitted request, stops the loop and frees it; loads
 * that could never be admitted (nothing running, nothing left to free) end
 * with E_NOMEM.  The traces it loaded stay resident in the context.
 * Errors: E_INVALID. */
int thapi_server_destroy(thapi_server *s);

/* Static description of a status code (no paper counterpart). */
const char *thapi_strerror(int code);

#ifdef __cplusplus
}
#endif

#endif /* THAPI_H */

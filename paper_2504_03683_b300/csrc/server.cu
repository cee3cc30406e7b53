// server.cu — the serving loop: requests arrive over time and are served with
// continuous batching over the traces a context keeps resident.
//
// The paper's analysis runs beside the traced job on its node and keeps up
// with it (Sec. 3.7, on-node processing; Sec. 3.4, the tally and timeline
// views).  Served here, that means: a trace arrives (LOAD) and is decoded
// into resident tally rows and timeline; queries ask for a trace's tally
// (TALLY) or for the intervals of a time range of its timeline (WINDOW); a
// trace leaves (FREE).  Requests that arrive while others are on the GPU do
// not wait for them: a request starts as soon as a slot of its class is free
// and, for a load, as soon as the context's device-memory cap has room for
// the load's coarse peak (admission by HBM footprint; loads are admitted in
// arrival order, queries and frees pass waiting loads).  Every slot is a host
// thread with its own CUDA stream (query slots at the highest stream
// priority, load slots at the lowest), so the kernels and copies of
// different requests overlap on the device.
//
// Order per trace: a query names a resident trace, or the ticket of the load
// that brings it in (it starts once that load completes); a FREE waits for
// the queries of its trace submitted before it, and queries submitted after
// it are refused.  Results go to the caller's memory (host or device), or,
// without one, to pinned host memory the server owns until the ticket is
// released.  Every result equals that of the plain entry points
// (thapi_trace_load, thapi_tally, thapi_timeline): the same kernels run, only
// on other streams and at other times.
#include <algorithm>
#include <chrono>
#include <iterator>
#include <condition_variable>
#include <deque>
#include <map>
#include <mutex>
#include <new>
#include <set>
#include <thread>
#include <vector>

#include "internal.cuh"

// the ABI's struct layouts (include/thapi.h), as the binding reads them
static_assert(sizeof(thapi_request) == 72, "request");
static_assert(sizeof(thapi_result) == 64, "result");
static_assert(sizeof(thapi_server_stats) == 48, "server stats");

namespace {

using Clock = std::chrono::steady_clock;
constexpr uint64_t kIdKey = 1ull << 63;      // trace key of a trace the server did not load: id | kIdKey
constexpr uint64_t kArenaAlign = 256;
// results above this many intervals go through the slot's device staging buffer
// (smaller ones are written through the pinned memory's mapping)
constexpr uint64_t kStageMinIntervals = (1ull << 20) / sizeof(thapi_interval);

// Pinned, device-mapped host memory for results the server owns: one block
// pinned when the server starts (pinning pages is slow, and freeing pinned
// memory waits for the whole device), handed out first-fit and coalesced on
// return.  A result that finds no room gets its own pinned allocation (the
// slow path, released with cudaFreeHost).
struct HostArena {
  std::mutex mu;
  uint8_t *base = nullptr;
  uint64_t size = 0;
  std::map<uint64_t, uint64_t> idle;  // offset -> bytes, disjoint and coalesced
  uint64_t own_allocs = 0;            // results that took the slow path
  bool init(uint64_t bytes) {
    bytes = (bytes + kArenaAlign - 1) / kArenaAlign * kArenaAlign;
    void *p = nullptr;
    if (cudaHostAlloc(&p, bytes, cudaHostAllocMapped | cudaHostAllocPortable) != cudaSuccess) {
      cudaGetLastError();
      return false;
    }
    base = static_cast<uint8_t *>(p);
    size = bytes;
    idle[0] = bytes;
    return true;
  }
  // *own: the memory is a separate allocation (not from the block)
  void *get(uint64_t bytes, bool *own) {
    bytes = std::max<uint64_t>(kArenaAlign, (bytes + kArenaAlign - 1) / kArenaAlign * kArenaAlign);
    {
      std::lock_guard<std::mutex> g(mu);
      for (auto it = idle.begin(); it != idle.end(); ++it) {
        if (it->second < bytes) continue;
        const uint64_t off = it->first, left = it->second - bytes;
        idle.erase(it);
        if (left) idle[off + bytes] = left;
        *own = false;
        return base + off;
      }
      own_allocs += 1;
    }
    void *p = nullptr;
    if (cudaHostAlloc(&p, bytes, cudaHostAllocMapped | cudaHostAllocPortable) != cudaSuccess) {
      cudaGetLastError();
      return nullptr;
    }
    *own = true;
    return p;
  }
  void put(void *p, uint64_t bytes, bool own) {
    if (!p) return;
    if (own) {
      cudaFreeHost(p);
      return;
    }
    bytes = std::max<uint64_t>(kArenaAlign, (bytes + kArenaAlign - 1) / kArenaAlign * kArenaAlign);
    std::lock_guard<std::mutex> g(mu);
    uint64_t off = static_cast<uint8_t *>(p) - base;
    auto nx = idle.lower_bound(off);
    if (nx != idle.end() && off + bytes == nx->first) {  // merge with the next free range
      bytes += nx->second;
      nx = idle.erase(nx);
    }
    if (nx != idle.begin()) {  // and with the previous one
      auto pv = std::prev(nx);
      if (pv->first + pv->second == off) {
        pv->second += bytes;
        return;
      }
    }
    idle[off] = bytes;
  }
  ~HostArena() {
    if (base) cudaFreeHost(base);
  }
};

struct Req {
  uint64_t ticket = 0;
  thapi_request r{};
  uint64_t charge = 0;       // LOAD: what admission charges against the cap
  uint64_t key = 0;          // the trace's key (its load ticket, or id | kIdKey)
  bool counted = false;      // TALLY / WINDOW counted in pending[key]
  bool auto_release = false; // drop a server-owned result at completion (replay without keep)
  bool waited = false;       // LOAD: admission waited for memory at least once
  int state = 0;             // 0 waiting, 1 running, 2 done
  thapi_trace_id trace = 0;  // resolved trace
  thapi_result res{};
  void *buf = nullptr;       // server-owned result
  uint64_t buf_bytes = 0;
  bool buf_own = false;      // a separate pinned allocation, not arena memory
};

struct Slot {
  bool query = false;
  cudaStream_t stream = nullptr;
  std::thread th;
  thapi::WinWork *w = nullptr;               // device
  unsigned long long *total_h = nullptr;     // pinned, device-mapped count word
  unsigned long long *total_d = nullptr;     // its device view
  thapi_interval *stage = nullptr;           // device staging for pageable destinations
  uint64_t stage_bytes = 0;
};

}  // namespace

struct thapi_server {
  thapi_ctx *ctx = nullptr;
  int device = 0;
  std::mutex mu;
  std::condition_variable cv;       // workers: a request may have become startable
  std::condition_variable cv_done;  // waiters: a request completed
  std::map<uint64_t, Req *> reqs;   // every ticket not released
  std::deque<Req *> waiting;        // submitted, not started, in ticket order
  std::map<uint64_t, std::pair<int, thapi_trace_id>> loads;  // completed loads: status, trace
  std::map<thapi_trace_id, uint64_t> id_key;                 // traces this server loaded -> load ticket
  std::map<uint64_t, uint64_t> pending;                      // trace key -> queries submitted, not completed
  std::set<uint64_t> leaving;                                // trace keys with a FREE submitted
  uint64_t next_ticket = 1, reserved = 0;
  uint32_t running = 0;
  bool stop = false;
  Clock::time_point t0;
  std::vector<Slot *> slots;
  cudaStream_t head_stream = nullptr;  // reads the file heads of device traces at submission
  std::mutex head_mu;
  HostArena arena;
  thapi_server_stats st{};
};

namespace {

double secs(const thapi_server *S, Clock::time_point t) {
  return std::chrono::duration<double>(t - S->t0).count();
}

void note_memory(thapi_server *S) {  // under S->mu
  uint64_t cap = 0, used = 0;
  thapi::ctx_memory(S->ctx, &cap, &used);
  if (used + S->reserved > S->st.peak_committed) S->st.peak_committed = used + S->reserved;
}

// Completes a request (under S->mu): records its result and the per-trace state.
void complete(thapi_server *S, Req *q, int status) {
  q->res.status = status;
  q->res.kind = q->r.kind;
  q->res.t_done = secs(S, Clock::now());
  q->state = 2;
  const uint32_t k = q->r.kind;
  if (k == THAPI_REQ_LOAD) {
    S->loads[q->ticket] = std::make_pair(status, q->trace);
    if (status == THAPI_OK) S->id_key[q->trace] = q->ticket;
  } else if (k == THAPI_REQ_FREE) {
    if (status == THAPI_OK) {
      S->id_key.erase(q->trace);
      S->pending.erase(q->key);
    }
  }
  if (q->counted) {
    auto it = S->pending.find(q->key);
    if (it != S->pending.end() && it->second && --it->second == 0) S->pending.erase(it);
    q->counted = false;
  }
  if (q->auto_release && q->buf) {
    S->arena.put(q->buf, q->buf_bytes, q->buf_own);
    q->buf = nullptr;
    q->res.data = nullptr;
  }
  S->st.completed += 1;
  S->cv.notify_all();
  S->cv_done.notify_all();
}

// The next request a slot of this class may start (under S->mu), or null.
// Requests whose load failed complete here with that load's status.
Req *pick(thapi_server *S, bool query) {
  bool load_blocked = false;
  for (auto it = S->waiting.begin(); it != S->waiting.end();) {
    Req *q = *it;
    const bool is_load = q->r.kind == THAPI_REQ_LOAD;
    if (is_load == query) {
      ++it;
      continue;
    }
    if (is_load) {
      if (load_blocked) {
        ++it;
        continue;
      }
      uint64_t cap = 0, used = 0;
      thapi::ctx_memory(S->ctx, &cap, &used);
      if (cap && used + S->reserved + q->charge > cap) {  // arrival order among loads: later ones wait too
        if (!q->waited) S->st.load_waits += 1;
        q->waited = true;
        load_blocked = true;
        ++it;
        continue;
      }
      S->reserved += q->charge;
      S->waiting.erase(it);
      return q;
    }
    if (q->r.after) {
      auto l = S->loads.find(q->r.after);
      if (l == S->loads.end()) {  // its load has not completed
        ++it;
        continue;
      }
      if (l->second.first != THAPI_OK) {
        it = S->waiting.erase(it);
        complete(S, q, l->second.first);
        continue;
      }
      q->trace = l->second.second;
    }
    if (q->r.kind == THAPI_REQ_FREE) {
      auto p = S->pending.find(q->key);
      if (p != S->pending.end() && p->second) {  // queries of the trace submitted before it come first
        ++it;
        continue;
      }
    }
    S->waiting.erase(it);
    return q;
  }
  return nullptr;
}

int grow_stage(thapi_server *S, Slot *sl, uint64_t bytes) {
  if (sl->stage_bytes >= bytes) return THAPI_OK;
  if (sl->stage) thapi::ctx_free(S->ctx, sl->stage, sl->stage_bytes, sl->stream);
  sl->stage_bytes = 0;
  sl->stage = static_cast<thapi_interval *>(thapi::ctx_alloc(S->ctx, bytes, sl->stream));
  if (!sl->stage) return THAPI_E_NOMEM;
  sl->stage_bytes = bytes;
  return THAPI_OK;
}

// Runs one window query on the slot's stream; the count lands in *n.
int window_once(thapi_server *S, Slot *sl, thapi_trace_id id, const thapi_request &r, thapi_interval *dst,
                uint64_t cap, uint64_t *n) {
  int rc = thapi::window_enqueue_id(S->ctx, id, r.t0, r.t1, dst, cap, sl->w, sl->total_d, sl->stream);
  if (rc != THAPI_OK) return rc;
  if (cudaStreamSynchronize(sl->stream) != cudaSuccess) {
    cudaGetLastError();
    return THAPI_E_CUDA;
  }
  *n = *reinterpret_cast<volatile unsigned long long *>(sl->total_h);
  return THAPI_OK;
}

// Does the work of one request on a slot (no server lock held).
int execute(thapi_server *S, Slot *sl, Req *q) {
  thapi_result &res = q->res;
  const thapi_request &r = q->r;
  if (r.kind == THAPI_REQ_LOAD) {
    const uint8_t *b = static_cast<const uint8_t *>(r.bytes);
    int rc = thapi::load_admitted(S->ctx, r.on_device ? nullptr : b, r.on_device ? b : nullptr, r.nbytes, sl->stream,
                                  &q->trace);
    if (rc == THAPI_OK) {
      uint64_t rows, ivs;
      thapi::trace_sizes(S->ctx, q->trace, &rows, &ivs, &res.events);
    }
    res.trace = q->trace;
    return rc;
  }
  res.trace = q->trace;
  if (r.kind == THAPI_REQ_FREE) return thapi::free_trace_on(S->ctx, q->trace, sl->stream);
  uint64_t rows = 0, ivs = 0;
  int rc = thapi::trace_sizes(S->ctx, q->trace, &rows, &ivs, &res.events);
  if (rc != THAPI_OK) return rc;
  if (r.kind == THAPI_REQ_TALLY) {
    void *dst = r.out;
    uint64_t cap = r.cap;
    if (!dst) {
      q->buf_bytes = rows * sizeof(thapi_tally_row);
      q->buf = S->arena.get(q->buf_bytes, &q->buf_own);
      if (!q->buf) return THAPI_E_NOMEM;
      dst = q->buf;
      cap = rows;
    }
    rc = thapi::tally_enqueue(S->ctx, q->trace, static_cast<thapi_tally_row *>(dst), cap, &res.n, sl->stream);
    if (rc == THAPI_OK && cudaStreamSynchronize(sl->stream) != cudaSuccess) rc = THAPI_E_CUDA;
    if (rc == THAPI_OK) res.data = dst;
    return rc;
  }
  // WINDOW: a device destination takes the matches in the counting pass; host
  // destinations (the caller's, or the server's pinned result memory) are
  // written once the count is known.  The whole time range is the whole
  // ordered timeline: one copy, no counting pass.
  cudaPointerAttributes pa{};
  const bool to_device = r.out && cudaPointerGetAttributes(&pa, r.out) == cudaSuccess &&
                         (pa.type == cudaMemoryTypeDevice || pa.type == cudaMemoryTypeManaged);
  cudaGetLastError();
  if (r.t0 == 0 && r.t1 == ~0ull) {
    res.n = ivs;
    void *dst = r.out;
    if (dst && res.n > r.cap) return THAPI_E_RANGE;
    if (!dst && res.n) {
      q->buf_bytes = res.n * sizeof(thapi_interval);
      q->buf = S->arena.get(q->buf_bytes, &q->buf_own);
      if (!q->buf) return THAPI_E_NOMEM;
      dst = q->buf;
    }
    rc = thapi::timeline_copy_id(S->ctx, q->trace, dst, res.n, to_device, sl->stream);
    if (rc == THAPI_OK && cudaStreamSynchronize(sl->stream) != cudaSuccess) rc = THAPI_E_CUDA;
    if (rc == THAPI_OK) res.data = dst;
    return rc;
  }
  if ((rc = window_once(S, sl, q->trace, r, to_device ? static_cast<thapi_interval *>(r.out) : nullptr,
                        to_device ? r.cap : 0, &res.n)) != THAPI_OK)
    return rc;
  if (to_device) {
    if (res.n > r.cap) return THAPI_E_RANGE;
    res.data = r.out;
    return THAPI_OK;
  }
  void *dst = r.out;
  if (dst && res.n > r.cap) return THAPI_E_RANGE;
  if (!dst && res.n) {
    q->buf_bytes = res.n * sizeof(thapi_interval);
    q->buf = S->arena.get(q->buf_bytes, &q->buf_own);
    if (!q->buf) return THAPI_E_NOMEM;
    dst = q->buf;
  }
  if (res.n > kStageMinIntervals && (rc = grow_stage(S, sl, res.n * sizeof(thapi_interval))) != THAPI_OK) return rc;
  rc = thapi::window_to_host_id(S->ctx, q->trace, r.t0, r.t1, dst, res.n,
                                res.n > kStageMinIntervals ? sl->stage : nullptr, sl->w, sl->total_d, sl->stream);
  if (rc == THAPI_OK) res.data = dst;
  return rc;
}

void run_slot(thapi_server *S, Slot *sl) {
  cudaSetDevice(S->device);
  std::unique_lock<std::mutex> lk(S->mu);
  for (;;) {
    Req *q = S->stop ? nullptr : pick(S, sl->query);
    if (!q) {
      if (S->stop) return;
      S->cv.wait(lk);
      continue;
    }
    q->state = 1;
    q->res.t_admit = secs(S, Clock::now());
    S->running += 1;
    if (S->running > S->st.peak_running) S->st.peak_running = S->running;
    note_memory(S);
    lk.unlock();
    const int rc = execute(S, sl, q);
    lk.lock();
    S->running -= 1;
    if (q->r.kind == THAPI_REQ_LOAD) S->reserved -= q->charge;
    complete(S, q, rc);
  }
}

void destroy_slot(thapi_server *S, Slot *sl) {
  if (sl->w) thapi::ctx_free(S->ctx, sl->w, sizeof(thapi::WinWork), sl->stream);
  if (sl->stage) thapi::ctx_free(S->ctx, sl->stage, sl->stage_bytes, sl->stream);
  if (sl->stream) cudaStreamSynchronize(sl->stream);
  if (sl->total_h) cudaFreeHost(sl->total_h);
  if (sl->stream) cudaStreamDestroy(sl->stream);
  delete sl;
}

int submit(thapi_server *S, const thapi_request &r, bool auto_release, double arrival, uint64_t *ticket) {
  if (r.kind > THAPI_REQ_FREE) return THAPI_E_INVALID;
  if (r.kind == THAPI_REQ_LOAD && !r.bytes) return THAPI_E_INVALID;
  if ((r.kind == THAPI_REQ_TALLY || r.kind == THAPI_REQ_WINDOW) && r.cap && !r.out) return THAPI_E_INVALID;
  Req *q = new (std::nothrow) Req();
  if (!q) return THAPI_E_NOMEM;
  q->r = r;
  q->auto_release = auto_release;
  int refuse = THAPI_OK;
  if (r.kind == THAPI_REQ_LOAD) {  // the admission charge, from the file header and tables
    cudaSetDevice(S->device);
    const uint8_t *b = static_cast<const uint8_t *>(r.bytes);
    std::lock_guard<std::mutex> hg(S->head_mu);
    refuse = thapi::load_charge(S->ctx, r.on_device ? nullptr : b, r.on_device ? b : nullptr, r.nbytes,
                                S->head_stream, &q->charge);
    uint64_t cap = 0, used = 0;
    thapi::ctx_memory(S->ctx, &cap, &used);
    if (refuse == THAPI_OK && cap && q->charge > cap) refuse = THAPI_E_NOMEM;  // can never fit
  }
  std::lock_guard<std::mutex> g(S->mu);
  if (r.kind != THAPI_REQ_LOAD) {
    if (r.after) {
      auto it = S->reqs.find(r.after);
      const bool was_load = (it != S->reqs.end() && it->second->r.kind == THAPI_REQ_LOAD) || S->loads.count(r.after);
      if (!was_load || r.after >= S->next_ticket) {
        delete q;
        return THAPI_E_INVALID;
      }
      q->key = r.after;
    } else {
      auto k = S->id_key.find(r.trace);
      q->key = k != S->id_key.end() ? k->second : (r.trace | kIdKey);
      q->trace = r.trace;
    }
    if (S->leaving.count(q->key)) refuse = THAPI_E_INVALID;  // the trace has been freed (or is being freed)
  }
  q->ticket = S->next_ticket++;
  q->res.t_arrival = arrival >= 0 ? arrival : secs(S, Clock::now());
  S->reqs[q->ticket] = q;
  S->st.submitted += 1;
  *ticket = q->ticket;
  if (refuse != THAPI_OK) {
    q->res.trace = q->trace;
    complete(S, q, refuse);
    return THAPI_OK;
  }
  if (r.kind == THAPI_REQ_TALLY || r.kind == THAPI_REQ_WINDOW) {
    S->pending[q->key] += 1;
    q->counted = true;
  } else if (r.kind == THAPI_REQ_FREE) {
    S->leaving.insert(q->key);
  }
  S->waiting.push_back(q);
  S->cv.notify_all();
  return THAPI_OK;
}

int wait_ticket(thapi_server *S, uint64_t ticket, uint32_t wait_ms, thapi_result *res) {
  std::unique_lock<std::mutex> lk(S->mu);
  auto it = S->reqs.find(ticket);
  if (it == S->reqs.end()) return THAPI_E_INVALID;
  Req *q = it->second;
  if (q->state != 2) {
    auto done = [&]() { return q->state == 2; };
    if (wait_ms == UINT32_MAX)
      S->cv_done.wait(lk, done);
    else if (!S->cv_done.wait_for(lk, std::chrono::milliseconds(wait_ms), done))
      return THAPI_PENDING;
  }
  *res = q->res;
  return THAPI_OK;
}

int release(thapi_server *S, uint64_t ticket) {
  std::lock_guard<std::mutex> g(S->mu);
  auto it = S->reqs.find(ticket);
  if (it == S->reqs.end() || it->second->state != 2) return THAPI_E_INVALID;
  Req *q = it->second;
  if (q->buf) S->arena.put(q->buf, q->buf_bytes, q->buf_own);
  S->reqs.erase(it);
  delete q;
  return THAPI_OK;
}

}  // namespace

extern "C" {

int thapi_server_create(thapi_ctx *ctx, uint32_t load_slots, uint32_t query_slots, uint64_t result_bytes,
                        thapi_server **out) {
  if (!ctx || !out || load_slots == 0 || query_slots == 0 || load_slots + query_slots > 64) return THAPI_E_INVALID;
  *out = nullptr;
  thapi_server *S = new (std::nothrow) thapi_server();
  if (!S) return THAPI_E_NOMEM;
  S->ctx = ctx;
  S->device = thapi::ctx_device(ctx);
  S->t0 = Clock::now();
  if (cudaSetDevice(S->device) != cudaSuccess) {
    delete S;
    return THAPI_E_CUDA;
  }
  int least = 0, greatest = 0;
  cudaDeviceGetStreamPriorityRange(&least, &greatest);
  int rc = THAPI_OK;
  if (!S->arena.init(result_bytes ? result_bytes : (1ull << 30)) ||
      cudaStreamCreateWithFlags(&S->head_stream, cudaStreamNonBlocking) != cudaSuccess) {
    cudaGetLastError();
    delete S;
    return THAPI_E_CUDA;
  }
  for (uint32_t i = 0; i < load_slots + query_slots && rc == THAPI_OK; ++i) {
    Slot *sl = new (std::nothrow) Slot();
    if (!sl) {
      rc = THAPI_E_NOMEM;
      break;
    }
    sl->query = i >= load_slots;
    S->slots.push_back(sl);
    void *h = nullptr;
    if (cudaStreamCreateWithPriority(&sl->stream, cudaStreamNonBlocking, sl->query ? greatest : least) !=
            cudaSuccess ||
        cudaHostAlloc(&h, 64, cudaHostAllocMapped | cudaHostAllocPortable) != cudaSuccess) {
      cudaGetLastError();
      rc = THAPI_E_CUDA;
      break;
    }
    sl->total_h = static_cast<unsigned long long *>(h);
    sl->total_d = static_cast<unsigned long long *>(thapi::device_view(h));
    if (sl->query) {
      sl->w = static_cast<thapi::WinWork *>(thapi::ctx_alloc(ctx, sizeof(thapi::WinWork), sl->stream));
      if (!sl->w || !sl->total_d) rc = THAPI_E_NOMEM;
    }
  }
  if (rc == THAPI_OK)
    for (Slot *sl : S->slots) sl->th = std::thread(run_slot, S, sl);
  if (rc != THAPI_OK) {
    for (Slot *sl : S->slots) destroy_slot(S, sl);
    cudaStreamDestroy(S->head_stream);
    delete S;
    return rc;
  }
  *out = S;
  return THAPI_OK;
}

int thapi_server_submit(thapi_server *s, const thapi_request *req, uint64_t *ticket) {
  if (!s || !req || !ticket) return THAPI_E_INVALID;
  return submit(s, *req, false, -1.0, ticket);
}

int thapi_server_poll(thapi_server *s, uint64_t ticket, uint32_t wait_ms, thapi_result *res) {
  if (!s || !res) return THAPI_E_INVALID;
  return wait_ticket(s, ticket, wait_ms, res);
}

int thapi_server_release(thapi_server *s, uint64_t ticket) {
  if (!s) return THAPI_E_INVALID;
  return release(s, ticket);
}

double thapi_server_now(thapi_server *s) { return s ? secs(s, Clock::now()) : 0.0; }

int thapi_server_replay(thapi_server *s, const thapi_request *reqs, const double *arrival_s, uint64_t n, int keep,
                        thapi_result *results) {
  if (!s || (n && (!reqs || !arrival_s || !results))) return THAPI_E_INVALID;
  for (uint64_t i = 0; i < n; ++i)  // `after` names an earlier request of the schedule (index + 1)
    if (reqs[i].after > i || (i && arrival_s[i] < arrival_s[i - 1])) return THAPI_E_INVALID;
  std::vector<uint64_t> tk(n, 0);
  const Clock::time_point start = Clock::now();
  const double start_s = secs(s, start);
  for (uint64_t i = 0; i < n; ++i) {
    std::this_thread::sleep_until(start + std::chrono::duration_cast<Clock::duration>(
                                              std::chrono::duration<double>(arrival_s[i])));
    thapi_request r = reqs[i];
    if (r.after) r.after = tk[r.after - 1];
    results[i] = thapi_result{};
    const int rc = (reqs[i].after && !r.after) ? THAPI_E_INVALID : submit(s, r, keep == 0, start_s + arrival_s[i], &tk[i]);
    if (rc != THAPI_OK) {
      tk[i] = 0;
      results[i].status = rc;
      results[i].kind = reqs[i].kind;
      results[i].t_arrival = results[i].t_done = start_s + arrival_s[i];
    }
  }
  for (uint64_t i = 0; i < n; ++i) {
    if (!tk[i]) continue;
    wait_ticket(s, tk[i], UINT32_MAX, &results[i]);
    if (!keep) release(s, tk[i]);
  }
  return THAPI_OK;
}

int thapi_server_stats_get(thapi_server *s, thapi_server_stats *st) {
  if (!s || !st) return THAPI_E_INVALID;
  std::lock_guard<std::mutex> g(s->mu);
  *st = s->st;
  std::lock_guard<std::mutex> ga(s->arena.mu);
  st->result_allocs = s->arena.own_allocs;
  return THAPI_OK;
}

int thapi_server_destroy(thapi_server *s) {
  if (!s) return THAPI_E_INVALID;
  {
    std::unique_lock<std::mutex> lk(s->mu);
    // every request completes; loads that can never be admitted (nothing
    // running, nothing left to free) are refused with E_NOMEM
    size_t last = ~size_t(0);
    while (!s->waiting.empty() || s->running) {
      s->cv_done.wait_for(lk, std::chrono::milliseconds(200));
      if (!s->running && s->waiting.size() == last) {
        while (!s->waiting.empty()) {
          Req *q = s->waiting.front();
          s->waiting.pop_front();
          complete(s, q, q->r.kind == THAPI_REQ_LOAD ? THAPI_E_NOMEM : THAPI_E_INVALID);
        }
      }
      last = s->waiting.size();
    }
    s->stop = true;
    s->cv.notify_all();
  }
  for (Slot *sl : s->slots)
    if (sl->th.joinable()) sl->th.join();
  cudaSetDevice(s->device);
  for (Slot *sl : s->slots) destroy_slot(s, sl);
  cudaStreamDestroy(s->head_stream);
  for (auto &kv : s->reqs) {
    if (kv.second->buf) s->arena.put(kv.second->buf, kv.second->buf_bytes, kv.second->buf_own);
    delete kv.second;
  }
  delete s;
  return THAPI_OK;
}

}  // extern "C"

// sst_server.cpp -- the served path: continuous batching of events submitted one at
// a time (arXiv 2101.11489, section 3: many events processed concurrently on one
// GPU, with transfers overlapped with computation and a caching allocator for
// device memory).
//
// Memory: at start the server carves `max_inflight` batch slots out of the device
// budget.  A slot owns a stream, the batched kernels' scratch, a device raw arena,
// device cluster arrays and pinned host mirrors for its results; events waiting for
// a slot sit in a pinned host pool.  Nothing is allocated per event.
//
// Admission (sst_submit): the device budget is fixed at start (the slots); an event
// is taken when a request slot is free (else BUSY) and its bytes fit in the pinned
// host pool that holds events waiting for a slot (else BUDGET, retry after
// polling); an event larger than a slot's raw arena is never admissible
// (TOO_LARGE).
//
// Lifetime: callers inside sst_submit / sst_poll are counted; sst_server_stop
// detaches the server from the context (later calls get STATE), wakes waiting
// pollers and frees the server only once no caller is inside.
//
// The loop thread launches a batch as soon as a slot is free and events are
// pending (FIFO, up to max_batch_events and the slot's raw arena): it copies the
// events into the slot's arena (in place mode: the kernels read them from the
// callers' pinned buffers instead, one copy-engine transfer per event saved), runs the batched unpack + cluster kernels, packs
// the events' clusters back to back and reads back the statuses; when those are
// in, it reads back exactly the packed clusters into a pinned results pool and
// frees the slot.  Batches on different slots overlap on the GPU.  sst_poll
// copies an event's results out of the pool.  The pool is sized for the worst
// case of every admitted event (a cluster needs at least two payload bytes, so at
// most 8 bytes of results per raw byte), so a batch never waits for the client to
// poll, whatever order the client polls in.
#include <chrono>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <map>
#include <thread>
#include <vector>

#include "sst_internal.h"

namespace {

// The context's server, counted as in use until release_server (nullptr when no
// server runs).
sst_server* acquire_server(sst_ctx* ctx);
void release_server(sst_ctx* ctx, sst_server* sv);

double now_us() {
  using namespace std::chrono;
  return duration_cast<duration<double, std::micro>>(steady_clock::now().time_since_epoch()).count();
}

// First-fit allocator of byte ranges (host pool), 256-byte granules.
class RangeAlloc {
 public:
  void reset(size_t cap) {
    free_.clear();
    cap_ = cap;
    if (cap) free_[0] = cap;
  }
  bool alloc(size_t n, size_t* off) {
    n = (n + 255) & ~size_t(255);
    if (n == 0) n = 256;
    for (auto it = free_.begin(); it != free_.end(); ++it) {
      if (it->second >= n) {
        *off = it->first;
        const size_t rest = it->second - n, at = it->first + n;
        free_.erase(it);
        if (rest) free_[at] = rest;
        return true;
      }
    }
    return false;
  }
  void release(size_t off, size_t n) {
    n = (n + 255) & ~size_t(255);
    if (n == 0) n = 256;
    auto next = free_.lower_bound(off);
    if (next != free_.end() && off + n == next->first) {
      n += next->second;
      free_.erase(next);
    }
    auto it = free_.lower_bound(off);
    if (it != free_.begin()) {
      auto prev = std::prev(it);
      if (prev->first + prev->second == off) {
        prev->second += n;
        return;
      }
    }
    free_[off] = n;
  }

 private:
  std::map<size_t, size_t> free_;
  size_t cap_ = 0;
};

enum class ReqState { kFree, kPending, kLaunched, kDone, kCollecting };
enum class SlotState { kFree, kRunning, kReading };

struct Req {
  ReqState state = ReqState::kFree;
  uint64_t ticket = 0;
  size_t host_off = 0;   // raw bytes in the host pool (reserved also in zero-copy mode, for admission)
  const uint8_t* src = nullptr;  // zero-copy modes: the caller's bytes
  uint64_t bytes = 0;
  std::vector<uint32_t> fed_len;
  double t_submit = 0, t_done = 0;
  int slot = -1;
  uint32_t index = 0;    // position in its batch
  sst_event_status status{};
  size_t res_off = 0;    // its batch's results region in the results pool
  uint64_t res_total = 0;  // records in that region
  uint64_t first = 0;    // its first record in the region
};

struct Slot {
  SlotState state = SlotState::kFree;
  cudaStream_t st = nullptr;
  cudaEvent_t ev_status = nullptr, ev_done = nullptr;
  cudaEvent_t ev_comp = nullptr;  // the batch's kernels done (the next batch's kernels wait for it)
  sst::Scratch scratch;
  uint8_t* d_raw = nullptr;
  size_t raw_cap = 0;
  uint64_t* d_event_off = nullptr;
  uint64_t* d_event_end = nullptr;  // in-place batches: each event's end (events need not follow one another)
  uint32_t* d_fed_len = nullptr;
  uint64_t* d_clu_off = nullptr;
  sst_event_status* d_status = nullptr;
  uint64_t* d_pack_off = nullptr;
  sst_clusters d_out{};  // the batch's clusters, events back to back (d_pack_off)
  size_t clu_cap = 0;
  uint64_t* h_event_off = nullptr;
  uint64_t* h_event_end = nullptr;
  uint32_t* h_fed_len = nullptr;
  uint64_t* h_clu_off = nullptr;
  sst_event_status* h_status = nullptr;
  uint64_t* h_pack_off = nullptr;
  std::vector<int> reqs;   // requests of the current batch, in batch order
  size_t res_off = 0;      // results region of the current batch
  uint64_t res_total = 0;
};

}  // namespace

struct sst_server {
  sst_ctx* ctx = nullptr;
  sst_server_opts opts{};
  std::mutex mu;
  std::condition_variable cv_loop, cv_done;
  std::thread loop;
  bool stop = false;
  std::string fatal;  // CUDA error seen by the loop; every later call reports it
  std::vector<Slot> slots;
  std::vector<Req> reqs;
  std::deque<int> pending;
  std::vector<int> free_reqs;  // request slots not in use (a stack)
  uint64_t next_seq = 1;       // tickets: sequence number << 20 | request slot
  uint8_t* host_pool = nullptr;
  size_t host_cap = 0;
  RangeAlloc host_alloc;
  uint8_t* res_pool = nullptr;  // results of finished batches (pinned)
  size_t res_cap = 0;
  RangeAlloc res_alloc;
  std::map<size_t, std::pair<size_t, int>> regions;  // results region -> (bytes, events not yet polled)
  size_t max_event_bytes = 0;
  int last_launch = -1;  // slot of the batch launched last (loop thread only)
  int users = 0;  // callers inside sst_submit / sst_poll (under ctx->mu)
  std::condition_variable cv_users;
};

namespace {

template <typename T>
cudaError_t dalloc(T** p, size_t n) {
  return cudaMalloc(reinterpret_cast<void**>(p), (n ? n : 1) * sizeof(T));
}
template <typename T>
cudaError_t halloc(T** p, size_t n) {
  return cudaHostAlloc(reinterpret_cast<void**>(p), (n ? n : 1) * sizeof(T), cudaHostAllocDefault);
}

void free_slot(Slot& s) {
  if (s.st) cudaStreamSynchronize(s.st);
  sst::free_scratch(s.scratch);
  cudaFree(s.d_raw);
  cudaFree(s.d_event_off);
  cudaFree(s.d_event_end);
  cudaFree(s.d_fed_len);
  cudaFree(s.d_clu_off);
  cudaFree(s.d_status);
  cudaFree(s.d_pack_off);
  cudaFree(s.d_out.det);
  cudaFree(s.d_out.first);
  cudaFree(s.d_out.width);
  cudaFree(s.d_out.charge);
  cudaFree(s.d_out.barycenter);
  cudaFreeHost(s.h_event_off);
  cudaFreeHost(s.h_event_end);
  cudaFreeHost(s.h_fed_len);
  cudaFreeHost(s.h_clu_off);
  cudaFreeHost(s.h_status);
  cudaFreeHost(s.h_pack_off);
  if (s.ev_status) cudaEventDestroy(s.ev_status);
  if (s.ev_done) cudaEventDestroy(s.ev_done);
  if (s.ev_comp) cudaEventDestroy(s.ev_comp);
  if (s.st) cudaStreamDestroy(s.st);
  s = Slot{};
}

cudaError_t alloc_clusters(sst_clusters* c, size_t n, bool /*host*/) {
  cudaError_t e;
  c->capacity = n;
  if ((e = dalloc(&c->det, n)) || (e = dalloc(&c->first, n)) || (e = dalloc(&c->width, n)) ||
      (e = dalloc(&c->charge, n)) || (e = dalloc(&c->barycenter, n)))
    return e;
  return cudaSuccess;
}

// The five arrays of `n` packed records of a results region, in the pool.
struct HostClusters {
  uint32_t* det;
  uint16_t* first;
  uint16_t* width;
  uint32_t* charge;
  float* bary;
};
HostClusters region_arrays(uint8_t* base, uint64_t n) {
  HostClusters h;
  h.det = reinterpret_cast<uint32_t*>(base);
  h.charge = reinterpret_cast<uint32_t*>(base + 4 * n);
  h.bary = reinterpret_cast<float*>(base + 8 * n);
  h.first = reinterpret_cast<uint16_t*>(base + 12 * n);
  h.width = reinterpret_cast<uint16_t*>(base + 14 * n);
  return h;
}

cudaError_t init_slot(Slot& s, const sst_server_opts& o, size_t raw_cap, uint32_t n_feds, int n_sm) {
  cudaError_t e;
  const uint32_t E = o.max_batch_events;
  s.raw_cap = raw_cap;
  s.clu_cap = raw_cap / 2 + E;
  if ((e = cudaStreamCreateWithFlags(&s.st, cudaStreamNonBlocking))) return e;
  if ((e = cudaEventCreateWithFlags(&s.ev_status, cudaEventDisableTiming))) return e;
  if ((e = cudaEventCreateWithFlags(&s.ev_done, cudaEventDisableTiming))) return e;
  if ((e = cudaEventCreateWithFlags(&s.ev_comp, cudaEventDisableTiming))) return e;
  if ((e = sst::ensure_scratch(s.scratch, (size_t)E * n_feds * sst::kFe, E, s.clu_cap))) return e;
  if ((e = sst::ensure_spill(s.scratch, (size_t)n_sm * sst::kMaxWarpsPerSm))) return e;
  if ((e = dalloc(&s.d_raw, raw_cap))) return e;
  if ((e = dalloc(&s.d_event_off, E + 1)) || (e = dalloc(&s.d_event_end, E)) || (e = dalloc(&s.d_fed_len, (size_t)E * n_feds)) ||
      (e = dalloc(&s.d_clu_off, E + 1)) || (e = dalloc(&s.d_status, E)) || (e = dalloc(&s.d_pack_off, E + 1)))
    return e;
  if ((e = alloc_clusters(&s.d_out, s.clu_cap, false))) return e;
  if ((e = halloc(&s.h_event_off, E + 1)) || (e = halloc(&s.h_event_end, E)) || (e = halloc(&s.h_fed_len, (size_t)E * n_feds)) ||
      (e = halloc(&s.h_clu_off, E + 1)) || (e = halloc(&s.h_status, E)) || (e = halloc(&s.h_pack_off, E + 1)))
    return e;
  return cudaSuccess;
}

void loop_main(sst_server* sv);

}  // namespace

namespace {

// One event of a batch being formed: where its bytes and FED lengths are (stable
// while its request is launched: only the loop thread touches such a request).
struct Part {
  const uint8_t* src;
  uint64_t bytes;
  const uint32_t* fed_len;
};

// Takes the next batch off the pending queue for slot si (FIFO, up to
// max_batch_events and the slot's raw arena).  Lock held.  Returns false when
// nothing was pending.
bool take_batch(sst_server* sv, int si, std::vector<Part>* parts) {
  Slot& s = sv->slots[si];
  s.reqs.clear();
  parts->clear();
  uint64_t bytes = 0;
  while (!sv->pending.empty() && s.reqs.size() < sv->opts.max_batch_events) {
    Req& r = sv->reqs[sv->pending.front()];
    if (bytes + r.bytes > s.raw_cap) break;
    bytes += r.bytes;
    r.state = ReqState::kLaunched;
    r.slot = si;
    r.index = (uint32_t)s.reqs.size();
    parts->push_back(Part{r.src ? r.src : sv->host_pool + r.host_off, r.bytes, r.fed_len.data()});
    s.reqs.push_back(sv->pending.front());
    sv->pending.pop_front();
  }
  return !s.reqs.empty();
}

// Launches a taken batch on slot si: copies the events into the slot's arena,
// runs the batched unpack + cluster kernels, packs the events' clusters back to
// back and reads back the statuses.  Called WITHOUT the lock (CUDA calls only,
// on slot state that only the loop thread touches).
cudaError_t launch_batch_on(sst_server* sv, int si, const std::vector<Part>& parts) {
  Slot& s = sv->slots[si];
  const uint32_t nf = sv->opts.n_feds;
  const uint32_t E = (uint32_t)parts.size();
  // in place (zero_copy 2): the kernels read every event from the caller's pinned
  // buffer over the host link, with offsets from the lowest of the buffers
  const bool in_place = sv->opts.zero_copy == 2;
  const uint8_t* base = in_place ? parts[0].src : s.d_raw;
  for (uint32_t i = 1; in_place && i < E; i++)
    if (parts[i].src < base) base = parts[i].src;
  uint64_t off = 0, coff = 0;
  cudaError_t e = cudaSuccess;
  for (uint32_t i = 0; i < E; i++) {
    s.h_event_off[i] = in_place ? (uint64_t)((uintptr_t)parts[i].src - (uintptr_t)base) : off;
    s.h_event_end[i] = s.h_event_off[i] + parts[i].bytes;
    s.h_clu_off[i] = coff;
    std::memcpy(s.h_fed_len + (size_t)i * nf, parts[i].fed_len, nf * sizeof(uint32_t));
    if (!in_place && !e)
      e = cudaMemcpyAsync(s.d_raw + off, parts[i].src, parts[i].bytes, cudaMemcpyHostToDevice, s.st);
    off += parts[i].bytes;
    coff += parts[i].bytes / 2 + 1;
  }
  s.h_event_off[E] = in_place ? s.h_event_end[E - 1] : off;
  s.h_clu_off[E] = coff;
  if (!e) e = cudaMemcpyAsync(s.d_event_off, s.h_event_off, (E + 1) * sizeof(uint64_t), cudaMemcpyHostToDevice, s.st);
  if (!e && in_place)
    e = cudaMemcpyAsync(s.d_event_end, s.h_event_end, E * sizeof(uint64_t), cudaMemcpyHostToDevice, s.st);
  if (!e) e = cudaMemcpyAsync(s.d_fed_len, s.h_fed_len, (size_t)E * nf * sizeof(uint32_t), cudaMemcpyHostToDevice, s.st);
  if (!e) e = cudaMemcpyAsync(s.d_clu_off, s.h_clu_off, (E + 1) * sizeof(uint64_t), cudaMemcpyHostToDevice, s.st);
  sst_clusters out = s.d_out;
  out.capacity = s.clu_cap;
  // one batch's kernels at a time: each persistent launch fills the GPU, so
  // batches run back to back at full speed and finish one after another, and a
  // batch's copies overlap the next one's kernels (kernels of several slots
  // running at once would finish together and leave the GPU idle while all of
  // them copy their results back)
  if (!e && sv->last_launch >= 0) e = cudaStreamWaitEvent(s.st, sv->slots[sv->last_launch].ev_comp, 0);
  if (!e) e = sst::launch_batch(base, s.d_event_off, s.d_fed_len, E, nf, s.d_clu_off, out, s.d_status,
                                sst::kparams(sv->ctx), s.scratch, sv->ctx->shape, sv->ctx->n_sm, s.st, s.d_pack_off,
                                nullptr, nullptr, in_place ? s.d_event_end : nullptr);
  if (!e) e = cudaEventRecord(s.ev_comp, s.st);
  sv->last_launch = si;
  if (!e) e = cudaMemcpyAsync(s.h_status, s.d_status, E * sizeof(sst_event_status), cudaMemcpyDeviceToHost, s.st);
  if (!e) e = cudaMemcpyAsync(s.h_pack_off, s.d_pack_off, (E + 1) * sizeof(uint64_t), cudaMemcpyDeviceToHost, s.st);
  if (!e) e = cudaEventRecord(s.ev_status, s.st);
  return e;
}

// Issues the read-back of a finished batch's packed clusters into its results
// region.  Called WITHOUT the lock.
cudaError_t read_back(sst_server* sv, Slot& s) {
  const uint64_t total = s.res_total;
  const sst_clusters& d = s.d_out;
  const HostClusters h = region_arrays(sv->res_pool + s.res_off, total);
  cudaError_t e = cudaSuccess;
  if (total) {
    e = cudaMemcpyAsync(h.det, d.det, total * 4, cudaMemcpyDeviceToHost, s.st);
    if (!e) e = cudaMemcpyAsync(h.first, d.first, total * 2, cudaMemcpyDeviceToHost, s.st);
    if (!e) e = cudaMemcpyAsync(h.width, d.width, total * 2, cudaMemcpyDeviceToHost, s.st);
    if (!e) e = cudaMemcpyAsync(h.charge, d.charge, total * 4, cudaMemcpyDeviceToHost, s.st);
    if (!e) e = cudaMemcpyAsync(h.bary, d.barycenter, total * 4, cudaMemcpyDeviceToHost, s.st);
  }
  if (!e) e = cudaEventRecord(s.ev_done, s.st);
  return e;
}

void set_fatal(sst_server* sv, const char* what, cudaError_t e) {  // lock held
  if (sv->fatal.empty()) sv->fatal = std::string(what) + cudaGetErrorString(e);
}

// The loop thread.  The lock guards the requests, the pending queue, the pools'
// allocators and the stop flag; the slots belong to this thread.  Each pass
// queries the slots' CUDA events without the lock, takes the lock once to account
// for what finished and to take new batches off the queue, and issues the
// read-backs and launches without it: a slow driver call never holds up
// sst_submit / sst_poll, and the lock changes hands twice per pass.
void loop_main(sst_server* sv) {
  cudaSetDevice(sv->ctx->device);
  const size_t ns = sv->slots.size();
  std::vector<std::vector<Part>> parts(ns);
  std::vector<cudaError_t> q(ns), err(ns);
  enum Todo : char { kNothing, kReadBack, kLaunch };
  std::vector<Todo> todo(ns, kNothing);
  std::unique_lock<std::mutex> lock(sv->mu);
  while (!sv->stop) {
    lock.unlock();
    for (size_t si = 0; si < ns; si++) {
      const Slot& s = sv->slots[si];
      q[si] = s.state == SlotState::kRunning   ? cudaEventQuery(s.ev_status)
              : s.state == SlotState::kReading ? cudaEventQuery(s.ev_done)
                                               : cudaSuccess;
    }
    const double t = now_us();
    lock.lock();
    bool progress = false;
    for (size_t si = 0; si < ns; si++) {
      Slot& s = sv->slots[si];
      todo[si] = kNothing;
      if (q[si] == cudaErrorNotReady) continue;
      if (s.state == SlotState::kRunning) {
        if (q[si]) set_fatal(sv, "served batch: ", q[si]);
        s.res_total = q[si] ? 0 : s.h_pack_off[s.reqs.size()];
        s.res_off = 0;
        if (!q[si] && !sv->res_alloc.alloc(16 * s.res_total, &s.res_off)) {
          sv->fatal = "served batch: results pool exhausted";  // excluded by its sizing
          s.res_total = 0;
        }
        s.state = SlotState::kReading;
        todo[si] = kReadBack;
        progress = true;
        continue;
      }
      if (s.state == SlotState::kReading) {
        if (q[si]) set_fatal(sv, "served batch: ", q[si]);
        sv->regions[s.res_off] = std::make_pair((size_t)(16 * s.res_total), (int)s.reqs.size());
        for (size_t i = 0; i < s.reqs.size(); i++) {
          Req& r = sv->reqs[s.reqs[i]];
          r.state = ReqState::kDone;
          r.t_done = t;
          r.status = s.h_status[i];
          r.res_off = s.res_off;
          r.res_total = s.res_total;
          r.first = s.h_pack_off[i];
        }
        s.reqs.clear();
        s.state = SlotState::kFree;
        progress = true;
        sv->cv_done.notify_all();
      }
      if (s.state == SlotState::kFree && sv->fatal.empty() && take_batch(sv, (int)si, &parts[si])) {
        s.state = SlotState::kRunning;
        todo[si] = kLaunch;
        progress = true;
      }
    }
    if (!progress) {
      if (sv->stop) break;
      bool busy = false;
      for (const Slot& s : sv->slots)
        busy |= s.state == SlotState::kRunning || s.state == SlotState::kReading;
      // new events notify cv_loop; batches in flight are polled every 20 us
      if (busy)
        sv->cv_loop.wait_for(lock, std::chrono::microseconds(20));
      else
        sv->cv_loop.wait_for(lock, std::chrono::milliseconds(5),
                             [&] { return sv->stop || (!sv->pending.empty() && sv->fatal.empty()); });
      continue;
    }
    lock.unlock();
    for (size_t si = 0; si < ns; si++) {
      err[si] = todo[si] == kReadBack ? read_back(sv, sv->slots[si])
                : todo[si] == kLaunch ? launch_batch_on(sv, (int)si, parts[si])
                                      : cudaSuccess;
    }
    lock.lock();
    for (size_t si = 0; si < ns; si++)
      if (err[si]) set_fatal(sv, todo[si] == kLaunch ? "served batch launch: " : "served batch: ", err[si]);
  }
}

// Releases a finished request: its raw bytes and its share of its results region.
// Lock held.
void release(sst_server* sv, int ri) {
  Req& r = sv->reqs[ri];
  sv->host_alloc.release(r.host_off, r.bytes);
  auto it = sv->regions.find(r.res_off);
  const bool finished = r.state == ReqState::kDone || r.state == ReqState::kCollecting;
  if (finished && it != sv->regions.end() && --it->second.second == 0) {
    sv->res_alloc.release(it->first, it->second.first);
    sv->regions.erase(it);
  }
  r = Req{};
  sv->free_reqs.push_back(ri);
}

}  // namespace

namespace {
sst_status submit_one(sst_ctx* ctx, sst_server* sv, const uint8_t* raw, uint64_t raw_bytes, const uint32_t* fed_len,
                      uint64_t* ticket);
sst_status poll_one(sst_ctx* ctx, sst_server* sv, uint64_t ticket, int64_t timeout_us, sst_result_info* info,
                    uint32_t* det, uint16_t* first, uint16_t* width, uint32_t* charge, float* barycenter,
                    uint64_t capacity);
}  // namespace

extern "C" {

sst_status sst_server_stop(sst_ctx* ctx);

sst_status sst_server_start(sst_ctx* ctx, const sst_server_opts* opts) {
  if (!ctx || !opts) return SST_ERR_INVALID_ARG;
  {
    std::lock_guard<std::mutex> g(ctx->mu);
    if (ctx->server) return sst::set_err(ctx, SST_ERR_STATE, "sst_server_start: already running");
  }
  if (!ctx->has_calib) return sst::set_err(ctx, SST_ERR_NO_CALIB, "sst_server_start: no calibration");
  const sst_server_opts& o = *opts;
  if (o.mem_budget_bytes < (64ull << 20) || o.max_batch_events == 0 || o.max_batch_events > 4096 ||
      o.max_inflight == 0 || o.max_inflight > 8 || o.max_requests == 0 || o.max_requests > (1u << 20) ||
      o.n_feds == 0 || o.n_feds > ctx->n_feds || o.zero_copy > 2)
    return sst::set_err(ctx, SST_ERR_INVALID_ARG,
                        "sst_server_start: need budget >= 64 MiB, 1..4096 events per batch, 1..8 in flight, "
                        "1..2^20 requests, 1..context FEDs per event and zero_copy 0, 1 or 2");
  int prev = -1;
  cudaGetDevice(&prev);
  cudaSetDevice(ctx->device);
  auto* sv = new sst_server();
  sv->ctx = ctx;
  sv->opts = o;
  // per slot: raw arena r, cluster records r/2 three times over (per-event
  // output, packed output, staging) at 16 bytes each, pinned host results: ~25 r
  const size_t raw_cap = (size_t)(o.mem_budget_bytes / (25ull * o.max_inflight)) & ~size_t(255);
  sv->max_event_bytes = raw_cap;
  sv->host_cap = raw_cap * (o.max_inflight + 1);
  if (sv->host_cap > (size_t(2) << 30)) sv->host_cap = size_t(2) << 30;
  cudaError_t e = cudaHostAlloc(reinterpret_cast<void**>(&sv->host_pool), sv->host_cap, cudaHostAllocDefault);
  sv->host_alloc.reset(sv->host_cap);
  // every admitted event's results fit at once: at most raw/2 + 1 records of 16
  // bytes per event, plus one 256-byte granule of rounding per batch
  sv->res_cap = 8 * sv->host_cap + (size_t)(16 + 256) * o.max_requests + 256 * o.max_inflight;
  if (!e) e = cudaHostAlloc(reinterpret_cast<void**>(&sv->res_pool), sv->res_cap, cudaHostAllocDefault);
  sv->res_alloc.reset(sv->res_cap);
  sv->slots.resize(o.max_inflight);
  for (uint32_t i = 0; i < o.max_inflight && !e; i++) e = init_slot(sv->slots[i], o, raw_cap, o.n_feds, ctx->n_sm);
  if (e) {
    for (Slot& s : sv->slots) free_slot(s);
    if (sv->host_pool) cudaFreeHost(sv->host_pool);
    if (sv->res_pool) cudaFreeHost(sv->res_pool);
    delete sv;
    if (prev >= 0) cudaSetDevice(prev);
    return sst::cuda_err(ctx, e, "sst_server_start");
  }
  sv->reqs.resize(o.max_requests);
  sv->free_reqs.reserve(o.max_requests);
  for (uint32_t i = o.max_requests; i-- > 0;) sv->free_reqs.push_back((int)i);
  sv->loop = std::thread(loop_main, sv);
  {
    std::lock_guard<std::mutex> g(ctx->mu);
    ctx->server = sv;
  }
  if (prev >= 0) cudaSetDevice(prev);
  return SST_OK;
}

sst_status sst_server_stop(sst_ctx* ctx) {
  if (!ctx) return SST_ERR_INVALID_ARG;
  sst_server* sv = nullptr;
  {
    std::unique_lock<std::mutex> g(ctx->mu);
    sv = ctx->server;
    if (!sv) return SST_OK;
    ctx->server = nullptr;  // new submit / poll calls get STATE from here on
    {
      std::lock_guard<std::mutex> lock(sv->mu);
      sv->stop = true;
    }
    sv->cv_loop.notify_all();
    sv->cv_done.notify_all();  // pollers waiting without a timeout return
    sv->cv_users.wait(g, [&] { return sv->users == 0; });
  }
  sv->loop.join();
  int prev = -1;
  cudaGetDevice(&prev);
  cudaSetDevice(ctx->device);
  for (Slot& s : sv->slots) free_slot(s);
  if (sv->host_pool) cudaFreeHost(sv->host_pool);
  if (sv->res_pool) cudaFreeHost(sv->res_pool);
  if (prev >= 0) cudaSetDevice(prev);
  delete sv;
  return SST_OK;
}

sst_status sst_submit(sst_ctx* ctx, const uint8_t* raw, uint64_t raw_bytes, const uint32_t* fed_len,
                      uint64_t* ticket) {
  if (!ctx || !raw || !fed_len || !ticket) return SST_ERR_INVALID_ARG;
  sst_server* sv = acquire_server(ctx);
  if (!sv) return sst::set_err(ctx, SST_ERR_STATE, "sst_submit: server not running");
  const sst_status r = submit_one(ctx, sv, raw, raw_bytes, fed_len, ticket);
  release_server(ctx, sv);
  return r;
}

sst_status sst_poll(sst_ctx* ctx, uint64_t ticket, int64_t timeout_us, sst_result_info* info, uint32_t* det,
                    uint16_t* first, uint16_t* width, uint32_t* charge, float* barycenter, uint64_t capacity) {
  if (!ctx) return SST_ERR_INVALID_ARG;
  sst_server* sv = acquire_server(ctx);
  if (!sv) return sst::set_err(ctx, SST_ERR_STATE, "sst_poll: server not running");
  const sst_status r = poll_one(ctx, sv, ticket, timeout_us, info, det, first, width, charge, barycenter, capacity);
  release_server(ctx, sv);
  return r;
}

}  // extern "C"

namespace {

sst_server* acquire_server(sst_ctx* ctx) {
  std::lock_guard<std::mutex> g(ctx->mu);
  sst_server* sv = ctx->server;
  if (sv) sv->users++;
  return sv;
}

void release_server(sst_ctx* ctx, sst_server* sv) {
  std::lock_guard<std::mutex> g(ctx->mu);
  if (--sv->users == 0) sv->cv_users.notify_all();
}

// Whether the kernels may read [p, p + n) in place: 16-byte aligned, a multiple of
// 16 bytes, and its first and last bytes in page-locked host memory that the
// device sees at the same address (the caller guarantees that the whole span is one
// such allocation).  Returns null when it may, else what is wrong.  The query runs
// with the server's device current (the calling thread's device is restored).
const char* pinned_span(int device, const uint8_t* p, uint64_t n) {
  if (n == 0) return nullptr;
  if ((uintptr_t)p & 15u) return "not 16-byte aligned";
  if (n & 15u) return "length not a multiple of 16 bytes";
  int prev = -1;
  cudaGetDevice(&prev);
  cudaSetDevice(device);  // also binds the device's context to a thread that has made no CUDA call yet
  const char* why = nullptr;
  for (const uint8_t* q : {p, p + n - 1}) {
    cudaPointerAttributes a{};
    const cudaError_t e = cudaPointerGetAttributes(&a, q);
    if (e != cudaSuccess) {
      cudaGetLastError();  // not a pointer the runtime knows: not readable in place
      why = "unknown to the CUDA runtime";
    } else if (a.type != cudaMemoryTypeHost) {
      why = "not page-locked host memory";
    } else if (a.devicePointer != (const void*)q) {
      why = "mapped at another address on the device";
    }
    if (why) break;
  }
  if (prev >= 0 && prev != device) cudaSetDevice(prev);
  return why;
}

sst_status submit_one(sst_ctx* ctx, sst_server* sv, const uint8_t* raw, uint64_t raw_bytes, const uint32_t* fed_len,
                      uint64_t* ticket) {
  if (raw_bytes > sv->max_event_bytes) return SST_ERR_TOO_LARGE;
  if (sv->opts.zero_copy == 2) {
    const char* why = pinned_span(ctx->device, raw, raw_bytes);
    if (why)
      return sst::set_err(ctx, SST_ERR_INVALID_ARG,
                          std::string("sst_submit: an event read in place must be a 16-byte aligned span of pinned "
                                      "host memory, a multiple of 16 bytes long: ") + why);
  }
  std::vector<uint32_t> fl(fed_len, fed_len + sv->opts.n_feds);
  const bool lend = sv->opts.zero_copy != 0;
  int ri = -1;
  size_t off = 0;
  {
    std::lock_guard<std::mutex> lock(sv->mu);
    if (!sv->fatal.empty()) return sst::set_err(ctx, SST_ERR_CUDA, sv->fatal);
    if (sv->free_reqs.empty()) return SST_ERR_BUSY;
    if (!sv->host_alloc.alloc(raw_bytes, &off)) return SST_ERR_BUDGET;
    ri = sv->free_reqs.back();
    sv->free_reqs.pop_back();
    Req& r = sv->reqs[ri];
    r.state = ReqState::kPending;  // reserved; queued below (at once when the caller lends its buffer)
    r.host_off = off;
    r.bytes = raw_bytes;
    r.ticket = (sv->next_seq++ << 20) | (uint64_t)ri;
    *ticket = r.ticket;
    if (lend) {
      r.src = raw;
      r.fed_len.swap(fl);
      r.t_submit = now_us();
      sv->pending.push_back(ri);
    }
  }
  if (!lend) {  // copy outside the lock, then queue
    std::memcpy(sv->host_pool + off, raw, raw_bytes);
    std::lock_guard<std::mutex> lock(sv->mu);
    Req& r = sv->reqs[ri];
    r.fed_len.swap(fl);
    r.t_submit = now_us();
    sv->pending.push_back(ri);
  }
  sv->cv_loop.notify_one();
  return SST_OK;
}

sst_status poll_one(sst_ctx* ctx, sst_server* sv, uint64_t ticket, int64_t timeout_us, sst_result_info* info,
                    uint32_t* det, uint16_t* first, uint16_t* width, uint32_t* charge, float* barycenter,
                    uint64_t capacity) {
  std::unique_lock<std::mutex> lock(sv->mu);
  const uint64_t slot = ticket & ((1u << 20) - 1u);  // a ticket names its request slot
  const int ri = slot < sv->reqs.size() ? (int)slot : -1;
  if (ri < 0 || sv->reqs[ri].ticket != ticket || sv->reqs[ri].state == ReqState::kFree ||
      sv->reqs[ri].state == ReqState::kCollecting)
    return sst::set_err(ctx, SST_ERR_INVALID_ARG, "sst_poll: unknown ticket");
  // gone: another caller collected this ticket meanwhile
  auto gone = [&] { return sv->reqs[ri].ticket != ticket || sv->reqs[ri].state == ReqState::kCollecting; };
  auto done = [&] { return gone() || sv->reqs[ri].state == ReqState::kDone || !sv->fatal.empty() || sv->stop; };
  if (timeout_us < 0)
    sv->cv_done.wait(lock, done);
  else if (timeout_us > 0)
    sv->cv_done.wait_for(lock, std::chrono::microseconds(timeout_us), done);
  if (!sv->fatal.empty()) return sst::set_err(ctx, SST_ERR_CUDA, sv->fatal);
  if (gone()) return sst::set_err(ctx, SST_ERR_INVALID_ARG, "sst_poll: unknown ticket");
  Req& r = sv->reqs[ri];
  if (r.state != ReqState::kDone)
    return sv->stop ? sst::set_err(ctx, SST_ERR_STATE, "sst_poll: server stopped") : SST_ERR_NOT_READY;
  // the results are copied out without the lock: the request is marked as being
  // collected, which keeps its results region allocated and other callers off it
  r.state = ReqState::kCollecting;
  const sst_event_status st = r.status;
  const uint64_t a = r.first;
  const uint64_t n = st.n_clusters < capacity ? st.n_clusters : capacity;
  const HostClusters h = region_arrays(sv->res_pool + r.res_off, r.res_total);
  if (info) {
    info->status = st;
    info->t_submit_us = r.t_submit;
    info->t_done_us = r.t_done;
  }
  if (n == 0 || !(det || first || width || charge || barycenter)) {  // nothing to copy
    release(sv, ri);
    return SST_OK;
  }
  lock.unlock();
  if (det) std::memcpy(det, h.det + a, n * sizeof(uint32_t));
  if (first) std::memcpy(first, h.first + a, n * sizeof(uint16_t));
  if (width) std::memcpy(width, h.width + a, n * sizeof(uint16_t));
  if (charge) std::memcpy(charge, h.charge + a, n * sizeof(uint32_t));
  if (barycenter) std::memcpy(barycenter, h.bary + a, n * sizeof(float));
  lock.lock();
  release(sv, ri);
  return SST_OK;
}

}  // namespace


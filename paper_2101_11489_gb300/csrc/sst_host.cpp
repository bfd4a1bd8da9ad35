// sst_host.cpp -- sst_batch_host: batched unpack + cluster of events that live in
// host memory, with the host->device copies, the kernels and the device->host
// copies of successive chunks of events overlapped (arXiv 2101.11489, section 3:
// transfers overlapped with computation on CUDA streams).
//
// The batch is cut into chunks of consecutive events, and the work runs on four
// streams of the context: one for host->device copies, one for the kernels (in
// chunk order), one for the small status copies and one for the cluster copies
// (apart, so that a chunk's cluster copy never queues behind the status copy of
// a later chunk, which waits for that chunk's kernels).  Chunk j uses the device arenas
// of pipeline slot j mod kSlots:
//   H2D   the chunk's raw bytes, FED lengths and (rebased) event offsets, once
//         the slot's previous chunk has finished its kernels;
//   GPU   the batched kernels in packed mode (events back to back, pack_off),
//         once the copies are in and the slot's previous clusters are out;
//   D2H   the statuses and pack_off, then an event the host waits on.
// Before slot k takes chunk j + kSlots, the host waits for chunk j's statuses,
// which gives it chunk j's cluster count, and enqueues the exact-size copies of
// chunk j's clusters into the caller's arrays right after the ones before it.
// The kernels of the next chunks are already queued, so the GPU does not wait
// for the host, and a chunk's copies overlap the kernels of the chunks after it.
//
// Batches are submitted to a worker thread of the context (sst_batch_host_submit)
// and processed in submission order as one continuous stream of chunks: the next
// batch's first chunks are copied in and computed while the previous batch's
// last chunks are still being copied out, so consecutive batches overlap.
// sst_batch_host_wait returns when a batch's results are in the caller's arrays;
// sst_batch_host is submit + wait.
//
// Device arenas grow on demand (a cudaMalloc only when a batch needs more than
// any batch before it on this context; the worker drains the pipeline first) and
// live until sst_destroy.
#include <condition_variable>
#include <cstring>
#include <deque>
#include <map>
#include <thread>
#include <vector>

#include "sst_internal.h"

namespace {

constexpr int kSlots = 3;

template <typename T>
cudaError_t dgrow(T*& p, size_t& cap, size_t need) {
  if (need <= cap) return cudaSuccess;
  if (p) cudaFree(p);
  p = nullptr;
  cap = 0;
  need = need ? need : 1;
  const cudaError_t e = cudaMalloc(reinterpret_cast<void**>(&p), need * sizeof(T));
  if (e == cudaSuccess) cap = need;
  return e;
}

template <typename T>
cudaError_t hgrow(T*& p, size_t& cap, size_t need) {
  if (need <= cap) return cudaSuccess;
  if (p) cudaFreeHost(p);
  p = nullptr;
  cap = 0;
  need = need ? need : 1;
  const cudaError_t e = cudaHostAlloc(reinterpret_cast<void**>(&p), need * sizeof(T), cudaHostAllocDefault);
  if (e == cudaSuccess) cap = need;
  return e;
}

struct PipeSlot {
  cudaEvent_t ev_h2d = nullptr;     // inputs copied in
  cudaEvent_t ev_comp = nullptr;    // kernels done (inputs free, outputs ready)
  cudaEvent_t ev_status = nullptr;  // statuses and pack_off copied out
  cudaEvent_t ev_d2h = nullptr;     // clusters copied out (outputs free)
  uint8_t* d_raw = nullptr;
  size_t raw_cap = 0;
  uint64_t* d_event_off = nullptr;
  size_t eo_cap = 0;
  uint32_t* d_fed_len = nullptr;
  size_t fl_cap = 0;
  uint64_t* d_clu_off = nullptr;
  size_t co_cap = 0;
  sst_event_status* d_status = nullptr;
  size_t st_cap = 0;
  uint64_t* d_pack_off = nullptr;
  size_t po_cap = 0;
  uint32_t* d_det = nullptr;
  uint16_t* d_first = nullptr;
  uint16_t* d_width = nullptr;
  uint32_t* d_charge = nullptr;
  float* d_bary = nullptr;
  size_t clu_cap = 0;
  uint64_t* h_event_off = nullptr;
  size_t h_eo_cap = 0;
  uint64_t* h_clu_off = nullptr;
  size_t h_co_cap = 0;
  sst_event_status* h_status = nullptr;
  size_t h_st_cap = 0;
  uint64_t* h_pack_off = nullptr;
  size_t h_po_cap = 0;
  // amplitudes (batches that ask for them): the chunk's amplitude arena, its
  // clusters' amp_first and its events' slices (rebased to the chunk's first)
  uint8_t* d_amp = nullptr;
  size_t amp_cap = 0;
  uint32_t* d_amp_first = nullptr;
  size_t af_cap = 0;
  uint64_t* d_amp_off = nullptr;
  size_t ao_cap = 0;
  uint64_t* h_amp_off = nullptr;
  size_t h_ao_cap = 0;
  // the chunk in flight: chunk `chunk` of `job`, or job == null when the slot is idle
  struct HostJob* job = nullptr;
  size_t chunk = 0;
};

// One chunk's sizes.
struct Chunk {
  uint32_t e0, e1;
  uint64_t base;       // first raw byte copied (event_off[e0] rounded down to 16)
  uint64_t bytes;      // raw bytes copied
  uint64_t clu_total;  // staging records (sum over events of bytes / 2 + 1)
  uint64_t amp_base = 0, amp_bytes = 0;  // amplitudes: the chunk's range of the caller's amp array
};

// A batch submitted with sst_batch_host_submit: the caller's buffers, its chunks
// and how far the pipeline has got with it.
struct HostJob {
  uint64_t ticket = 0;
  const uint8_t* raw = nullptr;
  const uint64_t* event_off = nullptr;
  const uint32_t* fed_len = nullptr;
  uint32_t n_events = 0, n_feds = 0;
  sst_clusters out{};
  uint64_t* event_first = nullptr;
  sst_event_status* status = nullptr;
  std::vector<Chunk> chunks;
  uint32_t max_e = 0;
  uint64_t max_bytes = 0, max_clu = 0;
  bool amps = false;     // out.amp given: amplitudes too (out.amp_off: host, the events' slices)
  uint64_t max_amp = 0;  // largest chunk amplitude range
  size_t next = 0;      // next chunk to issue
  size_t finished = 0;  // chunks whose clusters are on their way to the caller
  uint64_t pos = 0;     // clusters stored so far
  cudaEvent_t done = nullptr;  // recorded after the batch's last copies
  bool recorded = false;
  cudaError_t err = cudaSuccess;
};

bool slot_fits(const PipeSlot& s, uint32_t E, uint32_t nf, uint64_t bytes, uint64_t clu, uint64_t amp) {
  if (amp && (s.amp_cap < amp || s.af_cap < clu || s.ao_cap < E + 1u || s.h_ao_cap < E + 1u)) return false;
  return s.raw_cap >= bytes && s.fl_cap >= (size_t)E * nf && s.eo_cap >= E + 1u && s.co_cap >= E + 1u &&
         s.st_cap >= E && s.po_cap >= E + 1u && s.clu_cap >= clu && s.h_eo_cap >= E + 1u && s.h_co_cap >= E + 1u &&
         s.h_st_cap >= E && s.h_po_cap >= E + 1u && s.ev_h2d != nullptr;
}

cudaError_t grow_slot(PipeSlot& s, uint32_t E, uint32_t nf, uint64_t bytes, uint64_t clu, uint64_t amp) {
  cudaError_t e;
  if (amp) {
    if ((e = dgrow(s.d_amp, s.amp_cap, amp))) return e;
    if ((e = dgrow(s.d_amp_first, s.af_cap, clu))) return e;
    if ((e = dgrow(s.d_amp_off, s.ao_cap, E + 1))) return e;
    if ((e = hgrow(s.h_amp_off, s.h_ao_cap, E + 1))) return e;
  }
  for (cudaEvent_t* ev : {&s.ev_h2d, &s.ev_comp, &s.ev_status, &s.ev_d2h})
    if (!*ev && (e = cudaEventCreateWithFlags(ev, cudaEventDisableTiming))) return e;
  if ((e = dgrow(s.d_raw, s.raw_cap, bytes))) return e;
  if ((e = dgrow(s.d_event_off, s.eo_cap, E + 1))) return e;
  if ((e = dgrow(s.d_fed_len, s.fl_cap, (size_t)E * nf))) return e;
  if ((e = dgrow(s.d_clu_off, s.co_cap, E + 1))) return e;
  if ((e = dgrow(s.d_status, s.st_cap, E))) return e;
  if ((e = dgrow(s.d_pack_off, s.po_cap, E + 1))) return e;
  if (clu > s.clu_cap) {
    size_t c1 = s.clu_cap, c2 = s.clu_cap, c3 = s.clu_cap, c4 = s.clu_cap, c5 = s.clu_cap;
    if ((e = dgrow(s.d_det, c1, clu)) || (e = dgrow(s.d_first, c2, clu)) || (e = dgrow(s.d_width, c3, clu)) ||
        (e = dgrow(s.d_charge, c4, clu)) || (e = dgrow(s.d_bary, c5, clu)))
      return e;
    s.clu_cap = clu;
  }
  if ((e = hgrow(s.h_event_off, s.h_eo_cap, E + 1))) return e;
  if ((e = hgrow(s.h_clu_off, s.h_co_cap, E + 1))) return e;
  if ((e = hgrow(s.h_status, s.h_st_cap, E))) return e;
  if ((e = hgrow(s.h_pack_off, s.h_po_cap, E + 1))) return e;
  return cudaSuccess;
}

void free_slot(PipeSlot& s) {
  cudaFree(s.d_raw);
  cudaFree(s.d_event_off);
  cudaFree(s.d_fed_len);
  cudaFree(s.d_clu_off);
  cudaFree(s.d_status);
  cudaFree(s.d_pack_off);
  cudaFree(s.d_det);
  cudaFree(s.d_first);
  cudaFree(s.d_width);
  cudaFree(s.d_charge);
  cudaFree(s.d_bary);
  cudaFreeHost(s.h_event_off);
  cudaFreeHost(s.h_clu_off);
  cudaFreeHost(s.h_status);
  cudaFreeHost(s.h_pack_off);
  cudaFree(s.d_amp);
  cudaFree(s.d_amp_first);
  cudaFree(s.d_amp_off);
  cudaFreeHost(s.h_amp_off);
  for (cudaEvent_t ev : {s.ev_h2d, s.ev_comp, s.ev_status, s.ev_d2h})
    if (ev) cudaEventDestroy(ev);
  s = PipeSlot{};
}

}  // namespace

struct sst_host_pipe {
  cudaStream_t h2d = nullptr, comp = nullptr, stat = nullptr, d2h = nullptr;
  sst::Scratch scratch;  // the kernels' scratch, shared by the slots (one chunk runs at a time)
  PipeSlot slots[kSlots];
  // worker
  sst_ctx* ctx = nullptr;
  std::mutex mu;
  std::condition_variable cv_work, cv_done;
  std::thread worker;
  bool stop = false;
  std::deque<HostJob*> queue;            // batches with chunks still to issue, in order
  std::map<uint64_t, HostJob*> jobs;     // every batch not yet waited for
  uint64_t next_ticket = 1;
  uint64_t issued = 0, retired = 0;      // chunks issued / finished; chunk g uses slot g % kSlots
  cudaError_t fatal = cudaSuccess;       // a CUDA error ends the pipeline; later calls report it
};

namespace sst {

void free_host_pipe(sst_ctx* ctx) {
  sst_host_pipe* p = ctx->pipe;
  if (!p) return;
  {
    std::lock_guard<std::mutex> lock(p->mu);
    p->stop = true;
  }
  p->cv_work.notify_all();
  if (p->worker.joinable()) p->worker.join();
  for (auto& kv : p->jobs) {
    if (kv.second->done) cudaEventDestroy(kv.second->done);
    delete kv.second;
  }
  for (cudaStream_t st : {p->h2d, p->comp, p->stat, p->d2h})
    if (st) cudaStreamSynchronize(st);
  for (PipeSlot& s : p->slots) free_slot(s);
  sst::free_scratch(p->scratch);
  for (cudaStream_t st : {p->h2d, p->comp, p->stat, p->d2h})
    if (st) cudaStreamDestroy(st);
  delete p;
  ctx->pipe = nullptr;
}

}  // namespace sst

namespace {

// Enqueues chunk c on slot s: host staging of the rebased offsets, the H2D
// copies, the batched kernels in packed mode and the D2H of statuses and
// pack_off, with the events that order them across the three streams.
cudaError_t enqueue_chunk(sst_ctx* ctx, sst_host_pipe& p, PipeSlot& s, HostJob* job, size_t ci) {
  const Chunk& c = job->chunks[ci];
  const uint8_t* raw = job->raw;
  const uint64_t* event_off = job->event_off;
  const uint32_t* fed_len = job->fed_len;
  const uint32_t nf = job->n_feds;
  const uint32_t E = c.e1 - c.e0;
  uint64_t co = 0;
  for (uint32_t i = 0; i <= E; i++) {
    s.h_event_off[i] = event_off[c.e0 + i] - c.base;
    s.h_clu_off[i] = co;
    if (i < E) co += (event_off[c.e0 + i + 1] - event_off[c.e0 + i]) / 2 + 1;
  }
  cudaError_t e;
  // inputs, once the slot's previous chunk has finished reading them
  if ((e = cudaStreamWaitEvent(p.h2d, s.ev_comp, 0))) return e;
  if ((e = cudaMemcpyAsync(s.d_raw, raw + c.base, c.bytes, cudaMemcpyHostToDevice, p.h2d))) return e;
  if ((e = cudaMemcpyAsync(s.d_fed_len, fed_len + (size_t)c.e0 * nf, (size_t)E * nf * sizeof(uint32_t),
                           cudaMemcpyHostToDevice, p.h2d)))
    return e;
  if ((e = cudaMemcpyAsync(s.d_event_off, s.h_event_off, (E + 1) * sizeof(uint64_t), cudaMemcpyHostToDevice, p.h2d)))
    return e;
  if ((e = cudaMemcpyAsync(s.d_clu_off, s.h_clu_off, (E + 1) * sizeof(uint64_t), cudaMemcpyHostToDevice, p.h2d)))
    return e;
  if (job->amps) {  // the events' amplitude slices, rebased to the chunk's first byte
    for (uint32_t i = 0; i <= E; i++) s.h_amp_off[i] = job->out.amp_off[c.e0 + i] - c.amp_base;
    if ((e = cudaMemcpyAsync(s.d_amp_off, s.h_amp_off, (E + 1) * sizeof(uint64_t), cudaMemcpyHostToDevice, p.h2d)))
      return e;
  }
  if ((e = cudaEventRecord(s.ev_h2d, p.h2d))) return e;
  // kernels, once the inputs are in and the slot's previous clusters are out
  if ((e = cudaStreamWaitEvent(p.comp, s.ev_h2d, 0))) return e;
  if ((e = cudaStreamWaitEvent(p.comp, s.ev_d2h, 0))) return e;
  sst_clusters out{};
  out.det = s.d_det;
  out.first = s.d_first;
  out.width = s.d_width;
  out.charge = s.d_charge;
  out.barycenter = s.d_bary;
  out.capacity = c.clu_total;
  if (job->amps) {
    out.amp = s.d_amp;
    out.amp_first = s.d_amp_first;
    out.amp_off = s.d_amp_off;
    out.amp_capacity = c.amp_bytes ? c.amp_bytes : 1;
  }
  if ((e = sst::launch_batch(s.d_raw, s.d_event_off, s.d_fed_len, E, nf, s.d_clu_off, out, s.d_status,
                             sst::kparams(ctx), p.scratch, ctx->shape, ctx->n_sm, p.comp, s.d_pack_off)))
    return e;
  // amp_first: from the chunk's arena to the caller's array
  if (job->amps && c.amp_base &&
      (e = sst::rebase_amp_first(s.d_amp_first, s.d_pack_off + E, (uint32_t)c.amp_base, ctx->n_sm, p.comp)))
    return e;
  if ((e = cudaEventRecord(s.ev_comp, p.comp))) return e;
  // statuses and event starts back to the host
  if ((e = cudaStreamWaitEvent(p.stat, s.ev_comp, 0))) return e;
  if ((e = cudaMemcpyAsync(s.h_status, s.d_status, E * sizeof(sst_event_status), cudaMemcpyDeviceToHost, p.stat)))
    return e;
  if ((e = cudaMemcpyAsync(s.h_pack_off, s.d_pack_off, (E + 1) * sizeof(uint64_t), cudaMemcpyDeviceToHost, p.stat)))
    return e;
  if ((e = cudaEventRecord(s.ev_status, p.stat))) return e;
  s.job = job;
  s.chunk = ci;
  return cudaSuccess;
}

// Waits for slot s's statuses, writes them and the event starts, and enqueues
// the D2H copies of the chunk's clusters at the job's next position in the
// caller's arrays (truncated to out.capacity, the cut events flagged).  After a
// job's last chunk, writes event_first[n_events] and records the job's event.
cudaError_t finish_chunk(sst_host_pipe& p, PipeSlot& s) {
  HostJob* job = s.job;
  if (!job) return cudaSuccess;
  const Chunk& c = job->chunks[s.chunk];
  cudaError_t e = cudaEventSynchronize(s.ev_status);
  if (e) return e;
  const sst_clusters* out = &job->out;
  const uint32_t E = c.e1 - c.e0;
  const uint64_t total = s.h_pack_off[E];
  const uint64_t room = out->capacity > job->pos ? out->capacity - job->pos : 0;
  const uint64_t stored = total < room ? total : room;
  for (uint32_t i = 0; i < E; i++) {
    sst_event_status st = s.h_status[i];
    const uint64_t a = s.h_pack_off[i];
    const uint64_t b = a + st.n_clusters;
    if (b > stored) {
      st.n_clusters = (uint32_t)(a < stored ? stored - a : 0);
      st.flags |= SST_EV_CLUSTER_CAPACITY;
    }
    job->status[c.e0 + i] = st;
    job->event_first[c.e0 + i] = job->pos + (a < stored ? a : stored);
  }
  if (stored) {
    const uint64_t q = job->pos;
    if ((e = cudaMemcpyAsync(out->det + q, s.d_det, stored * 4, cudaMemcpyDeviceToHost, p.d2h))) return e;
    if ((e = cudaMemcpyAsync(out->first + q, s.d_first, stored * 2, cudaMemcpyDeviceToHost, p.d2h))) return e;
    if ((e = cudaMemcpyAsync(out->width + q, s.d_width, stored * 2, cudaMemcpyDeviceToHost, p.d2h))) return e;
    if ((e = cudaMemcpyAsync(out->charge + q, s.d_charge, stored * 4, cudaMemcpyDeviceToHost, p.d2h))) return e;
    if ((e = cudaMemcpyAsync(out->barycenter + q, s.d_bary, stored * 4, cudaMemcpyDeviceToHost, p.d2h))) return e;
    if (job->amps &&
        (e = cudaMemcpyAsync(out->amp_first + q, s.d_amp_first, stored * 4, cudaMemcpyDeviceToHost, p.d2h)))
      return e;
  }
  if (job->amps && c.amp_bytes &&
      (e = cudaMemcpyAsync(out->amp + c.amp_base, s.d_amp, c.amp_bytes, cudaMemcpyDeviceToHost, p.d2h)))
    return e;
  if ((e = cudaEventRecord(s.ev_d2h, p.d2h))) return e;
  job->pos += stored;
  s.job = nullptr;
  if (++job->finished == job->chunks.size()) {
    job->event_first[job->n_events] = job->pos;
    if ((e = cudaEventRecord(job->done, p.d2h))) return e;
    {
      std::lock_guard<std::mutex> lock(p.mu);
      job->recorded = true;
    }
    p.cv_done.notify_all();
  }
  std::lock_guard<std::mutex> lock(p.mu);
  p.retired++;
  return cudaSuccess;
}

// Chunk boundaries: with a tuned chunk size, equal chunks; otherwise chunks of
// about a quarter of the batch (at most 32 events), except that the first and
// the last are a quarter of that, so that the copies nothing overlaps (the first
// chunk's inputs, the last chunk's clusters) stay short.
std::vector<uint32_t> plan_chunks(uint32_t n_events, int tuned) {
  std::vector<uint32_t> cut{0};
  if (tuned > 0) {
    for (uint32_t e = 0; e < n_events;) {
      e = e + (uint32_t)tuned < n_events ? e + (uint32_t)tuned : n_events;
      cut.push_back(e);
    }
    return cut;
  }
  uint32_t per = (n_events + 3) / 4;
  if (per > 32) per = 32;
  const uint32_t edge = per / 4 ? per / 4 : 1;
  uint32_t e = n_events < edge ? n_events : edge;
  cut.push_back(e);
  while (n_events - e > per + edge) {
    e += per;
    cut.push_back(e);
  }
  if (n_events - e > edge) cut.push_back(n_events - edge);
  if (cut.back() != n_events) cut.push_back(n_events);
  return cut;
}

// Finishes every chunk in flight, in order, and waits for all copies.
cudaError_t drain(sst_host_pipe& p) {
  cudaError_t e = cudaSuccess;
  while (!e) {
    uint64_t r, n;
    {
      std::lock_guard<std::mutex> lock(p.mu);
      r = p.retired;
      n = p.issued;
    }
    if (r == n) break;
    e = finish_chunk(p, p.slots[r % kSlots]);
  }
  for (cudaStream_t st : {p.h2d, p.comp, p.stat, p.d2h})
    if (!e) e = cudaStreamSynchronize(st);
  return e;
}

// Before a job's first chunk: grow the arenas when the job needs more than they
// hold (after draining the pipeline, so that no chunk in flight uses them).
cudaError_t prepare_job(sst_host_pipe& p, const HostJob* job) {
  const uint32_t nf = job->n_feds;
  bool fits = p.scratch.items_cap >= (size_t)job->max_e * nf * sst::kFe && p.scratch.ev_cap >= job->max_e &&
              p.scratch.stage_cap >= job->max_clu;
  const uint64_t amp = job->amps ? (job->max_amp ? job->max_amp : 1) : 0;
  if (amp)
    fits = fits && p.scratch.amp_items_cap >= (size_t)job->max_e * nf * sst::kFe && p.scratch.amp_ev_cap >= job->max_e &&
           p.scratch.amp_stage_cap >= amp;
  for (const PipeSlot& s : p.slots) fits = fits && slot_fits(s, job->max_e, nf, job->max_bytes, job->max_clu, amp);
  if (fits) return cudaSuccess;
  cudaError_t e = drain(p);
  if (!e) e = sst::ensure_scratch(p.scratch, (size_t)job->max_e * nf * sst::kFe, job->max_e, job->max_clu);
  if (!e) e = sst::ensure_spill(p.scratch, (size_t)p.ctx->n_sm * sst::kMaxWarpsPerSm);
  if (!e && amp) e = sst::ensure_amp_scratch(p.scratch, (size_t)job->max_e * nf * sst::kFe, job->max_e, amp);
  for (PipeSlot& s : p.slots)
    if (!e) e = grow_slot(s, job->max_e, nf, job->max_bytes, job->max_clu, amp);
  return e;
}

// Marks every job not yet complete as failed with e; the pipeline stays failed.
void fail_all(sst_host_pipe& p, cudaError_t e) {
  {
    std::lock_guard<std::mutex> lock(p.mu);
    p.fatal = e;
    for (auto& kv : p.jobs)
      if (!kv.second->recorded) kv.second->err = e;
    p.queue.clear();
    p.issued = p.retired;
  }
  for (PipeSlot& s : p.slots) s.job = nullptr;
  p.cv_done.notify_all();
}

// The worker: issues the queued jobs' chunks in order, each into the slot whose
// previous chunk it first finishes; with nothing left to issue, finishes the
// chunks still in flight.
void pipe_main(sst_host_pipe* p) {
  cudaSetDevice(p->ctx->device);
  for (;;) {
    HostJob* job = nullptr;
    bool in_flight;
    {
      std::unique_lock<std::mutex> lock(p->mu);
      p->cv_work.wait(lock, [&] { return p->stop || !p->queue.empty() || p->retired < p->issued; });
      in_flight = p->retired < p->issued;
      if (p->queue.empty() && !in_flight) return;  // stop requested, nothing left
      if (!p->queue.empty()) job = p->queue.front();
    }
    cudaError_t e = cudaSuccess;
    if (job) {
      if (job->next == 0) e = prepare_job(*p, job);
      if (!e) {
        uint64_t g;
        {
          std::lock_guard<std::mutex> lock(p->mu);
          g = p->issued;
        }
        PipeSlot& s = p->slots[g % kSlots];
        if (s.job) e = finish_chunk(*p, s);  // the chunk issued kSlots before
        if (!e) e = enqueue_chunk(p->ctx, *p, s, job, job->next);
        if (!e) {
          std::lock_guard<std::mutex> lock(p->mu);
          job->next++;
          p->issued++;
          if (job->next == job->chunks.size()) p->queue.pop_front();
        }
      }
    } else {
      uint64_t r;
      {
        std::lock_guard<std::mutex> lock(p->mu);
        r = p->retired;
      }
      e = finish_chunk(*p, p->slots[r % kSlots]);
    }
    if (e) fail_all(*p, e);
  }
}

}  // namespace

namespace sst {
uint32_t host_chunks(uint32_t n_events, int tuned) { return (uint32_t)plan_chunks(n_events, tuned).size() - 1; }
}  // namespace sst

using namespace sst;

extern "C" {

sst_status sst_batch_host_submit(sst_ctx* ctx, const uint8_t* raw, const uint64_t* event_off,
                                 const uint32_t* fed_len, uint32_t n_events, uint32_t n_feds,
                                 const sst_clusters* out, uint64_t* event_first, sst_event_status* status,
                                 uint64_t* ticket) {
  if (!ctx) return SST_ERR_INVALID_ARG;
  if (!ctx->has_calib) return set_err(ctx, SST_ERR_NO_CALIB, "sst_batch_host: no calibration");
  if (!raw || !event_off || !fed_len || !out || !event_first || !status || !ticket || !out->det || !out->first ||
      !out->width || !out->charge || !out->barycenter)
    return set_err(ctx, SST_ERR_INVALID_ARG, "sst_batch_host: null pointer");
  if (n_events == 0 || n_feds == 0 || n_feds > ctx->n_feds)
    return set_err(ctx, SST_ERR_INVALID_ARG, "sst_batch_host: bad n_events / n_feds");
  for (uint32_t i = 0; i < n_events; i++)
    if (event_off[i + 1] < event_off[i])
      return set_err(ctx, SST_ERR_INVALID_ARG, "sst_batch_host: event_off decreases");
  if (out->amp) {
    bool ok = out->amp_first && out->amp_off && out->amp_capacity > 0 && out->amp_capacity < kNoAmp &&
              out->amp_off[n_events] <= out->amp_capacity;
    for (uint32_t i = 0; ok && i < n_events; i++) ok = out->amp_off[i + 1] >= out->amp_off[i];
    if (!ok)
      return set_err(ctx, SST_ERR_INVALID_ARG,
                     "sst_batch_host: amp needs amp_first and a non-decreasing host amp_off within "
                     "1 <= amp_capacity < 2^32 - 1");
  }
  auto* job = new HostJob();
  job->raw = raw;
  job->event_off = event_off;
  job->fed_len = fed_len;
  job->n_events = n_events;
  job->n_feds = n_feds;
  job->out = *out;
  job->event_first = event_first;
  job->status = status;
  job->amps = out->amp != nullptr;
  // chunks of consecutive events
  const std::vector<uint32_t> cut = plan_chunks(n_events, ctx->shape.host_chunk);
  for (size_t k = 0; k + 1 < cut.size(); k++) {
    const uint32_t e0 = cut[k], e1 = cut[k + 1];
    Chunk c{e0, e1, event_off[e0] & ~15ull, 0, 0};
    c.bytes = event_off[e1] - c.base;
    if (job->amps) {
      c.amp_base = out->amp_off[e0];
      c.amp_bytes = out->amp_off[e1] - c.amp_base;
      if (c.amp_bytes > job->max_amp) job->max_amp = c.amp_bytes;
    }
    for (uint32_t i = e0; i < e1; i++) c.clu_total += (event_off[i + 1] - event_off[i]) / 2 + 1;
    job->chunks.push_back(c);
    if (e1 - e0 > job->max_e) job->max_e = e1 - e0;
    if (c.bytes > job->max_bytes) job->max_bytes = c.bytes;
    if (c.clu_total > job->max_clu) job->max_clu = c.clu_total;
  }
  if ((uint64_t)job->max_e * n_feds * sst::kFe >= (1ull << 31)) {
    delete job;
    return set_err(ctx, SST_ERR_INVALID_ARG, "sst_batch_host: too many FE units in one chunk (2^31)");
  }
  DeviceGuard g(ctx->device);
  cudaError_t e = cudaEventCreateWithFlags(&job->done, cudaEventDisableTiming);
  if (e) {
    delete job;
    return cuda_err(ctx, e, "sst_batch_host event");
  }
  sst_host_pipe* p;
  {
    std::lock_guard<std::mutex> lock(ctx->mu);  // creates the pipeline once
    if (!ctx->pipe) {
      p = new sst_host_pipe();
      p->ctx = ctx;
      for (cudaStream_t* st : {&p->h2d, &p->comp, &p->stat, &p->d2h})
        if (!e && !*st) e = cudaStreamCreateWithFlags(st, cudaStreamNonBlocking);
      if (!e) {
        ctx->pipe = p;
        p->worker = std::thread(pipe_main, p);
      } else {
        for (cudaStream_t st : {p->h2d, p->comp, p->stat, p->d2h})
          if (st) cudaStreamDestroy(st);
        delete p;
      }
    }
    p = ctx->pipe;
  }
  if (e) {
    cudaEventDestroy(job->done);
    delete job;
    return cuda_err(ctx, e, "sst_batch_host streams");
  }
  {
    std::lock_guard<std::mutex> lock(p->mu);
    if (p->fatal) {
      cudaEventDestroy(job->done);
      delete job;
      return cuda_err(ctx, p->fatal, "sst_batch_host (an earlier batch failed)");
    }
    job->ticket = p->next_ticket++;
    *ticket = job->ticket;
    p->jobs[job->ticket] = job;
    p->queue.push_back(job);
  }
  p->cv_work.notify_all();
  return SST_OK;
}

sst_status sst_batch_host_wait(sst_ctx* ctx, uint64_t ticket) {
  if (!ctx) return SST_ERR_INVALID_ARG;
  sst_host_pipe* p = ctx->pipe;
  if (!p) return set_err(ctx, SST_ERR_INVALID_ARG, "sst_batch_host_wait: unknown ticket");
  HostJob* job;
  {
    std::unique_lock<std::mutex> lock(p->mu);
    auto it = p->jobs.find(ticket);
    if (it == p->jobs.end()) return set_err(ctx, SST_ERR_INVALID_ARG, "sst_batch_host_wait: unknown ticket");
    job = it->second;
    p->cv_done.wait(lock, [&] { return job->recorded || job->err != cudaSuccess; });
  }
  cudaError_t e = job->err;
  if (!e) e = cudaEventSynchronize(job->done);
  {
    std::lock_guard<std::mutex> lock(p->mu);
    p->jobs.erase(ticket);
  }
  cudaEventDestroy(job->done);
  delete job;
  return cuda_err(ctx, e, "sst_batch_host");
}

sst_status sst_batch_host(sst_ctx* ctx, const uint8_t* raw, const uint64_t* event_off, const uint32_t* fed_len,
                          uint32_t n_events, uint32_t n_feds, const sst_clusters* out, uint64_t* event_first,
                          sst_event_status* status) {
  uint64_t t = 0;
  const sst_status r = sst_batch_host_submit(ctx, raw, event_off, fed_len, n_events, n_feds, out, event_first, status,
                                             &t);
  return r == SST_OK ? sst_batch_host_wait(ctx, t) : r;
}

}  // extern "C"

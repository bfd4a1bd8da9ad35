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
// Device arenas grow on demand (a cudaMalloc only when a call needs more than
// any call before it on this context) and live until sst_destroy.
#include <cstring>
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
  // the chunk in flight: events [e0, e1), or e1 == e0 when the slot is idle
  uint32_t e0 = 0, e1 = 0;
};

// One chunk's sizes.
struct Chunk {
  uint32_t e0, e1;
  uint64_t base;       // first raw byte copied (event_off[e0] rounded down to 16)
  uint64_t bytes;      // raw bytes copied
  uint64_t clu_total;  // staging records (sum over events of bytes / 2 + 1)
};

cudaError_t grow_slot(PipeSlot& s, uint32_t E, uint32_t nf, uint64_t bytes, uint64_t clu) {
  cudaError_t e;
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
  for (cudaEvent_t ev : {s.ev_h2d, s.ev_comp, s.ev_status, s.ev_d2h})
    if (ev) cudaEventDestroy(ev);
  s = PipeSlot{};
}

}  // namespace

struct sst_host_pipe {
  cudaStream_t h2d = nullptr, comp = nullptr, stat = nullptr, d2h = nullptr;
  sst::Scratch scratch;  // the kernels' scratch, shared by the slots (one chunk runs at a time)
  PipeSlot slots[kSlots];
};

namespace sst {

void free_host_pipe(sst_ctx* ctx) {
  sst_host_pipe* p = ctx->pipe;
  if (!p) return;
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
cudaError_t enqueue_chunk(sst_ctx* ctx, sst_host_pipe& p, PipeSlot& s, const Chunk& c, const uint8_t* raw,
                          const uint64_t* event_off, const uint32_t* fed_len, uint32_t nf) {
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
  if ((e = sst::launch_batch(s.d_raw, s.d_event_off, s.d_fed_len, E, nf, s.d_clu_off, out, s.d_status,
                             sst::kparams(ctx), p.scratch, ctx->shape, ctx->n_sm, p.comp, s.d_pack_off)))
    return e;
  if ((e = cudaEventRecord(s.ev_comp, p.comp))) return e;
  // statuses and event starts back to the host
  if ((e = cudaStreamWaitEvent(p.stat, s.ev_comp, 0))) return e;
  if ((e = cudaMemcpyAsync(s.h_status, s.d_status, E * sizeof(sst_event_status), cudaMemcpyDeviceToHost, p.stat)))
    return e;
  if ((e = cudaMemcpyAsync(s.h_pack_off, s.d_pack_off, (E + 1) * sizeof(uint64_t), cudaMemcpyDeviceToHost, p.stat)))
    return e;
  if ((e = cudaEventRecord(s.ev_status, p.stat))) return e;
  s.e0 = c.e0;
  s.e1 = c.e1;
  return cudaSuccess;
}

// Waits for slot s's statuses, writes them and the event starts, and enqueues
// the D2H copies of the chunk's clusters at *pos in the caller's arrays
// (truncated to out->capacity, the cut events flagged).
cudaError_t finish_chunk(sst_host_pipe& p, PipeSlot& s, const sst_clusters* out, uint64_t* event_first,
                         sst_event_status* status, uint64_t* pos) {
  if (s.e1 == s.e0) return cudaSuccess;
  cudaError_t e = cudaEventSynchronize(s.ev_status);
  if (e) return e;
  const uint32_t E = s.e1 - s.e0;
  const uint64_t total = s.h_pack_off[E];
  const uint64_t room = out->capacity > *pos ? out->capacity - *pos : 0;
  const uint64_t stored = total < room ? total : room;
  for (uint32_t i = 0; i < E; i++) {
    sst_event_status st = s.h_status[i];
    const uint64_t a = s.h_pack_off[i];
    const uint64_t b = a + st.n_clusters;
    if (b > stored) {
      st.n_clusters = (uint32_t)(a < stored ? stored - a : 0);
      st.flags |= SST_EV_CLUSTER_CAPACITY;
    }
    status[s.e0 + i] = st;
    event_first[s.e0 + i] = *pos + (a < stored ? a : stored);
  }
  if (stored) {
    const uint64_t q = *pos;
    if ((e = cudaMemcpyAsync(out->det + q, s.d_det, stored * 4, cudaMemcpyDeviceToHost, p.d2h))) return e;
    if ((e = cudaMemcpyAsync(out->first + q, s.d_first, stored * 2, cudaMemcpyDeviceToHost, p.d2h))) return e;
    if ((e = cudaMemcpyAsync(out->width + q, s.d_width, stored * 2, cudaMemcpyDeviceToHost, p.d2h))) return e;
    if ((e = cudaMemcpyAsync(out->charge + q, s.d_charge, stored * 4, cudaMemcpyDeviceToHost, p.d2h))) return e;
    if ((e = cudaMemcpyAsync(out->barycenter + q, s.d_bary, stored * 4, cudaMemcpyDeviceToHost, p.d2h))) return e;
  }
  if ((e = cudaEventRecord(s.ev_d2h, p.d2h))) return e;
  *pos += stored;
  s.e0 = s.e1 = 0;
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

}  // namespace

using namespace sst;

extern "C" sst_status sst_batch_host(sst_ctx* ctx, const uint8_t* raw, const uint64_t* event_off,
                                     const uint32_t* fed_len, uint32_t n_events, uint32_t n_feds,
                                     const sst_clusters* out, uint64_t* event_first, sst_event_status* status) {
  if (!ctx) return SST_ERR_INVALID_ARG;
  if (!ctx->has_calib) return set_err(ctx, SST_ERR_NO_CALIB, "sst_batch_host: no calibration");
  if (!raw || !event_off || !fed_len || !out || !event_first || !status || !out->det || !out->first ||
      !out->width || !out->charge || !out->barycenter)
    return set_err(ctx, SST_ERR_INVALID_ARG, "sst_batch_host: null pointer");
  if (n_events == 0 || n_feds == 0 || n_feds > ctx->n_feds)
    return set_err(ctx, SST_ERR_INVALID_ARG, "sst_batch_host: bad n_events / n_feds");
  if (out->amp)
    return set_err(ctx, SST_ERR_INVALID_ARG, "sst_batch_host: amplitudes are produced by sst_batch and sst_cluster");
  for (uint32_t i = 0; i < n_events; i++)
    if (event_off[i + 1] < event_off[i])
      return set_err(ctx, SST_ERR_INVALID_ARG, "sst_batch_host: event_off decreases");
  // chunks of consecutive events
  const std::vector<uint32_t> cut = plan_chunks(n_events, ctx->shape.host_chunk);
  std::vector<Chunk> chunks;
  uint32_t max_e = 0;
  uint64_t max_bytes = 0, max_clu = 0;
  for (size_t k = 0; k + 1 < cut.size(); k++) {
    const uint32_t e0 = cut[k], e1 = cut[k + 1];
    Chunk c{e0, e1, event_off[e0] & ~15ull, 0, 0};
    c.bytes = event_off[e1] - c.base;
    for (uint32_t i = e0; i < e1; i++) c.clu_total += (event_off[i + 1] - event_off[i]) / 2 + 1;
    chunks.push_back(c);
    if (e1 - e0 > max_e) max_e = e1 - e0;
    if (c.bytes > max_bytes) max_bytes = c.bytes;
    if (c.clu_total > max_clu) max_clu = c.clu_total;
  }
  if ((uint64_t)max_e * n_feds >= (1ull << 31))
    return set_err(ctx, SST_ERR_INVALID_ARG, "sst_batch_host: too many FED records in one chunk");
  std::lock_guard<std::mutex> lock(ctx->mu);
  DeviceGuard g(ctx->device);
  cudaError_t e = cudaSuccess;
  if (!ctx->pipe) ctx->pipe = new sst_host_pipe();
  sst_host_pipe& p = *ctx->pipe;
  for (cudaStream_t* st : {&p.h2d, &p.comp, &p.stat, &p.d2h})
    if (!e && !*st) e = cudaStreamCreateWithFlags(st, cudaStreamNonBlocking);
  if (!e) e = ensure_scratch(p.scratch, (size_t)max_e * n_feds * kFe, max_e, max_clu);
  PipeSlot* slots = p.slots;
  const int used = chunks.size() < (size_t)kSlots ? (int)chunks.size() : kSlots;
  for (int k = 0; k < used && !e; k++) e = grow_slot(slots[k], max_e, n_feds, max_bytes, max_clu);
  uint64_t pos = 0;
  for (size_t j = 0; j < chunks.size() && !e; j++) {
    PipeSlot& s = slots[j % kSlots];
    e = finish_chunk(p, s, out, event_first, status, &pos);
    if (!e) e = enqueue_chunk(ctx, p, s, chunks[j], raw, event_off, fed_len, n_feds);
  }
  // the remaining chunks, in order, then every copy
  for (size_t j = chunks.size() > (size_t)kSlots ? chunks.size() - kSlots : 0; j < chunks.size() && !e; j++)
    e = finish_chunk(p, slots[j % kSlots], out, event_first, status, &pos);
  for (cudaStream_t st : {p.h2d, p.comp, p.stat, p.d2h}) {
    const cudaError_t q = st ? cudaStreamSynchronize(st) : cudaSuccess;
    if (!e) e = q;
  }
  for (int k = 0; k < kSlots; k++) slots[k].e0 = slots[k].e1 = 0;
  if (e) return cuda_err(ctx, e, "sst_batch_host");
  event_first[n_events] = pos;
  return SST_OK;
}

// sst_api.cu -- host side of the C ABI declared in include/sst.h: contexts,
// calibration upload (arXiv 2101.11489 section 2: noise and gain per strip, here
// plus the bad-strip list), argument checks and kernel launches.
#include <chrono>
#include <cmath>
#include <cstring>
#include <vector>

#include "sst_internal.h"

namespace sst {

sst_status set_err(sst_ctx* c, sst_status code, const std::string& msg) {
  if (c) c->err = msg;
  return code;
}

sst_status cuda_err(sst_ctx* c, cudaError_t e, const char* where) {
  if (e == cudaSuccess) return SST_OK;
  return set_err(c, SST_ERR_CUDA, std::string(where) + ": " + cudaGetErrorString(e));
}

KParams kparams(const sst_ctx* c) {
  KParams k;
  k.t_cluster = c->params.t_cluster;
  k.max_holes = c->params.max_seq_holes;
  k.max_bad = c->params.max_seq_bad;
  k.max_adj = c->params.max_adj_bad;
  k.calq = c->calq;
  k.badmask = c->badmask;
  k.qmul = c->qmul;
  return k;
}

// Gain-corrected charge of a non-saturated ADC (section 2: charge corrected by the
// strip's gain): the ADC divided by the APV gain, rounded half up, capped at 254;
// each operation one binary32 rounding.  `mul` selects the form the kernels use
// with a certified multiplier m: the ADC times m instead of divided by the gain.
static uint32_t charge_of(uint32_t adc, float g, bool mul) {
  const float a = (float)adc;
  const float x = mul ? a * g : a / g;
  const float y = x + 0.5f;
  return y >= 254.0f ? 254u : (uint32_t)y;  // (uint32_t)y truncates; y >= 0
}

// A multiplier for one APV: the binary32 reciprocal of the gain, or a neighbour of
// it within a few units in the last place, that gives exactly the quotient form's
// charge for every ADC 0..253 (checked here, exhaustively).  When none does, -gain:
// the kernels then divide.  Needs binary32 arithmetic without contraction (the
// library's host code is compiled with -ffp-contract=off).
static float certified_multiplier(float g) {
  uint32_t want[254];
  for (uint32_t a = 0; a < 254; a++) want[a] = charge_of(a, g, false);
  const float r = 1.0f / g;
  float cand[9];
  cand[0] = r;
  float up = r, dn = r;
  for (int k = 1; k <= 4; k++) {
    up = std::nextafter(up, INFINITY);
    dn = std::nextafter(dn, 0.0f);
    cand[2 * k - 1] = up;
    cand[2 * k] = dn;
  }
  for (float m : cand) {
    if (!(m > 0.f) || !std::isfinite(m)) continue;
    bool ok = true;
    for (uint32_t a = 1; a < 254 && ok; a++) ok = charge_of(a, m, true) == want[a];
    if (ok) return m;
  }
  return -g;
}

template <typename T>
static cudaError_t grow(T*& p, size_t& cap, size_t need) {
  if (need <= cap) return cudaSuccess;
  if (p) cudaFree(p);
  p = nullptr;
  cap = 0;
  cudaError_t e = cudaMalloc(&p, need * sizeof(T));
  if (e == cudaSuccess) cap = need;
  return e;
}

cudaError_t ensure_scratch(Scratch& s, size_t items, size_t events, size_t stage_records) {
  cudaError_t e = cudaSuccess;
  if (!s.tickets) {
    if ((e = cudaMalloc(&s.tickets, 16 * sizeof(uint32_t)))) return e;
    if ((e = cudaMemset(s.tickets, 0, 16 * sizeof(uint32_t)))) return e;
  }
  items = items ? items : 1;
  events = events ? events : 1;
  stage_records = stage_records ? stage_records : 1;
  if (items > s.items_cap || events > s.ev_cap || stage_records > s.stage_cap) {
    // growing: wait for all work that may still use the old buffers
    if ((e = cudaDeviceSynchronize())) return e;
    if (items > s.items_cap) {
      size_t cap = s.items_cap, c2 = s.items_cap, c3 = s.items_cap, c4 = s.items_cap, c5 = s.items_cap;
      size_t c6 = s.items_cap, c7 = s.items_cap;
      if ((e = grow(s.lb, cap, items))) return e;
      if ((e = grow(s.fed_off, c2, items))) return e;
      if ((e = grow(s.fed_cnt, c3, items))) return e;
      if ((e = grow(s.fed_start, c4, items))) return e;
      if ((e = grow(s.fed_dest, c5, items))) return e;
      if ((e = grow(s.unit_desc, c6, items))) return e;
      if ((e = grow(s.big_list, c7, items))) return e;
      s.items_cap = items;
    }
    if ((e = grow(s.ev_alloc, s.ev_cap, events))) return e;
    if ((e = grow(s.stage, s.stage_cap, stage_records))) return e;
  }
  return cudaSuccess;
}

cudaError_t ensure_spill(Scratch& s, size_t warps) {
  if (warps <= s.spill_warps) return cudaSuccess;
  cudaError_t e = cudaDeviceSynchronize();  // growing: wait for all work that may still use the old area
  if (e) return e;
  if (s.spill) cudaFree(s.spill);
  s.spill = nullptr;
  s.spill_warps = 0;
  if ((e = cudaMalloc(&s.spill, warps * kSpillRecords * sizeof(uint4)))) return e;
  s.spill_warps = warps;
  return cudaSuccess;
}

cudaError_t ensure_amp_scratch(Scratch& s, size_t items, size_t events, size_t amp_bytes) {
  items = items ? items : 1;
  events = events ? events : 1;
  amp_bytes = amp_bytes ? amp_bytes : 1;
  if (items <= s.amp_items_cap && events <= s.amp_ev_cap && amp_bytes <= s.amp_stage_cap) return cudaSuccess;
  cudaError_t e = cudaDeviceSynchronize();  // growing: wait for all work that may still use the old buffers
  if (e) return e;
  if (items > s.amp_items_cap) {
    size_t c1 = s.amp_items_cap, c2 = s.amp_items_cap, c3 = s.amp_items_cap;
    if ((e = grow(s.seg_amp_cnt, c1, items))) return e;
    if ((e = grow(s.seg_amp_start, c2, items))) return e;
    if ((e = grow(s.seg_amp_dest, c3, items))) return e;
    s.amp_items_cap = items;
  }
  if ((e = grow(s.amp_alloc, s.amp_ev_cap, events))) return e;
  return grow(s.amp_stage, s.amp_stage_cap, amp_bytes);
}

void free_scratch(Scratch& s) {
  if (s.lb) cudaFree(s.lb);
  if (s.fed_off) cudaFree(s.fed_off);
  if (s.fed_cnt) cudaFree(s.fed_cnt);
  if (s.fed_start) cudaFree(s.fed_start);
  if (s.fed_dest) cudaFree(s.fed_dest);
  if (s.unit_desc) cudaFree(s.unit_desc);
  if (s.big_list) cudaFree(s.big_list);
  if (s.ev_alloc) cudaFree(s.ev_alloc);
  if (s.stage) cudaFree(s.stage);
  if (s.tickets) cudaFree(s.tickets);
  if (s.spill) cudaFree(s.spill);
  for (void* p : {(void*)s.amp_stage, (void*)s.amp_alloc, (void*)s.seg_amp_cnt, (void*)s.seg_amp_start,
                  (void*)s.seg_amp_dest})
    if (p) cudaFree(p);
  s = Scratch{};
}

static bool params_ok(const sst_params* p) {
  if (!p) return false;
  auto fin = [](float x) { return std::isfinite(x); };
  return fin(p->t_channel) && fin(p->t_seed) && fin(p->t_cluster) && p->t_channel > 0.f &&
         p->t_seed >= p->t_channel && p->t_cluster >= 0.f && p->reserved == 0;
}

}  // namespace sst

using namespace sst;

extern "C" {

sst_status sst_create(sst_ctx** out, int device, uint32_t n_feds) {
  if (!out) return SST_ERR_INVALID_ARG;
  *out = nullptr;
  if (n_feds == 0 || n_feds > SST_MAX_FEDS) return SST_ERR_INVALID_ARG;
  int count = 0;
  if (cudaGetDeviceCount(&count) != cudaSuccess || device < 0 || device >= count) return SST_ERR_CUDA;
  auto* c = new sst_ctx();
  c->device = device;
  c->n_feds = n_feds;
  c->shape = default_shape();
  DeviceGuard g(device);
  cudaError_t e = cudaDeviceGetAttribute(&c->n_sm, cudaDevAttrMultiProcessorCount, device);
  if (e == cudaSuccess) e = ensure_scratch(c->scratch, (size_t)n_feds, 1, 1);
  if (e != cudaSuccess) {
    free_scratch(c->scratch);
    delete c;
    return SST_ERR_CUDA;
  }
  *out = c;
  return SST_OK;
}

sst_status sst_server_stop(sst_ctx* ctx);

sst_status sst_destroy(sst_ctx* ctx) {
  if (!ctx) return SST_ERR_INVALID_ARG;
  if (ctx->server) sst_server_stop(ctx);
  DeviceGuard g(ctx->device);
  cudaDeviceSynchronize();
  free_host_pipe(ctx);
  for (auto& pr : ctx->prof_events) ctx->prof_free.push_back(pr);
  for (auto& pr : ctx->prof_free) {
    cudaEventDestroy(pr.first);
    cudaEventDestroy(pr.second);
  }
  free_scratch(ctx->scratch);
  if (ctx->calq) cudaFree(ctx->calq);
  if (ctx->badmask) cudaFree(ctx->badmask);
  if (ctx->qmul) cudaFree(ctx->qmul);
  if (ctx->pitch) cudaFree(ctx->pitch);
  delete ctx;
  return SST_OK;
}

const char* sst_last_error(const sst_ctx* ctx) {
  if (!ctx) return "null context";
  return ctx->err.c_str();
}

sst_status sst_calib_upload(sst_ctx* ctx, const float* noise, const float* gain, const uint8_t* bad,
                            const sst_params* params, void* stream) {
  if (!ctx) return SST_ERR_INVALID_ARG;
  if (!noise || !gain || !bad) return set_err(ctx, SST_ERR_INVALID_ARG, "sst_calib_upload: null table");
  if (!params_ok(params))
    return set_err(ctx, SST_ERR_INVALID_ARG,
                   "sst_calib_upload: thresholds must be finite with 0 < t_channel <= t_seed, t_cluster >= 0");
  const uint64_t n = (uint64_t)ctx->n_feds * kCh * kStrips;
  const uint64_t n_apv = n / kApv;
  for (uint64_t i = 0; i < n; i++)
    if (!(noise[i] >= 0.f) || !std::isfinite(noise[i]))
      return set_err(ctx, SST_ERR_INVALID_ARG, "sst_calib_upload: noise must be finite and >= 0");
  for (uint64_t i = 0; i < n_apv; i++)
    if (!(gain[i] > 0.f) || !std::isfinite(gain[i]))
      return set_err(ctx, SST_ERR_INVALID_ARG, "sst_calib_upload: gain must be finite and > 0");
  std::vector<float> qmul(n_apv);
  for (uint64_t i = 0; i < n_apv; i++) qmul[i] = certified_multiplier(gain[i]);
  DeviceGuard g(ctx->device);
  cudaStream_t st = (cudaStream_t)stream;
  cudaError_t e = cudaSuccess;
  if (!ctx->calq) {
    if ((e = cudaMalloc(&ctx->calq, n * sizeof(uint2)))) return cuda_err(ctx, e, "cudaMalloc calq");
    if ((e = cudaMalloc(&ctx->badmask, n / 8))) return cuda_err(ctx, e, "cudaMalloc badmask");
    if ((e = cudaMalloc(&ctx->qmul, n_apv * sizeof(float)))) return cuda_err(ctx, e, "cudaMalloc qmul");
  }
  // staging of the raw tables, freed once the kernels' tables are built
  uint8_t* bad_dev = nullptr;
  float* noise_dev = nullptr;
  if ((e = cudaMalloc(&bad_dev, n))) return cuda_err(ctx, e, "cudaMalloc bad");
  if ((e = cudaMalloc(&noise_dev, n * sizeof(float)))) {
    cudaFree(bad_dev);
    return cuda_err(ctx, e, "cudaMalloc noise");
  }
  // Copies are stream-ordered after earlier work on `st`; synchronise before the
  // host buffers go out of the caller's hands and before freeing the staging.
  if (!e) e = cudaMemcpyAsync(noise_dev, noise, n * sizeof(float), cudaMemcpyHostToDevice, st);
  if (!e) e = cudaMemcpyAsync(ctx->qmul, qmul.data(), n_apv * sizeof(float), cudaMemcpyHostToDevice, st);
  if (!e) e = cudaMemcpyAsync(bad_dev, bad, n, cudaMemcpyHostToDevice, st);
  if (!e) e = build_badmask(bad_dev, ctx->badmask, n, st);
  if (!e) e = build_calib(noise_dev, ctx->badmask, ctx->calq, n, *params, st);
  if (!e) e = cudaStreamSynchronize(st);
  cudaFree(bad_dev);
  cudaFree(noise_dev);
  if (e) return cuda_err(ctx, e, "sst_calib_upload");
  ctx->params = *params;
  ctx->has_calib = true;
  return SST_OK;
}

sst_status sst_unpack(sst_ctx* ctx, const uint8_t* raw, uint64_t raw_bytes, const uint32_t* fed_len, uint32_t n_feds,
                      const sst_digis* out, void* stream) {
  if (!ctx) return SST_ERR_INVALID_ARG;
  if (!raw || !fed_len || !out || !out->strip || !out->adc || !out->chan_off || !out->chan_status || !out->status)
    return set_err(ctx, SST_ERR_INVALID_ARG, "sst_unpack: null pointer");
  if (((uintptr_t)raw & 15u) != 0) return set_err(ctx, SST_ERR_INVALID_ARG, "sst_unpack: raw not 16-byte aligned");
  if (n_feds == 0 || n_feds > ctx->n_feds)
    return set_err(ctx, SST_ERR_INVALID_ARG, "sst_unpack: n_feds outside 1..context FEDs");
  DeviceGuard g(ctx->device);
  cudaError_t e = ensure_scratch(ctx->scratch, n_feds, 1, 1);
  if (e) return cuda_err(ctx, e, "sst_unpack scratch");
  e = launch_unpack(raw, raw_bytes, fed_len, n_feds, *out, ctx->scratch, ctx->shape, (cudaStream_t)stream);
  return cuda_err(ctx, e, "sst_unpack");
}

sst_status sst_cluster(sst_ctx* ctx, const sst_digis* in, uint32_t n_feds, const sst_clusters* out, void* stream) {
  if (!ctx) return SST_ERR_INVALID_ARG;
  if (!ctx->has_calib) return set_err(ctx, SST_ERR_NO_CALIB, "sst_cluster: no calibration");
  if (!in || !in->strip || !in->adc || !in->chan_off || !in->status || !out || !out->det || !out->first ||
      !out->width || !out->charge || !out->barycenter)
    return set_err(ctx, SST_ERR_INVALID_ARG, "sst_cluster: null pointer");
  if (n_feds == 0 || n_feds > ctx->n_feds)
    return set_err(ctx, SST_ERR_INVALID_ARG, "sst_cluster: n_feds outside 1..context FEDs");
  if (out->amp && (!out->amp_first || out->amp_capacity == 0 || out->amp_capacity >= kNoAmp))
    return set_err(ctx, SST_ERR_INVALID_ARG, "sst_cluster: amp needs amp_first and 1 <= amp_capacity < 2^32 - 1");
  DeviceGuard g(ctx->device);
  cudaError_t e = ensure_scratch(ctx->scratch, (size_t)n_feds * kFe, 1, out->capacity);
  if (!e && out->amp) e = ensure_amp_scratch(ctx->scratch, (size_t)n_feds * kFe, 1, out->amp_capacity);
  if (!e) e = ensure_spill(ctx->scratch, (size_t)n_feds * kFe);
  if (e) return cuda_err(ctx, e, "sst_cluster scratch");
  e = launch_cluster(*in, n_feds, *out, kparams(ctx), ctx->scratch, ctx->shape, (cudaStream_t)stream);
  return cuda_err(ctx, e, "sst_cluster");
}

sst_status sst_batch(sst_ctx* ctx, const uint8_t* raw, const uint64_t* event_off, const uint32_t* fed_len,
                     uint32_t n_events, uint32_t n_feds, const uint64_t* clu_off, const sst_clusters* out,
                     sst_event_status* status, void* stream) {
  if (!ctx) return SST_ERR_INVALID_ARG;
  if (!ctx->has_calib) return set_err(ctx, SST_ERR_NO_CALIB, "sst_batch: no calibration");
  if (!raw || !event_off || !fed_len || !clu_off || !out || !status || !out->det || !out->first || !out->width ||
      !out->charge || !out->barycenter)
    return set_err(ctx, SST_ERR_INVALID_ARG, "sst_batch: null pointer");
  if (((uintptr_t)raw & 15u) != 0) return set_err(ctx, SST_ERR_INVALID_ARG, "sst_batch: raw not 16-byte aligned");
  if (n_events == 0 || n_feds == 0 || n_feds > ctx->n_feds)
    return set_err(ctx, SST_ERR_INVALID_ARG, "sst_batch: bad n_events / n_feds");
  if ((uint64_t)n_events * n_feds * kFe >= (1ull << 31))
    return set_err(ctx, SST_ERR_INVALID_ARG, "sst_batch: too many FE units in one batch (2^31)");
  if (out->amp && (!out->amp_first || !out->amp_off || out->amp_capacity == 0 || out->amp_capacity >= kNoAmp))
    return set_err(ctx, SST_ERR_INVALID_ARG,
                   "sst_batch: amp needs amp_first, amp_off and 1 <= amp_capacity < 2^32 - 1");
  DeviceGuard g(ctx->device);
  const size_t items = (size_t)n_events * n_feds;
  cudaError_t e = ensure_scratch(ctx->scratch, items * kFe, n_events, out->capacity);
  if (!e && out->amp) e = ensure_amp_scratch(ctx->scratch, items * kFe, n_events, out->amp_capacity);
  if (!e) e = ensure_spill(ctx->scratch, (size_t)ctx->n_sm * kMaxWarpsPerSm);
  if (e) return cuda_err(ctx, e, "sst_batch scratch");
  cudaEvent_t eb = nullptr, ee = nullptr;
  if (ctx->profiling) {
    if (!ctx->prof_free.empty()) {
      eb = ctx->prof_free.back().first;
      ee = ctx->prof_free.back().second;
      ctx->prof_free.pop_back();
    } else {
      if ((e = cudaEventCreate(&eb))) return cuda_err(ctx, e, "sst_batch profile event");
      if ((e = cudaEventCreate(&ee))) {
        cudaEventDestroy(eb);
        return cuda_err(ctx, e, "sst_batch profile event");
      }
    }
  }
  e = launch_batch(raw, event_off, fed_len, n_events, n_feds, clu_off, *out, status, kparams(ctx), ctx->scratch,
                   ctx->shape, ctx->n_sm, (cudaStream_t)stream, nullptr, eb, ee);
  if (eb) {
    if (e == cudaSuccess)
      ctx->prof_events.emplace_back(eb, ee);
    else
      ctx->prof_free.emplace_back(eb, ee);
  }
  return cuda_err(ctx, e, "sst_batch");
}

sst_status sst_testing_set_wait(sst_ctx* ctx, uint32_t spin_limit, int32_t withhold_fed) {
  if (!ctx) return SST_ERR_INVALID_ARG;
  if (spin_limit > (1u << 20) || withhold_fed < -1)
    return set_err(ctx, SST_ERR_INVALID_ARG, "sst_testing_set_wait: spin_limit above 2^20 or withhold_fed below -1");
  ctx->scratch.lb_spin_limit = spin_limit;
  ctx->scratch.lb_withhold = withhold_fed;
  return SST_OK;
}

sst_status sst_profile_enable(sst_ctx* ctx, int enable) {
  if (!ctx) return SST_ERR_INVALID_ARG;
  ctx->profiling = enable != 0;
  return SST_OK;
}

sst_status sst_profile_read(sst_ctx* ctx, uint64_t* launches, double* total_ms, int reset) {
  if (!ctx) return SST_ERR_INVALID_ARG;
  DeviceGuard g(ctx->device);
  double sum = 0.0;
  for (auto& pr : ctx->prof_events) {
    cudaError_t e = cudaEventSynchronize(pr.second);
    float ms = 0.f;
    if (!e) e = cudaEventElapsedTime(&ms, pr.first, pr.second);
    if (e) return cuda_err(ctx, e, "sst_profile_read");
    sum += ms;
  }
  if (launches) *launches = ctx->prof_events.size();
  if (total_ms) *total_ms = sum;
  if (reset) {
    for (auto& pr : ctx->prof_events) ctx->prof_free.push_back(pr);
    ctx->prof_events.clear();
  }
  return SST_OK;
}

sst_status sst_set_tune(sst_ctx* ctx, const sst_tune* t) {
  if (!ctx || !t) return SST_ERR_INVALID_ARG;
  if (t->host_chunk_events > 4096u) return set_err(ctx, SST_ERR_INVALID_ARG, "sst_set_tune: host_chunk_events > 4096");
  Shape s{(int)t->block, (int)t->tile_digis, (int)t->lanes_per_channel, (int)t->ctas_per_sm,
          (int)t->host_chunk_events, (int)t->units_per_warp};
  if (!shape_valid(s)) return set_err(ctx, SST_ERR_INVALID_ARG, "sst_set_tune: unsupported launch shape");
  ctx->shape = s;
  return SST_OK;
}

sst_status sst_get_tune(const sst_ctx* ctx, sst_tune* t) {
  if (!ctx || !t) return SST_ERR_INVALID_ARG;
  t->block = (uint32_t)ctx->shape.block;
  t->ctas_per_sm = (uint32_t)ctx->shape.ctas_per_sm;
  t->units_per_warp = (uint32_t)ctx->shape.units;
  t->host_chunk_events = (uint32_t)ctx->shape.host_chunk;
  t->tile_digis = (uint32_t)ctx->shape.tile;
  t->lanes_per_channel = (uint32_t)ctx->shape.lanes;
  return SST_OK;
}

sst_status sst_get_launch_info(sst_ctx* ctx, uint32_t n_events, uint32_t n_feds, sst_launch_info* info) {
  if (!ctx || !info || n_events == 0 || n_feds == 0) return SST_ERR_INVALID_ARG;
  DeviceGuard g(ctx->device);
  int grid = 0, ipf = 0;
  size_t smem = 0;
  const cudaError_t e = batch_launch_info(ctx->shape, n_events, n_feds, ctx->n_sm, &grid, &smem, &ipf);
  if (e) return cuda_err(ctx, e, "sst_get_launch_info");
  info->grid = (uint32_t)grid;
  info->block = (uint32_t)ctx->shape.block;
  info->smem_bytes = (uint32_t)smem;
  info->items_per_fed = (uint32_t)ipf;
  info->host_chunks = host_chunks(n_events, ctx->shape.host_chunk);
  return SST_OK;
}

sst_status sst_autotune(sst_ctx* ctx, const uint8_t* raw, const uint64_t* event_off, const uint32_t* fed_len,
                        uint32_t n_events, uint32_t n_feds, const uint64_t* clu_off, const sst_clusters* out,
                        sst_event_status* status, void* stream, sst_tune* best, float* best_us) {
  if (!ctx) return SST_ERR_INVALID_ARG;
  const Shape keep = ctx->shape;
  cudaStream_t st = (cudaStream_t)stream;
  // one untimed call sizes the scratch and checks the arguments
  sst_status r = sst_batch(ctx, raw, event_off, fed_len, n_events, n_feds, clu_off, out, status, stream);
  if (r != SST_OK) return r;
  DeviceGuard g(ctx->device);
  cudaEvent_t e0, e1;
  if (cudaEventCreate(&e0) != cudaSuccess) return cuda_err(ctx, cudaGetLastError(), "autotune event");
  if (cudaEventCreate(&e1) != cudaSuccess) {
    cudaEventDestroy(e0);
    return cuda_err(ctx, cudaGetLastError(), "autotune event");
  }
  const int blocks[] = {128, 256};
  const int widths[] = {1, 2};
  const int per_sm[] = {2, 3, 4, 6, 8};
  float best_t = 1e30f;
  Shape best_s = keep;
  std::vector<std::pair<int, Shape>> timed;  // (effective grid, shape) already measured
  cudaError_t ce = cudaSuccess;
  for (int b : blocks)
    for (int u : widths)
      for (int p : per_sm) {
        Shape s = keep;
        s.block = b;
        s.units = u;
        s.ctas_per_sm = p;
        if (!shape_valid(s) || batch_smem(u, b) * (size_t)p > 227u * 1024u) continue;
        int grid = 0, ipf = 0;
        size_t smem = 0;
        if ((ce = batch_launch_info(s, n_events, n_feds, ctx->n_sm, &grid, &smem, &ipf))) break;
        bool dup = false;  // the occupancy clamps p: the same launch was timed already
        for (auto& pr : timed)
          if (pr.first == grid && pr.second.block == b && pr.second.units == u) dup = true;
        if (dup) continue;
        timed.emplace_back(grid, s);
        float ms_total = 0.f;
        for (int rep = 0; rep < 3 && ce == cudaSuccess; rep++) {
          ce = cudaEventRecord(e0, st);
          if (!ce) ce = launch_batch(raw, event_off, fed_len, n_events, n_feds, clu_off, *out, status, kparams(ctx),
                                     ctx->scratch, s, ctx->n_sm, st);
          if (!ce) ce = cudaEventRecord(e1, st);
          if (!ce) ce = cudaEventSynchronize(e1);
          float ms = 0.f;
          if (!ce) ce = cudaEventElapsedTime(&ms, e0, e1);
          if (rep > 0) ms_total += ms;  // the first launch is a warm-up
        }
        if (ce != cudaSuccess) break;
        const float us = ms_total * 1000.f / 2.f;
        if (us < best_t) {
          best_t = us;
          best_s = s;
        }
      }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (ce != cudaSuccess) {
    ctx->shape = keep;
    return cuda_err(ctx, ce, "sst_autotune");
  }
  ctx->shape = best_s;
  if (best) sst_get_tune(ctx, best);
  if (best_us) *best_us = best_t;
  return SST_OK;
}

sst_status sst_autotune_host(sst_ctx* ctx, const uint8_t* raw, const uint64_t* event_off, const uint32_t* fed_len,
                             uint32_t n_events, uint32_t n_feds, const sst_clusters* out, uint64_t* event_first,
                             sst_event_status* status, uint32_t* best_chunk, float* best_us) {
  if (!ctx) return SST_ERR_INVALID_ARG;
  const int keep = ctx->shape.host_chunk;
  sst_status r = sst_batch_host(ctx, raw, event_off, fed_len, n_events, n_feds, out, event_first, status);
  if (r != SST_OK) return r;
  const int chunks[] = {0, 4, 8, 16, 32, 64, 128};
  double best_t = 1e30;
  int best_c = keep;
  for (int c : chunks) {
    if ((uint32_t)c > n_events) continue;
    ctx->shape.host_chunk = c;
    r = sst_batch_host(ctx, raw, event_off, fed_len, n_events, n_feds, out, event_first, status);  // untimed
    double total = 0;
    for (int rep = 0; rep < 2 && r == SST_OK; rep++) {
      const auto t0 = std::chrono::steady_clock::now();
      r = sst_batch_host(ctx, raw, event_off, fed_len, n_events, n_feds, out, event_first, status);
      total += std::chrono::duration<double, std::micro>(std::chrono::steady_clock::now() - t0).count();
    }
    if (r != SST_OK) {
      ctx->shape.host_chunk = keep;
      return r;
    }
    if (total / 2 < best_t) {
      best_t = total / 2;
      best_c = c;
    }
  }
  ctx->shape.host_chunk = best_c;
  if (best_chunk) *best_chunk = (uint32_t)best_c;
  if (best_us) *best_us = (float)best_t;
  return SST_OK;
}

}  // extern "C"

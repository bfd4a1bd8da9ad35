// sst_internal.h -- internal declarations shared by the library's translation units.
#pragma once

#include <cuda_runtime.h>

#include <cstdint>
#include <mutex>
#include <string>
#include <utility>
#include <vector>

#include "../../include/sst.h"

namespace sst {

constexpr int kCh = SST_CH_PER_FED;          // channels per FED
constexpr int kStrips = SST_STRIPS_PER_CH;   // strips per channel (module)
constexpr int kFe = SST_FE_PER_FED;          // FE units per FED
constexpr int kChPerFe = SST_CH_PER_FE;      // channels per FE unit
constexpr int kApv = SST_STRIPS_PER_APV;     // strips per APV
constexpr int kHdr = SST_FED_HEADER_BYTES;   // FED header bytes
constexpr int kFedStrips = kCh * kStrips;    // 24,576 strips per FED
constexpr int kMaskWords = kStrips / 32;     // 8 words of 32 strips per channel

// Calibration and thresholds as the kernels see them.  The per-strip tables are
// built on the device at calibration upload (k_calib_pack) from the noise, the
// bad-strip flags and the parameters; the per-APV multipliers on the host.
struct KParams {
  float t_cluster;
  int max_holes, max_bad, max_adj;
  const uint2* calq;        // [n_strips]: {thr_ch | thr_seed << 8 | gap << 16, noise^2 (binary32 bits)}
                            // (see k_calib_pack); one 8-byte load per recorded strip
  const uint32_t* badmask;  // [n_strips / 32], bit (s & 31) of word s / 32
  const float* qmul;        // [n_strips / 128]: per APV, a multiplier certified to give the
                            // gain-corrected charge of every ADC 0..253, or -gain (divide)
  uint4* spill = nullptr;   // the launch's spill areas (one per warp of the grid, kSpillRecords records each)
  uint32_t spill_warps = 0; // warps that have one
  const uint32_t* big_list = nullptr;  // batched launches: the work items too large to stage (their
                                       // ticket-order indices; how many: tickets[2], from the prologue)
};


// Launch shape of the kernels.
struct Shape {
  int block;        // batched kernel: threads per CTA
  int tile;         // per-event unpack kernel: digis per on-chip tile
  int lanes;        // per-event unpack kernel: lanes per channel when copying runs
  int ctas_per_sm;  // batched kernel: persistent CTAs per SM
  int host_chunk = 0;  // events per chunk of sst_batch_host (0: automatic)
  int units = 2;       // batched kernel: FE units per warp work item (1 or 2)
};

// Device scratch for one stream of work, owned by a context (or by one server
// stream): look-back states of the per-event unpack, work tickets, per-(event,
// FED) byte offsets and cluster bookkeeping, and the cluster staging buffer.
struct Scratch {
  unsigned long long* lb = nullptr;  // look-back states, one per FED (per-event unpack)
  uint64_t* fed_off = nullptr;       // absolute byte offset per (event, FED)
  uint32_t* fed_cnt = nullptr;       // clusters found per work item (event, FED, pair of FE units)
  uint32_t* fed_start = nullptr;     // staging offset per work item, within its event's slice
  uint32_t* fed_dest = nullptr;      // output offset per work item, within its event's slice
  uint2* unit_desc = nullptr;        // per (event, FED, FE unit): offset in the FED record, length | status
  uint32_t* big_list = nullptr;      // work items too large to stage (batched path; count in tickets[2])
  size_t items_cap = 0;
  uint32_t* ev_alloc = nullptr;      // staging allocation counter per event
  size_t ev_cap = 0;
  uint4* stage = nullptr;            // staged cluster records (16 bytes each)
  size_t stage_cap = 0;
  uint32_t* tickets = nullptr;       // [16] work counters
  uint4* spill = nullptr;            // per warp, kSpillRecords cluster records of a chunked work item
  size_t spill_warps = 0;            // warps that have a spill area (a warp beyond them counts its chunks twice)
  uint32_t lb_spin_limit = 0;        // polls before a look-back wait gives up (0: the default, about a second)
  int32_t lb_withhold = -1;          // failure tests: the FED that never publishes its count (-1: none)
  // optional cluster amplitudes
  uint8_t* amp_stage = nullptr;      // staged amplitudes, sliced per event like the output
  size_t amp_stage_cap = 0;
  uint32_t* amp_alloc = nullptr;     // amplitude allocation counter per event
  uint32_t* seg_amp_cnt = nullptr;   // amplitudes per work item; 0 when they did not fit
  uint32_t* seg_amp_start = nullptr; // their offset in the event's slice, or kNoAmp
  uint32_t* seg_amp_dest = nullptr;  // their offset in the event's output slice
  size_t amp_items_cap = 0, amp_ev_cap = 0;
};
constexpr uint32_t kNoAmp = 0xFFFFFFFFu;
constexpr uint32_t kSpillRecords = 1024;  // records per warp spill area (16 KiB)
constexpr int kMaxWarpsPerSm = 32;        // resident warps of the batched kernel per SM (its register use)

size_t smem_bytes(int tile);
size_t batch_smem(int units, int block);  // shared memory per CTA of the batched kernel
// Grid, shared memory per CTA and work items per FED of the batched kernel's
// launch for a shape and batch (the occupancy look-up may call the driver once).
cudaError_t batch_launch_info(const Shape& sh, uint32_t n_events, uint32_t n_feds, int n_sm, int* grid, size_t* smem,
                              int* items_per_fed);
// Chunks sst_batch_host cuts a batch of n_events into (tuned: events per chunk, 0 = automatic).
uint32_t host_chunks(uint32_t n_events, int tuned);
Shape default_shape();
bool shape_valid(const Shape& s);

// Kernel launchers (sst_kernels.cu).  They only enqueue work on `st`.
cudaError_t launch_unpack(const uint8_t* raw, uint64_t raw_bytes, const uint32_t* fed_len, uint32_t n_feds,
                          const sst_digis& out, const Scratch& s, const Shape& sh, cudaStream_t st);
cudaError_t launch_cluster(const sst_digis& in, uint32_t n_feds, const sst_clusters& out, const KParams& kp,
                           const Scratch& s, const Shape& sh, cudaStream_t st);
// Kernels launched per batched call: k_fed_scan, k_batch, k_order; one more
// (k_clu_scan) for packed output or amplitudes (then k_compact instead of k_order).
// Batched unpack + cluster.  Event e's clusters are staged in, and by default
// written to, the slice [clu_off[e], clu_off[e+1]) of `out` (bounded by
// out.capacity).  With pack_off (device, n_events + 1 values) the events' clusters
// are written back to back instead, event e from pack_off[e], which the launch
// computes.  With event_end (device, n_events values) event e's bytes are
// [event_off[e], event_end[e]) of raw, so that the events need not follow one
// another (raw may then be pinned host memory read in place).
cudaError_t launch_batch(const uint8_t* raw, const uint64_t* event_off, const uint32_t* fed_len, uint32_t n_events,
                         uint32_t n_feds, const uint64_t* clu_off, const sst_clusters& out, sst_event_status* status,
                         const KParams& kp, const Scratch& s, const Shape& sh, int n_sm, cudaStream_t st,
                         uint64_t* pack_off = nullptr, cudaEvent_t ev_begin = nullptr, cudaEvent_t ev_end = nullptr,
                         const uint64_t* event_end = nullptr);
cudaError_t build_badmask(const uint8_t* bad_dev, uint32_t* mask_dev, uint64_t n_strips, cudaStream_t st);
// Adds base to the first *count (device) values of amp_first, kNoAmp excepted.
cudaError_t rebase_amp_first(uint32_t* amp_first, const uint64_t* count, uint32_t base, int n_sm, cudaStream_t st);
cudaError_t build_calib(const float* noise_dev, const uint32_t* mask_dev, uint2* calq_dev,
                        uint64_t n_strips, const sst_params& p, cudaStream_t st);

}  // namespace sst

struct sst_server;
struct sst_host_pipe;

struct sst_ctx {
  int device = 0;
  uint32_t n_feds = 0;
  int n_sm = 0;
  bool has_calib = false;
  sst_params params{};
  uint2* calq = nullptr;       // per strip: channel and seed thresholds as ADC limits and linking gap; noise^2
  uint32_t* badmask = nullptr;
  float* qmul = nullptr;       // per APV: certified multiplier or -gain
  sst::Scratch scratch;
  sst::Shape shape{};
  std::string err;
  std::mutex mu;
  sst_server* server = nullptr;
  sst_host_pipe* pipe = nullptr;  // streams and arenas of sst_batch_host, made on first use
  float* pitch = nullptr;         // strip pitch per module (sst_pitch_upload), or null
  bool profiling = false;
  std::vector<std::pair<cudaEvent_t, cudaEvent_t>> prof_events;  // recorded launches
  std::vector<std::pair<cudaEvent_t, cudaEvent_t>> prof_free;    // reusable pairs
};

namespace sst {
sst_status set_err(sst_ctx* c, sst_status code, const std::string& msg);
sst_status cuda_err(sst_ctx* c, cudaError_t e, const char* where);
KParams kparams(const sst_ctx* c);
cudaError_t ensure_scratch(Scratch& s, size_t items, size_t events, size_t stage_records);
// Spill areas for `warps` warps (the batched kernel's resident warps, or one per FE
// unit for the per-event cluster kernel); grows only.
cudaError_t ensure_spill(Scratch& s, size_t warps);
cudaError_t ensure_amp_scratch(Scratch& s, size_t items, size_t events, size_t amp_bytes);
void free_scratch(Scratch& s);
void free_host_pipe(sst_ctx* ctx);

// Makes `dev` current for the guard's lifetime.
struct DeviceGuard {
  int prev = -1;
  explicit DeviceGuard(int dev) {
    if (cudaGetDevice(&prev) != cudaSuccess) prev = -1;
    if (prev != dev) cudaSetDevice(dev);
  }
  ~DeviceGuard() {
    int cur = -1;
    if (prev >= 0 && cudaGetDevice(&cur) == cudaSuccess && cur != prev) cudaSetDevice(prev);
  }
};
}  // namespace sst

// sst_noalloc.cu -- sst_unpack_noalloc: per-event unpacking that allocates no
// memory at all.
//
// Who needs it: code that may not call cudaMalloc once it is running.  A trigger
// or data-acquisition process typically reserves all device memory up front for
// its own caching allocator, so a library allocation can fail or steal from that
// reserve; cudaMalloc / cudaFree also synchronise the device, which stalls every
// other stream of a real-time pipeline; and some callers run where allocation is
// not allowed at all.  sst_unpack keeps its scratch (look-back states, FED offsets,
// work tickets) in the context and grows it on demand, and a context itself is
// created with cudaMalloc.  This entry point needs neither: its scratch lives in
// the fixed array below, which every GPU that loads the library holds until the
// process exits.
#include <mutex>

#include "sst_internal.h"

namespace {

constexpr uint32_t kMaxFeds = SST_NOALLOC_MAX_FEDS;
constexpr int kMaxDevices = 64;

// Scratch for one call: kMaxFeds look-back states, kMaxFeds FED byte offsets, and
// 8 words of work tickets (16 KiB + 64 B).
static __device__ __align__(256) unsigned long long g_scratch[2 * kMaxFeds + 8];

std::mutex g_mu;
void* g_addr[kMaxDevices];  // device address of g_scratch, per device, once known

// Device address of g_scratch on the current device (looked up on the first call
// for that device).
cudaError_t scratch_address(int dev, void** out) {
  std::lock_guard<std::mutex> lock(g_mu);
  if (!g_addr[dev]) {
    void* p = nullptr;
    const cudaError_t e = cudaGetSymbolAddress(&p, g_scratch);
    if (e != cudaSuccess) return e;
    g_addr[dev] = p;
  }
  *out = g_addr[dev];
  return cudaSuccess;
}

}  // namespace

extern "C" sst_status sst_unpack_noalloc(const uint8_t* raw, uint64_t raw_bytes, const uint32_t* fed_len,
                                         uint32_t n_feds, const sst_digis* out, void* stream) {
  if (!raw || !fed_len || !out || !out->strip || !out->adc || !out->chan_off || !out->chan_status || !out->status)
    return SST_ERR_INVALID_ARG;
  if (((uintptr_t)raw & 15u) != 0) return SST_ERR_INVALID_ARG;
  if (n_feds == 0) return SST_ERR_INVALID_ARG;
  if (n_feds > kMaxFeds) return SST_ERR_TOO_LARGE;
  int dev = -1;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) return SST_ERR_CUDA;
  void* base = nullptr;
  if (scratch_address(dev, &base) != cudaSuccess) return SST_ERR_CUDA;
  unsigned long long* words = static_cast<unsigned long long*>(base);
  sst::Scratch s;
  s.lb = words;
  s.fed_off = reinterpret_cast<uint64_t*>(words + kMaxFeds);
  s.tickets = reinterpret_cast<uint32_t*>(words + 2 * kMaxFeds);
  // the launcher clears the look-back states, the tickets and the event status
  // before its kernels run, on the caller's stream
  const cudaError_t e = sst::launch_unpack(raw, raw_bytes, fed_len, n_feds, *out, s, sst::default_shape(),
                                           static_cast<cudaStream_t>(stream));
  return e == cudaSuccess ? SST_OK : SST_ERR_CUDA;
}

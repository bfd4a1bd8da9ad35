// sst_geom.cu -- local positions of clusters (arXiv 2101.11489 section 4: the
// clusters become hits with positions for the track finder).  The detector
// geometry is not available, so every module gets a strip pitch from the caller
// (a synthetic geometry); the local x of a cluster is measured from the module's
// centre, between strips 127 and 128: x = (barycenter - 128) * pitch[det], one
// binary32 subtraction and one binary32 multiplication, both rounded to nearest.
#include <cmath>

#include "sst_internal.h"

namespace {

__global__ void k_local_x(const uint32_t* __restrict__ det, const float* __restrict__ bary, uint64_t n,
                          const float* __restrict__ pitch, uint32_t n_modules, float* __restrict__ x) {
  const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
  for (uint64_t k = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; k < n; k += stride) {
    const uint32_t m = det[k];
    // a module id outside the detector has no position
    x[k] = m < n_modules ? __fmul_rn(__fsub_rn(bary[k], 128.0f), pitch[m]) : __int_as_float(0x7fc00000);
  }
}

}  // namespace

using namespace sst;

extern "C" {

sst_status sst_pitch_upload(sst_ctx* ctx, const float* pitch) {
  if (!ctx) return SST_ERR_INVALID_ARG;
  if (!pitch) return set_err(ctx, SST_ERR_INVALID_ARG, "sst_pitch_upload: null pitch");
  const uint32_t n = ctx->n_feds * kCh;
  for (uint32_t i = 0; i < n; i++)
    if (!(pitch[i] > 0.f) || !std::isfinite(pitch[i]))
      return set_err(ctx, SST_ERR_INVALID_ARG, "sst_pitch_upload: pitch must be finite and > 0");
  DeviceGuard g(ctx->device);
  cudaError_t e = cudaSuccess;
  if (!ctx->pitch && (e = cudaMalloc(&ctx->pitch, n * sizeof(float)))) return cuda_err(ctx, e, "cudaMalloc pitch");
  if ((e = cudaMemcpy(ctx->pitch, pitch, n * sizeof(float), cudaMemcpyHostToDevice)))
    return cuda_err(ctx, e, "sst_pitch_upload");
  return SST_OK;
}

sst_status sst_local_x(sst_ctx* ctx, const uint32_t* det, const float* barycenter, uint64_t n, float* x,
                       void* stream) {
  if (!ctx) return SST_ERR_INVALID_ARG;
  if (!ctx->pitch) return set_err(ctx, SST_ERR_STATE, "sst_local_x: no pitch uploaded");
  if (n == 0) return SST_OK;
  if (!det || !barycenter || !x) return set_err(ctx, SST_ERR_INVALID_ARG, "sst_local_x: null pointer");
  DeviceGuard g(ctx->device);
  const uint64_t want = (n + 255) / 256;
  const uint64_t cap = (uint64_t)(ctx->n_sm > 0 ? ctx->n_sm : 1) * 16;
  const unsigned grid = (unsigned)(want < cap ? want : cap);
  k_local_x<<<grid, 256, 0, (cudaStream_t)stream>>>(det, barycenter, n, ctx->pitch, ctx->n_feds * kCh, x);
  return cuda_err(ctx, cudaGetLastError(), "sst_local_x");
}

}  // extern "C"

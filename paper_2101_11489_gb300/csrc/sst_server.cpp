// sst_server.cpp -- served path (continuous batching).  Placeholder until the
// request loop lands: every entry point reports SST_ERR_STATE.
#include "sst_internal.h"

extern "C" {
sst_status sst_server_start(sst_ctx* ctx, const sst_server_opts*) {
  return sst::set_err(ctx, SST_ERR_STATE, "server not available");
}
sst_status sst_server_stop(sst_ctx* ctx) { return ctx ? SST_OK : SST_ERR_INVALID_ARG; }
sst_status sst_submit(sst_ctx* ctx, const uint8_t*, uint64_t, const uint32_t*, uint64_t*) {
  return sst::set_err(ctx, SST_ERR_STATE, "server not running");
}
sst_status sst_poll(sst_ctx* ctx, uint64_t, int64_t, sst_result_info*, uint32_t*, uint16_t*, uint16_t*, uint32_t*,
                    float*, uint64_t) {
  return sst::set_err(ctx, SST_ERR_STATE, "server not running");
}
}

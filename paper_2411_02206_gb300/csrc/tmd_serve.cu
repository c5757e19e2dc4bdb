// tmd_serve.cu -- serving: admission by memory budget, resident buffers,
// continuous batching (filled in by the serving milestone).
#include "tmd_api_internal.h"

void tmd_serve_shutdown(tmd_handle*) {}

extern "C" int tmd_submit(tmd_handle* h, const tmd_frame_in*, uint64_t*) {
  return tmd_set_error(h, TMD_ERR_STATE, "serving is not available in this build");
}
extern "C" int tmd_poll(tmd_handle* h, uint64_t, uint32_t, tmd_frame_out*) {
  return tmd_set_error(h, TMD_ERR_STATE, "serving is not available in this build");
}
extern "C" int tmd_release(tmd_handle* h, uint64_t) {
  return tmd_set_error(h, TMD_ERR_STATE, "serving is not available in this build");
}

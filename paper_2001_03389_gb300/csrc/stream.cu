// stream.cu -- streaming service (continuous batching of beam chunks).
#include <cuda_runtime.h>

#include "runtime.h"

namespace rfim {
struct StreamService {};
void stream_service_destroy(StreamService* s) { delete s; }
}  // namespace rfim

using namespace rfim;

extern "C" {
rfim_status rfim_stream_open(rfim_ctx* ctx, int, int, int, rfim_dtype, const rfim_cut*, const rfim_cut*) {
  if (!ctx) return RFIM_ERR_ARG;
  ctx_set_error(ctx, "streaming service not available in this build");
  return RFIM_ERR_STATE;
}
rfim_status rfim_stream_push(rfim_ctx* ctx, int, const void*, double, unsigned long long*) {
  if (!ctx) return RFIM_ERR_ARG;
  return RFIM_ERR_STATE;
}
rfim_status rfim_stream_poll(rfim_ctx* ctx, unsigned long long, void**, void**, int) {
  if (!ctx) return RFIM_ERR_ARG;
  return RFIM_ERR_STATE;
}
rfim_status rfim_stream_release(rfim_ctx* ctx, unsigned long long) {
  if (!ctx) return RFIM_ERR_ARG;
  return RFIM_ERR_STATE;
}
rfim_status rfim_stream_stats(rfim_ctx* ctx, double*, double*, double*, double*, unsigned long long*, int) {
  if (!ctx) return RFIM_ERR_ARG;
  return RFIM_ERR_STATE;
}
rfim_status rfim_stream_close(rfim_ctx* ctx) {
  if (!ctx) return RFIM_ERR_ARG;
  return RFIM_ERR_STATE;
}
}

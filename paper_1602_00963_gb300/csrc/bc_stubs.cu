// Temporary entry points for subsystems not built yet (replaced as they land).
#include "bc_internal.h"

namespace bcl {
void server_stop(Ctx *) {}
bool server_graph_busy(Ctx *, Graph *) { return false; }
}  // namespace bcl

extern "C" {
bc_status bc_autotune(bc_graph *, int32_t, uint64_t, bc_tune_result *) {
  return bcl::fail(BC_EINVAL, "autotuner not available in this build");
}
bc_status bc_stream_submit(bc_ctx *, const bc_request *, uint64_t *) {
  return bcl::fail(BC_EINVAL, "serving not available in this build");
}
bc_status bc_stream_poll(bc_ctx *, uint64_t, int32_t, bc_result *) {
  return bcl::fail(BC_EINVAL, "serving not available in this build");
}
bc_status bc_stream_cancel(bc_ctx *, uint64_t) {
  return bcl::fail(BC_EINVAL, "serving not available in this build");
}
}

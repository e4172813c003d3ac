// Serving loop (placeholder until the scheduler lands).
#include "dd_solver.cuh"

namespace dd {
void destroy_server(void *) {}
int server_magic_ok(void *) { return 0; }
}  // namespace dd

extern "C" {
int dd_server_create(const dd_server_params *, dd_server_t *) {
  dd::set_error("dd_server_create: not available");
  return DD_EINVAL;
}
int dd_submit(dd_server_t, const dd_request *, uint64_t *) { return DD_EINVAL; }
int dd_poll(dd_server_t, uint64_t, int *, double *, dd_solve_info *) { return DD_EINVAL; }
int dd_cancel(dd_server_t, uint64_t) { return DD_EINVAL; }
int dd_server_get_stats(dd_server_t, dd_server_stats *) { return DD_EINVAL; }
}

// Batched local BA (persistent launch over many small problems).
#include "handle.h"

struct ba_batch {};

namespace ba {
void destroy_batch(ba_handle* h) {
  delete h->batch;
  h->batch = nullptr;
}
}  // namespace ba

extern "C" {
ba_status ba_solve_batch(ba_handle* h, int32_t, const ba_problem*, ba_result*) {
  if (h) h->err = "ba_solve_batch: not available";
  return BA_ERR_STATE;
}
ba_status ba_get_batch_schedule(const ba_handle*, int32_t*, int32_t*) { return BA_ERR_STATE; }
ba_status ba_set_batch_schedule(ba_handle*, int32_t, int32_t) { return BA_ERR_STATE; }
ba_status ba_tune_batch(ba_handle*, int32_t, const ba_problem*, int32_t*, int32_t*) {
  return BA_ERR_STATE;
}
}

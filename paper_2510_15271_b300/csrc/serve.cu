// Served local BA (continuous batching of requests).
#include "handle.h"

struct ba_server {};

namespace ba {
void destroy_server(ba_handle* h) {
  delete h->server;
  h->server = nullptr;
}
}  // namespace ba

extern "C" {
ba_status ba_create_server(const ba_options*, ba_handle**) { return BA_ERR_STATE; }
ba_status ba_submit(ba_handle*, const ba_problem*, uint64_t*) { return BA_ERR_STATE; }
ba_status ba_poll(ba_handle*, uint64_t, ba_result*) { return BA_ERR_STATE; }
}

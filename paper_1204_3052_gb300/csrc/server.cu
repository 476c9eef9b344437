// Request server (continuous batching) -- entry points; scheduler to follow.
#include "internal.cuh"
#include "plan.h"

using namespace mp;

extern "C" matpow_status matpow_server_create(matpow_server_t* server, const matpow_server_desc*) {
  if (server) *server = nullptr;
  return fail(nullptr, MATPOW_EUNSUPPORTED, "matpow_server: not built yet");
}
extern "C" matpow_status matpow_submit(matpow_server_t, const matpow_request*, uint64_t*) {
  return fail(nullptr, MATPOW_EUNSUPPORTED, "matpow_server: not built yet");
}
extern "C" matpow_status matpow_poll(matpow_server_t, uint64_t, uint32_t) {
  return fail(nullptr, MATPOW_EUNSUPPORTED, "matpow_server: not built yet");
}
extern "C" int64_t matpow_server_latencies(matpow_server_t, double*, int64_t) { return 0; }
extern "C" matpow_status matpow_server_destroy(matpow_server_t) { return MATPOW_OK; }

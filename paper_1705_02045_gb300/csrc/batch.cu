// Batched and served computation (filled in by the persistent batched kernel).
#include "engine.h"

namespace ecc {
struct Request {};
void serve_shutdown(ecc_handle*) {}
}  // namespace ecc

using namespace ecc;

extern "C" {
int ecc_compute_batch(ecc_handle* h, int, const ecc_image*, ecc_result*) {
  return set_err(h, ECC_ERR_STATE, "batched computation not built yet");
}
int ecc_submit(ecc_handle* h, const void*, const int64_t*, int, ecc_dtype, uint64_t*) {
  return set_err(h, ECC_ERR_STATE, "serving not built yet");
}
int ecc_poll(ecc_handle* h, uint64_t, ecc_result*, int64_t) {
  return set_err(h, ECC_ERR_STATE, "serving not built yet");
}
int ecc_request_latency_us(ecc_handle* h, uint64_t, double*) {
  return set_err(h, ECC_ERR_STATE, "serving not built yet");
}
}

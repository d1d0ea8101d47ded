// Streaming (placeholder until the slab ring is in).
#include "engine.h"

using namespace ecc;

extern "C" {
int ecc_stream_begin(ecc_handle* h, const int64_t*, int, ecc_dtype, ecc_stream** out) {
  if (out) *out = nullptr;
  return set_err(h, ECC_ERR_STATE, "streaming not built yet");
}
int ecc_stream_push_slab(ecc_stream*, const void*, int64_t, int64_t) { return ECC_ERR_STATE; }
int ecc_stream_finish(ecc_stream*, ecc_result*) { return ECC_ERR_STATE; }
void ecc_stream_abort(ecc_stream*) {}
}

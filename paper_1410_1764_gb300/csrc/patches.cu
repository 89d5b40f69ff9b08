// Batched patches (placeholder until the persistent batched kernel lands).
#include "internal.h"

namespace chemora {
void destroy_batch(chemora_batch*) {}
}  // namespace chemora

using namespace chemora;

extern "C" {
int chemora_patches_create(int, const int*, int, double, int, const chemora_params*,
                           chemora_batch** out) {
  if (out) *out = nullptr;
  return set_error(CHEMORA_EUNSUPPORTED, "batched patches not built yet");
}
int chemora_patches_state(chemora_batch*, int, double**) {
  return set_error(CHEMORA_EUNSUPPORTED, "batched patches not built yet");
}
int chemora_patches_step(chemora_batch*, double, int, int, void*) {
  return set_error(CHEMORA_EUNSUPPORTED, "batched patches not built yet");
}
int chemora_adjoint_rk4(chemora_system*, const double*, const double*, double, int, int,
                        const int64_t*, int, const double*, double*, double*, double*, void*) {
  return set_error(CHEMORA_EUNSUPPORTED, "adjoint not built yet");
}
}

// Passes for sides 256 384 512.
#include "kernels_inst.cuh"

namespace sgp {
static SGP_DEFINE_TWIDDLE_INIT(twiddle_init_mid_b)
void register_mid_b(Registry& R) {
  register_side<256>(R);
  register_side<384>(R);
  register_side<512>(R);
  R.twiddle_init[6] = &twiddle_init_mid_b;
}
}  // namespace sgp

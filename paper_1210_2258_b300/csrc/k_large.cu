// Passes for sides 768 1024.
#include "kernels_inst.cuh"

namespace sgp {
static SGP_DEFINE_TWIDDLE_INIT(twiddle_init_large)
void register_large(Registry& R) {
  register_side<768>(R);
  register_side<1024>(R);
  R.twiddle_init[2] = &twiddle_init_large;
}
}  // namespace sgp

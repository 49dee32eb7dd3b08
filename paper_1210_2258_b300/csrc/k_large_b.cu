// Passes for sides 1536 2048.
#include "kernels_inst.cuh"

namespace sgp {
static SGP_DEFINE_TWIDDLE_INIT(twiddle_init_large_b)
void register_large_b(Registry& R) {
  register_side<1536>(R);
  register_side<2048>(R);
  R.twiddle_init[7] = &twiddle_init_large_b;
}
}  // namespace sgp

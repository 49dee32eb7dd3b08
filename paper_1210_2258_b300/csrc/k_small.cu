// Passes for sides 16 24 32 48 64.
#include "kernels_inst.cuh"

namespace sgp {
static SGP_DEFINE_TWIDDLE_INIT(twiddle_init_small)
void register_small(Registry& R) {
  register_side<16>(R);
  register_side<24>(R);
  register_side<32>(R);
  register_side<48>(R);
  register_side<64>(R);
  R.twiddle_init[0] = &twiddle_init_small;
}
}  // namespace sgp

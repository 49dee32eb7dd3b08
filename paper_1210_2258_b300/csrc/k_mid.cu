// Passes for sides 96 128 192.
#include "kernels_inst.cuh"

namespace sgp {
static SGP_DEFINE_TWIDDLE_INIT(twiddle_init_mid)
void register_mid(Registry& R) {
  register_side<96>(R);
  register_side<128>(R);
  register_side<192>(R);
  R.twiddle_init[1] = &twiddle_init_mid;
}
}  // namespace sgp

// Multi-size SGP pass K6 (the scans K7 and K8 are in k_multi_scan_*.cu, one unit each so that the
// units compile in parallel).
#include "multi_common.cuh"

namespace sgp {
#define B4(N) b_sgp_ad_armijo<N, FP64>(imgs, items, n_items)
SGP_MULTI_ROW(km_sgp_ad_armijo, B4)

static SGP_DEFINE_TWIDDLE_INIT(twiddle_init_multi_sgp_b)

void register_multi_sgp_b(Registry& R) {
  R.row_multi[ROP_SGP_AD][0] = (const void*)&km_sgp_ad_armijo<false>;
  R.row_multi[ROP_SGP_AD][1] = (const void*)&km_sgp_ad_armijo<true>;
  R.twiddle_init[5] = &twiddle_init_multi_sgp_b;
}

}  // namespace sgp

// Multi-size SGP passes (K6, K7, K8).
#include "multi_common.cuh"

namespace sgp {
#define B4(N) b_sgp_ad_armijo<N, FP64>(imgs, items, n_items)
SGP_MULTI_ROW(km_sgp_ad_armijo, B4)
#define B5(N) b_sgp_lambda_scan<N, FP64, false>(imgs, items, n_items)
SGP_MULTI_ROW(km_sgp_armijo_extra, B5)
#define B9(N) b_sgp_lambda_scan<N, FP64, true>(imgs, items, n_items)
SGP_MULTI_ROW(km_sgp_land, B9)

static SGP_DEFINE_TWIDDLE_INIT(twiddle_init_multi_sgp_b)

void register_multi_sgp_b(Registry& R) {
#define REG(OP, K) R.row_multi[OP][0] = (const void*)&K<false>; R.row_multi[OP][1] = (const void*)&K<true>;
  REG(ROP_SGP_AD, km_sgp_ad_armijo)
  REG(ROP_SGP_ARMX, km_sgp_armijo_extra)
  REG(ROP_SGP_LAND, km_sgp_land)
#undef REG
  R.twiddle_init[5] = &twiddle_init_multi_sgp_b;
}

}  // namespace sgp

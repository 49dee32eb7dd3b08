// Multi-size SGP pass K8 (the landing step lengths), plain FP32 reductions.
#include "multi_common.cuh"

namespace sgp {
#define BS(N) b_sgp_lambda_scan<N, false, true>(imgs, items, n_items)
SGP_MULTI_ROW_FIXED(km_land_f, BS, false)

void register_multi_land_f(Registry& R) { R.row_multi[ROP_SGP_LAND][0] = (const void*)&km_land_f; }

}  // namespace sgp

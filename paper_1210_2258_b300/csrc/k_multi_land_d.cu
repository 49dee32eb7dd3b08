// Multi-size SGP pass K8 (the landing step lengths), float-pair / FP64 reductions.
#include "multi_common.cuh"

namespace sgp {
#define BS(N) b_sgp_lambda_scan<N, true, true>(imgs, items, n_items)
SGP_MULTI_ROW_FIXED(km_land_d, BS, true)

void register_multi_land_d(Registry& R) { R.row_multi[ROP_SGP_LAND][1] = (const void*)&km_land_d; }

}  // namespace sgp

// Multi-size SGP pass K7 (the remaining Armijo step lengths), float-pair / FP64 reductions.
#include "multi_common.cuh"

namespace sgp {
#define BS(N) b_sgp_lambda_scan<N, true, false>(imgs, items, n_items)
SGP_MULTI_ROW_FIXED(km_armx_d, BS, true)

void register_multi_armx_d(Registry& R) { R.row_multi[ROP_SGP_ARMX][1] = (const void*)&km_armx_d; }

}  // namespace sgp

// Multi-size SGP pass K7 (the remaining Armijo step lengths), plain FP32 reductions.
#include "multi_common.cuh"

namespace sgp {
#define BS(N) b_sgp_lambda_scan<N, false, false>(imgs, items, n_items)
SGP_MULTI_ROW_FIXED(km_armx_f, BS, false)

void register_multi_armx_f(Registry& R) { R.row_multi[ROP_SGP_ARMX][0] = (const void*)&km_armx_f; }

}  // namespace sgp

// Explicit instantiation of the size-templated passes for a group of sides (one translation unit
// per group so the groups compile in parallel).
#pragma once
#include "colops.cuh"
#include "registry.h"
#include "rowops.cuh"

namespace sgp {

template <int N>
void register_side(Registry& R) {
  const int s = side_index(N);
#define SGP_ROW_BOTH(OP, KER)                                        \
  R.row[OP][0][s] = reinterpret_cast<const void*>(&KER<N, false>); \
  R.row[OP][1][s] = reinterpret_cast<const void*>(&KER<N, true>);
  SGP_ROW_BOTH(ROP_SGP_UPDATE, k_sgp_update_ratio)
  SGP_ROW_BOTH(ROP_SGP_GRAD, k_sgp_grad_bb)
  SGP_ROW_BOTH(ROP_SGP_Y, k_sgp_y)
  SGP_ROW_BOTH(ROP_SGP_AD, k_sgp_ad_armijo)
  SGP_ROW_BOTH(ROP_SGP_ARMX, k_sgp_armijo_extra)
  SGP_ROW_BOTH(ROP_SGP_LAND, k_sgp_land)
  SGP_ROW_BOTH(ROP_RL_UPDATE, k_rl_update)
  SGP_ROW_BOTH(ROP_RL_RATIO, k_rl_ratio)
#undef SGP_ROW_BOTH
  R.row[ROP_MINMAX][0][s] = R.row[ROP_MINMAX][1][s] = reinterpret_cast<const void*>(&k_rl_step_minmax<N>);
  R.row[ROP_R2C][0][s] = R.row[ROP_R2C][1][s] = reinterpret_cast<const void*>(&k_row_r2c<N>);
  R.row[ROP_C2R][0][s] = R.row[ROP_C2R][1][s] = reinterpret_cast<const void*>(&k_row_c2r<N>);
  R.col[COL_KHAT][s] = reinterpret_cast<const void*>(&k_col<N, COL_KHAT>);
  R.col[COL_1TOP][s] = reinterpret_cast<const void*>(&k_col<N, COL_1TOP>);
  R.col[COL_1TOP_CONJ][s] = reinterpret_cast<const void*>(&k_col<N, COL_1TOP_CONJ>);
  R.col[COL_PTO1][s] = reinterpret_cast<const void*>(&k_col<N, COL_PTO1, 0>);
  R.col[COL_PTOV][s] = reinterpret_cast<const void*>(&k_col<N, COL_PTOV>);
  R.col[kColPto1P1][s] = reinterpret_cast<const void*>(&k_col<N, COL_PTO1, 1>);
  R.row_smem[s] = RowGeo<N>::SMEM;
  R.row_rows[s] = RowGeo<N>::ROWS;
  R.col_smem[s] = ColGeo<N>::SMEM;
  R.col_cols[s] = ColGeo<N>::C;
  if constexpr (N == kNarrowSide) {   // the narrow column variant (ColPlanNarrow)
    R.col_narrow[COL_KHAT] = reinterpret_cast<const void*>(&k_col<N, COL_KHAT, 0, true>);
    R.col_narrow[COL_1TOP] = reinterpret_cast<const void*>(&k_col<N, COL_1TOP, 0, true>);
    R.col_narrow[COL_1TOP_CONJ] = reinterpret_cast<const void*>(&k_col<N, COL_1TOP_CONJ, 0, true>);
    R.col_narrow[COL_PTO1] = reinterpret_cast<const void*>(&k_col<N, COL_PTO1, 0, true>);
    R.col_narrow[COL_PTOV] = reinterpret_cast<const void*>(&k_col<N, COL_PTOV, 0, true>);
    R.col_narrow[kColPto1P1] = reinterpret_cast<const void*>(&k_col<N, COL_PTO1, 1, true>);
    R.col_narrow_smem = ColGeo<N, true>::SMEM;
    R.col_narrow_cols = ColGeo<N, true>::C;
  }
}

}  // namespace sgp

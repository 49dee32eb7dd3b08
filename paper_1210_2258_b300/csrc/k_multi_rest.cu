// Multi-size RL, set-up and column passes.
#include "multi_common.cuh"

namespace sgp {
#define B6(N) b_rl_update<N, FP64>(imgs, items, n_items, extra)
SGP_MULTI_ROW(km_rl_update, B6)
#define B7(N) b_rl_ratio<N, FP64>(imgs, items, n_items, extra)
SGP_MULTI_ROW(km_rl_ratio, B7)
#define B8(N) b_rl_step_minmax<N>(imgs, items, n_items)
SGP_MULTI_ROW(km_rl_step_minmax, B8)

template <int MODE, int NV>
__global__ void __launch_bounds__(kColBlock) km_col(const ColJob* __restrict__ jobs, const int2* __restrict__ items,
                                                   int n_items) {
  const int it = blockIdx.x;
  if (it >= n_items) return;
  const int H = jobs[items[it].x].H;
#define BC(N) b_col<N, MODE, NV>(jobs, items, n_items)
  SGP_SWITCH_SIDE(H, BC)
#undef BC
}

static SGP_DEFINE_TWIDDLE_INIT(twiddle_init_multi_rest)

void register_multi_rest(Registry& R) {
#define REG(OP, K) R.row_multi[OP][0] = (const void*)&K<false>; R.row_multi[OP][1] = (const void*)&K<true>;
  REG(ROP_RL_UPDATE, km_rl_update)
  REG(ROP_RL_RATIO, km_rl_ratio)
  REG(ROP_MINMAX, km_rl_step_minmax)
#undef REG
  R.col_multi[0] = (const void*)&km_col<COL_1TOP, 0>;
  R.col_multi[1] = (const void*)&km_col<COL_PTO1, 0>;
  R.col_multi[2] = (const void*)&km_col<COL_PTO1, 1>;
  R.col_multi_smem = max_col_smem();
  R.twiddle_init[4] = &twiddle_init_multi_rest;
}

}  // namespace sgp

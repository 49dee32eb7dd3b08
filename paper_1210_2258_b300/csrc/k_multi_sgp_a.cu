// Multi-size SGP passes (K1, K3, K4).
#include "multi_common.cuh"

namespace sgp {
#define B1(N) b_sgp_update_ratio<N, FP64>(imgs, items, n_items)
SGP_MULTI_ROW(km_sgp_update_ratio, B1)
#define B2(N) b_sgp_grad_bb<N, FP64>(imgs, items, n_items)
SGP_MULTI_ROW(km_sgp_grad_bb, B2)
#define B3(N) b_sgp_y<N, FP64>(imgs, items, n_items)
SGP_MULTI_ROW(km_sgp_y, B3)

static SGP_DEFINE_TWIDDLE_INIT(twiddle_init_multi_sgp_a)

void register_multi_sgp_a(Registry& R) {
#define REG(OP, K) R.row_multi[OP][0] = (const void*)&K<false>; R.row_multi[OP][1] = (const void*)&K<true>;
  REG(ROP_SGP_UPDATE, km_sgp_update_ratio)
  REG(ROP_SGP_GRAD, km_sgp_grad_bb)
  REG(ROP_SGP_Y, km_sgp_y)
#undef REG
  R.row_multi_smem = max_row_smem();
  R.twiddle_init[3] = &twiddle_init_multi_sgp_a;
}

}  // namespace sgp

// Shared pieces of the multi-size passes: one launch covers problems of different sides; every
// block reads the side of its work item's problem and runs the body instantiated for that side.
#pragma once
#include "kernels_inst.cuh"

namespace sgp {
#define SGP_SWITCH_SIDE(N_, CALL) \
  switch (N_) { case 16: CALL(16); break; case 24: CALL(24); break; case 32: CALL(32); break; case 48: CALL(48); break; case 64: CALL(64); break; case 96: CALL(96); break; case 128: CALL(128); break; case 192: CALL(192); break; case 256: CALL(256); break; case 384: CALL(384); break; case 512: CALL(512); break; case 768: CALL(768); break; case 1024: CALL(1024); break; case 1536: CALL(1536); break; case 2048: CALL(2048); break; default: break; }

template <int N> constexpr size_t row_smem_of() { return RowGeo<N>::SMEM; }
constexpr size_t max_row_smem() {
  size_t m = 0;
  const size_t v[] = {RowGeo<16>::SMEM, RowGeo<24>::SMEM, RowGeo<32>::SMEM, RowGeo<48>::SMEM, RowGeo<64>::SMEM,
                      RowGeo<96>::SMEM, RowGeo<128>::SMEM, RowGeo<192>::SMEM, RowGeo<256>::SMEM, RowGeo<384>::SMEM,
                      RowGeo<512>::SMEM, RowGeo<768>::SMEM, RowGeo<1024>::SMEM, RowGeo<1536>::SMEM, RowGeo<2048>::SMEM};
  for (size_t x : v) m = x > m ? x : m;
  return m;
}
constexpr size_t max_col_smem() {
  size_t m = 0;
  const size_t v[] = {ColGeo<16>::SMEM, ColGeo<24>::SMEM, ColGeo<32>::SMEM, ColGeo<48>::SMEM, ColGeo<64>::SMEM,
                      ColGeo<96>::SMEM, ColGeo<128>::SMEM, ColGeo<192>::SMEM, ColGeo<256>::SMEM, ColGeo<384>::SMEM,
                      ColGeo<512>::SMEM, ColGeo<768>::SMEM, ColGeo<1024>::SMEM, ColGeo<1536>::SMEM, ColGeo<2048>::SMEM};
  for (size_t x : v) m = x > m ? x : m;
  return m;
}

#define SGP_MULTI_ROW(NAME, BODY)                                                                          \
  template <bool FP64>                                                                                    \
  __global__ void __launch_bounds__(kRowBlock, 2) NAME(const ImgDesc* __restrict__ imgs, const int2* __restrict__ items, \
                                                    int n_items, int extra) {                              \
    const int it = blockIdx.x;                                                                            \
    if (it >= n_items) return;                                                                            \
    const int W = imgs[items[it].x].W;                                                                    \
    (void)extra;                                                                                          \
    SGP_SWITCH_SIDE(W, BODY)                                                                              \
  }

// the same with the reduction precision fixed (a plain kernel, for units that build one variant)
#define SGP_MULTI_ROW_FIXED(NAME, BODY, FP64V)                                                            \
  __global__ void __launch_bounds__(kRowBlock, 2) NAME(const ImgDesc* __restrict__ imgs, const int2* __restrict__ items, \
                                                    int n_items, int extra) {                              \
    constexpr bool FP64 = FP64V;                                                                          \
    const int it = blockIdx.x;                                                                            \
    if (it >= n_items) return;                                                                            \
    const int W = imgs[items[it].x].W;                                                                    \
    (void)extra;                                                                                          \
    SGP_SWITCH_SIDE(W, BODY)                                                                              \
  }

}  // namespace sgp

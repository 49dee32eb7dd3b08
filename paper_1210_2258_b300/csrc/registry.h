// Kernel registry: function pointers and launch geometry of the size-templated passes.
#pragma once
#include <cuda_runtime.h>
#include <stddef.h>

namespace sgp {

constexpr int kNumSides = 15;
constexpr int kSides[kNumSides] = {16, 24, 32, 48, 64, 96, 128, 192, 256, 384, 512, 768, 1024, 1536, 2048};
inline int side_index(int n) {
  for (int i = 0; i < kNumSides; ++i)
    if (kSides[i] == n) return i;
  return -1;
}

enum RowOp {
  ROP_SGP_UPDATE = 0, ROP_SGP_GRAD, ROP_SGP_Y, ROP_SGP_AD, ROP_SGP_ARMX, ROP_RL_UPDATE, ROP_RL_RATIO,
  ROP_MINMAX, ROP_R2C, ROP_C2R, ROP_SGP_LAND, ROP_COUNT
};
// column variants: COL_KHAT, COL_1TOP, COL_1TOP_CONJ, COL_PTO1 (any p), COL_PTOV, COL_PTO1 for p = 1
constexpr int kColModes = 6;
constexpr int kColPto1P1 = 5;

constexpr int kTwiddleUnits = 8;   // translation units with their own twiddle table (null: none)

struct Registry {
  const void* row[ROP_COUNT][2][kNumSides];   // [op][fp64][side]
  const void* col[kColModes][kNumSides];      // [variant][side]
  size_t row_smem[kNumSides], col_smem[kNumSides];
  int row_rows[kNumSides], col_cols[kNumSides];
  // narrow column variant of the one side that has it (kNarrowSide): [variant]
  const void* col_narrow[kColModes];
  size_t col_narrow_smem;
  int col_narrow_cols;
  cudaError_t (*twiddle_init[kTwiddleUnits])(const float2*);
  // multi-size kernels (one launch covers problems of different sides): row ops, and the column
  // passes 1 -> p (index 0), p -> 1 for any p (index 1) and for p = 1 (index 2); dynamic shared
  // memory = max over the sides
  const void* row_multi[ROP_COUNT][2];
  const void* col_multi[3];
  size_t row_multi_smem, col_multi_smem;
};

// one per translation unit; register_all (runtime.cu) calls every one
void register_small(Registry&);
void register_mid(Registry&);
void register_mid_b(Registry&);
void register_large(Registry&);
void register_large_b(Registry&);
void register_multi_sgp_a(Registry&);
void register_multi_sgp_b(Registry&);
void register_multi_armx_f(Registry&);
void register_multi_armx_d(Registry&);
void register_multi_land_f(Registry&);
void register_multi_land_d(Registry&);
void register_multi_rest(Registry&);

}  // namespace sgp

// Verification kernel of the reductions: pixel terms of one kind, computed by the same device
// functions as the row passes (KL term, Armijo difference, scaled-BB terms), summed by the same
// per-thread accumulator, block reduction and fixed-order controller sum (reduce.cuh), so that a
// test can compare the library's sum of FP32 terms with an exact sum of the very same terms.
#pragma once
#include "rowops.cuh"
#include "state.cuh"

namespace sgp {

enum SumKind { SUM_VALUES = 0, SUM_KL = 1, SUM_ARMIJO = 2, SUM_BB0 = 3 };   // SUM_BB0 + 0..3: BB terms
constexpr int kSumPerThread = 32;   // terms per thread, as in a 2048-wide row pass (16 pixel pairs)

template <bool FP64>
__global__ void __launch_bounds__(kRowBlock) k_sum_terms(int kind, const float* __restrict__ a,
                                                        const float* __restrict__ b, const float* __restrict__ c,
                                                        size_t n, float lam, float* __restrict__ terms,
                                                        double* __restrict__ part, CtrlState* cs, int nblocks,
                                                        double* __restrict__ out) {
  Acc<FP64> acc[1];
  const size_t base = size_t(blockIdx.x) * kRowBlock * kSumPerThread;
  for (int q = 0; q < kSumPerThread; ++q) {
    const size_t i = base + threadIdx.x + size_t(q) * kRowBlock;
    if (i >= n) break;
    float t = 0.0f;
    if (kind == SUM_VALUES) {
      t = a[i];
    } else if (kind == SUM_KL) {
      float rm;
      t = kl_ratio(a[i], b[i], rm);                  // g, u0 = A f + b
    } else if (kind == SUM_ARMIJO) {                 // g, u0, A d
      const float g = a[i], u0 = b[i], ad = c[i];
      if (g < 0.0f) t = 0.0f;
      else if (g == 0.0f) t = lam * ad;
      else if (u0 <= 0.0f) t = f_inf();
      else t = armijo_term(lam, fdiv(ad, u0), u0 - g, g);
    } else {                                         // s, z, D
      const float D = c[i];
      if (D > 0.0f) {
        float tb[4];
        bb_terms(a[i], b[i], D, tb);
        t = tb[(kind - SUM_BB0) & 3];
      }
    }
    if (terms) terms[i] = t;
    acc[0].add(t);
  }
  block_sum_store<1, FP64>(acc, part + size_t(blockIdx.x) * kPartStride);
  if (arrive_last(cs, nblocks)) {
    ImgDesc d = {};
    d.part = part;
    d.n_row_items = nblocks;
    double r[1];
    ctrl_sum<1, FP64>(d, 0, r, false);
    if (threadIdx.x == 0) *out = r[0];
  }
}

}  // namespace sgp

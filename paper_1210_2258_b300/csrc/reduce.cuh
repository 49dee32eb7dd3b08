// Reductions of the row passes and of the controllers.
//
// Per thread, the "mixed" variant (FP64 = true) accumulates its pixel terms error-free: each term
// is added to a running FP32 value hi with Knuth's two-sum, which also yields the exact rounding
// error of that addition, and the errors are summed in a second FP32 value lo.  The pair hi + lo
// is the sum to about (n u)^2 of the sum of |terms| (u = 2^-24, n <= 48 terms a thread), far below
// the 1e-12 an FP64 sum of the same FP32 terms carries.  Above the thread every sum travels as an
// unevaluated pair of FP32 values (hi + lo, combined with the same two-sum: about 48 significand
// bits) and is converted to FP64 only for the controller's scalar logic: FP64 arithmetic is slow
// on this part, FP32 is not.  The plain-FP32 variant (FP64 = false) sums single FP32 values from
// the thread up and takes the decisions in FP32.
//
// A block stores its NS sums as float2 (hi, lo) in consecutive 8-byte slots of its item's
// partial-sum record; the controller of a problem adds the records of all its items in a fixed
// order (deterministic, no atomics on values).  The controller runs at the end of a row pass in
// the block that finishes last (arrive_last), so no separate launch is needed for it.
#pragma once
#include <math.h>
#include "state.cuh"

namespace sgp {

// value hi + lo with |lo| <= ulp(hi)/2 after ff_add
struct FF {
  float hi, lo;
};

// Per-thread accumulator of pixel terms (see the top of this file).
template <bool FP64> struct Acc;
template <> struct Acc<true> {
  float hi = 0.0f, lo = 0.0f;   // value hi + lo
  __device__ __forceinline__ void add(float x) {
    const float s = hi + x;                          // two-sum: s + e = hi + x exactly
    const float bv = s - hi;
    const float e = (hi - (s - bv)) + (x - bv);
    lo += e;
    hi = s;
  }
  __device__ __forceinline__ FF pair() const {      // renormalised: |lo| <= ulp(hi)/2
    const float s = hi + lo, bv = s - hi;
    return FF{s, (hi - (s - bv)) + (lo - bv)};
  }
};
template <> struct Acc<false> {
  float hi = 0.0f;
  __device__ __forceinline__ void add(float x) { hi += x; }
  __device__ __forceinline__ FF pair() const { return FF{hi, 0.0f}; }
};
__device__ __forceinline__ FF ff_add(FF a, FF b) {
  const float s = a.hi + b.hi;                       // two-sum: s + e = a.hi + b.hi exactly
  const float bv = s - a.hi;
  const float e = (a.hi - (s - bv)) + (b.hi - bv);
  const float lo = e + (a.lo + b.lo);
  const float hi = s + lo;                           // fast two-sum renormalisation
  return FF{hi, lo - (hi - s)};
}
__device__ __forceinline__ FF ff_shfl_xor(FF a, int o) {
  return FF{__shfl_xor_sync(0xffffffffu, a.hi, o), __shfl_xor_sync(0xffffffffu, a.lo, o)};
}
__device__ __forceinline__ FF ff_warp_sum(FF v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v = ff_add(v, ff_shfl_xor(v, o));
  return v;
}
__device__ __forceinline__ float warp_sum(float v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}
__device__ __forceinline__ double ff_value(FF a) { return double(a.hi) + double(a.lo); }

// a partial-sum slot holds one float2 (hi, lo)
__device__ __forceinline__ void slot_store(double* slot, FF v) {
  *reinterpret_cast<float2*>(slot) = make_float2(v.hi, v.lo);
}
__device__ __forceinline__ FF slot_load(const double* slot) {
  const float2 v = __ldcg(reinterpret_cast<const float2*>(slot));   // L2: written by other blocks
  return FF{v.x, v.y};
}

// Sum NS per-thread values over the block; thread 0 stores them to out[0..NS).
template <int NS, bool FP64>
__device__ __forceinline__ void block_sum_store(const Acc<FP64> (&loc)[NS], double* out) {
  __shared__ FF red[NS][kRowBlock / 32];
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
#pragma unroll
  for (int s = 0; s < NS; ++s) {
    FF v;
    if (FP64) v = ff_warp_sum(loc[s].pair());
    else v = FF{warp_sum(loc[s].pair().hi), 0.0f};
    if (lane == 0) red[s][wid] = v;
  }
  __syncthreads();
  if (wid == 0) {
#pragma unroll
    for (int s = 0; s < NS; ++s) {
      FF v = lane < (int)(blockDim.x >> 5) ? red[s][lane] : FF{0.0f, 0.0f};
      if (FP64) v = ff_warp_sum(v);
      else v = FF{warp_sum(v.hi), 0.0f};
      if (lane == 0) slot_store(out + s, v);
    }
  }
  __syncthreads();
}

// Sum NA slots (from slotA) over list A and NB slots (from slotB) over list B of this problem's
// items (row list or row-view list) in a fixed order; the results are on every thread of the block.
// Pair arithmetic (or plain FP32 sums) throughout: each result is converted to double once, by
// one lane (an FP64 operation has a latency of about 60 cycles on this part, an FP32 one 4).
// This runs in the one block that finishes a pass last, while the rest of the GPU waits for it,
// so its latency is what counts.  Up to 8 sums: warp w sums slot w over all items, each lane 8
// items per load round (all loads in flight together), then one shuffle tree; a single global
// round trip and no block-level tree.  More sums: every thread loads all sums of one item, a
// shuffle tree per warp, a tree over the warps (at most 8).
template <int NA, int NB, bool FP64>
__device__ void ctrl_sums(const ImgDesc& d, int slotA, bool viewA, double* resA, int slotB, bool viewB,
                          double* resB) {
  constexpr int NS = NA + NB;
  static_assert(NS >= 1 && NS <= 32, "at most 32 sums per call");
  if constexpr (NS <= 8) {
    __shared__ double fin8[NS];
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = int(blockDim.x >> 5);
    for (int k = wid; k < NS; k += nw) {
      const bool isA = k < NA;
      const bool view = isA ? viewA : viewB;
      const int n = view ? d.n_rv_items : d.n_row_items;
      const double* b = (view ? d.partv : d.part) + (isA ? slotA + k : slotB + (k - NA));
      FF acc{0.0f, 0.0f};
      for (int i0 = 0; i0 < n; i0 += 256) {
        FF v[8];                                    // every load of the round before any use
#pragma unroll
        for (int q = 0; q < 8; ++q) {
          const int i = i0 + lane + 32 * q;
          v[q] = i < n ? slot_load(b + size_t(i) * kPartStride) : FF{0.0f, 0.0f};
        }
#pragma unroll
        for (int q = 0; q < 8; ++q) {
          if (FP64) acc = ff_add(acc, v[q]);
          else acc.hi += v[q].hi;
        }
      }
      acc = FP64 ? ff_warp_sum(acc) : FF{warp_sum(acc.hi), 0.0f};
      if (lane == 0) fin8[k] = FP64 ? ff_value(acc) : double(acc.hi);
    }
    __syncthreads();
#pragma unroll
    for (int k = 0; k < NA; ++k) resA[k] = fin8[k];
#pragma unroll
    for (int k = 0; k < NB; ++k) resB[k] = fin8[NA + k];
    __syncthreads();
  } else {
    static_assert(kCtrlBlock <= 256 && kRowBlock <= 256, "the tree over the warps takes at most 8 warps");
    __shared__ FF red[NS][8];
    __shared__ double fin[NS];
    const int nA = viewA ? d.n_rv_items : d.n_row_items;
    const int nB = viewB ? d.n_rv_items : d.n_row_items;
    const double* bA = (viewA ? d.partv : d.part) + slotA;
    const double* bB = (viewB ? d.partv : d.part) + slotB;
    const int n = NB > 0 ? max(nA, nB) : nA;
    FF loc[NS];
#pragma unroll
    for (int k = 0; k < NS; ++k) loc[k] = FF{0.0f, 0.0f};
    for (int i = threadIdx.x; i < n; i += blockDim.x) {
      FF v[NS];                                       // every load of the item before any use
#pragma unroll
      for (int k = 0; k < NA; ++k) v[k] = i < nA ? slot_load(bA + size_t(i) * kPartStride + k) : FF{0.0f, 0.0f};
#pragma unroll
      for (int k = 0; k < NB; ++k) v[NA + k] = i < nB ? slot_load(bB + size_t(i) * kPartStride + k) : FF{0.0f, 0.0f};
#pragma unroll
      for (int k = 0; k < NS; ++k) {
        if (FP64) loc[k] = ff_add(loc[k], v[k]);
        else loc[k].hi += v[k].hi;
      }
    }
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = int(blockDim.x >> 5);
#pragma unroll
    for (int k = 0; k < NS; ++k) {
      const FF v = FP64 ? ff_warp_sum(loc[k]) : FF{warp_sum(loc[k].hi), 0.0f};
      if (lane == 0) red[k][wid] = v;
    }
    __syncthreads();
    if (wid == 0) {
#pragma unroll
      for (int k = 0; k < NS; ++k) {
        FF v = lane < nw ? red[k][lane] : FF{0.0f, 0.0f};
#pragma unroll
        for (int o = 4; o > 0; o >>= 1) {          // lanes >= 8 hold zeros and never reach lanes < 8
          const FF w = ff_shfl_xor(v, o);
          if (FP64) v = ff_add(v, w);
          else v.hi += w.hi;
        }
        if (lane == 0) red[k][0] = v;
      }
      __syncwarp();
      if (lane < NS) fin[lane] = FP64 ? ff_value(red[lane][0]) : double(red[lane][0].hi);
    }
    __syncthreads();
#pragma unroll
    for (int k = 0; k < NA; ++k) resA[k] = fin[k];
#pragma unroll
    for (int k = 0; k < NB; ++k) resB[k] = fin[NA + k];
    __syncthreads();
  }
}
// Sum NS slots over this problem's items (row list or row-view list); see ctrl_sums.
template <int NS, bool FP64>
__device__ void ctrl_sum(const ImgDesc& d, int slot, double (&res)[NS], bool view_list) {
  ctrl_sums<NS, 0, FP64>(d, slot, view_list, res, 0, false, nullptr);
}

// min over SLOT_MIN and max over SLOT_MAX (plain doubles) of this problem's row items
__device__ inline void ctrl_minmax(const ImgDesc& d, double& mn, double& mx) {
  __shared__ double rmn[kCtrlBlock / 32], rmx[kCtrlBlock / 32];
  double a = INFINITY, b = 0.0;
  for (int i = threadIdx.x; i < d.n_row_items; i += blockDim.x) {
    const double* p = d.part + size_t(i) * kPartStride;
    a = fmin(a, __ldcg(p + SLOT_MIN));
    b = fmax(b, __ldcg(p + SLOT_MAX));
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    a = fmin(a, __shfl_xor_sync(0xffffffffu, a, o));
    b = fmax(b, __shfl_xor_sync(0xffffffffu, b, o));
  }
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  if (lane == 0) { rmn[wid] = a; rmx[wid] = b; }
  __syncthreads();
  mn = INFINITY; mx = 0.0;
  for (int w = 0; w < int(blockDim.x >> 5); ++w) { mn = fmin(mn, rmn[w]); mx = fmax(mx, rmx[w]); }
  __syncthreads();
}

// Called once by every block of a problem in a pass, after the block's partial sums are stored
// (by its thread 0).  True in the block that arrives last: it then sees every block's partials.
// The last block resets the counter, so the next pass starts from zero.  Nothing waits.
__device__ __forceinline__ bool arrive_last(CtrlState* c, int n_blocks) {
  __shared__ int s_last;
  __syncthreads();
  if (threadIdx.x == 0) {
    // acquire-release at device scope: thread 0 stored this block's partials before the add
    // (release); the last block then sees every other block's partials (acquire) and passes them
    // to its other threads through the barrier below
    unsigned prev;
    asm volatile("atom.add.acq_rel.gpu.global.u32 %0, [%1], 1;" : "=r"(prev) : "l"(&c->arrive) : "memory");
    const int last = prev == unsigned(n_blocks - 1);
    if (last) c->arrive = 0u;
    s_last = last;
  }
  __syncthreads();
  return s_last != 0;
}

}  // namespace sgp

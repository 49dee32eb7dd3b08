// Column passes: FFT down the columns of packed spectra, multiply by the PSF spectra, inverse FFT.
//
// A tile holds C adjacent spectrum columns x all H rows in shared memory (global loads and stores
// are C*8 contiguous bytes per row).  Column 0 carries the DC and Nyquist columns of the row
// transform as real / imaginary part; with Z its column FFT, F0[k] = (Z[k] + conj Z[-k])/2 and
// FM[k] = (Z[k] - conj Z[-k])/(2i), and a product with the PSF spectrum becomes
//     Z[k] P[k] + conj(Z[-k]) Q[k],   P = (K0 + KM)/2,  Q = (K0 - KM)/2
// (K0, KM the PSF spectrum on those two columns; conjugated for the transpose), which is again
// the packed spectrum of two real columns.
//
// Modes
//   COL_KHAT      : forward only; writes the PSF spectrum (P in column 0, Q in a side column),
//                   scaled by 1/(H*M*sum K) and, for centred PSFs, by (-1)^(kr+kc) (origin shift).
//   COL_1TOP      : one input plane -> nout planes, out_j = IFFT(FFT(in) . K_j)   (A_j f, Eq. projection)
//   COL_1TOP_CONJ : as COL_1TOP with conj K_j (correlation, used for alpha_j = K_j (x) M_S)
//   COL_PTO1      : nin planes -> one plane, out = IFFT(sum_j FFT(in_j) . conj K_j)
//                   (sum_j A_j^T y_j, Eq. backprojection)
//   COL_PTOV      : per view (one item per view and tile), out_{j+1} = IFFT(FFT(in_j) . conj K_j);
//                   with the column transform linear, a view sum afterwards (k_view_sum) gives
//                   COL_PTO1's plane with p times the parallelism
#pragma once
#include "fft.cuh"
#include "state.cuh"

namespace sgp {


// columns of 2048 (the iteration's column passes at the largest supported side, one block per SM
// over the PSF band: latency-bound) form their twiddles from fewer table entries (stage_twiddles)
template <int H> constexpr bool kColPowTwiddles = H == 2048;

template <int H, bool NARROW = false> struct ColGeo {
  using P = typename std::conditional<NARROW, ColPlanNarrow<H>, ColPlan<H>>::type;
  static constexpr int T = P::T, E = P::E;
  static constexpr int C = kColBlock / T;
  static constexpr int ROWSP = col_rows_padded<H>();
  static constexpr size_t SMEM = size_t(C) * ROWSP * sizeof(float2);
};

template <class P, int C>
__device__ __forceinline__ void col_load(const ColLayout<C>& x, const float2* __restrict__ src, int M, int t, bool act) {
  constexpr int T = P::T, E = P::E;
  constexpr bool IL = spec_interleaved(P::L);
  if (act) {
#pragma unroll
    for (int q = 0; q < E; ++q) {
      const int i = t + q * T;
      x(i) = src[spec_row_off(i, M, IL)];
    }
  }
}

// product of the column spectrum with the PSF spectrum for the element (row i) owned by a thread
template <int H, int C, bool CONJ>
__device__ __forceinline__ float2 col_product(const ColLayout<C>& x, int i, int col, float2 X,
                                              const float2* __restrict__ kh, const float2* __restrict__ kq, int M) {
  constexpr bool IL = spec_interleaved(H);
  float2 K = __ldg(&kh[spec_row_off(i, M, IL) + (IL ? 4 : 1) * col]);
  if (CONJ) K = cconj(K);
  if (col != 0) return cmul(X, K);
  float2 Q = __ldg(&kq[i]);
  if (CONJ) Q = cconj(Q);
  const float2 Xm = x((H - i) % H);
  return cadd(cmul(X, K), cmul(cconj(Xm), Q));
}

// MODE as above; NV = number of views summed by COL_PTO1 (0: any number, runtime loop).
// One block per item (job, col0 | view << 16): runtime loops around the transforms make the
// register allocator keep every stage's addresses live, so views are separate items where possible.
template <int H, int MODE, int NV = 0, bool NARROW = false>
__device__ __forceinline__ void b_col(const ColJob* __restrict__ jobs, const int2* __restrict__ items, int n_items) {
  pdl_enter();
  using G = ColGeo<H, NARROW>;
  using CP = typename G::P;
  constexpr int C = G::C, T = G::T, E = G::E;
  extern __shared__ float2 smem[];
  // lanes: for tiles of up to 8 columns, 4 consecutive lanes take 4 consecutive rows of one column,
  // then the next column, so a warp's global accesses are runs of 4 rows x C columns of the
  // interleaved spectrum layout; wider tiles keep the columns fastest (4 rows of a 16- or more
  // column tile would fall into the same shared-memory banks)
  // (the mapping only affects speed: addresses follow the plane's layout, spec_row_off)
  constexpr bool RUNS = T % 4 == 0 && C <= 8;
  constexpr bool IL = spec_interleaved(H);
  const int c = RUNS ? int(threadIdx.x >> 2) % C : int(threadIdx.x) % C;
  const int t = RUNS ? int(threadIdx.x & 3) + 4 * int(threadIdx.x / (4 * C)) : int(threadIdx.x) / C;
  const ColLayout<C> x{smem + c};
  {
    const int it = blockIdx.x;
    if (it >= n_items) return;
    const int2 item = items[it];
    const ColJob& jb = jobs[item.x];
    if (jb.ctrl && jb.ctrl->done >= 1) return;
    const int M = jb.M;
    const int col = (item.y & 0xffff) + c;
    const bool act = col < M;
    if (MODE == COL_KHAT) {
      col_load<CP, C>(x, jb.in + (IL ? 4 : 1) * col, M, t, act);
      __syncthreads();
      fft_inplace<H, false, ColLayout<C>, CP, kColPowTwiddles<H>>(x, t, act);
      if (act) {
        float2 outv[E], qv[E];
        const float s = jb.scale;
#pragma unroll
        for (int q = 0; q < E; ++q) {
          const int i = t + q * T;
          const float2 X = x(i);
          if (col == 0) {
            const float2 Xm = cconj(x((H - i) % H));
            float2 F0 = cscale(cadd(X, Xm), 0.5f);
            float2 FM = cscale(csub(X, Xm), 0.5f);
            FM = make_float2(FM.y, -FM.x);               // divide by i
            float s0 = s, sM = s;
            if (!jb.corner) {
              if (i & 1) { s0 = -s0; sM = -sM; }
              if (M & 1) sM = -sM;
            }
            F0 = cscale(F0, s0);
            FM = cscale(FM, sM);
            outv[q] = cscale(cadd(F0, FM), 0.5f);
            qv[q] = cscale(csub(F0, FM), 0.5f);
          } else {
            const float sg = (!jb.corner && ((i + col) & 1)) ? -s : s;
            outv[q] = cscale(X, sg);
            qv[q] = make_float2(0.0f, 0.0f);
          }
        }
#pragma unroll
        for (int q = 0; q < E; ++q) {
          const int i = t + q * T;
          jb.out[spec_row_off(i, M, IL) + (IL ? 4 : 1) * col] = outv[q];
          if (col == 0) jb.khatq[i] = qv[q];
        }
      }
      __syncthreads();
    } else if (MODE == COL_1TOP || MODE == COL_1TOP_CONJ || MODE == COL_PTOV) {
      constexpr bool CJ = MODE != COL_1TOP;
      {
        const int j = item.y >> 16;
        col_load<CP, C>(x, jb.in + (MODE == COL_PTOV ? size_t(j) * jb.plane_stride : size_t(0)) + (IL ? 4 : 1) * col,
                        M, t, act);
        __syncthreads();
        fft_inplace<H, false, ColLayout<C>, CP, kColPowTwiddles<H>>(x, t, act);
        float2 v[E];
        if (act) {
          const float2* kh = jb.khat + size_t(j) * jb.plane_stride;
          const float2* kq = jb.khatq + size_t(j) * H;
#pragma unroll
          for (int q = 0; q < E; ++q) {
            const int i = t + q * T;
            v[q] = col_product<H, C, CJ>(x, i, col, x(i), kh, kq, M);
          }
        }
        __syncthreads();
        if (act) {
#pragma unroll
          for (int q = 0; q < E; ++q) x(t + q * T) = v[q];
        }
        __syncthreads();
        fft_inplace<H, true, ColLayout<C>, CP, kColPowTwiddles<H>>(x, t, act);
        if (act) {
          float2* dst = jb.out + size_t(MODE == COL_PTOV ? j + 1 : j) * jb.plane_stride + (IL ? 4 : 1) * col;
#pragma unroll
          for (int q = 0; q < E; ++q) {
            const int i = t + q * T;
            dst[spec_row_off(i, M, IL)] = x(i);
          }
        }
        __syncthreads();
      }
    } else if (NV == 1) {  // COL_PTO1, one view: the product goes straight back to x
      col_load<CP, C>(x, jb.in + (IL ? 4 : 1) * col, M, t, act);
      __syncthreads();
      fft_inplace<H, false, ColLayout<C>, CP, kColPowTwiddles<H>>(x, t, act);
      float2 v[E];
      if (act) {
#pragma unroll
        for (int q = 0; q < E; ++q) {
          const int i = t + q * T;
          v[q] = col_product<H, C, true>(x, i, col, x(i), jb.khat, jb.khatq, M);
        }
      }
      __syncthreads();
      if (act) {
#pragma unroll
        for (int q = 0; q < E; ++q) x(t + q * T) = v[q];
      }
      __syncthreads();
      fft_inplace<H, true, ColLayout<C>, CP, kColPowTwiddles<H>>(x, t, act);
      if (act) {
        float2* dst = jb.out + (IL ? 4 : 1) * col;
#pragma unroll
        for (int q = 0; q < E; ++q) {
          const int i = t + q * T;
          dst[spec_row_off(i, M, IL)] = x(i);
        }
      }
      __syncthreads();
    } else {  // COL_PTO1, p views: the sum over views accumulates in the output column (L2-resident;
              // a register accumulator live across the p transforms spilled), then back into x
      const int nin = NV > 0 ? NV : jb.nin;
      float2* o = jb.out + (IL ? 4 : 1) * col;
#pragma unroll 1
      for (int j = 0; j < nin; ++j) {
        col_load<CP, C>(x, jb.in + size_t(j) * jb.plane_stride + (IL ? 4 : 1) * col, M, t, act);
        __syncthreads();
        fft_inplace<H, false, ColLayout<C>, CP, kColPowTwiddles<H>>(x, t, act);
        if (act) {
          const float2* kh = jb.khat + size_t(j) * jb.plane_stride;
          const float2* kq = jb.khatq + size_t(j) * H;
#pragma unroll
          for (int q = 0; q < E; ++q) {
            const int i = t + q * T;
            const float2 pr = col_product<H, C, true>(x, i, col, x(i), kh, kq, M);
            const size_t oi = spec_row_off(i, M, IL);
            o[oi] = j == 0 ? pr : cadd(o[oi], pr);   // this thread's own elements only
          }
        }
        __syncthreads();
      }
      if (act) {
#pragma unroll
        for (int q = 0; q < E; ++q) {
          const int i = t + q * T;
          x(i) = o[spec_row_off(i, M, IL)];
        }
      }
      __syncthreads();
      fft_inplace<H, true, ColLayout<C>, CP, kColPowTwiddles<H>>(x, t, act);
      if (act) {
        float2* dst = jb.out + (IL ? 4 : 1) * col;
#pragma unroll
        for (int q = 0; q < E; ++q) {
          const int i = t + q * T;
          dst[spec_row_off(i, M, IL)] = x(i);
        }
      }
      __syncthreads();
    }
  }
}

template <int H, int MODE, int NV = 0, bool NARROW = false>
__global__ void __launch_bounds__(kColBlock) k_col(const ColJob* __restrict__ jobs, const int2* __restrict__ items,
                                                  int n_items) {
  b_col<H, MODE, NV, NARROW>(jobs, items, n_items);

}

}  // namespace sgp

// Row passes: packed real FFTs along image rows with the method's pointwise work fused in.
//
// A row of W reals is handled as M = W/2 complex values z[n] = x[2n] + i x[2n+1]; one complex
// FFT of length M plus a pairwise (k, M-k) post-processing gives the half spectrum X[0..M]; X[0]
// and X[M] are real and are stored together in slot 0 (re = X[0], im = X[M]), so a spectrum row is
// exactly M complex values (16-byte aligned, the same bytes as the real row).
//
// Pointwise formulas (Sect. 1, 2.1-2.4):
//   ratio      r = g / (A f + b)                     (0 where g = 0 or outside S)
//   KL term    g ln(g/u) + u - g = g phi((u-g)/g),   phi(t) = t - log(1+t), u = A f + b
//   Armijo     J(f + lam d) - J(f) = sum lam Ad - g log(1 + lam Ad / u)
//              = sum (u - g) q + g phi(q),  q = lam Ad / u         (no cancellation)
//   scaling    D = w clip(f, L1, L2), w = 1/p (periodic) or M_R/alpha (boundary), Eq. (Dk),(Dkbound)
//   gradient   grad = sum_j A_j^T (1 - r_j) on R (0 outside R), Eq. (KLgrad),(gradientboundary);
//              the row passes transform r - 1, so no 1 - A^T r cancellation
//   step       y = P_+(f - alpha D grad), d = y - f, Eq. (diry); flux mode y = max(0, x - mu D)
#pragma once
#include "control.cuh"
#include "fft.cuh"
#include "state.cuh"

namespace sgp {

// Row tiling of width W: T threads per row holding E complex values each, ROWS rows per block of
// kRowBlock threads.  Rows of 2048 reals run one warp per row (WARP: the four-step transform of
// warp_fft1024, no block barrier inside the transform, 32 values per lane); the other widths run
// the block Stockham transform of their Plan.  The launch bounds ask for BLOCKS_HOT (the passes
// whose registers are held to 64 for the block transform) or BLOCKS_MIN (the others) resident
// blocks per SM: 2 for the warp rows, i.e. at most 128 registers per thread.
template <int W> struct RowGeo {
  static constexpr int M = W / 2;
  using P = Plan<M>;
  static constexpr bool WARP = (M == 1024);
  static constexpr int T = WARP ? 32 : P::T, E = WARP ? 32 : P::E;
  static constexpr int ROWS = kRowBlock / T;
  static constexpr int PITCH = RowLayout<M>::pitch;
  static constexpr size_t SMEM = size_t(ROWS) * PITCH * sizeof(float2);
  static constexpr int BLOCKS_HOT = WARP ? 2 : 4;
  static constexpr int BLOCKS_MIN = WARP ? 2 : 1;
};

// Pixel pairs per thread whose global loads are issued together, before any of them is used and
// before any global store: a store in between would keep the compiler from moving later loads
// above it (it cannot rule out aliasing), leaving one load latency per pixel pair.  The batch loop
// itself is not unrolled (code size), and the passes that use it are held to 64 registers
// (4 blocks per SM) by their launch bounds.
template <int E, int WANT> constexpr int batch_of() {
  return E % WANT == 0 ? WANT : (E % 4 == 0 ? 4 : (E % 2 == 0 ? 2 : 1));
}

// ------------------------------------------------------------------------------ pointwise math
// Divisions whose result only enters a sum of pixel terms (the KL value, the Armijo differences)
// use the fast form a * rcp(b) (error <= 2 ulp for the normal, positive divisors that reach it);
// the ratio and the BB sums, which steer the iteration, keep correctly rounded division.
__device__ __forceinline__ float fdiv(float a, float b) { return __fdividef(a, b); }

// phi(t) = t - log1p(t); for |t| < 1/8 the alternating series t^2 sum_{n>=2} (-t)^(n-2)/n
// (truncated after n = 9: relative error < 1.3e-8, below FP32 rounding) avoids the cancellation
// of the direct form.
__device__ __forceinline__ float phi_series(float t) {
  float p = -1.0f / 9.0f;
  p = fmaf(t, p, 1.0f / 8.0f);
  p = fmaf(t, p, -1.0f / 7.0f);
  p = fmaf(t, p, 1.0f / 6.0f);
  p = fmaf(t, p, -1.0f / 5.0f);
  p = fmaf(t, p, 1.0f / 4.0f);
  p = fmaf(t, p, -1.0f / 3.0f);
  p = fmaf(t, p, 0.5f);
  return t * t * p;
}
__device__ __forceinline__ float phi_t(float t) {
  if (fabsf(t) < 0.125f) return phi_series(t);
  return t - log1pf(t);
}
// true on every active lane of the warp when p holds on all of them (the warp then takes a
// branch-free path; the lanes of a row pass share their loop bounds)
__device__ __forceinline__ bool warp_all(bool p) { return __all_sync(__activemask(), p); }
__device__ __forceinline__ float f_inf() { return __int_as_float(0x7f800000); }

// KL pixel term g ln(g/u0) + u0 - g and the ratio r - 1 = (g - u0)/u0 (r = 0 where g = 0 or
// u0 <= 0; g < 0 marks a pixel outside S: both 0).  With z = (u0 - g)/(u0 + g), ln(u0/g) =
// 2 atanh(z) = 2 (z + z^3/3 + z^5/5 + ...) and u0 - g = 2 g z/(1 - z), so the term is
// (u0 - g) z - 2 g z^3 S(z^2), S(w) = sum_k w^k/(2k+3): both parts are O(z^2), no cancellation.
// For |z| < 1/3 (1/2 < u0/g < 2) S is truncated after w^6 (relative error < 4e-8 of the second
// part, itself < 8 % of the term); outside, the direct form has no cancellation to speak of.
// The series branch of kl_ratio at a pixel with g > 0, u0 > 0: z = (u0 - g)/(u0 + g) from the caller,
// which checked |z| < 1/3 (the same operations as kl_ratio takes there)
__device__ __forceinline__ float kl_series(float g, float u0, float z, float& rm1) {
  const float dlt = u0 - g;
  rm1 = -dlt / u0;
  const float w = z * z;
  float S = 1.0f / 15.0f;
  S = fmaf(w, S, 1.0f / 13.0f);
  S = fmaf(w, S, 1.0f / 11.0f);
  S = fmaf(w, S, 1.0f / 9.0f);
  S = fmaf(w, S, 1.0f / 7.0f);
  S = fmaf(w, S, 1.0f / 5.0f);
  S = fmaf(w, S, 1.0f / 3.0f);
  return fmaf(dlt, z, -2.0f * g * z * w * S);
}
__device__ __forceinline__ float kl_ratio(float g, float u0, float& rm1) {
  if (g < 0.0f) { rm1 = 0.0f; return 0.0f; }
  if (g == 0.0f) { rm1 = -1.0f; return u0; }
  if (u0 <= 0.0f) { rm1 = -1.0f; return f_inf(); }
  const float dlt = u0 - g;
  rm1 = -dlt / u0;
  const float z = fdiv(dlt, u0 + g);
  if (fabsf(z) < 1.0f / 3.0f) {
    const float w = z * z;
    float S = 1.0f / 15.0f;
    S = fmaf(w, S, 1.0f / 13.0f);
    S = fmaf(w, S, 1.0f / 11.0f);
    S = fmaf(w, S, 1.0f / 9.0f);
    S = fmaf(w, S, 1.0f / 7.0f);
    S = fmaf(w, S, 1.0f / 5.0f);
    S = fmaf(w, S, 1.0f / 3.0f);
    return fmaf(dlt, z, -2.0f * g * z * w * S);
  }
  return dlt - g * logf(fdiv(u0, g));
}
// One Armijo pixel term J(f + lam d) - J(f) at a pixel with g > 0 and u0 = A f + b > 0, from
// qb = A d / u0 and gm = u0 - g: (u0 - g) q + g phi(q), q = lam qb (+inf when u0 + lam A d <= 0).
__device__ __forceinline__ float armijo_term(float lam, float qb, float gm, float g) {
  const float q = lam * qb;                   // u0 + lam ad <= 0  <=>  q <= -1
  return q <= -1.0f ? f_inf() : fmaf(gm, q, g * phi_t(q));
}
// The four pixel terms of the scaled BB sums (Eq. BB1, BB2) at a pixel with D > 0:
// s^2 / D^2, s z / D, s z D, z^2 D^2.
__device__ __forceinline__ void bb_terms(float s, float z, float D, float (&t)[4]) {
  const float sd = s / D, zd = z * D;
  t[0] = sd * sd; t[1] = sd * z; t[2] = s * zd; t[3] = zd * zd;
}
// Armijo pixel terms J(f + lam d) - J(f) for the step lengths lam[0..N) at one pixel, u0 = A f + b,
// ad = A d; q = lam ad / u0 shares one division over the step lengths
template <int N, class A>
__device__ __forceinline__ void armijo_add(A (&acc)[N], const float (&lam)[N], float g, float u0, float ad) {
  if (g < 0.0f) return;                       // outside S
  if (g == 0.0f) {
#pragma unroll
    for (int l = 0; l < N; ++l) acc[l].add(lam[l] * ad);
    return;
  }
  if (u0 <= 0.0f) {
#pragma unroll
    for (int l = 0; l < N; ++l) acc[l].add(f_inf());
    return;
  }
  const float qb = fdiv(ad, u0), gm = u0 - g;
#pragma unroll
  for (int l = 0; l < N; ++l) acc[l].add(armijo_term(lam[l], qb, gm, g));
}
// Armijo terms at a pixel with g > 0, u0 > 0 and |qb| < 1/8, qb = fdiv(A d, u0): every
// |lam qb| < 1/8 as well (lam <= 1), so the terms are the series branch of armijo_term
template <int N, class A>
__device__ __forceinline__ void armijo_series(A (&acc)[N], const float (&lam)[N], float g, float u0, float qb) {
  const float gm = u0 - g;
#pragma unroll
  for (int l = 0; l < N; ++l) {
    const float q = lam[l] * qb;
    acc[l].add(fmaf(gm, q, g * phi_series(q)));
  }
}
// the same for the step lengths lam0 th^l (GEOM) or lam0 + l th (arithmetic), l = 0..N-1, as
// running products or sums (few registers)
template <int N, bool GEOM, class A>
__device__ __forceinline__ void armijo_add_prog(A (&acc)[N], float lam0, float th, float g, float u0, float ad) {
  if (g < 0.0f) return;
  float a;
  if (g == 0.0f) a = ad;                      // q = lam A d here
  else if (u0 > 0.0f) a = fdiv(ad, u0);
  else {
#pragma unroll
    for (int l = 0; l < N; ++l) acc[l].add(f_inf());
    return;
  }
  const float gm = u0 - g, dq = th * a;
  float q = lam0 * a;
#pragma unroll
  for (int l = 0; l < N; ++l) {
    if (g == 0.0f) acc[l].add(q);
    else acc[l].add(q <= -1.0f ? f_inf() : fmaf(gm, q, g * phi_t(q)));
    q = GEOM ? q * th : q + dq;
  }
}
// The row passes transform r - 1 on S (0 outside S) instead of r, so that
// sum_j A_j^T (r_j - 1) = -grad J_0 (Eq. gradientboundary with A_j^T 1 moved inside) is computed
// without the cancellation of 1 - A^T r when A^T r -> 1.

// ------------------------------------------------------------------------------ reductions
// min over strictly positive values and max, stored to out[0], out[1]
__device__ __forceinline__ void block_minmax_store(float mn, float mx, double* out) {
  __shared__ float rmn[kRowBlock / 32], rmx[kRowBlock / 32];
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    mn = fminf(mn, __shfl_xor_sync(0xffffffffu, mn, o));
    mx = fmaxf(mx, __shfl_xor_sync(0xffffffffu, mx, o));
  }
  if (lane == 0) { rmn[wid] = mn; rmx[wid] = mx; }
  __syncthreads();
  if (wid == 0) {
    mn = lane < (int)(blockDim.x >> 5) ? rmn[lane] : f_inf();
    mx = lane < (int)(blockDim.x >> 5) ? rmx[lane] : 0.0f;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      mn = fminf(mn, __shfl_xor_sync(0xffffffffu, mn, o));
      mx = fmaxf(mx, __shfl_xor_sync(0xffffffffu, mx, o));
    }
    if (lane == 0) { out[0] = mn; out[1] = mx; }
  }
  __syncthreads();
}

// ------------------------------------------------------------------------------ row FFT pieces
// Spectrum rows: only the columns < cb of the PSF band are stored and loaded; the loaded row is
// zero beyond (the PSF spectrum is zero there, so is every product with it).  cb = W/2: all.
template <int W>
__device__ __forceinline__ void row_load(const RowLayout<W / 2>& x, const float2* __restrict__ src, int t, bool act,
                                         int cb, bool il) {
  using G = RowGeo<W>;
  if (act) {
#pragma unroll
    for (int q = 0; q < G::E; ++q) {
      const int i = t + q * G::T;
      x(i) = i < cb ? src[il ? 4 * i : i] : make_float2(0.0f, 0.0f);
    }
  }
}
template <int W>
__device__ __forceinline__ void row_store(const RowLayout<W / 2>& x, float2* __restrict__ dst, int t, bool act,
                                          int cb, bool il) {
  using G = RowGeo<W>;
  if (act) {
#pragma unroll
    for (int q = 0; q < G::E; ++q) {
      const int i = t + q * G::T;
      if (i < cb) dst[il ? 4 * i : i] = x(i);
    }
  }
}

// packed half spectrum X -> Z with IFFT_M(Z) = M (x[2n] + i x[2n+1])
template <int W>
__device__ __forceinline__ void c2r_pre(const RowLayout<W / 2>& x, int t, bool act) {
  constexpr int M = W / 2, T = RowGeo<W>::T;
  if (!act) return;
  for (int k = t; k <= M / 2; k += T) {
    if (k == 0) {
      const float2 a = x(0);
      x(0) = make_float2(0.5f * (a.x + a.y), 0.5f * (a.x - a.y));
    } else {
      const float2 a = x(k), b = x(M - k);
      const float2 w = twl<W, true>(k);                       // exp(+2 pi i k / W)
      const float2 e1 = make_float2(a.x + b.x, a.y - b.y);    // a + conj b
      const float2 o1 = make_float2(a.x - b.x, a.y + b.y);    // a - conj b
      const float2 wo = cmul(w, o1);
      const float2 zk = make_float2(0.5f * (e1.x - wo.y), 0.5f * (e1.y + wo.x));   // (e1 + i w o1)/2
      const float2 e2 = make_float2(b.x + a.x, b.y - a.y);    // b + conj a
      const float2 o2 = make_float2(b.x - a.x, b.y + a.y);    // b - conj a
      const float2 wo2 = cmul(cconj(w), o2);
      const float2 zm = make_float2(0.5f * (e2.x + wo2.y), 0.5f * (e2.y - wo2.x));  // (e2 - i conj(w) o2)/2
      x(k) = zk;
      x(M - k) = zm;
    }
  }
}

// Z = FFT_M(z) -> packed half spectrum X
template <int W>
__device__ __forceinline__ void r2c_post(const RowLayout<W / 2>& x, int t, bool act) {
  constexpr int M = W / 2, T = RowGeo<W>::T;
  if (!act) return;
  for (int k = t; k <= M / 2; k += T) {
    if (k == 0) {
      const float2 a = x(0);
      x(0) = make_float2(a.x + a.y, a.x - a.y);
    } else {
      const float2 a = x(k), b = x(M - k);
      const float2 w = twl<W, false>(k);                      // exp(-2 pi i k / W)
      const float2 e1 = make_float2(a.x + b.x, a.y - b.y);
      const float2 o1 = make_float2(a.x - b.x, a.y + b.y);
      const float2 wo = cmul(w, o1);
      const float2 xk = make_float2(0.5f * (e1.x + wo.y), 0.5f * (e1.y - wo.x));   // (e1 - i w o1)/2
      const float2 e2 = make_float2(b.x + a.x, b.y - a.y);
      const float2 o2 = make_float2(b.x - a.x, b.y + a.y);
      const float2 wo2 = cmul(cconj(w), o2);
      const float2 xm = make_float2(0.5f * (e2.x - wo2.y), 0.5f * (e2.y + wo2.x));  // (e2 + i conj(w) o2)/2
      x(k) = xk;
      x(M - k) = xm;
    }
  }
}

// Block-cooperative store to the interleaved spectrum layout: when the block's rows form whole
// groups of 4 (rows per block a multiple of 4; the first row is then a multiple of 4 too), the
// block writes each group as one contiguous run (4 rows x the band's columns), thread e taking row
// e % 4, column e / 4.  s_rows[r] is row r's start in the plane (nullptr for a row beyond H).
template <int W>
__device__ __forceinline__ bool rows_grouped(bool il) {
  return !RowGeo<W>::WARP && il && (blockDim.x / RowGeo<W>::T) % 4 == 0;
}
template <int W>
__device__ __forceinline__ void rows_store_grouped(float2* const* s_rows, int cb) {
  using G = RowGeo<W>;
  extern __shared__ float2 smem[];
  const int R = blockDim.x / G::T;
  for (int g = 0; g < R / 4; ++g)
    for (int e = threadIdx.x; e < 4 * cb; e += blockDim.x) {
      const int rr = e & 3, i = e >> 2;
      float2* p = s_rows[4 * g + rr];
      if (p) p[4 * i] = smem[(4 * g + rr) * G::PITCH + i + (i >> 4)];
    }
}
// ------------------------------------------------------------------------------ warp rows (W = 2048)
// One warp per row of 2048 reals (M = 1024 complex values, 32 per lane; warp_fft1024).  Lane t
// holds the pixel pairs t + 32 q, q = 0..31, the same pairs the pointwise loops visit with T = 32.
//
// C2R: the packed half spectrum X of the row (global, band columns < cb) -> x(t + 32 q) = M times
// the real pixel pair.  The pre-processing of c2r_pre is applied while loading: for k = 1..M-1
//   Z[k] = (X[k] + conj X[M-k] + i e^{+2 pi i k / W} (X[k] - conj X[M-k])) / 2,
// (the pair form of c2r_pre for k and M - k is this one expression at both indices) and
// Z[0] = ((X0 + XM) / 2, (X0 - XM) / 2) from the packed slot 0.  Lane t loads X[k] and X[M - k]
// for its own k = t + 32 q only (both 0 outside the band), so no exchange precedes the transform.
// The result stays in v (lane t: pixel pairs t + 32 q); tb is the warp's transpose buffer.  Loads
// whose whole warp lies outside the band are skipped by a warp-uniform test.
__device__ __forceinline__ void warp_c2r_1024_v(float2 (&v)[32], const float2* __restrict__ src, int t, int cb,
                                                bool il, float2* tb) {
  constexpr int M = 1024;
  const int s = il ? 4 : 1;
  const float2 wt = twl<2048, true>(t);                     // e^{+2 pi i t / 2048}
#pragma unroll
  for (int q = 0; q < 32; ++q) {
    const int k = t + 32 * q, km = M - k;
    const float2 z2 = make_float2(0.0f, 0.0f);
    float2 a = z2, b = z2;
    if (32 * q < cb) a = k < cb ? src[k * s] : z2;                               // some lane: k < cb
    if (M - 32 * q - 31 < cb) b = (q > 0 || t > 0) && km < cb ? src[km * s] : z2; // some lane: M - k < cb
    if (q == 0 && t == 0) {
      v[q] = make_float2(0.5f * (a.x + a.y), 0.5f * (a.x - a.y));
    } else {
      const float2 w = cmul(wt, c_w64[q]);                  // e^{+2 pi i (t + 32 q) / 2048}
      const float2 e1 = make_float2(a.x + b.x, a.y - b.y);  // a + conj b
      const float2 o1 = make_float2(a.x - b.x, a.y + b.y);  // a - conj b
      const float2 wo = cmul(w, o1);
      v[q] = make_float2(0.5f * (e1.x - wo.y), 0.5f * (e1.y + wo.x));
    }
  }
  warp_fft1024<true>(v, tb, t);
}
__device__ __forceinline__ void warp_c2r_1024(const RowLayout<1024>& x, const float2* __restrict__ src, int t,
                                              int cb, bool il) {
  float2 v[32];
  warp_c2r_1024_v(v, src, t, cb, il, x.base);
  __syncwarp();
#pragma unroll
  for (int q = 0; q < 32; ++q) x(t + 32 * q) = v[q];
  __syncwarp();
}
// R2C: x(t + 32 q) (the lane's own pixel pairs) -> the packed half spectrum, band columns < cb
// stored to dst (stride 4 when interleaved).  r2c_post per index k = 1..M-1:
//   X[k] = (Z[k] + conj Z[M-k] - i e^{-2 pi i k / W} (Z[k] - conj Z[M-k])) / 2,
// slot 0 = (Re Z0 + Im Z0, Re Z0 - Im Z0) (X[0] and X[M]), with Z[M - k] read from the lane that
// holds it through the row buffer.
__device__ __forceinline__ void warp_r2c_1024(const RowLayout<1024>& x, float2* __restrict__ dst, int t, int cb,
                                              bool il) {
  constexpr int M = 1024;
  const int s = il ? 4 : 1;
  float2 v[32];
#pragma unroll
  for (int q = 0; q < 32; ++q) v[q] = x(t + 32 * q);
  warp_fft1024<false>(v, x.base, t);
  __syncwarp();
#pragma unroll
  for (int q = 0; q < 32; ++q) x(t + 32 * q) = v[q];
  __syncwarp();
  const float2 wt = twl<2048, false>(t);                    // e^{-2 pi i t / 2048}
#pragma unroll
  for (int q = 0; q < 32; ++q) {
    const int k = t + 32 * q;
    if (k < cb) {
      const float2 a = v[q];
      float2 X;
      if (q == 0 && t == 0) {
        X = make_float2(a.x + a.y, a.x - a.y);
      } else {
        const float2 b = x(M - k);
        const float2 w = cmulc(wt, c_w64[q]);               // e^{-2 pi i (t + 32 q) / 2048}
        const float2 e1 = make_float2(a.x + b.x, a.y - b.y);
        const float2 o1 = make_float2(a.x - b.x, a.y + b.y);
        const float2 wo = cmul(w, o1);
        X = make_float2(0.5f * (e1.x + wo.y), 0.5f * (e1.y - wo.x));
      }
      dst[k * s] = X;
    }
  }
  __syncwarp();
}

// spectrum row (global) -> real values (times M) in shared memory; ends synchronised
// (warp rows: each warp transforms its own row; the lane reads back only its own pixel pairs, so
// no block barrier is needed)
template <int W>
__device__ __forceinline__ void row_spec_to_real(const RowLayout<W / 2>& x, const float2* src, int t, bool act,
                                                 bool il, int cb = W / 2) {
  if constexpr (RowGeo<W>::WARP) {
    if (act) warp_c2r_1024(x, src, t, cb, il);
  } else {
    row_load<W>(x, src, t, act, cb, il);   // (a block-cooperative load measured slower: K6 49 -> 72 us)
    __syncthreads();
    c2r_pre<W>(x, t, act);
    __syncthreads();
    fft_inplace<W / 2, true>(x, t, act);
  }
}
// real values in shared memory -> spectrum row (global); starts with a barrier
template <int W>
__device__ __forceinline__ void row_real_to_spec(const RowLayout<W / 2>& x, float2* dst, int t, bool act,
                                                 bool il, int cb = W / 2) {
  if constexpr (RowGeo<W>::WARP) {
    if (act) warp_r2c_1024(x, dst, t, cb, il);
    __syncthreads();
  } else {
    __syncthreads();
    fft_inplace<W / 2, false>(x, t, act);
    r2c_post<W>(x, t, act);
    if (rows_grouped<W>(il)) {
      __shared__ float2* s_rows[kRowBlock];
      if (t == 0) s_rows[threadIdx.x / RowGeo<W>::T] = act ? dst : nullptr;
      __syncthreads();
      rows_store_grouped<W>(s_rows, cb);
    } else {
      __syncthreads();
      row_store<W>(x, dst, t, act, cb, il);
    }
    __syncthreads();
  }
}

// ------------------------------------------------------------------------------ generic passes
// out[v] = R2C(max(in[v], 0) if clamp else in[v]) for nviews planes of H x W
template <int W>
__global__ void __launch_bounds__(kRowBlock, RowGeo<W>::BLOCKS_MIN) k_row_r2c(const float* __restrict__ in, size_t in_vs,
                                                      float2* __restrict__ out, size_t out_vs,
                                                      int H, int nviews, int clamp) {
  using G = RowGeo<W>;
  extern __shared__ float2 smem[];
  const int r = threadIdx.x / G::T, t = threadIdx.x % G::T;
  const RowLayout<G::M> x{smem + r * G::PITCH};
  const int per_view = (H + G::ROWS - 1) / G::ROWS;
  {
    const int it = blockIdx.x;
    if (it >= nviews * per_view) return;
    const int v = it / per_view;
    const int row = (it % per_view) * G::ROWS + r;
    const bool act = row < H;
    const float2* src = reinterpret_cast<const float2*>(in + v * in_vs + size_t(row) * W);
    if (act) {
#pragma unroll
      for (int q = 0; q < G::E; ++q) {
        float2 z = src[t + q * G::T];
        if (clamp) { z.x = fmaxf(z.x, 0.0f); z.y = fmaxf(z.y, 0.0f); }
        x(t + q * G::T) = z;
      }
    }
    const bool il = spec_interleaved(H);
    row_real_to_spec<W>(x, out + v * out_vs + spec_row_off(row, G::M, il), t, act, il);
  }
}

// out[v] = scale * C2R(in[v])
template <int W>
__global__ void __launch_bounds__(kRowBlock, RowGeo<W>::BLOCKS_MIN) k_row_c2r(const float2* __restrict__ in, size_t in_vs,
                                                      float* __restrict__ out, size_t out_vs,
                                                      int H, int nviews, float scale) {
  using G = RowGeo<W>;
  extern __shared__ float2 smem[];
  const int r = threadIdx.x / G::T, t = threadIdx.x % G::T;
  const RowLayout<G::M> x{smem + r * G::PITCH};
  const int per_view = (H + G::ROWS - 1) / G::ROWS;
  {
    const int it = blockIdx.x;
    if (it >= nviews * per_view) return;
    const int v = it / per_view;
    const int row = (it % per_view) * G::ROWS + r;
    const bool act = row < H;
    const bool il = spec_interleaved(H);
    row_spec_to_real<W>(x, in + v * in_vs + spec_row_off(row, G::M, il), t, act, il);
    float2* dst = reinterpret_cast<float2*>(out + v * out_vs + size_t(row) * W);
    if (act) {
#pragma unroll
      for (int q = 0; q < G::E; ++q) dst[t + q * G::T] = cscale(x(t + q * G::T), scale);
    }
    __syncthreads();
  }
}

// ------------------------------------------------------------------------------ hot passes
__device__ __forceinline__ float2 ld2(const float* p, size_t i) { return reinterpret_cast<const float2*>(p)[i]; }
__device__ __forceinline__ void st2(float* p, size_t i, float2 v) { reinterpret_cast<float2*>(p)[i] = v; }
__device__ __forceinline__ float clipf(float f, float L1, float L2) { return fminf(L2, fmaxf(L1, f)); }
__device__ __forceinline__ float2 w_pair(const ImgDesc& d, size_t i) {
  return d.w ? ld2(d.w, i) : make_float2(d.w_scalar, d.w_scalar);
}
__device__ __forceinline__ float2 b_pair(const ImgDesc& d, int j, size_t i) {
  return d.b ? ld2(d.b + size_t(j) * d.P, i) : make_float2(d.bs[j], d.bs[j]);
}
// Scaling of the SGP step: D = w clip(f, L1, L2), Eq. (Dk)/(Dkbound) (w = 1/p, or M_R/alpha with a
// boundary); with the Tikhonov term beta/2 ||f||^2 the split-gradient scaling D = w c / (1 + beta w c),
// c = clip(f, L1, L2) (the split grad = V - U with V = sum_j A_j^T 1 + beta f, D = c / V(c)).
// (the regularised form divides with the fast reciprocal, error <= 2 ulp: D only has to be one
// consistent positive scaling, and a correctly rounded division on this path would be evaluated
// for every pixel of the unregularised passes too)
__device__ __forceinline__ float scale_of(float f, float w, float L1, float L2, float beta) {
  const float c = w * clipf(f, L1, L2);
  return beta > 0.0f ? __fdividef(c, fmaf(beta, c, 1.0f)) : c;
}
// y = P(f - alpha D grad): non-negativity (mu = 0) or flux (mu from the search)
__device__ __forceinline__ float proj_step(float f, float gr, float w, float alpha, float mu, float L1, float L2,
                                          float beta) {
  const float D = scale_of(f, w, L1, L2, beta);
  return fmaxf(f - D * fmaf(alpha, gr, mu), 0.0f);
}
__device__ __forceinline__ float2* spec_plane(const ImgDesc& d, int plane) {
  return reinterpret_cast<float2*>(d.spec) + (size_t(plane) * d.P) / 2;
}
__device__ __forceinline__ double* part_of(const ImgDesc& d, int it) {
  return d.part + size_t(it - d.row_item0) * kPartStride;
}
__device__ __forceinline__ double* partv_of(const ImgDesc& d, int it) {
  return d.partv + size_t(it - d.rv_item0) * kPartStride;
}
// view-list items carry the view index in the high bits of .y
__device__ __forceinline__ int item_row(int2 item) { return item.y & 0xffff; }
__device__ __forceinline__ int item_view(int2 item) { return item.y >> 16; }

// SGP K1: apply the pending update f <- f + lambda d and A_j f <- A_j f + lambda A_j d (Alg. 1,
// step 6), then r_j = g_j / (A_j f + b_j) -> R2C into planes 1..p, with the KL (and rho) partials.
template <int W, bool FP64>
__device__ __forceinline__ void b_sgp_update_ratio(const ImgDesc* __restrict__ imgs,
                                                               const int2* __restrict__ items, int n_items) {
  pdl_enter();
  using G = RowGeo<W>;
  extern __shared__ float2 smem[];
  const int r = threadIdx.x / G::T, t = threadIdx.x % G::T;
  const RowLayout<G::M> x{smem + r * G::PITCH};
  const int it = blockIdx.x;
  if (it >= n_items) return;
  const int2 item = items[it];
  const ImgDesc& d = imgs[item.x];
  const CtrlState* c = d.ctrl;
  const int done = c->done;
  if (done >= 2) return;
  const int j = item_view(item);
  const int k = c->k, fresh = c->fresh, ke = k + (fresh ? 0 : 1);
  const int row = item_row(item) + r;
  const bool act = row < d.H;
  const size_t off = size_t(row) * G::M;
  Acc<FP64> acc[2];
  const float lam = float(c->lambda);
  if (j == 0 && act) {
    float* fcur = d.f[ke & 1];
    if (!fresh && f_update_in_k1(c, done)) {
      const float* fo = d.f[k & 1];
      const float* go = d.grad[k & 1];
      const float alpha = float(c->alpha), mu = float(c->mu);
      const float L1 = float(c->L1), L2 = float(c->L2);
      constexpr int B = batch_of<G::E, 4>();
#pragma unroll 1
      for (int q0 = 0; q0 < G::E; q0 += B) {
        float2 f[B], gr[B], w[B];
#pragma unroll
        for (int b = 0; b < B; ++b) {
          const size_t i = off + t + (q0 + b) * G::T;
          f[b] = ld2(fo, i); gr[b] = ld2(go, i); w[b] = w_pair(d, i);
        }
#pragma unroll
        for (int b = 0; b < B; ++b) {
          float2 fn;
          fn.x = fmaf(lam, proj_step(f[b].x, gr[b].x, w[b].x, alpha, mu, L1, L2, d.reg_beta) - f[b].x, f[b].x);
          fn.y = fmaf(lam, proj_step(f[b].y, gr[b].y, w[b].y, alpha, mu, L1, L2, d.reg_beta) - f[b].y, f[b].y);
          st2(fcur, off + t + (q0 + b) * G::T, fn);
        }
      }
    }
    if (done == 0 && d.ftrue && c->stop_kind == STOP_MIN_ERROR) {
      for (int q = 0; q < G::E; ++q) {
        const size_t i = off + t + q * G::T;
        const float2 f = ld2(fcur, i), ft = ld2(d.ftrue, i);
        acc[1].add((f.x - ft.x) * (f.x - ft.x) + (f.y - ft.y) * (f.y - ft.y));
      }
    }
  }
  float* uj = d.u + size_t(j) * d.P;
  const float* adj = d.Ad + size_t(j) * d.P;
  const float* gj = d.g + size_t(j) * d.P;
  if (act) {
    constexpr int B = batch_of<G::E, 4>();
#pragma unroll 1
    for (int q0 = 0; q0 < G::E; q0 += B) {
      float2 u[B], a[B], g[B], bk[B];
#pragma unroll
      for (int b = 0; b < B; ++b) {
        const size_t i = off + t + (q0 + b) * G::T;
        u[b] = ld2(uj, i);
        a[b] = fresh ? make_float2(0.0f, 0.0f) : ld2(adj, i);
        g[b] = done == 0 ? ld2(gj, i) : make_float2(0.0f, 0.0f);
        bk[b] = b_pair(d, j, i);
      }
#pragma unroll
      for (int b = 0; b < B; ++b) {
        const size_t i = off + t + (q0 + b) * G::T;
        if (!fresh) {
          u[b].x = fmaf(lam, a[b].x, u[b].x);
          u[b].y = fmaf(lam, a[b].y, u[b].y);
          st2(uj, i, u[b]);
        }
      }
      if (done == 0) {
        // batches whose pixels all take the series branch of kl_ratio (g > 0, u0 > 0,
        // |(u0 - g)/(u0 + g)| < 1/3 on the whole warp) run it without the per-pixel branches
        float2 u0[B], z[B];
        bool series = true;
#pragma unroll
        for (int b = 0; b < B; ++b) {
          u0[b] = make_float2(u[b].x + bk[b].x, u[b].y + bk[b].y);
          z[b] = make_float2(fdiv(u0[b].x - g[b].x, u0[b].x + g[b].x), fdiv(u0[b].y - g[b].y, u0[b].y + g[b].y));
          series = series && g[b].x > 0.0f && u0[b].x > 0.0f && fabsf(z[b].x) < 1.0f / 3.0f &&
                   g[b].y > 0.0f && u0[b].y > 0.0f && fabsf(z[b].y) < 1.0f / 3.0f;
        }
        if (warp_all(series)) {
#pragma unroll
          for (int b = 0; b < B; ++b) {
            float2 rm;
            acc[0].add(kl_series(g[b].x, u0[b].x, z[b].x, rm.x));
            acc[0].add(kl_series(g[b].y, u0[b].y, z[b].y, rm.y));
            x(t + (q0 + b) * G::T) = rm;
          }
        } else {
#pragma unroll
          for (int b = 0; b < B; ++b) {
            float2 rm;
            acc[0].add(kl_ratio(g[b].x, u0[b].x, rm.x));
            acc[0].add(kl_ratio(g[b].y, u0[b].y, rm.y));
            x(t + (q0 + b) * G::T) = rm;
          }
        }
      }
    }
  }
  if (done == 0) {
    row_real_to_spec<W>(x, spec_plane(d, j + 1) + spec_row_off(row, G::M, spec_interleaved(d.H)), t, act, spec_interleaved(d.H), d.cb);
    block_sum_store<2, FP64>(acc, partv_of(d, it) + SLOT_KL);
  }
  {  // the controller: real in the last block, dry in the others when d.dry_rv (control.cuh)
    const bool last = arrive_last(d.ctrl, d.n_rv_items);
    if constexpr (RowGeo<W>::WARP) {
      if (last || d.dry_rv) ctrl_sgp_begin_nl<FP64>(d, !last);
    } else if (last) {
      ctrl_sgp_begin<FP64>(d, false);
    }
  }
}
template <int W, bool FP64>
__global__ void __launch_bounds__(kRowBlock, RowGeo<W>::BLOCKS_HOT) k_sgp_update_ratio(const ImgDesc* __restrict__ imgs,
                                                               const int2* __restrict__ items, int n_items) {
  b_sgp_update_ratio<W, FP64>(imgs, items, n_items);
}

// SGP K3: C2R of plane 0 (= sum_j A_j^T r_j) -> gradient, and the four scaled-BB partial sums.
// With f_pending it first forms f^(k) = f^(k-1) + lambda d from f^(k-1) and grad^(k-1) (the step
// of the previous iteration: its alpha, mu and lambda are still in the state) and stores it.
template <int W, bool FP64>
__device__ __forceinline__ void b_sgp_grad_bb(const ImgDesc* __restrict__ imgs,
                                                          const int2* __restrict__ items, int n_items) {
  pdl_enter();
  using G = RowGeo<W>;
  extern __shared__ float2 smem[];
  const int r = threadIdx.x / G::T, t = threadIdx.x % G::T;
  const RowLayout<G::M> x{smem + r * G::PITCH};
  {
    const int it = blockIdx.x;
    if (it >= n_items) return;
    const int2 item = items[it];
    const ImgDesc& d = imgs[item.x];
    const CtrlState* c = d.ctrl;
    if (c->done >= 1) return;
    const int ke = c->k + (c->fresh ? 0 : 1);
    const int row = item_row(item) + r;
    const bool act = row < d.H;
    const size_t off = size_t(row) * G::M;
    row_spec_to_real<W>(x, spec_plane(d, 0) + spec_row_off(row, G::M, spec_interleaved(d.H)), t, act, spec_interleaved(d.H), d.cb);
    Acc<FP64> acc[4];
    if (act) {
      float* f = d.f[ke & 1];
      const float* fp = d.f[(ke + 1) & 1];
      const float* gp = d.grad[(ke + 1) & 1];
      float* gn = d.grad[ke & 1];
      const float L1 = float(c->L1), L2 = float(c->L2);
      const bool bb = ke >= 1;
      const bool pend = c->f_pending != 0;
      const float rb = d.reg_beta;                  // the gradient gains beta f with regularisation
      const bool need_f = bb || rb > 0.0f;
      const float lam = float(c->lambda), alpha = float(c->alpha), mu = float(c->mu);
      constexpr int B = batch_of<G::E, 4>();
#pragma unroll 1
      for (int q0 = 0; q0 < G::E; q0 += B) {
        float2 wv[B], fcv[B], fov[B], gov[B];
#pragma unroll
        for (int b = 0; b < B; ++b) {
          const size_t i = off + t + (q0 + b) * G::T;
          wv[b] = w_pair(d, i);
          const float2 z2 = make_float2(0.0f, 0.0f);
          fcv[b] = need_f && !pend ? ld2(f, i) : z2; fov[b] = bb ? ld2(fp, i) : z2; gov[b] = bb ? ld2(gp, i) : z2;
        }
        if (pend) {   // f^(k) = f^(k-1) + lambda (P(f^(k-1) - alpha D grad^(k-1)) - f^(k-1)), as K1 forms it
#pragma unroll
          for (int b = 0; b < B; ++b) {
            const float2 fo = fov[b], go = gov[b], w = wv[b];
            float2 fn;
            fn.x = fmaf(lam, proj_step(fo.x, go.x, w.x, alpha, mu, L1, L2, rb) - fo.x, fo.x);
            fn.y = fmaf(lam, proj_step(fo.y, go.y, w.y, alpha, mu, L1, L2, rb) - fo.y, fo.y);
            fcv[b] = fn;
            st2(f, off + t + (q0 + b) * G::T, fn);
          }
        }
#pragma unroll
        for (int b = 0; b < B; ++b) {
        const size_t i = off + t + (q0 + b) * G::T;
        const float2 v = x(t + (q0 + b) * G::T), w = wv[b];   // v = sum_j A_j^T (r_j - 1)
        float2 gr;
        if (rb > 0.0f) {                            // grad J_0 + beta f on R
          gr.x = w.x > 0.0f ? fmaf(rb, fcv[b].x, -v.x) : 0.0f;
          gr.y = w.y > 0.0f ? fmaf(rb, fcv[b].y, -v.y) : 0.0f;
        } else {
          gr.x = w.x > 0.0f ? -v.x : 0.0f;
          gr.y = w.y > 0.0f ? -v.y : 0.0f;
        }
        st2(gn, i, gr);
        if (bb) {
          const float2 fc = fcv[b], fo = fov[b], go = gov[b];
          const float sx = fc.x - fo.x, sy = fc.y - fo.y, zx = gr.x - go.x, zy = gr.y - go.y;
          const float Dx = scale_of(fc.x, w.x, L1, L2, rb), Dy = scale_of(fc.y, w.y, L1, L2, rb);
          float tb[4];
          if (Dx > 0.0f) {
            bb_terms(sx, zx, Dx, tb);
            acc[0].add(tb[0]); acc[1].add(tb[1]); acc[2].add(tb[2]); acc[3].add(tb[3]);
          }
          if (Dy > 0.0f) {
            bb_terms(sy, zy, Dy, tb);
            acc[0].add(tb[0]); acc[1].add(tb[1]); acc[2].add(tb[2]); acc[3].add(tb[3]);
          }
        }
        }
      }
    }
    block_sum_store<4, FP64>(acc, part_of(d, it) + SLOT_BB);
    const bool last = arrive_last(d.ctrl, d.n_row_items);
    if constexpr (RowGeo<W>::WARP) {
      if (last || d.dry_row) ctrl_sgp_alpha_nl<FP64>(d, !last);
    } else if (last) {
      ctrl_sgp_alpha<FP64>(d, false);
    }
  }
}
template <int W, bool FP64>
__global__ void __launch_bounds__(kRowBlock, RowGeo<W>::BLOCKS_HOT) k_sgp_grad_bb(const ImgDesc* __restrict__ imgs,
                                                          const int2* __restrict__ items, int n_items) {
  b_sgp_grad_bb<W, FP64>(imgs, items, n_items);
}

// SGP K4: y = P(f - alpha D grad) (Alg. 1 step 2), d = y - f -> R2C into plane 0, grad'd partials.
template <int W, bool FP64>
__device__ __forceinline__ void b_sgp_y(const ImgDesc* __restrict__ imgs,
                                                    const int2* __restrict__ items, int n_items) {
  pdl_enter();
  using G = RowGeo<W>;
  extern __shared__ float2 smem[];
  const int r = threadIdx.x / G::T, t = threadIdx.x % G::T;
  const RowLayout<G::M> x{smem + r * G::PITCH};
  {
    const int it = blockIdx.x;
    if (it >= n_items) return;
    const int2 item = items[it];
    const ImgDesc& d = imgs[item.x];
    const CtrlState* c = d.ctrl;
    if (c->done >= 1) return;
    const int k = c->k;
    const int row = item_row(item) + r;
    const bool act = row < d.H;
    const size_t off = size_t(row) * G::M;
    Acc<FP64> acc[1], accr[2];                      // g'd; f'd and d'd with regularisation
    const float rb = d.reg_beta;
    if (act) {
      const float* f = d.f[k & 1];
      const float* gr = d.grad[k & 1];
      const float alpha = float(c->alpha), mu = float(c->mu), L1 = float(c->L1), L2 = float(c->L2);
      constexpr int B = batch_of<G::E, 4>();
#pragma unroll 1
      for (int q0 = 0; q0 < G::E; q0 += B) {
        float2 fv[B], gv[B], w[B];
#pragma unroll
        for (int b = 0; b < B; ++b) {
          const size_t i = off + t + (q0 + b) * G::T;
          fv[b] = ld2(f, i); gv[b] = ld2(gr, i); w[b] = w_pair(d, i);
        }
#pragma unroll
        for (int b = 0; b < B; ++b) {
          const float yx = proj_step(fv[b].x, gv[b].x, w[b].x, alpha, mu, L1, L2, rb);
          const float yy = proj_step(fv[b].y, gv[b].y, w[b].y, alpha, mu, L1, L2, rb);
          const float dx = yx - fv[b].x, dy = yy - fv[b].y;
          acc[0].add(gv[b].x * dx);
          acc[0].add(gv[b].y * dy);
          if (rb > 0.0f) {
            accr[0].add(fv[b].x * dx); accr[0].add(fv[b].y * dy);
            accr[1].add(dx * dx); accr[1].add(dy * dy);
          }
          x(t + (q0 + b) * G::T) = make_float2(dx, dy);   // A d is transformed directly (no A y - A f cancellation)
        }
      }
    }
    row_real_to_spec<W>(x, spec_plane(d, 0) + spec_row_off(row, G::M, spec_interleaved(d.H)), t, act, spec_interleaved(d.H), d.cb);
    block_sum_store<1, FP64>(acc, part_of(d, it) + SLOT_GTD);
    if (rb > 0.0f) block_sum_store<2, FP64>(accr, part_of(d, it) + SLOT_REG);
  }
}
template <int W, bool FP64>
__global__ void __launch_bounds__(kRowBlock, RowGeo<W>::BLOCKS_MIN) k_sgp_y(const ImgDesc* __restrict__ imgs,
                                                    const int2* __restrict__ items, int n_items) {
  b_sgp_y<W, FP64>(imgs, items, n_items);
}

// K6 pixel loop for the first N step lengths (the other sums stay 0): stores A d, adds the Armijo
// terms
template <int W, int N, class A>
__device__ __forceinline__ void sgp_armijo_rows(const RowLayout<W / 2>& x, A (&acc)[kArmMain],
                                                const float (&lam)[kArmMain], const float* uj, float* adj,
                                                const float* gj, const ImgDesc& d, int j, size_t off, int t) {
  using G = RowGeo<W>;
  A (&accN)[N] = reinterpret_cast<A (&)[N]>(acc);
  const float (&lamN)[N] = reinterpret_cast<const float (&)[N]>(lam);
  constexpr int B = batch_of<G::E, 4>();
  // software pipeline: the loads of the next batch are issued before this batch is used (the pass
  // holds no transform data in registers here; K1, K3 and K4 measured slower with the same change)
  float2 un[B], gn[B];
  auto load = [&](int q0) {
#pragma unroll
    for (int b = 0; b < B; ++b) {
      const size_t i = off + t + (q0 + b) * G::T;
      un[b] = ld2(uj, i); gn[b] = ld2(gj, i);
    }
  };
  load(0);
#pragma unroll 1
  for (int q0 = 0; q0 < G::E; q0 += B) {
    float2 u[B], g[B], bk[B];
#pragma unroll
    for (int b = 0; b < B; ++b) {
      u[b] = un[b]; g[b] = gn[b]; bk[b] = b_pair(d, j, off + t + (q0 + b) * G::T);
    }
    if (q0 + B < G::E) load(q0 + B);
    // batches whose pixels all take the series branch (g > 0, u0 > 0, |A d / u0| < 1/8 on the
    // whole warp: the usual case) run it without the per-pixel branches; identical terms
    float2 ad[B], u0[B], qb[B];
    bool series = true;
#pragma unroll
    for (int b = 0; b < B; ++b) {
      ad[b] = x(t + (q0 + b) * G::T);
      st2(adj, off + t + (q0 + b) * G::T, ad[b]);
      u0[b] = make_float2(u[b].x + bk[b].x, u[b].y + bk[b].y);
      qb[b] = make_float2(fdiv(ad[b].x, u0[b].x), fdiv(ad[b].y, u0[b].y));
      series = series && g[b].x > 0.0f && u0[b].x > 0.0f && fabsf(qb[b].x) < 0.125f &&
               g[b].y > 0.0f && u0[b].y > 0.0f && fabsf(qb[b].y) < 0.125f;
    }
    if (warp_all(series)) {
#pragma unroll
      for (int b = 0; b < B; ++b) {
        armijo_series<N>(accN, lamN, g[b].x, u0[b].x, qb[b].x);
        armijo_series<N>(accN, lamN, g[b].y, u0[b].y, qb[b].y);
      }
    } else {
#pragma unroll
      for (int b = 0; b < B; ++b) {
        armijo_add<N>(accN, lamN, g[b].x, u0[b].x, ad[b].x);
        armijo_add<N>(accN, lamN, g[b].y, u0[b].y, ad[b].y);
      }
    }
  }
}

// SGP K6: per view, C2R of plane j+1 (= A_j d) -> stored A_j d (A(f + lam d) = A f + lam A d: no FFT
// per backtrack) and the Armijo partial sums Delta J(theta^i), i = 0..3 (Alg. 1 step 5).
template <int W, bool FP64>
__device__ __forceinline__ void b_sgp_ad_armijo(const ImgDesc* __restrict__ imgs,
                                                            const int2* __restrict__ items, int n_items) {
  pdl_enter();
  using G = RowGeo<W>;
  extern __shared__ float2 smem[];
  const int r = threadIdx.x / G::T, t = threadIdx.x % G::T;
  const RowLayout<G::M> x{smem + r * G::PITCH};
  const int it = blockIdx.x;
  if (it >= n_items) return;
  const int2 item = items[it];
  const ImgDesc& d = imgs[item.x];
  const CtrlState* c = d.ctrl;
  if (c->done >= 1) return;
  const int j = item_view(item);
  const int row = item_row(item) + r;
  const bool act = row < d.H;
  const size_t off = size_t(row) * G::M;
  const float th = float(c->theta);
  float lam[kArmMain];
  lam[0] = 1.0f;
#pragma unroll
  for (int l = 1; l < kArmMain; ++l) lam[l] = lam[l - 1] * th;
  Acc<FP64> acc[kArmMain];
  row_spec_to_real<W>(x, spec_plane(d, j + 1) + spec_row_off(row, G::M, spec_interleaved(d.H)), t, act, spec_interleaved(d.H), d.cb);
  if (act) {
    const float* uj = d.u + size_t(j) * d.P;
    float* adj = d.Ad + size_t(j) * d.P;
    const float* gj = d.g + size_t(j) * d.P;
    const int nl = arm_count(c);
    if (nl == kArmMain) sgp_armijo_rows<W, kArmMain>(x, acc, lam, uj, adj, gj, d, j, off, t);
    else if (nl == 2) sgp_armijo_rows<W, 2>(x, acc, lam, uj, adj, gj, d, j, off, t);
    else sgp_armijo_rows<W, 1>(x, acc, lam, uj, adj, gj, d, j, off, t);
  }
  block_sum_store<kArmMain, FP64>(acc, partv_of(d, it) + SLOT_ARM);
  const bool last = arrive_last(d.ctrl, d.n_rv_items);
  if constexpr (RowGeo<W>::WARP) {
    if (last || d.dry_rv) ctrl_sgp_lambda_nl<FP64>(d, !last);
  } else if (last) {
    ctrl_sgp_lambda<FP64>(d, false);
  }
}
template <int W, bool FP64>
__global__ void __launch_bounds__(kRowBlock, RowGeo<W>::BLOCKS_MIN) k_sgp_ad_armijo(const ImgDesc* __restrict__ imgs,
                                                            const int2* __restrict__ items, int n_items) {
  b_sgp_ad_armijo<W, FP64>(imgs, items, n_items);
}

// SGP K7 (only when no lambda of the main pass was accepted): Delta J(theta^i), i = arm_nl..30.
// K8 (LAND, landed discrepancy stop only): Delta J at kLandCand equally spaced step lengths inside
// the current landing bracket.  Both read A f, A d, g of every view.
template <int W, bool FP64, bool LAND>
__device__ __forceinline__ void b_sgp_lambda_scan(const ImgDesc* __restrict__ imgs,
                                                  const int2* __restrict__ items, int n_items) {
  pdl_enter();
  using G = RowGeo<W>;
  const int r = threadIdx.x / G::T, t = threadIdx.x % G::T;
  {
    const int it = blockIdx.x;
    if (it >= n_items) return;
    const int2 item = items[it];
    const ImgDesc& d = imgs[item.x];
    const CtrlState* c = d.ctrl;
    if (c->done >= 1) return;
    if (LAND ? c->land_pass < 1 : !c->need_more) return;
    const int row = item_row(item) + r;
    const bool act = row < d.H;
    const size_t off = size_t(row) * G::M;
    float lam0, step;
    if (LAND) {
      const double h = (c->land_hi - c->land_lo) / double(kLandCand + 1);
      lam0 = float(c->land_lo + h);
      step = float(h);
    } else {
      step = float(c->theta);
      lam0 = 1.0f;
      const int nl = arm_count(c);
      for (int l = 0; l < nl; ++l) lam0 *= step;
    }
    Acc<FP64> acc[kArmExtra];
    if (act) {
      for (int j = 0; j < d.p; ++j) {
        const float* uj = d.u + size_t(j) * d.P;
        const float* adj = d.Ad + size_t(j) * d.P;
        const float* gj = d.g + size_t(j) * d.P;
        for (int q = 0; q < G::E; ++q) {
          const size_t i = off + t + q * G::T;
          const float2 u = ld2(uj, i), ad = ld2(adj, i), g = ld2(gj, i), b = b_pair(d, j, i);
          armijo_add_prog<kArmExtra, !LAND>(acc, lam0, step, g.x, u.x + b.x, ad.x);
          armijo_add_prog<kArmExtra, !LAND>(acc, lam0, step, g.y, u.y + b.y, ad.y);
        }
      }
    }
    block_sum_store<kArmExtra, FP64>(acc, part_of(d, it) + SLOT_ARMX);
    if (arrive_last(d.ctrl, d.n_row_items)) {
      if (LAND) ctrl_sgp_land<FP64>(d);
      else ctrl_sgp_lambda_extra<FP64>(d);
    }
  }
}
template <int W, bool FP64>
__global__ void __launch_bounds__(kRowBlock, RowGeo<W>::BLOCKS_MIN) k_sgp_armijo_extra(const ImgDesc* __restrict__ imgs,
                                                               const int2* __restrict__ items, int n_items) {
  b_sgp_lambda_scan<W, FP64, false>(imgs, items, n_items);
}
template <int W, bool FP64>
__global__ void __launch_bounds__(kRowBlock, RowGeo<W>::BLOCKS_MIN) k_sgp_land(const ImgDesc* __restrict__ imgs,
                                                       const int2* __restrict__ items, int n_items) {
  b_sgp_lambda_scan<W, FP64, true>(imgs, items, n_items);
}

// RL K1: if plane 0 holds v = sum_j A_j^T r_j, f <- w f v (Eq. RL / multipleRL / boundaryRL);
// then R2C of the current iterate into plane 0 (and the rho partial).
// OSEM sub-step (wview = j >= 0, Algorithm 2): plane j+1 holds v_j = A_j^T (r_j - 1) of view j
// only, and h <- w_j h A_j^T r_j = h (1 + w_j v_j) with w_j = 1 / A_j^T 1 = 1 (periodic, unit-volume
// PSF; Eq. OSEMstep) or M_R / alpha_j (Eq. boundaryOSEM); the R2C of h still goes to plane 0.
template <int W, bool FP64>
__device__ __forceinline__ void b_rl_update(const ImgDesc* __restrict__ imgs,
                                                        const int2* __restrict__ items, int n_items, int wview) {
  pdl_enter();
  using G = RowGeo<W>;
  extern __shared__ float2 smem[];
  const int r = threadIdx.x / G::T, t = threadIdx.x % G::T;
  const RowLayout<G::M> x{smem + r * G::PITCH};
  {
    const int it = blockIdx.x;
    if (it >= n_items) return;
    const int2 item = items[it];
    const ImgDesc& d = imgs[item.x];
    const CtrlState* c = d.ctrl;
    if (c->done >= 2) return;
    const int k = c->k, hv = c->have_v, ke = k + hv;
    const int row = item_row(item) + r;
    const bool act = row < d.H;
    const size_t off = size_t(row) * G::M;
    float2* sp = spec_plane(d, 0) + spec_row_off(row, G::M, spec_interleaved(d.H));
    const bool osem = wview >= 0;
    if (hv) row_spec_to_real<W>(x, osem ? spec_plane(d, wview + 1) + spec_row_off(row, G::M, spec_interleaved(d.H)) : sp, t, act, spec_interleaved(d.H), d.cb);
    Acc<FP64> acc[1], accq[1];                      // rho; f'f for the Tikhonov term at set-up
    const bool fsq = d.reg_beta > 0.0f;
    if (act) {
      const float* fo = d.f[k & 1];
      float* fn = d.f[ke & 1];
      const bool rho = d.ftrue && c->stop_kind == STOP_MIN_ERROR;
#pragma unroll 4
      for (int q = 0; q < G::E; ++q) {
        const size_t i = off + t + q * G::T;
        float2 f = ld2(fo, i);
        if (hv) {   // w f sum_j A_j^T r_j = f (1 + w v) on R, v = sum_j A_j^T (r_j - 1)
          const float2 v = x(t + q * G::T);
          const float2 w = !osem ? w_pair(d, i)
                                 : (d.wv ? ld2(d.wv + size_t(wview) * d.P, i) : make_float2(1.0f, 1.0f));
          f.x = w.x > 0.0f ? fmaf(f.x * w.x, v.x, f.x) : 0.0f;
          f.y = w.y > 0.0f ? fmaf(f.y * w.y, v.y, f.y) : 0.0f;
          st2(fn, i, f);
        }
        if (rho) {
          const float2 ft = ld2(d.ftrue, i);
          acc[0].add((f.x - ft.x) * (f.x - ft.x) + (f.y - ft.y) * (f.y - ft.y));
        }
        if (fsq) { accq[0].add(f.x * f.x); accq[0].add(f.y * f.y); }
        x(t + q * G::T) = f;
      }
    }
    row_real_to_spec<W>(x, sp, t, act, spec_interleaved(d.H), d.cb);
    block_sum_store<1, FP64>(acc, part_of(d, it) + SLOT_RHO);
    if (fsq) block_sum_store<1, FP64>(accq, part_of(d, it) + SLOT_FSQ);
  }
}
template <int W, bool FP64>
__global__ void __launch_bounds__(kRowBlock, RowGeo<W>::BLOCKS_MIN) k_rl_update(const ImgDesc* __restrict__ imgs,
                                                        const int2* __restrict__ items, int n_items, int wview) {
  b_rl_update<W, FP64>(imgs, items, n_items, wview);
}

// RL K3 (also a set-up pass): per view, C2R of plane j+1 (= A_j f) -> KL partials and
// r_j = g_j/(A_j f + b_j) -> R2C back into plane j+1.  write_u: 0 RL iteration (RL controller),
// 1 set-up (stores A_j f into u), 2 OSEM sub-step (the items of one view, in a view-major list: no
// partial sums; the last block of a problem counts the update, see osem_tick).
template <int W, bool FP64>
__device__ __forceinline__ void b_rl_ratio(const ImgDesc* __restrict__ imgs,
                                                       const int2* __restrict__ items, int n_items, int write_u) {
  pdl_enter();
  using G = RowGeo<W>;
  extern __shared__ float2 smem[];
  const int r = threadIdx.x / G::T, t = threadIdx.x % G::T;
  const RowLayout<G::M> x{smem + r * G::PITCH};
  const int it = blockIdx.x;
  if (it >= n_items) return;
  const int2 item = items[it];
  const ImgDesc& d = imgs[item.x];
  if (d.ctrl->done >= 2) return;
  const int j = item_view(item);
  const int row = item_row(item) + r;
  const bool act = row < d.H;
  const size_t off = size_t(row) * G::M;
  Acc<FP64> acc[1];
  float2* sp = spec_plane(d, j + 1) + spec_row_off(row, G::M, spec_interleaved(d.H));
  row_spec_to_real<W>(x, sp, t, act, spec_interleaved(d.H), d.cb);
  if (act) {
    float* uj = d.u + size_t(j) * d.P;
    const float* gj = d.g + size_t(j) * d.P;
#pragma unroll 4
    for (int q = 0; q < G::E; ++q) {
      const size_t i = off + t + q * G::T;
      const float2 u = x(t + q * G::T), g = ld2(gj, i), b = b_pair(d, j, i);
      if (write_u == 1) st2(uj, i, u);
      const float u0x = u.x + b.x, u0y = u.y + b.y;
      float2 rm;
      acc[0].add(kl_ratio(g.x, u0x, rm.x));
      acc[0].add(kl_ratio(g.y, u0y, rm.y));
      x(t + q * G::T) = rm;
    }
  }
  row_real_to_spec<W>(x, sp, t, act, spec_interleaved(d.H), d.cb);
  if (write_u == 2) {
    if (arrive_last(d.ctrl, d.n_row_items)) osem_tick(d.ctrl, 1);
    return;
  }
  block_sum_store<1, FP64>(acc, partv_of(d, it) + SLOT_KL);
  if (!write_u) {   // RL iteration (not set-up)
    const bool last = arrive_last(d.ctrl, d.n_rv_items);
    if constexpr (RowGeo<W>::WARP) {
      if (last || d.dry_rv) ctrl_rl_nl<FP64>(d, !last);
    } else if (last) {
      ctrl_rl<FP64>(d, false);
    }
  }
}
template <int W, bool FP64>
__global__ void __launch_bounds__(kRowBlock, RowGeo<W>::BLOCKS_HOT) k_rl_ratio(const ImgDesc* __restrict__ imgs,
                                                       const int2* __restrict__ items, int n_items, int write_u) {
  b_rl_ratio<W, FP64>(imgs, items, n_items, write_u);
}

// Set-up: y = w f v from plane 0 (one RL step from f^(0), Sect. 3.2); min over positive y and max y.
template <int W>
__device__ __forceinline__ void b_rl_step_minmax(const ImgDesc* __restrict__ imgs,
                                                             const int2* __restrict__ items, int n_items) {
  pdl_enter();
  using G = RowGeo<W>;
  extern __shared__ float2 smem[];
  const int r = threadIdx.x / G::T, t = threadIdx.x % G::T;
  const RowLayout<G::M> x{smem + r * G::PITCH};
  {
    const int it = blockIdx.x;
    if (it >= n_items) return;
    const int2 item = items[it];
    const ImgDesc& d = imgs[item.x];
    const int row = item_row(item) + r;
    const bool act = row < d.H;
    const size_t off = size_t(row) * G::M;
    row_spec_to_real<W>(x, spec_plane(d, 0) + spec_row_off(row, G::M, spec_interleaved(d.H)), t, act, spec_interleaved(d.H), d.cb);
    float mn = f_inf(), mx = 0.0f;
    if (act) {
      const float* f = d.f[d.ctrl->k & 1];
      for (int q = 0; q < G::E; ++q) {
        const size_t i = off + t + q * G::T;
        const float2 v = x(t + q * G::T), fv = ld2(f, i), w = w_pair(d, i);
        const float y0 = w.x > 0.0f ? fmaf(fv.x * w.x, v.x, fv.x) : 0.0f;
        const float y1 = w.y > 0.0f ? fmaf(fv.y * w.y, v.y, fv.y) : 0.0f;
        if (y0 > 0.0f) mn = fminf(mn, y0);
        if (y1 > 0.0f) mn = fminf(mn, y1);
        mx = fmaxf(mx, fmaxf(y0, y1));
      }
    }
    block_minmax_store(mn, mx, part_of(d, it) + SLOT_MIN);
  }
}
template <int W>
__global__ void __launch_bounds__(kRowBlock, RowGeo<W>::BLOCKS_MIN) k_rl_step_minmax(const ImgDesc* __restrict__ imgs,
                                                             const int2* __restrict__ items, int n_items) {
  b_rl_step_minmax<W>(imgs, items, n_items);
}

}  // namespace sgp

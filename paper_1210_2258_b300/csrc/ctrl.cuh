// Controller kernels outside the iteration (one block per problem) and the set-up and flux kernels.
// The per-iteration controllers run inside the row passes (control.cuh).
//   k_ctrl_setup   J_0 and the adaptive bounds L1, L2 of Sect. 3.2
//   k_ctrl_arm     (re)arms the stop rule of every problem
//   k_flux_pass / k_ctrl_flux  flux-constrained projection
#pragma once
#include <math.h>
#include "rowops.cuh"
#include "state.cuh"

namespace sgp {

// After the set-up passes: J_0 (from the ratio pass) and L1/L2 (Sect. 3.2) from one RL step.
template <bool FP64>
__global__ void __launch_bounds__(kCtrlBlock) k_ctrl_setup(const ImgDesc* __restrict__ imgs, int adaptive,
                                                          int want_bounds) {
  const ImgDesc& d = imgs[blockIdx.x];
  CtrlState* c = d.ctrl;
  double s[1];
  ctrl_sum<1, FP64>(d, SLOT_KL, s, true);
  double mn = 0.0, mx = 0.0;
  if (want_bounds) ctrl_minmax(d, mn, mx);
  double q[1] = {0.0};
  if (d.reg_beta > 0.0f) ctrl_sum<1, FP64>(d, SLOT_FSQ, q, false);   // f'f of the start
  if (threadIdx.x != 0) return;
  c->R = 0.5 * c->reg_beta * q[0];
  c->R_pred = c->R;
  c->J = s[0];
  c->J_prev = s[0];
  if (!isfinite(s[0])) { c->status = 8; c->done = 2; return; }
  if (want_bounds && adaptive) {
    if (!(mn < INFINITY) || mx <= 0.0) { c->status = 1; c->done = 2; return; }
    if (mx / mn < 50.0) { c->L1 = mn / 10.0; c->L2 = mx * 10.0; }
    else { c->L1 = mn; c->L2 = mx; }
  }
}

// (Re)arm the stop rule of every problem: kind, max_iter (relative to the current k or absolute).
__global__ void k_ctrl_arm(const ImgDesc* __restrict__ imgs, int n, int kind, int n_iter, double tol,
                           double eta, int relative) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  CtrlState* c = imgs[i].ctrl;
  if (c->status != 0) return;          // a failed problem stays stopped
  c->stop_kind = kind;
  c->capped = 0;
  c->max_iter = relative ? c->k + n_iter : n_iter;
  c->tol = tol;
  c->eta = eta;
  c->done = 0;
  c->result_prev = 0;
  c->need_more = 0;
  c->land_pass = 0;
}

// ------------------------------------------------------------------------------ flux projection
// Projection onto {y >= 0, sum y = c} in the D^-1 metric (SGP step 2 with the flux constraint):
// y_i = max(0, x_i - mu D_i), x = f - alpha D grad; pixels with D_i = 0 keep y_i = x_i.
// mu is the root of the non-increasing piecewise-linear phi(mu) = sum max(0, x - mu D) - c'.
// Passes: bounds (breakpoint range, sums) -> kFluxPasses candidate evaluations narrowing the bracket
// -> final exact solve on the active set.  Every pass reads f and grad of the current iterate.
__device__ __forceinline__ void flux_xd(const ImgDesc& d, const CtrlState* c, size_t i, float& x, float& D) {
  const float f = d.f[c->k & 1][i], gr = d.grad[c->k & 1][i];
  const float w = d.w ? d.w[i] : d.w_scalar;
  D = scale_of(f, w, float(c->L1), float(c->L2), d.reg_beta);
  x = f - float(c->alpha) * D * gr;
}

// mode 0: bounds; mode 1: candidate sums; mode 2: final active-set sums
template <bool FP64>
__global__ void __launch_bounds__(kRowBlock) k_flux_pass(const ImgDesc* __restrict__ imgs, const int2* __restrict__ items,
                                                        int n_items, int mode) {
  pdl_enter();
  const int it = blockIdx.x;
  if (it >= n_items) return;
  const int2 item = items[it];
  const ImgDesc& d = imgs[item.x];
  const CtrlState* c = d.ctrl;
  if (c->done >= 1 || c->constraint == 0) return;
  const int row0 = item.y & 0xffff;
  const int rows = min(d.rpi, d.H - row0);
  const size_t base = size_t(row0) * d.W, n = size_t(rows) * d.W;
  double* out = part_of(d, it);
  if (mode == 0) {
    Acc<FP64> acc[3];   // sum x (D > 0), sum D (D > 0), sum x (D = 0)
    float tmin = f_inf(), tmax = -f_inf();
    for (size_t q = threadIdx.x; q < n; q += blockDim.x) {
      float x, D;
      flux_xd(d, c, base + q, x, D);
      if (D > 0.0f) {
        acc[0].add(x); acc[1].add(D);
        const float t = x / D;
        tmin = fminf(tmin, t); tmax = fmaxf(tmax, t);
      } else {
        acc[2].add(x);
      }
    }
    block_sum_store<3, FP64>(acc, out + SLOT_PROJ);
    // min t into SLOT_MIN, -max t into SLOT_MAX (stored negated so both reduce as minima)
    __shared__ float rmn[kRowBlock / 32], rmx[kRowBlock / 32];
    float a = tmin, b = -tmax;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      a = fminf(a, __shfl_xor_sync(0xffffffffu, a, o));
      b = fminf(b, __shfl_xor_sync(0xffffffffu, b, o));
    }
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    if (lane == 0) { rmn[wid] = a; rmx[wid] = b; }
    __syncthreads();
    if (threadIdx.x == 0) {
      for (int w = 1; w < int(blockDim.x >> 5); ++w) { a = fminf(a, rmn[w]); b = fminf(b, rmx[w]); }
      a = fminf(rmn[0], a); b = fminf(rmx[0], b);
      out[SLOT_MIN] = a;
      out[SLOT_MAX] = b;
    }
  } else if (mode == 1) {
    Acc<FP64> acc[kFluxCand];
    float mu[kFluxCand];
    const double lo = c->mu_lo, hi = c->mu_hi;
#pragma unroll
    for (int q = 0; q < kFluxCand; ++q) mu[q] = float(lo + (hi - lo) * double(q + 1) / double(kFluxCand + 1));
    for (size_t q = threadIdx.x; q < n; q += blockDim.x) {
      float x, D;
      flux_xd(d, c, base + q, x, D);
      if (D > 0.0f) {
#pragma unroll
        for (int m = 0; m < kFluxCand; ++m) acc[m].add(fmaxf(x - mu[m] * D, 0.0f));
      }
    }
    block_sum_store<kFluxCand, FP64>(acc, out + SLOT_ARMX);
  } else {
    Acc<FP64> acc[2];   // sum x, sum D over the pixels with t > mu_lo (active just above mu_lo)
    const float a = float(c->mu_lo);
    for (size_t q = threadIdx.x; q < n; q += blockDim.x) {
      float x, D;
      flux_xd(d, c, base + q, x, D);
      if (D > 0.0f && x - a * D > 0.0f) { acc[0].add(x); acc[1].add(D); }
    }
    block_sum_store<2, FP64>(acc, out + SLOT_PROJ + 3);
  }
}

template <bool FP64>
__global__ void __launch_bounds__(kCtrlBlock) k_ctrl_flux(const ImgDesc* __restrict__ imgs, int mode) {
  pdl_enter();
  const ImgDesc& d = imgs[blockIdx.x];
  CtrlState* c = d.ctrl;
  if (c->done >= 1 || c->constraint == 0) return;
  if (mode == 0) {
    double s[3], mn = 0.0, mxneg = 0.0;
    ctrl_sum<3, FP64>(d, SLOT_PROJ, s, false);
    {   // minima of SLOT_MIN (min t) and SLOT_MAX (-max t)
      __shared__ double ra[kCtrlBlock / 32], rb[kCtrlBlock / 32];
      double a = INFINITY, b = INFINITY;
      for (int i = threadIdx.x; i < d.n_row_items; i += blockDim.x) {
        a = fmin(a, d.part[size_t(i) * kPartStride + SLOT_MIN]);
        b = fmin(b, d.part[size_t(i) * kPartStride + SLOT_MAX]);
      }
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) {
        a = fmin(a, __shfl_xor_sync(0xffffffffu, a, o));
        b = fmin(b, __shfl_xor_sync(0xffffffffu, b, o));
      }
      if ((threadIdx.x & 31) == 0) { ra[threadIdx.x >> 5] = a; rb[threadIdx.x >> 5] = b; }
      __syncthreads();
      mn = INFINITY; mxneg = INFINITY;
      for (int w = 0; w < int(blockDim.x >> 5); ++w) { mn = fmin(mn, ra[w]); mxneg = fmin(mxneg, rb[w]); }
      __syncthreads();
    }
    if (threadIdx.x != 0) return;
    const double cp = c->flux_c - s[2];
    c->phi_lo = cp;                              // target of the active part
    if (!(cp > 0.0) || !(s[1] > 0.0)) {          // nothing to distribute: y = 0 on D > 0
      c->mu = -mxneg + 1.0;
      c->mu_lo = c->mu_hi = c->mu;
      c->proj_pass = -1;
      return;
    }
    const double tmax = -mxneg;
    c->mu_hi = tmax;                                         // phi(mu_hi) = 0 <= cp
    c->mu_lo = fmin(mn, (s[0] - cp) / s[1]);                 // all active: phi = sum x - mu sum D >= cp
    c->proj_pass = 0;
  } else if (mode == 1) {
    double s[kFluxCand];
    ctrl_sum<kFluxCand, FP64>(d, SLOT_ARMX, s, false);
    if (threadIdx.x != 0 || c->proj_pass < 0) return;
    const double lo = c->mu_lo, hi = c->mu_hi, cp = c->phi_lo;
    double nlo = lo, nhi = hi;
    for (int q = 0; q < kFluxCand; ++q) {               // phi is non-increasing in mu
      const double m = lo + (hi - lo) * double(q + 1) / double(kFluxCand + 1);
      if (s[q] >= cp) nlo = m; else { nhi = m; break; }
    }
    c->mu_lo = nlo;
    c->mu_hi = nhi;
    c->proj_pass += 1;
  } else {
    double s[2];
    ctrl_sum<2, FP64>(d, SLOT_PROJ + 3, s, false);
    if (threadIdx.x != 0) return;
    if (c->proj_pass < 0) return;
    double mu = s[1] > 0.0 ? (s[0] - c->phi_lo) / s[1] : c->mu_hi;
    if (!(mu >= c->mu_lo)) mu = c->mu_lo;                 // clamp to the bracket
    if (!(mu <= c->mu_hi)) mu = c->mu_hi;
    c->mu = mu;
  }
}

// Plane 0 of the spectra = sum of planes 1..p (after the per-view adjoint column pass COL_PTOV),
// problems first .. first + gridDim.y - 1; skipped for a stopped problem when respect_done.
__global__ void k_view_sum(const ImgDesc* __restrict__ imgs, int first, int respect_done) {
  pdl_enter();
  const ImgDesc& d = imgs[first + blockIdx.y];
  if (respect_done && d.ctrl->done >= 1) return;
  const size_t n = d.P / 2;   // complex values per plane
  float2* s = reinterpret_cast<float2*>(d.spec);
  for (size_t i = blockIdx.x * size_t(blockDim.x) + threadIdx.x; i < n; i += size_t(gridDim.x) * blockDim.x) {
    float2 a = s[n + i];
    for (int j = 2; j <= d.p; ++j) {
      const float2 b = s[size_t(j) * n + i];
      a.x += b.x;
      a.y += b.y;
    }
    s[i] = a;
  }
}

// Scale f[0] by flux_c / sum f (flux-constrained start); sum from the set-up statistics
__global__ void k_scale(float* __restrict__ f, size_t P, const double* __restrict__ sum, double target) {
  const double s = sum[0];
  const float a = s > 0.0 ? float(target / s) : 1.0f;
  for (size_t i = blockIdx.x * size_t(blockDim.x) + threadIdx.x; i < P; i += size_t(gridDim.x) * blockDim.x)
    f[i] *= a;
}

// ------------------------------------------------------------------------------ set-up kernels
// g_int = g on S, -1 outside S (boundary); counts non-finite or negative samples.
__global__ void k_prepare_data(const float* __restrict__ g, const uint8_t* __restrict__ mask,
                               float* __restrict__ out, size_t P, int p, int* __restrict__ bad) {
  const size_t n = P * size_t(p);
  for (size_t i = blockIdx.x * size_t(blockDim.x) + threadIdx.x; i < n; i += size_t(gridDim.x) * blockDim.x) {
    float v = g[i];
    if (!isfinite(v) || v < 0.0f) { atomicAdd(bad, 1); v = 0.0f; }
    if (mask && !mask[i % P]) v = -1.0f;
    out[i] = v;
  }
}

// Grid-wide statistics in two stages (blocks x planes partials, then one block per plane).
// Stage 1, mode 0 (PSF): per plane sum, max, min, count of non-finite samples.
// Stage 1, mode 1 (data): per view sum over S of g (g >= 0 marks S), sum over S of b, |S|.
__global__ void __launch_bounds__(256) k_stats_partial(const float* __restrict__ x, const float* __restrict__ b,
                                                      const float* __restrict__ bconst, size_t P, int mode,
                                                      double* __restrict__ part) {
  const int plane = blockIdx.y;
  const float* a = x + size_t(plane) * P;
  const float* bj = b ? b + size_t(plane) * P : nullptr;
  const float bc = bconst ? bconst[plane] : 0.0f;
  // per thread: error-free FP32 two-sum accumulation (FP64 arithmetic is slow on this GPU) and FP32
  // max / min / counts (exact: a thread sees fewer than 2^24 pixels); FP64 from the block level up
  Acc<true> k0, k1;
  float m1 = mode ? 0.0f : -INFINITY, m2 = mode ? 0.0f : INFINITY, n2 = 0.0f, n3 = 0.0f;
  auto add = [&](float v, size_t i) {
    if (mode == 0) {
      if (!isfinite(v)) { n3 += 1.0f; return; }
      k0.add(v); m1 = fmaxf(m1, v); m2 = fminf(m2, v);
    } else {
      if (v < 0.0f) return;
      k0.add(v); k1.add(bj ? bj[i] : bc); n2 += 1.0f;
    }
  };
  const size_t stride = size_t(gridDim.x) * blockDim.x;
  // 16-byte loads of four samples, four of them in flight per thread, when the plane allows
  const bool vec = P % 4 == 0 && (reinterpret_cast<uintptr_t>(a) & 15) == 0;
  size_t i0 = 0;
  if (vec) {
    const float4* a4 = reinterpret_cast<const float4*>(a);
    const size_t P4 = P / 4;
    size_t j = blockIdx.x * size_t(blockDim.x) + threadIdx.x;
    for (; j + 3 * stride < P4; j += 4 * stride) {
      float4 v[4];
#pragma unroll
      for (int u = 0; u < 4; ++u) v[u] = a4[j + u * stride];
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        const size_t e = 4 * (j + u * stride);
        add(v[u].x, e); add(v[u].y, e + 1); add(v[u].z, e + 2); add(v[u].w, e + 3);
      }
    }
    for (; j < P4; j += stride) {
      const float4 v = a4[j];
      add(v.x, 4 * j); add(v.y, 4 * j + 1); add(v.z, 4 * j + 2); add(v.w, 4 * j + 3);
    }
    i0 = P;   // nothing left for the scalar loop
  }
  for (size_t i = i0 + blockIdx.x * size_t(blockDim.x) + threadIdx.x; i < P; i += stride) add(a[i], i);
  const double s0 = double(k0.hi) + double(k0.lo), s3 = n3;
  const double s1 = mode ? double(k1.hi) + double(k1.lo) : double(m1), s2 = mode ? double(n2) : double(m2);
  __shared__ double r[4][256];
  r[0][threadIdx.x] = s0; r[1][threadIdx.x] = s1; r[2][threadIdx.x] = s2; r[3][threadIdx.x] = s3;
  __syncthreads();
  for (int o = 128; o > 0; o >>= 1) {
    if (threadIdx.x < o) {
      r[0][threadIdx.x] += r[0][threadIdx.x + o];
      r[3][threadIdx.x] += r[3][threadIdx.x + o];
      if (mode == 0) {
        r[1][threadIdx.x] = fmax(r[1][threadIdx.x], r[1][threadIdx.x + o]);
        r[2][threadIdx.x] = fmin(r[2][threadIdx.x], r[2][threadIdx.x + o]);
      } else {
        r[1][threadIdx.x] += r[1][threadIdx.x + o];
        r[2][threadIdx.x] += r[2][threadIdx.x + o];
      }
    }
    __syncthreads();
  }
  if (threadIdx.x < 4) part[(size_t(plane) * gridDim.x + blockIdx.x) * 4 + threadIdx.x] = r[threadIdx.x][0];
}

// Stage 2: one block per plane combines the nb partials of stage 1 into out[4 * plane + 0..3].
__global__ void __launch_bounds__(256) k_stats_final(const double* __restrict__ part, int nb, int mode,
                                                    double* __restrict__ out) {
  const int plane = blockIdx.x;
  __shared__ double r[4][256];
  double s0 = 0.0, s1 = mode ? 0.0 : -INFINITY, s2 = mode ? 0.0 : INFINITY, s3 = 0.0;
  for (int i = threadIdx.x; i < nb; i += blockDim.x) {
    const double* q = part + (size_t(plane) * nb + i) * 4;
    s0 += q[0]; s3 += q[3];
    if (mode == 0) { s1 = fmax(s1, q[1]); s2 = fmin(s2, q[2]); }
    else { s1 += q[1]; s2 += q[2]; }
  }
  r[0][threadIdx.x] = s0; r[1][threadIdx.x] = s1; r[2][threadIdx.x] = s2; r[3][threadIdx.x] = s3;
  __syncthreads();
  for (int o = 128; o > 0; o >>= 1) {   // tree in a fixed pattern: deterministic
    if (threadIdx.x < o) {
      r[0][threadIdx.x] += r[0][threadIdx.x + o];
      r[3][threadIdx.x] += r[3][threadIdx.x + o];
      if (mode == 0) {
        r[1][threadIdx.x] = fmax(r[1][threadIdx.x], r[1][threadIdx.x + o]);
        r[2][threadIdx.x] = fmin(r[2][threadIdx.x], r[2][threadIdx.x + o]);
      } else {
        r[1][threadIdx.x] += r[1][threadIdx.x + o];
        r[2][threadIdx.x] += r[2][threadIdx.x + o];
      }
    }
    __syncthreads();
  }
  if (threadIdx.x < 4) out[4 * plane + threadIdx.x] = r[threadIdx.x][0];
}

// f = value on R (w > 0), 0 elsewhere; or f = max(src, 0) restricted to R when src != nullptr
__global__ void k_fill_start(float* __restrict__ f, const float* __restrict__ w, const float* __restrict__ src,
                             float value, size_t P) {
  for (size_t i = blockIdx.x * size_t(blockDim.x) + threadIdx.x; i < P; i += size_t(gridDim.x) * blockDim.x) {
    const bool inR = !w || w[i] > 0.0f;
    float v = src ? fmaxf(src[i], 0.0f) : value;
    if (!isfinite(v)) v = 0.0f;
    f[i] = inR ? v : 0.0f;
  }
}

// boundary set-up: R = {alpha_j >= sigma for every j}, w = M_R / sum_j alpha_j (Eq. Rdef, boundaryRL)
// and the per-view OSEM weights wv_j = M_R / alpha_j (Eq. boundaryOSEM)
__global__ void k_make_w(const float* __restrict__ alpha, int p, size_t P, float sigma, float* __restrict__ w,
                         float* __restrict__ wv) {
  for (size_t i = blockIdx.x * size_t(blockDim.x) + threadIdx.x; i < P; i += size_t(gridDim.x) * blockDim.x) {
    float s = 0.0f;
    bool inR = true;
    for (int j = 0; j < p; ++j) {
      const float a = alpha[size_t(j) * P + i];
      inR = inR && (a >= sigma);
      s += a;
    }
    w[i] = (inR && s > 0.0f) ? 1.0f / s : 0.0f;
    for (int j = 0; j < p; ++j) {
      const float a = alpha[size_t(j) * P + i];
      wv[size_t(j) * P + i] = (inR && a > 0.0f) ? 1.0f / a : 0.0f;
    }
  }
}

// Condition of the device-side solve loop (a WHILE node of a CUDA graph, see run_until): keep
// iterating while some problem has not stopped (done == 0) and fewer than `cap` bodies have
// run since the launch (counter, zeroed by the host before the launch).  One block; it is the last
// node of the loop body, so it sees the controllers' decisions of this iteration.  Launched as a
// programmatic dependent of the body's last pass: it waits for that pass before reading.
__global__ void k_loop_cond(const ImgDesc* __restrict__ imgs, int n, cudaGraphConditionalHandle h,
                            int* __restrict__ counter, int cap) {
  pdl_enter();
  __shared__ int running;
  if (threadIdx.x == 0) running = 0;
  __syncthreads();
  for (int i = threadIdx.x; i < n; i += blockDim.x)
    if (imgs[i].ctrl->done == 0) running = 1;
  __syncthreads();
  if (threadIdx.x == 0) {
    const int k = counter[0] + 1;
    counter[0] = k;
    cudaGraphSetConditional(h, (running && k < cap) ? 1u : 0u);
  }
}

// PSF band: out[c] = max over views j and rows r of max(|Re|, |Im|) of the PSF spectrum column c.
// Block (x, y) covers columns x * blockDim.x .. and the rows y, y + gridDim.y, ..; the partial
// maxima meet in out (zeroed by the caller) by an integer atomicMax, which orders non-negative
// floats like their bit patterns.
__global__ void k_khat_colmax(const float2* __restrict__ khat, int H, int M, int p, float* __restrict__ out) {
  const int col = blockIdx.x * blockDim.x + threadIdx.x;
  if (col >= M) return;
  float m = 0.0f;
  for (int j = 0; j < p; ++j)
    for (int r = blockIdx.y; r < H; r += gridDim.y) {
      const float2 v = khat[size_t(j) * H * M + spec_row_off(r, M, spec_interleaved(H)) + (spec_interleaved(H) ? 4 : 1) * col];
      m = fmaxf(m, fmaxf(fabsf(v.x), fabsf(v.y)));
    }
  atomicMax(reinterpret_cast<int*>(out) + col, __float_as_int(m));
}

// OSEM: count the pending update of every problem (after the last sub-step of a call)
__global__ void k_osem_tick(const ImgDesc* __restrict__ imgs, int n, int have_v_after) {
  const int i = blockIdx.x;
  if (i < n) osem_tick(imgs[i].ctrl, have_v_after);
}

__global__ void k_u8_to_float(const uint8_t* __restrict__ m, float* __restrict__ out, size_t P) {
  for (size_t i = blockIdx.x * size_t(blockDim.x) + threadIdx.x; i < P; i += size_t(gridDim.x) * blockDim.x)
    out[i] = m[i] ? 1.0f : 0.0f;
}

// x *= mask for nplanes planes: mask = (w > 0) [M_R] when w is given, (g >= 0) [M_S] when g is given
__global__ void k_apply_mask(float* __restrict__ x, size_t P, int nplanes, const float* __restrict__ w,
                             const float* __restrict__ g) {
  const size_t n = P * size_t(nplanes);
  for (size_t i = blockIdx.x * size_t(blockDim.x) + threadIdx.x; i < n; i += size_t(gridDim.x) * blockDim.x) {
    const size_t q = i % P;
    bool keep = true;
    if (w) keep = w[q] > 0.0f;
    if (g) keep = g[i] >= 0.0f;
    if (!keep) x[i] = 0.0f;
  }
}

// sum of squares of x (one block): out[0]
__global__ void __launch_bounds__(256) k_sumsq(const float* __restrict__ x, size_t P, double* __restrict__ out) {
  double s = 0.0;
  for (size_t i = threadIdx.x; i < P; i += blockDim.x) s += double(x[i]) * x[i];
  __shared__ double r[256];
  r[threadIdx.x] = s;
  __syncthreads();
  for (int o = 128; o > 0; o >>= 1) {
    if (threadIdx.x < o) r[threadIdx.x] += r[threadIdx.x + o];
    __syncthreads();
  }
  if (threadIdx.x == 0) out[0] = r[0];
}

}  // namespace sgp

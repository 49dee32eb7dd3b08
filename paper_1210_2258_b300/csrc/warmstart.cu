// Learned warm start: kernels of a small convolutional encoder-decoder that predicts the SGP
// starting point f^(0) from the detected image g (forward, backward and Adam).
//
// Tensors are NHWC with batch B; activations and the working copies of the weights are bf16,
// accumulation and master weights are FP32.  The 32 -> 32 channel 3x3 convolutions are implicit
// GEMMs on the tensor cores (mma.sync m16n8k16, bf16 in, FP32 accumulate):
//   forward  Y[p][co] = act(sum_{tap, ci} X[p + off(tap)][ci] W[co][tap][ci] + b[co])
//   dgrad    dX = the same kernel on dY with W'[ci][tap][co] = W[co][8 - tap][ci] (flipped taps),
//            times the ReLU mask of the layer below
//   wgrad    dW[co][tap][ci] = sum_p dY[p][co] X[p + off(tap)][ci]
// with "same" zero padding.  The 1 -> 32 input layer and the 32 -> 1 output layer are small and run on
// the FP32 pipes.  All declarations and contracts: include/warmstart.h.
#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include "../../include/warmstart.h"

namespace {

using bf16 = __nv_bfloat16;

__device__ __forceinline__ uint32_t ld32(const bf16* p) { return *reinterpret_cast<const uint32_t*>(p); }
__device__ __forceinline__ uint32_t pack2(bf16 lo, bf16 hi) {
  return uint32_t(__bfloat16_as_ushort(lo)) | (uint32_t(__bfloat16_as_ushort(hi)) << 16);
}
__device__ __forceinline__ void mma16816(float (&d)[4], uint32_t a0, uint32_t a1, uint32_t a2, uint32_t a3, uint32_t b0,
                                         uint32_t b1) {
  asm volatile(
      "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
      "{%0,%1,%2,%3};\n"
      : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
      : "r"(a0), "r"(a1), "r"(a2), "r"(a3), "r"(b0), "r"(b1));
}

constexpr int TW = 16, TH = 8;          // output tile: 8 rows x 16 columns = 128 pixels
constexpr int HX = TW + 2, HY = TH + 2;  // halo tile
constexpr int CP = 40;                   // channel pitch in shared memory (bank-conflict-free fragments)
constexpr int WP = 9 * 32 + 8;           // weight pitch per output channel

// Stage the input halo tile (zero outside the image) and the weights.
__device__ __forceinline__ void stage_tile(const bf16* __restrict__ x, bf16* sx, int b, int y0, int x0, int H, int W) {
  for (int i = threadIdx.x; i < HY * HX * 4; i += blockDim.x) {
    const int pix = i >> 2, q = i & 3;
    const int hy = pix / HX, hx = pix % HX;
    const int yy = y0 + hy - 1, xx = x0 + hx - 1;
    int4 v = make_int4(0, 0, 0, 0);
    if (yy >= 0 && yy < H && xx >= 0 && xx < W)
      v = reinterpret_cast<const int4*>(x + ((size_t(b) * H + yy) * W + xx) * 32)[q];
    *reinterpret_cast<int4*>(sx + pix * CP + q * 8) = v;
  }
}

// MODE: 0 bias + ReLU, 1 bias (linear), 2 multiply by (mask > 0), 3 plain
template <int MODE>
__global__ void __launch_bounds__(128) k_conv32(const bf16* __restrict__ x, const bf16* __restrict__ w,
                                               const float* __restrict__ bias, const bf16* __restrict__ mask,
                                               bf16* __restrict__ y, int H, int W) {
  __shared__ __align__(16) bf16 sx[HY * HX * CP];
  __shared__ __align__(16) bf16 sw[32 * WP];
  const int x0 = blockIdx.x * TW, y0 = blockIdx.y * TH, b = blockIdx.z;
  for (int i = threadIdx.x; i < 32 * 9 * 4; i += blockDim.x) {   // 32 co x 9 taps x 4 x 8 ci
    const int co = i / 36, r = i % 36;
    *reinterpret_cast<int4*>(sw + co * WP + r * 8) = reinterpret_cast<const int4*>(w)[i];
  }
  stage_tile(x, sx, b, y0, x0, H, W);
  __syncthreads();
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, g = lane >> 2, t = lane & 3;
  float acc[2][4][4];
#pragma unroll
  for (int i = 0; i < 2; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j)
#pragma unroll
      for (int k = 0; k < 4; ++k) acc[i][j][k] = 0.0f;
#pragma unroll
  for (int tap = 0; tap < 9; ++tap) {
    const int dy = tap / 3, dx = tap % 3;
#pragma unroll
    for (int h = 0; h < 2; ++h) {
      uint32_t bf[4][2];
#pragma unroll
      for (int nt = 0; nt < 4; ++nt) {
        const bf16* wp = sw + (8 * nt + g) * WP + tap * 32 + 16 * h + 2 * t;
        bf[nt][0] = ld32(wp);
        bf[nt][1] = ld32(wp + 8);
      }
#pragma unroll
      for (int mt = 0; mt < 2; ++mt) {
        const int r = 2 * warp + mt;
        const bf16* p0 = sx + ((r + dy) * HX + g + dx) * CP + 16 * h + 2 * t;
        const bf16* p1 = p0 + 8 * CP;
        const uint32_t a0 = ld32(p0), a1 = ld32(p1), a2 = ld32(p0 + 8), a3 = ld32(p1 + 8);
#pragma unroll
        for (int nt = 0; nt < 4; ++nt) mma16816(acc[mt][nt], a0, a1, a2, a3, bf[nt][0], bf[nt][1]);
      }
    }
  }
#pragma unroll
  for (int mt = 0; mt < 2; ++mt) {
    const int yy = y0 + 2 * warp + mt;
#pragma unroll
    for (int half = 0; half < 2; ++half) {
      const int xx = x0 + g + 8 * half;
      const size_t pix = (size_t(b) * H + yy) * W + xx;
#pragma unroll
      for (int nt = 0; nt < 4; ++nt) {
        const int co = 8 * nt + 2 * t;
        float v0 = acc[mt][nt][2 * half], v1 = acc[mt][nt][2 * half + 1];
        if (MODE <= 1) { v0 += bias[co]; v1 += bias[co + 1]; }
        if (MODE == 0) { v0 = fmaxf(v0, 0.0f); v1 = fmaxf(v1, 0.0f); }
        if (MODE == 2) {
          const bf16* m = mask + pix * 32 + co;
          if (!(__bfloat162float(m[0]) > 0.0f)) v0 = 0.0f;
          if (!(__bfloat162float(m[1]) > 0.0f)) v1 = 0.0f;
        }
        *reinterpret_cast<uint32_t*>(y + pix * 32 + co) = pack2(__float2bfloat16(v0), __float2bfloat16(v1));
      }
    }
  }
}

// dW[co][tap][ci] += sum_p dY[p][co] X[p + off(tap)][ci]  (32 x 288 GEMM with K = pixels), persistent
// blocks accumulate over tiles in registers and add once into the FP32 gradient.
__global__ void __launch_bounds__(128) k_conv32_wgrad(const bf16* __restrict__ dy, const bf16* __restrict__ x,
                                                     float* __restrict__ dw, int B, int H, int W) {
  __shared__ __align__(16) bf16 sx[HY * HX * CP];
  __shared__ __align__(16) bf16 sd[TH * TW * CP];
  const int tiles_x = W / TW, tiles_y = H / TH, ntiles = tiles_x * tiles_y * B;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, g = lane >> 2, t = lane & 3;
  float acc[2][9][4];
#pragma unroll
  for (int i = 0; i < 2; ++i)
#pragma unroll
    for (int j = 0; j < 9; ++j)
#pragma unroll
      for (int k = 0; k < 4; ++k) acc[i][j][k] = 0.0f;
  for (int tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
    const int b = tile / (tiles_x * tiles_y), rem = tile % (tiles_x * tiles_y);
    const int y0 = (rem / tiles_x) * TH, x0 = (rem % tiles_x) * TW;
    __syncthreads();
    stage_tile(x, sx, b, y0, x0, H, W);
    for (int i = threadIdx.x; i < TH * TW * 4; i += blockDim.x) {
      const int pix = i >> 2, q = i & 3;
      const int yy = y0 + pix / TW, xx = x0 + pix % TW;
      *reinterpret_cast<int4*>(sd + pix * CP + q * 8) =
          reinterpret_cast<const int4*>(dy + ((size_t(b) * H + yy) * W + xx) * 32)[q];
    }
    __syncthreads();
#pragma unroll 1
    for (int ks = 0; ks < TH; ++ks) {          // 16 pixels = one tile row per k-step
      uint32_t af[2][4];
#pragma unroll
      for (int mt = 0; mt < 2; ++mt) {
        const int co = 16 * mt + g;
        const bf16* d0 = sd + (ks * TW + 2 * t) * CP + co;
        af[mt][0] = pack2(d0[0], d0[CP]);
        af[mt][1] = pack2(d0[8], d0[CP + 8]);
        af[mt][2] = pack2(d0[8 * CP], d0[9 * CP]);
        af[mt][3] = pack2(d0[8 * CP + 8], d0[9 * CP + 8]);
      }
#pragma unroll
      for (int nt = 0; nt < 9; ++nt) {
        const int n = 8 * (9 * warp + nt) + g;
        const int tap = n >> 5, ci = n & 31, ddy = tap / 3, ddx = tap % 3;
        const bf16* xs = sx + ((ks + ddy) * HX + 2 * t + ddx) * CP + ci;
        const uint32_t b0 = pack2(xs[0], xs[CP]);
        const uint32_t b1 = pack2(xs[8 * CP], xs[9 * CP]);
#pragma unroll
        for (int mt = 0; mt < 2; ++mt) mma16816(acc[mt][nt], af[mt][0], af[mt][1], af[mt][2], af[mt][3], b0, b1);
      }
    }
  }
#pragma unroll
  for (int mt = 0; mt < 2; ++mt)
#pragma unroll
    for (int nt = 0; nt < 9; ++nt) {
      const int n = 8 * (9 * warp + nt) + 2 * t, co = 16 * mt + g;
      atomicAdd(dw + co * 288 + n, acc[mt][nt][0]);
      atomicAdd(dw + co * 288 + n + 1, acc[mt][nt][1]);
      atomicAdd(dw + (co + 8) * 288 + n, acc[mt][nt][2]);
      atomicAdd(dw + (co + 8) * 288 + n + 1, acc[mt][nt][3]);
    }
}

// W'[ci][tap][co] = W[co][8 - tap][ci]  (bf16 copy for the data-gradient pass)
__global__ void k_flip_weights(const bf16* __restrict__ w, bf16* __restrict__ wt) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= 32 * 9 * 32) return;
  const int ci = i / 288, tap = (i / 32) % 9, co = i % 32;
  wt[i] = w[(co * 9 + (8 - tap)) * 32 + ci];
}

// input layer 1 -> 32: Y[p][co] = relu(sum_tap X[p + off] W[co][tap] + b[co]), X fp32 single channel
__global__ void k_conv_in(const float* __restrict__ x, const float* __restrict__ w, const float* __restrict__ bias,
                          bf16* __restrict__ y, int B, int H, int W) {
  const size_t n = size_t(B) * H * W * 32;
  for (size_t i = blockIdx.x * size_t(blockDim.x) + threadIdx.x; i < n; i += size_t(gridDim.x) * blockDim.x) {
    const int co = int(i & 31);
    const size_t p = i >> 5;
    const int xx = int(p % W), yy = int((p / W) % H);
    const size_t bb = p / (size_t(W) * H);
    float s = bias[co];
#pragma unroll
    for (int tap = 0; tap < 9; ++tap) {
      const int u = yy + tap / 3 - 1, v = xx + tap % 3 - 1;
      if (u >= 0 && u < H && v >= 0 && v < W) s += x[(bb * H + u) * W + v] * w[co * 9 + tap];
    }
    y[i] = __float2bfloat16(fmaxf(s, 0.0f));
  }
}

// output layer 32 -> 1: Z[p] = sum_{tap, ci} X[p + off][ci] W[tap][ci] + b (FP32 out)
__global__ void k_conv_out(const bf16* __restrict__ x, const float* __restrict__ w, const float* __restrict__ bias,
                           float* __restrict__ z, int B, int H, int W) {
  const size_t n = size_t(B) * H * W;
  for (size_t p = blockIdx.x * size_t(blockDim.x) + threadIdx.x; p < n; p += size_t(gridDim.x) * blockDim.x) {
    const int xx = int(p % W), yy = int((p / W) % H);
    const size_t bb = p / (size_t(W) * H);
    float s = bias[0];
    for (int tap = 0; tap < 9; ++tap) {
      const int u = yy + tap / 3 - 1, v = xx + tap % 3 - 1;
      if (u < 0 || u >= H || v < 0 || v >= W) continue;
      const bf16* xp = x + ((bb * H + u) * W + v) * 32;
#pragma unroll
      for (int ci = 0; ci < 32; ++ci) s += __bfloat162float(xp[ci]) * w[tap * 32 + ci];
    }
    z[p] = s;
  }
}

// data gradient of the output layer, times the ReLU mask of its input:
// dX[q][ci] = (X[q][ci] > 0) sum_tap dZ[q - off(tap)] W[tap][ci]
__global__ void k_conv_out_dgrad(const float* __restrict__ dz, const float* __restrict__ w,
                                 const bf16* __restrict__ xin, bf16* __restrict__ dx, int B, int H, int W) {
  const size_t n = size_t(B) * H * W * 32;
  for (size_t i = blockIdx.x * size_t(blockDim.x) + threadIdx.x; i < n; i += size_t(gridDim.x) * blockDim.x) {
    const int ci = int(i & 31);
    const size_t q = i >> 5;
    const int xx = int(q % W), yy = int((q / W) % H);
    const size_t bb = q / (size_t(W) * H);
    float s = 0.0f;
#pragma unroll
    for (int tap = 0; tap < 9; ++tap) {
      const int u = yy - (tap / 3 - 1), v = xx - (tap % 3 - 1);
      if (u >= 0 && u < H && v >= 0 && v < W) s += dz[(bb * H + u) * W + v] * w[tap * 32 + ci];
    }
    dx[i] = __float2bfloat16(__bfloat162float(xin[i]) > 0.0f ? s : 0.0f);
  }
}

// Weight and bias gradients of the small layers, one thread per weight, blocks over pixel chunks:
// mode 0 (input layer): dW[co][tap] += sum_p dY[p][co] X[p + off(tap)] (X fp32, 1 channel), db[co] += sum dY
// mode 1 (output layer): dW[tap][ci] += sum_p dZ[p] X[p + off(tap)][ci] (X bf16, 32 channels), db += sum dZ
__global__ void __launch_bounds__(320) k_small_wgrad(const void* __restrict__ dyv, const void* __restrict__ xv,
                                                    float* __restrict__ dw, float* __restrict__ db, int B, int H, int W,
                                                    int mode, int chunk) {
  const int k = threadIdx.x;     // 0..287 weights, 288..319 bias entries
  const size_t n = size_t(B) * H * W;
  const size_t p0 = size_t(blockIdx.x) * chunk, p1 = p0 + chunk < n ? p0 + chunk : n;
  float s = 0.0f;
  if (mode == 0) {
    const bf16* dy = static_cast<const bf16*>(dyv);
    const float* x = static_cast<const float*>(xv);
    if (k < 288) {
      const int co = k / 9, tap = k % 9, oy = tap / 3 - 1, ox = tap % 3 - 1;
      for (size_t p = p0; p < p1; ++p) {
        const int xx = int(p % W), yy = int((p / W) % H);
        const int u = yy + oy, v = xx + ox;
        if (u >= 0 && u < H && v >= 0 && v < W)
          s += __bfloat162float(dy[p * 32 + co]) * x[(p / (size_t(W) * H) * H + u) * W + v];
      }
      atomicAdd(dw + k, s);
    } else {
      const int co = k - 288;
      for (size_t p = p0; p < p1; ++p) s += __bfloat162float(dy[p * 32 + co]);
      atomicAdd(db + co, s);
    }
  } else {
    const float* dz = static_cast<const float*>(dyv);
    const bf16* x = static_cast<const bf16*>(xv);
    if (k < 288) {
      const int tap = k / 32, ci = k % 32, oy = tap / 3 - 1, ox = tap % 3 - 1;
      for (size_t p = p0; p < p1; ++p) {
        const int xx = int(p % W), yy = int((p / W) % H);
        const int u = yy + oy, v = xx + ox;
        if (u >= 0 && u < H && v >= 0 && v < W)
          s += dz[p] * __bfloat162float(x[((p / (size_t(W) * H) * H + u) * W + v) * 32 + ci]);
      }
      atomicAdd(dw + k, s);
    } else if (k == 288) {
      for (size_t p = p0; p < p1; ++p) s += dz[p];
      atomicAdd(db, s);
    }
  }
}

// per-channel sum of dY (bias gradient of the 32 -> 32 layers)
__global__ void __launch_bounds__(256) k_bias_grad(const bf16* __restrict__ dy, float* __restrict__ db, size_t npix) {
  const int c = threadIdx.x & 31, row = threadIdx.x >> 5;
  float s = 0.0f;
  for (size_t p = blockIdx.x * size_t(8) + row; p < npix; p += size_t(gridDim.x) * 8) s += __bfloat162float(dy[p * 32 + c]);
  __shared__ float r[8][32];
  r[row][c] = s;
  __syncthreads();
  if (row == 0) {
    for (int q = 1; q < 8; ++q) s += r[q][c];
    atomicAdd(db + c, s);
  }
}

// 2x2 average pooling (forward) and its adjoint
__global__ void k_pool2(const bf16* __restrict__ x, bf16* __restrict__ y, int B, int H, int W) {
  const int h = H / 2, w = W / 2;
  const size_t n = size_t(B) * h * w * 32;
  for (size_t i = blockIdx.x * size_t(blockDim.x) + threadIdx.x; i < n; i += size_t(gridDim.x) * blockDim.x) {
    const int c = int(i & 31);
    const size_t q = i >> 5;
    const int xx = int(q % w), yy = int((q / w) % h);
    const size_t bb = q / (size_t(w) * h);
    const size_t base = ((bb * H + 2 * yy) * W + 2 * xx) * 32 + c;
    const float s = __bfloat162float(x[base]) + __bfloat162float(x[base + 32]) + __bfloat162float(x[base + size_t(W) * 32]) +
                    __bfloat162float(x[base + size_t(W) * 32 + 32]);
    y[i] = __float2bfloat16(0.25f * s);
  }
}

// nearest 2x upsampling (forward) of x (B, H/2, W/2) added to skip (B, H, W): y = up(x) + skip
__global__ void k_up2_add(const bf16* __restrict__ x, const bf16* __restrict__ skip, bf16* __restrict__ y, int B, int H,
                          int W) {
  const size_t n = size_t(B) * H * W * 32;
  for (size_t i = blockIdx.x * size_t(blockDim.x) + threadIdx.x; i < n; i += size_t(gridDim.x) * blockDim.x) {
    const int c = int(i & 31);
    const size_t p = i >> 5;
    const int xx = int(p % W), yy = int((p / W) % H);
    const size_t bb = p / (size_t(W) * H);
    const float v = __bfloat162float(x[((bb * (H / 2) + yy / 2) * (W / 2) + xx / 2) * 32 + c]) + __bfloat162float(skip[i]);
    y[i] = __float2bfloat16(v);
  }
}

// backward of the skip / pooling junction at full resolution:
// dZ2 = (dS5 + pool^T(dP2)) * (A2 > 0);  also dU = up^T(dS5) at half resolution (mode 1)
__global__ void k_junction_bwd(const bf16* __restrict__ ds5, const bf16* __restrict__ dp2, const bf16* __restrict__ a2,
                               bf16* __restrict__ dz2, int B, int H, int W) {
  const size_t n = size_t(B) * H * W * 32;
  for (size_t i = blockIdx.x * size_t(blockDim.x) + threadIdx.x; i < n; i += size_t(gridDim.x) * blockDim.x) {
    const int c = int(i & 31);
    const size_t p = i >> 5;
    const int xx = int(p % W), yy = int((p / W) % H);
    const size_t bb = p / (size_t(W) * H);
    float v = __bfloat162float(ds5[i]) + 0.25f * __bfloat162float(dp2[((bb * (H / 2) + yy / 2) * (W / 2) + xx / 2) * 32 + c]);
    dz2[i] = __float2bfloat16(__bfloat162float(a2[i]) > 0.0f ? v : 0.0f);
  }
}

// dA4 = up^T(dS5) (sum over each 2x2 block), times the ReLU mask of A4
__global__ void k_up2_bwd_mask(const bf16* __restrict__ ds5, const bf16* __restrict__ a4, bf16* __restrict__ dz4,
                               int B, int H, int W) {
  const int h = H / 2, w = W / 2;
  const size_t n = size_t(B) * h * w * 32;
  for (size_t i = blockIdx.x * size_t(blockDim.x) + threadIdx.x; i < n; i += size_t(gridDim.x) * blockDim.x) {
    const int c = int(i & 31);
    const size_t q = i >> 5;
    const int xx = int(q % w), yy = int((q / w) % h);
    const size_t bb = q / (size_t(w) * h);
    const size_t base = ((bb * H + 2 * yy) * W + 2 * xx) * 32 + c;
    const float s = __bfloat162float(ds5[base]) + __bfloat162float(ds5[base + 32]) +
                    __bfloat162float(ds5[base + size_t(W) * 32]) + __bfloat162float(ds5[base + size_t(W) * 32 + 32]);
    dz4[i] = __float2bfloat16(__bfloat162float(a4[i]) > 0.0f ? s : 0.0f);
  }
}

// squared-error loss between the output z and the target t; dz = 2 (z - t) / n; loss sum in out[0]
__global__ void __launch_bounds__(256) k_loss(const float* __restrict__ z, const float* __restrict__ t,
                                             float* __restrict__ dz, double* __restrict__ out, size_t n) {
  double s = 0.0;
  const float scale = 2.0f / float(n);
  for (size_t i = blockIdx.x * size_t(blockDim.x) + threadIdx.x; i < n; i += size_t(gridDim.x) * blockDim.x) {
    const float e = z[i] - t[i];
    s += double(e) * e;
    dz[i] = scale * e;
  }
  __shared__ double r[256];
  r[threadIdx.x] = s;
  __syncthreads();
  for (int o = 128; o > 0; o >>= 1) {
    if (threadIdx.x < o) r[threadIdx.x] += r[threadIdx.x + o];
    __syncthreads();
  }
  if (threadIdx.x == 0) atomicAdd(out, r[0]);
}

// Adam on FP32 master weights; the bf16 working copies of the 32 -> 32 layers are refreshed
__global__ void k_adam(float* __restrict__ p, float* __restrict__ m, float* __restrict__ v, const float* __restrict__ g,
                       int n, float lr, float b1, float b2, float eps, float c1, float c2) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const float gi = g[i];
  const float mi = b1 * m[i] + (1.0f - b1) * gi;
  const float vi = b2 * v[i] + (1.0f - b2) * gi * gi;
  m[i] = mi;
  v[i] = vi;
  p[i] -= lr * (mi / c1) / (sqrtf(vi / c2) + eps);
}

__global__ void k_to_bf16(const float* __restrict__ x, bf16* __restrict__ y, int n) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) y[i] = __float2bfloat16(x[i]);
}

// input normalisation x = (g - b) / s and target t = log(1 + max(f, 0) / s) - log(1 + max(x, 0)):
// the network predicts a correction to the log-transformed data (s per image)
__global__ void k_prep(const float* __restrict__ g, const float* __restrict__ f, const float* __restrict__ bvec,
                       const float* __restrict__ svec, float* __restrict__ x, float* __restrict__ t, int B, size_t P) {
  const size_t n = size_t(B) * P;
  for (size_t i = blockIdx.x * size_t(blockDim.x) + threadIdx.x; i < n; i += size_t(gridDim.x) * blockDim.x) {
    const size_t bb = i / P;
    const float s = svec[bb];
    const float xi = (g[i] - bvec[bb]) / s;
    x[i] = xi;
    if (f) t[i] = log1pf(fmaxf(f[i], 0.0f) / s) - log1pf(fmaxf(xi, 0.0f));
  }
}

// f0 = s expm1(clamp(z + log(1 + max(x, 0)), 0, 20)) (the inverse of the target transform, bounded)
__global__ void k_start(const float* __restrict__ z, const float* __restrict__ x, const float* __restrict__ svec,
                        float* __restrict__ f0, int B, size_t P) {
  const size_t n = size_t(B) * P;
  for (size_t i = blockIdx.x * size_t(blockDim.x) + threadIdx.x; i < n; i += size_t(gridDim.x) * blockDim.x)
    f0[i] = svec[i / P] * expm1f(fminf(fmaxf(z[i] + log1pf(fmaxf(x[i], 0.0f)), 0.0f), 20.0f));
}

// s[b] = 1 + mean over the image of max(g - b, 0) (input scale of the network), one block per image
__global__ void __launch_bounds__(256) k_scale(const float* __restrict__ g, const float* __restrict__ bvec,
                                              float* __restrict__ s, size_t P) {
  const float* gb = g + size_t(blockIdx.x) * P;
  const float bb = bvec[blockIdx.x];
  double acc = 0.0;
  for (size_t i = threadIdx.x; i < P; i += blockDim.x) acc += fmaxf(gb[i] - bb, 0.0f);
  __shared__ double r[256];
  r[threadIdx.x] = acc;
  __syncthreads();
  for (int o = 128; o > 0; o >>= 1) {
    if (threadIdx.x < o) r[threadIdx.x] += r[threadIdx.x + o];
    __syncthreads();
  }
  if (threadIdx.x == 0) s[blockIdx.x] = float(1.0 + r[0] / double(P));
}

int grid1(size_t n) {
  const size_t g = (n + 255) / 256;
  return int(g < 148 * 32 ? g : 148 * 32);
}

}  // namespace

extern "C" {

int ws_conv32(const void* x, const void* w, const float* bias, const void* mask, void* y, int B, int H, int W, int mode,
              void* stream) {
  if (H % TH || W % TW || B <= 0 || mode < 0 || mode > 3) return 1;
  const dim3 grid(W / TW, H / TH, B);
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  const bf16* xb = static_cast<const bf16*>(x);
  const bf16* wb = static_cast<const bf16*>(w);
  const bf16* mb = static_cast<const bf16*>(mask);
  bf16* yb = static_cast<bf16*>(y);
  switch (mode) {
    case 0: k_conv32<0><<<grid, 128, 0, s>>>(xb, wb, bias, mb, yb, H, W); break;
    case 1: k_conv32<1><<<grid, 128, 0, s>>>(xb, wb, bias, mb, yb, H, W); break;
    case 2: k_conv32<2><<<grid, 128, 0, s>>>(xb, wb, bias, mb, yb, H, W); break;
    default: k_conv32<3><<<grid, 128, 0, s>>>(xb, wb, bias, mb, yb, H, W); break;
  }
  return cudaPeekAtLastError() == cudaSuccess ? 0 : 4;
}

int ws_conv32_wgrad(const void* dy, const void* x, float* dw, int B, int H, int W, void* stream) {
  if (H % TH || W % TW || B <= 0) return 1;
  const int ntiles = (W / TW) * (H / TH) * B;
  const int grid = ntiles < 148 * 4 ? ntiles : 148 * 4;
  k_conv32_wgrad<<<grid, 128, 0, static_cast<cudaStream_t>(stream)>>>(static_cast<const bf16*>(dy),
                                                                     static_cast<const bf16*>(x), dw, B, H, W);
  return cudaPeekAtLastError() == cudaSuccess ? 0 : 4;
}

int ws_flip_weights(const void* w, void* wt, void* stream) {
  k_flip_weights<<<36, 256, 0, static_cast<cudaStream_t>(stream)>>>(static_cast<const bf16*>(w), static_cast<bf16*>(wt));
  return cudaPeekAtLastError() == cudaSuccess ? 0 : 4;
}

int ws_conv_in(const float* x, const float* w, const float* bias, void* y, int B, int H, int W, void* stream) {
  k_conv_in<<<grid1(size_t(B) * H * W * 32), 256, 0, static_cast<cudaStream_t>(stream)>>>(x, w, bias, static_cast<bf16*>(y), B, H, W);
  return cudaPeekAtLastError() == cudaSuccess ? 0 : 4;
}

int ws_conv_out(const void* x, const float* w, const float* bias, float* z, int B, int H, int W, void* stream) {
  k_conv_out<<<grid1(size_t(B) * H * W), 256, 0, static_cast<cudaStream_t>(stream)>>>(static_cast<const bf16*>(x), w, bias, z, B, H, W);
  return cudaPeekAtLastError() == cudaSuccess ? 0 : 4;
}

int ws_conv_out_dgrad(const float* dz, const float* w, const void* xin, void* dx, int B, int H, int W, void* stream) {
  k_conv_out_dgrad<<<grid1(size_t(B) * H * W * 32), 256, 0, static_cast<cudaStream_t>(stream)>>>(
      dz, w, static_cast<const bf16*>(xin), static_cast<bf16*>(dx), B, H, W);
  return cudaPeekAtLastError() == cudaSuccess ? 0 : 4;
}

int ws_small_wgrad(const void* dy, const void* x, float* dw, float* db, int B, int H, int W, int mode, void* stream) {
  const size_t n = size_t(B) * H * W;
  const int chunk = 1024;
  const int grid = int((n + chunk - 1) / chunk);
  k_small_wgrad<<<grid, 320, 0, static_cast<cudaStream_t>(stream)>>>(dy, x, dw, db, B, H, W, mode, chunk);
  return cudaPeekAtLastError() == cudaSuccess ? 0 : 4;
}

int ws_bias_grad(const void* dy, float* db, int B, int H, int W, void* stream) {
  const size_t np = size_t(B) * H * W;
  const int grid = int(np / 8 < 148 * 8 ? (np + 7) / 8 : 148 * 8);
  k_bias_grad<<<grid, 256, 0, static_cast<cudaStream_t>(stream)>>>(static_cast<const bf16*>(dy), db, np);
  return cudaPeekAtLastError() == cudaSuccess ? 0 : 4;
}

int ws_pool2(const void* x, void* y, int B, int H, int W, void* stream) {
  k_pool2<<<grid1(size_t(B) * H * W * 8), 256, 0, static_cast<cudaStream_t>(stream)>>>(
      static_cast<const bf16*>(x), static_cast<bf16*>(y), B, H, W);
  return cudaPeekAtLastError() == cudaSuccess ? 0 : 4;
}

int ws_up2_add(const void* x, const void* skip, void* y, int B, int H, int W, void* stream) {
  k_up2_add<<<grid1(size_t(B) * H * W * 32), 256, 0, static_cast<cudaStream_t>(stream)>>>(
      static_cast<const bf16*>(x), static_cast<const bf16*>(skip), static_cast<bf16*>(y), B, H, W);
  return cudaPeekAtLastError() == cudaSuccess ? 0 : 4;
}

int ws_junction_bwd(const void* ds5, const void* dp2, const void* a2, void* dz2, int B, int H, int W, void* stream) {
  k_junction_bwd<<<grid1(size_t(B) * H * W * 32), 256, 0, static_cast<cudaStream_t>(stream)>>>(
      static_cast<const bf16*>(ds5), static_cast<const bf16*>(dp2), static_cast<const bf16*>(a2), static_cast<bf16*>(dz2),
      B, H, W);
  return cudaPeekAtLastError() == cudaSuccess ? 0 : 4;
}

int ws_up2_bwd_mask(const void* ds5, const void* a4, void* dz4, int B, int H, int W, void* stream) {
  k_up2_bwd_mask<<<grid1(size_t(B) * H * W * 8), 256, 0, static_cast<cudaStream_t>(stream)>>>(
      static_cast<const bf16*>(ds5), static_cast<const bf16*>(a4), static_cast<bf16*>(dz4), B, H, W);
  return cudaPeekAtLastError() == cudaSuccess ? 0 : 4;
}

int ws_loss(const float* z, const float* t, float* dz, double* out, size_t n, void* stream) {
  k_loss<<<grid1(n) < 1024 ? grid1(n) : 1024, 256, 0, static_cast<cudaStream_t>(stream)>>>(z, t, dz, out, n);
  return cudaPeekAtLastError() == cudaSuccess ? 0 : 4;
}

int ws_adam(float* p, float* m, float* v, const float* g, int n, float lr, float b1, float b2, float eps, int step,
            void* stream) {
  const float c1 = 1.0f - powf(b1, float(step)), c2 = 1.0f - powf(b2, float(step));
  k_adam<<<(n + 255) / 256, 256, 0, static_cast<cudaStream_t>(stream)>>>(p, m, v, g, n, lr, b1, b2, eps, c1, c2);
  return cudaPeekAtLastError() == cudaSuccess ? 0 : 4;
}

int ws_to_bf16(const float* x, void* y, int n, void* stream) {
  k_to_bf16<<<(n + 255) / 256, 256, 0, static_cast<cudaStream_t>(stream)>>>(x, static_cast<bf16*>(y), n);
  return cudaPeekAtLastError() == cudaSuccess ? 0 : 4;
}

int ws_prep(const float* g, const float* f, const float* b, const float* s, float* x, float* t, int B, size_t P,
            void* stream) {
  k_prep<<<grid1(size_t(B) * P), 256, 0, static_cast<cudaStream_t>(stream)>>>(g, f, b, s, x, t, B, P);
  return cudaPeekAtLastError() == cudaSuccess ? 0 : 4;
}

int ws_start(const float* z, const float* x, const float* s, float* f0, int B, size_t P, void* stream) {
  k_start<<<grid1(size_t(B) * P), 256, 0, static_cast<cudaStream_t>(stream)>>>(z, x, s, f0, B, P);
  return cudaPeekAtLastError() == cudaSuccess ? 0 : 4;
}

int ws_scale(const float* g, const float* b, float* s, int B, size_t P, void* stream) {
  k_scale<<<B, 256, 0, static_cast<cudaStream_t>(stream)>>>(g, b, s, P);
  return cudaPeekAtLastError() == cudaSuccess ? 0 : 4;
}

int ws_zero(void* p, size_t bytes, void* stream) {
  return cudaMemsetAsync(p, 0, bytes, static_cast<cudaStream_t>(stream)) == cudaSuccess ? 0 : 4;
}

}  // extern "C"

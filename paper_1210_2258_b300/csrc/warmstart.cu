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
#include <algorithm>

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

// ------------------------------------------------------------------------------ tcgen05 convolution
// Forward (and data-gradient) 32 -> 32 3x3 convolution as an implicit GEMM on the 5th-generation
// tensor cores: a tile of M = 128 output pixels (16 image rows x 8 columns) times N = 32 output
// channels, K = 9 taps x 32 input channels, as 18 tcgen05.mma (kind::f16, bf16 in, FP32 accumulate
// in tensor memory) of K = 16 each, issued by one thread.
//
// Operands in shared memory, no swizzle, K-major "core matrices" of 8 rows x 16 bytes:
//   A: the tile's halo (18 x 10 pixels) stored [kc][halo pixel][8 channels] (kc = channel group of 8),
//      so that for tap (dy, dx) the 8-row group r (image row r of the tile, 8 consecutive pixels) starts
//      at halo pixel (r + dy) * 10 + dx: M-groups 160 bytes apart, K core matrices 180 * 16 bytes
//      apart -- every tap is the same buffer read at another start address, no copy per tap;
//   B: the weights stored [tap][kc][co][8 channels] (loaded once per block).
// Persistent blocks walk the tiles; the halo of tile i + 2 is fetched with cp.async (zero fill
// outside the image) while tile i is multiplied and tile i - 1 leaves tensor memory through the
// epilogue (two 32-column accumulators alternate).  Every wait on the MMA completion barrier has an
// iteration limit; a block that gives up records the error flag and still releases its tensor
// memory.
constexpr int TCR = 16, TCC = 8;                // output tile: 16 rows x 8 columns (M = 128)
constexpr int THC = TCC + 2;                    // halo columns
constexpr int THP = (TCR + 2) * THC;            // halo pixels (180)
constexpr int TA_BYTES = 4 * THP * 16;          // one A stage
constexpr int TB_BYTES = 9 * 4 * 32 * 16;       // weights
constexpr int TSTAGES = 3;
constexpr int TC_SMEM = TB_BYTES + TSTAGES * TA_BYTES;
constexpr int TC_BLOCKS_PER_SM = 4;             // 4 x 53 KB shared memory, 4 x 64 tensor-memory columns

__device__ __forceinline__ uint32_t smem_u32(const void* p) { return uint32_t(__cvta_generic_to_shared(p)); }

// tcgen05 shared-memory matrix descriptor: start address, byte distance between core matrices along
// K (leading) and along M/N (stride), the fixed version bits 46-48 = 0b001, no swizzle
__device__ __forceinline__ uint64_t umma_desc(uint32_t addr, uint32_t lead, uint32_t stride) {
  return uint64_t((addr & 0x3FFFF) >> 4) | (uint64_t((lead >> 4) & 0x3FFF) << 16) |
         (uint64_t((stride >> 4) & 0x3FFF) << 32) | (uint64_t(1) << 46);
}
// instruction descriptor of kind::f16: D FP32 (bits 4-5 = 1), A and B bf16 (bits 7-9, 10-12 = 1),
// both K-major, N = 32 (bits 17-22 = N / 8), M = 128 (bits 24-28 = M / 16)
constexpr uint32_t kConvIdesc = (1u << 4) | (1u << 7) | (1u << 10) | ((32u >> 3) << 17) | ((128u >> 4) << 24);

__device__ __forceinline__ bool mbar_wait_parity(uint64_t* m, uint32_t parity) {
  const uint32_t a = smem_u32(m);
  for (int i = 0; i < (1 << 22); ++i) {
    uint32_t ok;
    asm volatile("{ .reg .pred p; mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2; selp.u32 %0, 1, 0, p; }"
                 : "=r"(ok) : "r"(a), "r"(parity) : "memory");
    if (ok) return true;
  }
  return false;
}

__device__ __forceinline__ void tile_origin(int tile, int tiles_x, int tiles_yx, int& b, int& y0, int& x0) {
  b = tile / tiles_yx;
  const int rem = tile - b * tiles_yx;
  y0 = (rem / tiles_x) * TCR;
  x0 = (rem % tiles_x) * TCC;
}

// cp.async of one tile's halo into an A stage, 16 bytes per copy, zero fill outside the image
__device__ __forceinline__ void halo_async(const bf16* __restrict__ x, uint8_t* sa, int b, int y0, int x0, int H, int W) {
  const uint32_t base = smem_u32(sa);
  for (int i = threadIdx.x; i < THP * 4; i += blockDim.x) {
    const int hp = i >> 2, kc = i & 3;
    const int yy = y0 + hp / THC - 1, xx = x0 + hp % THC - 1;
    const bool in = yy >= 0 && yy < H && xx >= 0 && xx < W;
    const bf16* src = in ? x + ((size_t(b) * H + yy) * W + xx) * 32 + kc * 8 : x;
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;" ::"r"(base + (kc * THP + hp) * 16), "l"(src),
                 "r"(in ? 16 : 0) : "memory");
  }
}

// MODE: 0 bias + ReLU, 1 bias (linear), 2 multiply by (mask > 0), 3 plain
template <int MODE>
__global__ void __launch_bounds__(128, TC_BLOCKS_PER_SM) k_conv32(const bf16* __restrict__ x, const bf16* __restrict__ w,
                                                                 const float* __restrict__ bias,
                                                                 const bf16* __restrict__ mask, bf16* __restrict__ y,
                                                                 int B, int H, int W, int* __restrict__ err) {
  extern __shared__ __align__(128) uint8_t dsm[];
  uint8_t* sB = dsm;
  __shared__ __align__(8) uint64_t mbar[2];
  __shared__ uint32_t s_tmem;
  const int tiles_x = W / TCC, tiles_yx = tiles_x * (H / TCR), ntiles = tiles_yx * B;
  if (int(blockIdx.x) >= ntiles) return;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], 64;" ::"r"(smem_u32(&s_tmem))
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  if (threadIdx.x == 32) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(&mbar[0])) : "memory");
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(&mbar[1])) : "memory");
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  for (int i = threadIdx.x; i < 32 * 9 * 4; i += blockDim.x) {   // w[co][tap][ci] -> sB[tap][kc][co][8]
    const int co = i / 36, r = i % 36, tap = r >> 2, kc = r & 3;
    *reinterpret_cast<int4*>(sB + ((tap * 4 + kc) * 32 + co) * 16) = reinterpret_cast<const int4*>(w)[i];
  }
  // prologue: halos of this block's first two tiles
  for (int q = 0; q < 2; ++q) {
    const int tile = blockIdx.x + q * gridDim.x;
    if (tile < ntiles) {
      int b, y0, x0;
      tile_origin(tile, tiles_x, tiles_yx, b, y0, x0);
      halo_async(x, dsm + TB_BYTES + q * TA_BYTES, b, y0, x0, H, W);
    }
    asm volatile("cp.async.commit_group;" ::: "memory");
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const uint32_t tmem = s_tmem;
  bool ok = true;
  int prev_b = 0, prev_y0 = 0, prev_x0 = 0;
  int i = 0;
  auto epilogue = [&](int k, int b, int y0, int x0) {
    uint32_t v[32];
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,"
        "%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];"
        : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]), "=r"(v[7]),
          "=r"(v[8]), "=r"(v[9]), "=r"(v[10]), "=r"(v[11]), "=r"(v[12]), "=r"(v[13]), "=r"(v[14]), "=r"(v[15]),
          "=r"(v[16]), "=r"(v[17]), "=r"(v[18]), "=r"(v[19]), "=r"(v[20]), "=r"(v[21]), "=r"(v[22]), "=r"(v[23]),
          "=r"(v[24]), "=r"(v[25]), "=r"(v[26]), "=r"(v[27]), "=r"(v[28]), "=r"(v[29]), "=r"(v[30]), "=r"(v[31])
        : "r"(tmem + uint32_t((k & 1) * 32) + (uint32_t(32 * warp) << 16)));
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
    const int m = 32 * warp + lane;
    const size_t pix = (size_t(b) * H + y0 + m / TCC) * W + x0 + m % TCC;
    int4 mk[4];
    if (MODE == 2) {
#pragma unroll
      for (int q = 0; q < 4; ++q) mk[q] = reinterpret_cast<const int4*>(mask + pix * 32)[q];
    }
    uint32_t pk[16];
#pragma unroll
    for (int c = 0; c < 32; c += 2) {
      float v0 = __uint_as_float(v[c]), v1 = __uint_as_float(v[c + 1]);
      if (MODE <= 1) { v0 += bias[c]; v1 += bias[c + 1]; }
      if (MODE == 0) { v0 = fmaxf(v0, 0.0f); v1 = fmaxf(v1, 0.0f); }
      if (MODE == 2) {
        const uint32_t mw = reinterpret_cast<const uint32_t*>(mk)[c / 2];
        if (!(__bfloat162float(__ushort_as_bfloat16(uint16_t(mw & 0xffff))) > 0.0f)) v0 = 0.0f;
        if (!(__bfloat162float(__ushort_as_bfloat16(uint16_t(mw >> 16))) > 0.0f)) v1 = 0.0f;
      }
      pk[c / 2] = pack2(__float2bfloat16(v0), __float2bfloat16(v1));
    }
    int4* dst = reinterpret_cast<int4*>(y + pix * 32);
#pragma unroll
    for (int q = 0; q < 4; ++q) dst[q] = make_int4(int(pk[4 * q]), int(pk[4 * q + 1]), int(pk[4 * q + 2]), int(pk[4 * q + 3]));
  };
  for (int tile = blockIdx.x; tile < ntiles; tile += gridDim.x, ++i) {
    int b, y0, x0;
    tile_origin(tile, tiles_x, tiles_yx, b, y0, x0);
    // the halo of tile i has landed (only the group of tile i + 1 may still be in flight)
    asm volatile("cp.async.wait_group 1;" ::: "memory");
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    if (threadIdx.x == 0) {
      const uint32_t a0 = smem_u32(dsm + TB_BYTES + (i % TSTAGES) * TA_BYTES), b0 = smem_u32(sB);
      const uint32_t d = tmem + uint32_t((i & 1) * 32);
#pragma unroll 1
      for (int tap = 0; tap < 9; ++tap) {
        const int dy = tap / 3, dx = tap % 3;
#pragma unroll
        for (int ks = 0; ks < 2; ++ks) {
          const uint64_t ad = umma_desc(a0 + ((2 * ks) * THP + dy * THC + dx) * 16, THP * 16, THC * 16);
          const uint64_t bd = umma_desc(b0 + (tap * 4 + 2 * ks) * 32 * 16, 32 * 16, 8 * 16);
          const uint32_t accum = (tap | ks) ? 1u : 0u;
          asm volatile("{ .reg .pred p; setp.ne.b32 p, %4, 0; tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p; }"
                       ::"r"(d), "l"(ad), "l"(bd), "r"(kConvIdesc), "r"(accum) : "memory");
        }
      }
      asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];"
                   ::"r"(smem_u32(&mbar[i & 1])) : "memory");
    }
    if (i >= 1) {   // tile i - 1: its products are done, its stage is free, its accumulator is read out
      ok = ok && mbar_wait_parity(&mbar[(i - 1) & 1], uint32_t(((i - 1) >> 1) & 1));
      asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    }
    const int nt = tile + 2 * int(gridDim.x);
    if (nt < ntiles) {
      int nb, ny0, nx0;
      tile_origin(nt, tiles_x, tiles_yx, nb, ny0, nx0);
      halo_async(x, dsm + TB_BYTES + ((i + 2) % TSTAGES) * TA_BYTES, nb, ny0, nx0, H, W);
    }
    asm volatile("cp.async.commit_group;" ::: "memory");
    if (i >= 1) epilogue(i - 1, prev_b, prev_y0, prev_x0);
    prev_b = b; prev_y0 = y0; prev_x0 = x0;
  }
  ok = ok && mbar_wait_parity(&mbar[(i - 1) & 1], uint32_t(((i - 1) >> 1) & 1));
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  epilogue(i - 1, prev_b, prev_y0, prev_x0);
  asm volatile("cp.async.wait_group 0;" ::: "memory");
  if (!ok && lane == 0) atomicExch(err, 1);
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  if (warp == 0) {
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, 64;" ::"r"(tmem) : "memory");
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

// Pixel kernels: grid (ceil(W / 128), H, B), one thread per pixel (b, yy, xx); activations move as
// 64-byte rows of 32 bf16 channels (four 16-byte vectors).
__device__ __forceinline__ bool pix_of(int W, int& b, int& yy, int& xx) {
  xx = blockIdx.x * blockDim.x + threadIdx.x;
  yy = blockIdx.y;
  b = blockIdx.z;
  return xx < W;
}
__device__ __forceinline__ void load32(const bf16* p, float (&v)[32]) {
#pragma unroll
  for (int q = 0; q < 4; ++q) {
    const int4 t = reinterpret_cast<const int4*>(p)[q];
    const uint32_t w4[4] = {uint32_t(t.x), uint32_t(t.y), uint32_t(t.z), uint32_t(t.w)};
#pragma unroll
    for (int k = 0; k < 4; ++k) {
      v[8 * q + 2 * k] = __bfloat162float(__ushort_as_bfloat16(uint16_t(w4[k] & 0xffff)));
      v[8 * q + 2 * k + 1] = __bfloat162float(__ushort_as_bfloat16(uint16_t(w4[k] >> 16)));
    }
  }
}
__device__ __forceinline__ void store32(bf16* p, const float (&v)[32]) {
#pragma unroll
  for (int q = 0; q < 4; ++q)
    reinterpret_cast<int4*>(p)[q] = make_int4(
        int(pack2(__float2bfloat16(v[8 * q]), __float2bfloat16(v[8 * q + 1]))),
        int(pack2(__float2bfloat16(v[8 * q + 2]), __float2bfloat16(v[8 * q + 3]))),
        int(pack2(__float2bfloat16(v[8 * q + 4]), __float2bfloat16(v[8 * q + 5]))),
        int(pack2(__float2bfloat16(v[8 * q + 6]), __float2bfloat16(v[8 * q + 7]))));
}
dim3 pix_grid(int B, int H, int W) { return dim3((W + 127) / 128, H, B); }
// Block-wide store of 32 channels per pixel for the 128 consecutive pixels x0 .. x0 + 127 of one
// row (one per thread; pixels at or beyond W are skipped), staged in shared memory so that every
// warp store writes 512 contiguous bytes: stored directly, a thread's 64 bytes go out as four
// 16-byte pieces 64 bytes apart, half-sector writes.  Called by every thread of the block.
__device__ __forceinline__ void store32_block(bf16* row, int x0, int W, const float (&v)[32]) {
  __shared__ int4 tile[128 * 5];                   // 5 int4 per pixel: conflict-free both ways
  const int p = int(threadIdx.x);
#pragma unroll
  for (int q = 0; q < 4; ++q)
    tile[p * 5 + q] = make_int4(int(pack2(__float2bfloat16(v[8 * q]), __float2bfloat16(v[8 * q + 1]))),
                                int(pack2(__float2bfloat16(v[8 * q + 2]), __float2bfloat16(v[8 * q + 3]))),
                                int(pack2(__float2bfloat16(v[8 * q + 4]), __float2bfloat16(v[8 * q + 5]))),
                                int(pack2(__float2bfloat16(v[8 * q + 6]), __float2bfloat16(v[8 * q + 7]))));
  __syncthreads();
  int4* dst = reinterpret_cast<int4*>(row + size_t(x0) * 32);
#pragma unroll
  for (int j = 0; j < 4; ++j) {
    const int c = p + 128 * j;                      // 16-byte piece c: pixel c / 4, part c % 4
    if (x0 + c / 4 < W) dst[c] = tile[(c >> 2) * 5 + (c & 3)];
  }
}

// input layer 1 -> 32: Y[p][co] = relu(sum_tap X[p + off] W[co][tap] + b[co]), X fp32 single channel
__global__ void __launch_bounds__(128) k_conv_in(const float* __restrict__ x, const float* __restrict__ w,
                                                const float* __restrict__ bias, bf16* __restrict__ y, int H, int W) {
  __shared__ float sw[32 * 9 + 32];
  for (int i = threadIdx.x; i < 32 * 9 + 32; i += blockDim.x) sw[i] = i < 288 ? w[i] : bias[i - 288];
  __syncthreads();
  int b, yy, xx;
  const bool in = pix_of(W, b, yy, xx);            // (no early return: the store is block-wide)
  float xv[9];
#pragma unroll
  for (int tap = 0; tap < 9; ++tap) {
    const int u = yy + tap / 3 - 1, v = xx + tap % 3 - 1;
    xv[tap] = (in && u >= 0 && u < H && v >= 0 && v < W) ? x[(size_t(b) * H + u) * W + v] : 0.0f;
  }
  float o[32];
#pragma unroll
  for (int co = 0; co < 32; ++co) {
    float s = sw[288 + co];
#pragma unroll
    for (int tap = 0; tap < 9; ++tap) s = fmaf(xv[tap], sw[co * 9 + tap], s);
    o[co] = fmaxf(s, 0.0f);
  }
  store32_block(y + (size_t(b) * H + yy) * W * 32, int(blockIdx.x) * 128, W, o);
}

// output layer 32 -> 1: Z[p] = sum_{tap, ci} X[p + off][ci] W[tap][ci] + b (FP32 out), written as
// Z[p] = b + sum_tap u_tap[p + off(tap)] with u_tap[q] = X[q] . W[tap]: a block of 16 x 16 output
// pixels loads each pixel of its 18 x 18 halo once, forms its nine dot products in shared memory,
// and every output pixel adds the nine of its neighbours.
constexpr int OT = 16, OH = OT + 2;
__global__ void __launch_bounds__(256) k_conv_out(const bf16* __restrict__ x, const float* __restrict__ w,
                                                 const float* __restrict__ bias, float* __restrict__ z, int H, int W) {
  __shared__ float sw[288];
  __shared__ float u[9][OH * OH];
  for (int i = threadIdx.x; i < 288; i += blockDim.x) sw[i] = w[i];
  __syncthreads();
  const int x0 = blockIdx.x * OT, y0 = blockIdx.y * OT, b = blockIdx.z;
  for (int hp = threadIdx.x; hp < OH * OH; hp += blockDim.x) {
    const int yy = y0 + hp / OH - 1, xx = x0 + hp % OH - 1;
    float d[9];
#pragma unroll
    for (int t = 0; t < 9; ++t) d[t] = 0.0f;
    if (yy >= 0 && yy < H && xx >= 0 && xx < W) {
      const int4* src = reinterpret_cast<const int4*>(x + ((size_t(b) * H + yy) * W + xx) * 32);
#pragma unroll 1
      for (int q = 0; q < 4; ++q) {          // 8 channels at a time
        const int4 v = src[q];
        const uint32_t w4[4] = {uint32_t(v.x), uint32_t(v.y), uint32_t(v.z), uint32_t(v.w)};
#pragma unroll
        for (int k = 0; k < 8; ++k) {
          const uint16_t h = uint16_t(k & 1 ? w4[k >> 1] >> 16 : w4[k >> 1] & 0xffff);
          const float a = __bfloat162float(__ushort_as_bfloat16(h));
#pragma unroll
          for (int t = 0; t < 9; ++t) d[t] = fmaf(a, sw[t * 32 + 8 * q + k], d[t]);
        }
      }
    }
#pragma unroll
    for (int t = 0; t < 9; ++t) u[t][hp] = d[t];
  }
  __syncthreads();
  const int ty = threadIdx.x / OT, tx = threadIdx.x % OT;
  const int yy = y0 + ty, xx = x0 + tx;
  if (yy >= H || xx >= W) return;
  float s = bias[0];
#pragma unroll
  for (int t = 0; t < 9; ++t) s += u[t][(ty + t / 3) * OH + tx + t % 3];
  z[(size_t(b) * H + yy) * W + xx] = s;
}

// data gradient of the output layer, times the ReLU mask of its input:
// dX[q][ci] = (X[q][ci] > 0) sum_tap dZ[q - off(tap)] W[tap][ci]
__global__ void __launch_bounds__(128) k_conv_out_dgrad(const float* __restrict__ dz, const float* __restrict__ w,
                                                       const bf16* __restrict__ xin, bf16* __restrict__ dx, int H,
                                                       int W) {
  __shared__ float sw[288];
  for (int i = threadIdx.x; i < 288; i += blockDim.x) sw[i] = w[i];
  __syncthreads();
  int b, yy, xx;
  if (!pix_of(W, b, yy, xx)) return;
  float acc[32];
#pragma unroll
  for (int ci = 0; ci < 32; ++ci) acc[ci] = 0.0f;
#pragma unroll
  for (int tap = 0; tap < 9; ++tap) {
    const int u = yy - (tap / 3 - 1), v = xx - (tap % 3 - 1);
    if (u < 0 || u >= H || v < 0 || v >= W) continue;
    const float d = dz[(size_t(b) * H + u) * W + v];
#pragma unroll
    for (int ci = 0; ci < 32; ++ci) acc[ci] = fmaf(d, sw[tap * 32 + ci], acc[ci]);
  }
  const size_t q = ((size_t(b) * H + yy) * W + xx) * 32;
  float m[32];
  load32(xin + q, m);
#pragma unroll
  for (int ci = 0; ci < 32; ++ci) acc[ci] = m[ci] > 0.0f ? acc[ci] : 0.0f;
  store32(dx + q, acc);
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

// 2x2 average pooling (forward); grid over the half-resolution pixels
__global__ void __launch_bounds__(128) k_pool2(const bf16* __restrict__ x, bf16* __restrict__ y, int H, int W) {
  const int h = H / 2, w = W / 2;
  int b, yy, xx;
  if (!pix_of(w, b, yy, xx)) return;
  float s[32], a[32];
  const size_t base = (size_t(b) * H + 2 * yy) * W + 2 * xx;
  load32(x + base * 32, s);
  const size_t nb[3] = {base + 1, base + W, base + W + 1};
  for (int k = 0; k < 3; ++k) {
    load32(x + nb[k] * 32, a);
#pragma unroll
    for (int c = 0; c < 32; ++c) s[c] += a[c];
  }
#pragma unroll
  for (int c = 0; c < 32; ++c) s[c] *= 0.25f;
  store32(y + ((size_t(b) * h + yy) * w + xx) * 32, s);
}

// nearest 2x upsampling of x (B, H/2, W/2) added to skip (B, H, W): y = up(x) + skip
__global__ void __launch_bounds__(128) k_up2_add(const bf16* __restrict__ x, const bf16* __restrict__ skip,
                                                bf16* __restrict__ y, int H, int W) {
  int b, yy, xx;
  if (!pix_of(W, b, yy, xx)) return;
  float s[32], a[32];
  const size_t p = ((size_t(b) * H + yy) * W + xx) * 32;
  load32(skip + p, s);
  load32(x + ((size_t(b) * (H / 2) + yy / 2) * (W / 2) + xx / 2) * 32, a);
#pragma unroll
  for (int c = 0; c < 32; ++c) s[c] += a[c];
  store32(y + p, s);
}

// backward of the skip / pooling junction at full resolution: dZ2 = (dS5 + pool^T(dP2)) * (A2 > 0)
__global__ void __launch_bounds__(128) k_junction_bwd(const bf16* __restrict__ ds5, const bf16* __restrict__ dp2,
                                                     const bf16* __restrict__ a2, bf16* __restrict__ dz2, int H, int W) {
  int b, yy, xx;
  if (!pix_of(W, b, yy, xx)) return;
  float s[32], a[32], m[32];
  const size_t p = ((size_t(b) * H + yy) * W + xx) * 32;
  load32(ds5 + p, s);
  load32(dp2 + ((size_t(b) * (H / 2) + yy / 2) * (W / 2) + xx / 2) * 32, a);
  load32(a2 + p, m);
#pragma unroll
  for (int c = 0; c < 32; ++c) s[c] = m[c] > 0.0f ? s[c] + 0.25f * a[c] : 0.0f;
  store32(dz2 + p, s);
}

// dA4 = up^T(dS5) (sum over each 2x2 block), times the ReLU mask of A4; grid over half resolution
__global__ void __launch_bounds__(128) k_up2_bwd_mask(const bf16* __restrict__ ds5, const bf16* __restrict__ a4,
                                                     bf16* __restrict__ dz4, int H, int W) {
  const int h = H / 2, w = W / 2;
  int b, yy, xx;
  if (!pix_of(w, b, yy, xx)) return;
  float s[32], a[32];
  const size_t base = (size_t(b) * H + 2 * yy) * W + 2 * xx;
  load32(ds5 + base * 32, s);
  const size_t nb[3] = {base + 1, base + W, base + W + 1};
  for (int k = 0; k < 3; ++k) {
    load32(ds5 + nb[k] * 32, a);
#pragma unroll
    for (int c = 0; c < 32; ++c) s[c] += a[c];
  }
  const size_t q = ((size_t(b) * h + yy) * w + xx) * 32;
  load32(a4 + q, a);
#pragma unroll
  for (int c = 0; c < 32; ++c) s[c] = a[c] > 0.0f ? s[c] : 0.0f;
  store32(dz4 + q, s);
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
// the network predicts a correction to the log-transformed data (s per image); grid (chunks, B)
__global__ void k_prep(const float* __restrict__ g, const float* __restrict__ f, const float* __restrict__ bvec,
                       const float* __restrict__ svec, float* __restrict__ x, float* __restrict__ t, size_t P) {
  const size_t o = size_t(blockIdx.y) * P;
  const float s = svec[blockIdx.y], bb = bvec[blockIdx.y];
  for (size_t i = blockIdx.x * size_t(blockDim.x) + threadIdx.x; i < P; i += size_t(gridDim.x) * blockDim.x) {
    const float xi = (g[o + i] - bb) / s;
    x[o + i] = xi;
    if (f) t[o + i] = log1pf(fmaxf(f[o + i], 0.0f) / s) - log1pf(fmaxf(xi, 0.0f));
  }
}

// f0 = s expm1(clamp(z + log(1 + max(x, 0)), 0, 20)) (the inverse of the target transform, bounded)
__global__ void k_start(const float* __restrict__ z, const float* __restrict__ x, const float* __restrict__ svec,
                        float* __restrict__ f0, size_t P) {
  const size_t o = size_t(blockIdx.y) * P;
  const float s = svec[blockIdx.y];
  for (size_t i = blockIdx.x * size_t(blockDim.x) + threadIdx.x; i < P; i += size_t(gridDim.x) * blockDim.x)
    f0[o + i] = s * expm1f(fminf(fmaxf(z[o + i] + log1pf(fmaxf(x[o + i], 0.0f)), 0.0f), 20.0f));
}

// s[b] = 1 + mean over the image of max(g - b, 0) (input scale of the network): blocks (chunks, B)
// add FP64 block sums of FP32 per-thread sums into a per-image accumulator; k_scale_final divides.
constexpr int kScaleImages = 1024;            // images per ws_scale call
__device__ double g_scale_acc[kScaleImages];
__global__ void __launch_bounds__(256) k_scale(const float* __restrict__ g, const float* __restrict__ bvec, size_t P) {
  const float* gb = g + size_t(blockIdx.y) * P;
  const float bb = bvec[blockIdx.y];
  float acc = 0.0f;
  for (size_t i = blockIdx.x * size_t(blockDim.x) + threadIdx.x; i < P; i += size_t(gridDim.x) * blockDim.x)
    acc += fmaxf(gb[i] - bb, 0.0f);
  __shared__ double r[256];
  r[threadIdx.x] = acc;
  __syncthreads();
  for (int o = 128; o > 0; o >>= 1) {
    if (threadIdx.x < o) r[threadIdx.x] += r[threadIdx.x + o];
    __syncthreads();
  }
  if (threadIdx.x == 0) atomicAdd(&g_scale_acc[blockIdx.y], r[0]);
}
__global__ void k_scale_final(float* __restrict__ s, int B, size_t P) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= B) return;
  s[i] = float(1.0 + g_scale_acc[i] / double(P));
  g_scale_acc[i] = 0.0;
}

// device-side error flag of the warm-start kernels: 1 when a bounded wait for the tensor cores
// gave up (the results of that call are then undefined); read and cleared by ws_error
__device__ int g_ws_err;

int g_tc_ready[64] = {0};
int g_sm_count[64] = {0};

int grid1(size_t n) {
  const size_t g = (n + 255) / 256;
  return int(g < 148 * 32 ? g : 148 * 32);
}

}  // namespace

extern "C" {

int ws_conv32(const void* x, const void* w, const float* bias, const void* mask, void* y, int B, int H, int W, int mode,
              void* stream) {
  if (H % TCR || W % TCC || H <= 0 || W <= 0 || B <= 0 || mode < 0 || mode > 3) return 1;
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return 4;
  if (!g_tc_ready[dev]) {   // once per device: the kernels' shared-memory size and the SM count
    if (cudaFuncSetAttribute(k_conv32<0>, cudaFuncAttributeMaxDynamicSharedMemorySize, TC_SMEM) != cudaSuccess ||
        cudaFuncSetAttribute(k_conv32<1>, cudaFuncAttributeMaxDynamicSharedMemorySize, TC_SMEM) != cudaSuccess ||
        cudaFuncSetAttribute(k_conv32<2>, cudaFuncAttributeMaxDynamicSharedMemorySize, TC_SMEM) != cudaSuccess ||
        cudaFuncSetAttribute(k_conv32<3>, cudaFuncAttributeMaxDynamicSharedMemorySize, TC_SMEM) != cudaSuccess ||
        cudaDeviceGetAttribute(&g_sm_count[dev], cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
      return 4;
    g_tc_ready[dev] = 1;
  }
  const long long ntiles = (long long)(W / TCC) * (H / TCR) * B;
  if (ntiles > (1ll << 30)) return 1;
  const int grid = int(std::min<long long>(ntiles, (long long)g_sm_count[dev] * TC_BLOCKS_PER_SM));
  int* err = nullptr;
  if (cudaGetSymbolAddress(reinterpret_cast<void**>(&err), g_ws_err) != cudaSuccess) return 4;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  const bf16* xb = static_cast<const bf16*>(x);
  const bf16* wb = static_cast<const bf16*>(w);
  const bf16* mb = static_cast<const bf16*>(mask);
  bf16* yb = static_cast<bf16*>(y);
  switch (mode) {
    case 0: k_conv32<0><<<grid, 128, TC_SMEM, s>>>(xb, wb, bias, mb, yb, B, H, W, err); break;
    case 1: k_conv32<1><<<grid, 128, TC_SMEM, s>>>(xb, wb, bias, mb, yb, B, H, W, err); break;
    case 2: k_conv32<2><<<grid, 128, TC_SMEM, s>>>(xb, wb, bias, mb, yb, B, H, W, err); break;
    default: k_conv32<3><<<grid, 128, TC_SMEM, s>>>(xb, wb, bias, mb, yb, B, H, W, err); break;
  }
  return cudaPeekAtLastError() == cudaSuccess ? 0 : 4;
}

int ws_error(int* out) {
  int v = 0, zero = 0;
  if (cudaMemcpyFromSymbol(&v, g_ws_err, sizeof(int)) != cudaSuccess) return 4;
  if (cudaMemcpyToSymbol(g_ws_err, &zero, sizeof(int)) != cudaSuccess) return 4;
  if (out) *out = v;
  return 0;
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
  if (B <= 0 || H <= 0 || W <= 0) return 1;
  k_conv_in<<<pix_grid(B, H, W), 128, 0, static_cast<cudaStream_t>(stream)>>>(x, w, bias, static_cast<bf16*>(y), H, W);
  return cudaPeekAtLastError() == cudaSuccess ? 0 : 4;
}

int ws_conv_out(const void* x, const float* w, const float* bias, float* z, int B, int H, int W, void* stream) {
  if (B <= 0 || H <= 0 || W <= 0) return 1;
  if (B > 65535) return 1;
  k_conv_out<<<dim3((W + OT - 1) / OT, (H + OT - 1) / OT, B), 256, 0, static_cast<cudaStream_t>(stream)>>>(
      static_cast<const bf16*>(x), w, bias, z, H, W);
  return cudaPeekAtLastError() == cudaSuccess ? 0 : 4;
}

int ws_conv_out_dgrad(const float* dz, const float* w, const void* xin, void* dx, int B, int H, int W, void* stream) {
  if (B <= 0 || H <= 0 || W <= 0) return 1;
  k_conv_out_dgrad<<<pix_grid(B, H, W), 128, 0, static_cast<cudaStream_t>(stream)>>>(
      dz, w, static_cast<const bf16*>(xin), static_cast<bf16*>(dx), H, W);
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
  if (B <= 0 || H < 2 || W < 2 || H % 2 || W % 2) return 1;
  k_pool2<<<pix_grid(B, H / 2, W / 2), 128, 0, static_cast<cudaStream_t>(stream)>>>(
      static_cast<const bf16*>(x), static_cast<bf16*>(y), H, W);
  return cudaPeekAtLastError() == cudaSuccess ? 0 : 4;
}

int ws_up2_add(const void* x, const void* skip, void* y, int B, int H, int W, void* stream) {
  if (B <= 0 || H < 2 || W < 2 || H % 2 || W % 2) return 1;
  k_up2_add<<<pix_grid(B, H, W), 128, 0, static_cast<cudaStream_t>(stream)>>>(
      static_cast<const bf16*>(x), static_cast<const bf16*>(skip), static_cast<bf16*>(y), H, W);
  return cudaPeekAtLastError() == cudaSuccess ? 0 : 4;
}

int ws_junction_bwd(const void* ds5, const void* dp2, const void* a2, void* dz2, int B, int H, int W, void* stream) {
  if (B <= 0 || H < 2 || W < 2 || H % 2 || W % 2) return 1;
  k_junction_bwd<<<pix_grid(B, H, W), 128, 0, static_cast<cudaStream_t>(stream)>>>(
      static_cast<const bf16*>(ds5), static_cast<const bf16*>(dp2), static_cast<const bf16*>(a2), static_cast<bf16*>(dz2),
      H, W);
  return cudaPeekAtLastError() == cudaSuccess ? 0 : 4;
}

int ws_up2_bwd_mask(const void* ds5, const void* a4, void* dz4, int B, int H, int W, void* stream) {
  if (B <= 0 || H < 2 || W < 2 || H % 2 || W % 2) return 1;
  k_up2_bwd_mask<<<pix_grid(B, H / 2, W / 2), 128, 0, static_cast<cudaStream_t>(stream)>>>(
      static_cast<const bf16*>(ds5), static_cast<const bf16*>(a4), static_cast<bf16*>(dz4), H, W);
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
  if (B <= 0 || B > 65535 || P == 0) return 1;
  k_prep<<<dim3(unsigned((P + 255) / 256 < 1024 ? (P + 255) / 256 : 1024), B), 256, 0,
           static_cast<cudaStream_t>(stream)>>>(g, f, b, s, x, t, P);
  return cudaPeekAtLastError() == cudaSuccess ? 0 : 4;
}

int ws_start(const float* z, const float* x, const float* s, float* f0, int B, size_t P, void* stream) {
  if (B <= 0 || B > 65535 || P == 0) return 1;
  k_start<<<dim3(unsigned((P + 255) / 256 < 1024 ? (P + 255) / 256 : 1024), B), 256, 0,
            static_cast<cudaStream_t>(stream)>>>(z, x, s, f0, P);
  return cudaPeekAtLastError() == cudaSuccess ? 0 : 4;
}

int ws_scale(const float* g, const float* b, float* s, int B, size_t P, void* stream) {
  if (B <= 0 || B > kScaleImages || P == 0) return 1;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  const size_t per_image = (P + 255) / 256 < 1024 ? (P + 255) / 256 : 1024;
  const size_t chunks = std::max<size_t>(1, std::min<size_t>(per_image, (size_t(148) * 8 + B - 1) / B));
  k_scale<<<dim3(unsigned(chunks), B), 256, 0, st>>>(g, b, P);
  k_scale_final<<<(B + 127) / 128, 128, 0, st>>>(s, B, P);
  return cudaPeekAtLastError() == cudaSuccess ? 0 : 4;
}

int ws_zero(void* p, size_t bytes, void* stream) {
  return cudaMemsetAsync(p, 0, bytes, static_cast<cudaStream_t>(stream)) == cudaSuccess ? 0 : 4;
}

}  // extern "C"

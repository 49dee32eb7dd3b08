// Shared-memory Stockham FFT building blocks for real 2-D images on sm_103a.
//
// The convolutions A f = K * f and A^T y = K (x) y of the deconvolution methods (Sect. 2.2-2.4,
// Eq. projection / backprojection) are evaluated as
//      row R2C  ->  column FFT . (PSF spectrum) . column IFFT  ->  row C2R
// with every pass reading and writing HBM once.  This header provides the pieces:
//   * in-register DFTs of radix 2, 3, 4, 6, 8, 12, 16, 24, 32;
//   * one autosorting Stockham stage over data held in shared memory (radix R, sub-transform
//     length NS):  read x[j + m L/R], twiddle by w_{NS R}^{m (j mod NS)}, DFT_R, write to
//     (j - j mod NS) R + j mod NS + m NS.  The output is in natural order after the last stage,
//     so the spectrum multiply and the row post-processing need no reordering;
//   * per-length plans (radix sequences; E values per thread, T = L/E threads per transform);
//   * a twiddle table exp(-2 pi i q / L) for every supported length (filled once per device).
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

namespace sgp {

// ------------------------------------------------------------------------------ complex helpers
__device__ __forceinline__ float2 cadd(float2 a, float2 b) { return make_float2(a.x + b.x, a.y + b.y); }
__device__ __forceinline__ float2 csub(float2 a, float2 b) { return make_float2(a.x - b.x, a.y - b.y); }
__device__ __forceinline__ float2 cmul(float2 a, float2 b) {
  return make_float2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}
__device__ __forceinline__ float2 cmulc(float2 a, float2 b) {  // a * conj(b)
  return make_float2(a.x * b.x + a.y * b.y, a.y * b.x - a.x * b.y);
}
__device__ __forceinline__ float2 cconj(float2 a) { return make_float2(a.x, -a.y); }
__device__ __forceinline__ float2 cscale(float2 a, float s) { return make_float2(a.x * s, a.y * s); }
// multiply by -i (forward) or +i (inverse)
template <bool INV> __device__ __forceinline__ float2 mul_mi(float2 a) {
  return INV ? make_float2(-a.y, a.x) : make_float2(a.y, -a.x);
}

// ------------------------------------------------------------------------------ twiddles
// cos / sin (2 pi t / 48), t = 0..47: every in-register radix used here divides 48.
__constant__ float2 c_w48[48] = {
    {1.0f, 0.0f}, {9.91444861374e-1f, 1.3052619222e-1f}, {9.65925826289e-1f, 2.58819045103e-1f},
    {9.23879532511e-1f, 3.82683432365e-1f}, {8.66025403784e-1f, 5.0e-1f}, {7.93353340291e-1f, 6.08761429009e-1f},
    {7.07106781187e-1f, 7.07106781187e-1f}, {6.08761429009e-1f, 7.93353340291e-1f}, {5.0e-1f, 8.66025403784e-1f},
    {3.82683432365e-1f, 9.23879532511e-1f}, {2.58819045103e-1f, 9.65925826289e-1f}, {1.3052619222e-1f, 9.91444861374e-1f},
    {0.0f, 1.0f}, {-1.3052619222e-1f, 9.91444861374e-1f}, {-2.58819045103e-1f, 9.65925826289e-1f},
    {-3.82683432365e-1f, 9.23879532511e-1f}, {-5.0e-1f, 8.66025403784e-1f}, {-6.08761429009e-1f, 7.93353340291e-1f},
    {-7.07106781187e-1f, 7.07106781187e-1f}, {-7.93353340291e-1f, 6.08761429009e-1f}, {-8.66025403784e-1f, 5.0e-1f},
    {-9.23879532511e-1f, 3.82683432365e-1f}, {-9.65925826289e-1f, 2.58819045103e-1f}, {-9.91444861374e-1f, 1.3052619222e-1f},
    {-1.0f, 0.0f}, {-9.91444861374e-1f, -1.3052619222e-1f}, {-9.65925826289e-1f, -2.58819045103e-1f},
    {-9.23879532511e-1f, -3.82683432365e-1f}, {-8.66025403784e-1f, -5.0e-1f}, {-7.93353340291e-1f, -6.08761429009e-1f},
    {-7.07106781187e-1f, -7.07106781187e-1f}, {-6.08761429009e-1f, -7.93353340291e-1f}, {-5.0e-1f, -8.66025403784e-1f},
    {-3.82683432365e-1f, -9.23879532511e-1f}, {-2.58819045103e-1f, -9.65925826289e-1f}, {-1.3052619222e-1f, -9.91444861374e-1f},
    {0.0f, -1.0f}, {1.3052619222e-1f, -9.91444861374e-1f}, {2.58819045103e-1f, -9.65925826289e-1f},
    {3.82683432365e-1f, -9.23879532511e-1f}, {5.0e-1f, -8.66025403784e-1f}, {6.08761429009e-1f, -7.93353340291e-1f},
    {7.07106781187e-1f, -7.07106781187e-1f}, {7.93353340291e-1f, -6.08761429009e-1f}, {8.66025403784e-1f, -5.0e-1f},
    {9.23879532511e-1f, -3.82683432365e-1f}, {9.65925826289e-1f, -2.58819045103e-1f}, {9.91444861374e-1f, -1.3052619222e-1f},
};

// cos / sin (2 pi t / 64), t = 0..63: the radix-32 DFT and the 32 x 32 four-step transform.
__constant__ float2 c_w64[64] = {
    {1.0f, 0.0f}, {9.951847266722e-01f, 9.801714032956e-02f}, {9.807852804032e-01f, 1.950903220161e-01f}, {9.569403357322e-01f, 2.902846772545e-01f},
    {9.238795325113e-01f, 3.826834323651e-01f}, {8.819212643484e-01f, 4.713967368260e-01f}, {8.314696123025e-01f, 5.555702330196e-01f}, {7.730104533627e-01f, 6.343932841636e-01f},
    {7.071067811865e-01f, 7.071067811865e-01f}, {6.343932841636e-01f, 7.730104533627e-01f}, {5.555702330196e-01f, 8.314696123025e-01f}, {4.713967368260e-01f, 8.819212643484e-01f},
    {3.826834323651e-01f, 9.238795325113e-01f}, {2.902846772545e-01f, 9.569403357322e-01f}, {1.950903220161e-01f, 9.807852804032e-01f}, {9.801714032956e-02f, 9.951847266722e-01f},
    {0.0f, 1.0f}, {-9.801714032956e-02f, 9.951847266722e-01f}, {-1.950903220161e-01f, 9.807852804032e-01f}, {-2.902846772545e-01f, 9.569403357322e-01f},
    {-3.826834323651e-01f, 9.238795325113e-01f}, {-4.713967368260e-01f, 8.819212643484e-01f}, {-5.555702330196e-01f, 8.314696123025e-01f}, {-6.343932841636e-01f, 7.730104533627e-01f},
    {-7.071067811865e-01f, 7.071067811865e-01f}, {-7.730104533627e-01f, 6.343932841636e-01f}, {-8.314696123025e-01f, 5.555702330196e-01f}, {-8.819212643484e-01f, 4.713967368260e-01f},
    {-9.238795325113e-01f, 3.826834323651e-01f}, {-9.569403357322e-01f, 2.902846772545e-01f}, {-9.807852804032e-01f, 1.950903220161e-01f}, {-9.951847266722e-01f, 9.801714032956e-02f},
    {-1.0f, 0.0f}, {-9.951847266722e-01f, -9.801714032956e-02f}, {-9.807852804032e-01f, -1.950903220161e-01f}, {-9.569403357322e-01f, -2.902846772545e-01f},
    {-9.238795325113e-01f, -3.826834323651e-01f}, {-8.819212643484e-01f, -4.713967368260e-01f}, {-8.314696123025e-01f, -5.555702330196e-01f}, {-7.730104533627e-01f, -6.343932841636e-01f},
    {-7.071067811865e-01f, -7.071067811865e-01f}, {-6.343932841636e-01f, -7.730104533627e-01f}, {-5.555702330196e-01f, -8.314696123025e-01f}, {-4.713967368260e-01f, -8.819212643484e-01f},
    {-3.826834323651e-01f, -9.238795325113e-01f}, {-2.902846772545e-01f, -9.569403357322e-01f}, {-1.950903220161e-01f, -9.807852804032e-01f}, {-9.801714032956e-02f, -9.951847266722e-01f},
    {0.0f, -1.0f}, {9.801714032956e-02f, -9.951847266722e-01f}, {1.950903220161e-01f, -9.807852804032e-01f}, {2.902846772545e-01f, -9.569403357322e-01f},
    {3.826834323651e-01f, -9.238795325113e-01f}, {4.713967368260e-01f, -8.819212643484e-01f}, {5.555702330196e-01f, -8.314696123025e-01f}, {6.343932841636e-01f, -7.730104533627e-01f},
    {7.071067811865e-01f, -7.071067811865e-01f}, {7.730104533627e-01f, -6.343932841636e-01f}, {8.314696123025e-01f, -5.555702330196e-01f}, {8.819212643484e-01f, -4.713967368260e-01f},
    {9.238795325113e-01f, -3.826834323651e-01f}, {9.569403357322e-01f, -2.902846772545e-01f}, {9.807852804032e-01f, -1.950903220161e-01f}, {9.951847266722e-01f, -9.801714032956e-02f},
};

// v * w_R^e, w_R = exp(-/+ 2 pi i / R) (forward / inverse); e is a compile-time constant after unrolling
template <int R, bool INV>
__device__ __forceinline__ float2 twr(float2 v, int e) {
  if constexpr (48 % R == 0) {
    const int t = ((e % R) * (48 / R)) % 48;
    if (t == 0) return v;
    if (t == 24) return make_float2(-v.x, -v.y);
    if (t == 12) return mul_mi<INV>(v);
    if (t == 36) return mul_mi<!INV>(v);
    const float2 w = c_w48[t];
    return INV ? cmul(v, w) : cmulc(v, w);
  } else {
    static_assert(64 % R == 0, "in-register radix must divide 48 or 64");
    const int t = ((e % R) * (64 / R)) % 64;
    if (t == 0) return v;
    if (t == 32) return make_float2(-v.x, -v.y);
    if (t == 16) return mul_mi<INV>(v);
    if (t == 48) return mul_mi<!INV>(v);
    const float2 w = c_w64[t];
    return INV ? cmul(v, w) : cmulc(v, w);
  }
}

// supported transform lengths and the offsets of their tables exp(-2 pi i q / L), q < L, followed
// by the twiddles of the warp four-step transform (warp_fft1024) stored lane-fastest:
// entry kTw4Offset + 32 q + lane = exp(-2 pi i lane q / 1024), so that the 32 lanes of a warp read
// 256 contiguous bytes per q instead of 32 scattered entries
constexpr int kTw4Offset = 7148;
constexpr int kTwiddleTotal = kTw4Offset + 1024;
__host__ __device__ constexpr int tw_offset(int L) {
  return L == 8 ? 0 : L == 12 ? 8 : L == 16 ? 20 : L == 24 ? 36 : L == 32 ? 60 : L == 48 ? 92 :
         L == 64 ? 140 : L == 96 ? 204 : L == 128 ? 300 : L == 192 ? 428 : L == 256 ? 620 :
         L == 384 ? 876 : L == 512 ? 1260 : L == 768 ? 1772 : L == 1024 ? 2540 :
         L == 1536 ? 3564 : L == 2048 ? 5100 : -1;
}
// One copy per translation unit (internal linkage, no relocatable device code); every unit that
// launches FFT kernels defines an initialiser (SGP_DEFINE_TWIDDLE_INIT) that copies the table in.
namespace {
__device__ float2 g_twiddle[kTwiddleTotal];
}
#define SGP_DEFINE_TWIDDLE_INIT(NAME)                                                                 \
  cudaError_t NAME(const float2* host_table) {                                                       \
    return cudaMemcpyToSymbol(::sgp::g_twiddle, host_table, sizeof(float2) * ::sgp::kTwiddleTotal);  \
  }

template <bool INV>
__device__ __forceinline__ float2 tw4(int lane, int q) {  // exp(-/+ 2 pi i lane q / 1024), q < 32
  asm volatile("" : "+r"(lane));
  const float2 w = __ldg(&g_twiddle[kTw4Offset + 32 * q + lane]);
  return INV ? cconj(w) : w;
}
template <int L, bool INV>
__device__ __forceinline__ float2 twl(int q) {  // exp(-/+ 2 pi i q / L), 0 <= q < L
  // the empty asm keeps the load after the preceding barrier: read-only loads may otherwise be
  // hoisted across every stage of a transform, costing many live registers
  asm volatile("" : "+r"(q));
  const float2 w = __ldg(&g_twiddle[tw_offset(L) + q]);
  return INV ? cconj(w) : w;
}

// ------------------------------------------------------------------------------ register DFTs
// V[q] = sum_m v[m] w_R^{m q}
template <int R, bool INV> struct DFT;

template <bool INV> struct DFT<2, INV> {
  __device__ __forceinline__ static void run(float2* v) {
    const float2 a = v[0];
    v[0] = cadd(a, v[1]);
    v[1] = csub(a, v[1]);
  }
};
template <bool INV> struct DFT<4, INV> {
  __device__ __forceinline__ static void run(float2* v) {
    const float2 t0 = cadd(v[0], v[2]), t1 = csub(v[0], v[2]);
    const float2 t2 = cadd(v[1], v[3]), t3 = mul_mi<INV>(csub(v[1], v[3]));
    v[0] = cadd(t0, t2);
    v[2] = csub(t0, t2);
    v[1] = cadd(t1, t3);
    v[3] = csub(t1, t3);
  }
};
template <bool INV> struct DFT<3, INV> {
  __device__ __forceinline__ static void run(float2* v) {
    const float h = 0.866025403784438647f;  // sqrt(3)/2
    const float2 s = cadd(v[1], v[2]), d = csub(v[1], v[2]);
    const float2 m = make_float2(v[0].x - 0.5f * s.x, v[0].y - 0.5f * s.y);
    const float2 ihd = make_float2(-h * d.y, h * d.x);  // i h d
    v[0] = cadd(v[0], s);
    // forward: V1 = m - i h d, V2 = m + i h d; the inverse swaps the signs
    if (INV) { v[1] = cadd(m, ihd); v[2] = csub(m, ihd); }
    else     { v[1] = csub(m, ihd); v[2] = cadd(m, ihd); }
  }
};
// composite R = R1 * R2: input index m = R2 m1 + m2, output index q = q1 + R1 q2
template <int R1, int R2, bool INV> struct DFTComp {
  __device__ __forceinline__ static void run(float2* v) {
    constexpr int R = R1 * R2;
    float2 a[R2][R1];
#pragma unroll
    for (int m2 = 0; m2 < R2; ++m2) {
#pragma unroll
      for (int m1 = 0; m1 < R1; ++m1) a[m2][m1] = v[R2 * m1 + m2];
      DFT<R1, INV>::run(a[m2]);
#pragma unroll
      for (int q1 = 0; q1 < R1; ++q1) a[m2][q1] = twr<R, INV>(a[m2][q1], m2 * q1);
    }
#pragma unroll
    for (int q1 = 0; q1 < R1; ++q1) {
      float2 b[R2];
#pragma unroll
      for (int m2 = 0; m2 < R2; ++m2) b[m2] = a[m2][q1];
      DFT<R2, INV>::run(b);
#pragma unroll
      for (int q2 = 0; q2 < R2; ++q2) v[q1 + R1 * q2] = b[q2];
    }
  }
};
template <bool INV> struct DFT<6, INV> : DFTComp<2, 3, INV> {};
template <bool INV> struct DFT<8, INV> : DFTComp<2, 4, INV> {};
template <bool INV> struct DFT<12, INV> : DFTComp<4, 3, INV> {};
template <bool INV> struct DFT<16, INV> : DFTComp<4, 4, INV> {};
template <bool INV> struct DFT<24, INV> : DFTComp<8, 3, INV> {};
template <bool INV> struct DFT<32, INV> : DFTComp<4, 8, INV> {};

// ------------------------------------------------------------------------------ plans
template <int... Rs> struct RL {};
template <class A, class B> struct RevImpl;
template <int... Out> struct RevImpl<RL<>, RL<Out...>> { using type = RL<Out...>; };
template <int R, int... Rest, int... Out> struct RevImpl<RL<R, Rest...>, RL<Out...>> {
  using type = typename RevImpl<RL<Rest...>, RL<R, Out...>>::type;
};
template <class A> struct Rev { using type = typename RevImpl<A, RL<>>::type; };

// E: complex values held per thread in every stage (each radix divides E); T = L / E threads.
// The inverse runs the radices in reverse order.
template <int L> struct Plan;
#define SGP_PLAN(L_, E_, ...)                         \
  template <> struct Plan<L_> {                       \
    static constexpr int L = L_, E = E_, T = L_ / E_; \
    using Fwd = RL<__VA_ARGS__>;                      \
    using Inv = typename Rev<Fwd>::type;              \
  };
SGP_PLAN(8, 8, 8)
SGP_PLAN(12, 12, 12)
SGP_PLAN(16, 16, 16)
SGP_PLAN(24, 24, 8, 3)
SGP_PLAN(32, 16, 16, 2)
SGP_PLAN(48, 12, 4, 12)
SGP_PLAN(64, 16, 16, 4)
SGP_PLAN(96, 24, 8, 12)
SGP_PLAN(128, 16, 16, 8)
SGP_PLAN(192, 24, 8, 8, 3)
SGP_PLAN(256, 16, 16, 16)
SGP_PLAN(384, 24, 8, 8, 6)
SGP_PLAN(512, 16, 16, 16, 2)
SGP_PLAN(768, 24, 8, 8, 12)
SGP_PLAN(1024, 16, 16, 16, 4)
SGP_PLAN(1536, 24, 8, 8, 24)
SGP_PLAN(2048, 16, 16, 16, 8)
#undef SGP_PLAN

// Column transforms may use their own plan: fewer values per thread give more threads per column,
// fewer columns per block and so more blocks when the PSF band leaves few column tiles (rows of
// 2W reals keep Plan<W>, which measured faster with 16 values per thread).  Length 2048 has two
// column plans: ColPlan (16 values, 4 columns per block: faster over all columns) and
// ColPlanNarrow (8 values, 2 columns per block: faster when the band leaves half the columns or
// fewer); a context picks one at set-up.
template <int L> struct ColPlan : Plan<L> {};
template <> struct ColPlan<1024> {
  static constexpr int L = 1024, E = 8, T = 128;
  using Fwd = RL<8, 8, 8, 2>;
  using Inv = typename Rev<Fwd>::type;
};
template <int L> struct ColPlanNarrow : ColPlan<L> {};
template <> struct ColPlanNarrow<2048> {
  static constexpr int L = 2048, E = 8, T = 256;
  using Fwd = RL<8, 8, 8, 4>;
  using Inv = typename Rev<Fwd>::type;
};
constexpr int kNarrowSide = 2048;   // the one length with a narrow column variant

// ------------------------------------------------------------------------------ spectrum layout
// Packed spectra (and the PSF spectra) of H >= 1024 rows are stored interleaved by groups of 4
// rows: element (row r, column i) of an H x M plane at ((r / 4) M + i) 4 + r % 4.  A column pass
// (narrow tiles at these H) then reads and writes runs of 4 rows x its columns (64 - 128 contiguous
// bytes) instead of one 16 - 32-byte piece per row; a row is read with a stride of 4 elements.
// Fewer rows (small, L2-resident planes, where the strided row accesses cost more than the column
// runs save) keep the row-major layout: element (r, i) at r M + i.  The column passes know H at
// compile time, the row passes at run time.
__host__ __device__ constexpr bool spec_interleaved(int H) { return H >= 1024; }
__host__ __device__ __forceinline__ size_t spec_row_off(int row, int M, bool il) {   // start of row r
  return il ? size_t(row >> 2) * 4 * size_t(M) + (row & 3) : size_t(row) * M;
}

// ------------------------------------------------------------------------------ layouts
// Row layout: element i of a row at base[i + (i >> 4)] (one pad slot per 16 elements keeps the
// stride-R writes of the first stage free of bank conflicts).
template <int L> struct RowLayout {
  static constexpr int pitch = L + (L >> 4);
  float2* base;
  __device__ __forceinline__ float2& operator()(int i) const { return base[i + (i >> 4)]; }
};
// Column layout: element i of column c of a C-column tile at s[(i + (i >> 4)) * C + c]
// (base is already offset by c).
template <int C> struct ColLayout {
  float2* base;
  __device__ __forceinline__ float2& operator()(int i) const { return base[(i + (i >> 4)) * C]; }
};
template <int L> __host__ __device__ constexpr int col_rows_padded() { return L + (L >> 4); }

// ------------------------------------------------------------------------------ Stockham stage
// The twiddles w^(m e), m = 1..R-1, of one butterfly (w = exp(-/+ 2 pi i / L)).  Read from the table
// entry by entry, or (POW, radices 4 and 8) from the entries e, 2e and 4e and their products (at
// most two further roundings): the lanes of a warp hold few distinct e, and each distinct entry of
// a stage is a separate access (scattered table lines), so fewer entries per butterfly means less
// load traffic and latency per stage.
template <int L, int R, bool INV, bool POW>
__device__ __forceinline__ void stage_twiddles(int e, float2 (&w)[R]) {
  if constexpr (POW && (R == 4 || R == 8)) {
    w[1] = twl<L, INV>(e);
    w[2] = twl<L, INV>(2 * e);
    w[3] = cmul(w[2], w[1]);
    if constexpr (R == 8) {
      w[4] = twl<L, INV>(4 * e);
      w[5] = cmul(w[4], w[1]);
      w[6] = cmul(w[4], w[2]);
      w[7] = cmul(w[4], w[3]);
    }
  } else {
#pragma unroll
    for (int m = 1; m < R; ++m) w[m] = twl<L, INV>(m * e);
  }
}

// One radix-R stage of a length-L transform run by T threads (t in [0, T)).  Every thread of the
// block calls it (it synchronises); threads with act == false only synchronise.
template <int L, int R, int NS, int T, bool INV, class Lay, bool POW = false>
__device__ __forceinline__ void stockham_stage(const Lay& x0, int t, bool act) {
  // Opaque copies of the thread index and base pointer: without them the compiler hoists the
  // shared-memory addresses of every stage (and of every loop iteration around the transform)
  // to the top of the kernel and keeps them all live.
  asm volatile("" : "+r"(t));
  Lay x = x0;
  asm volatile("" : "+l"(x.base));
  constexpr int NB = L / R;
  constexpr int PER = NB / T;
  static_assert(PER * T == NB, "plan: each radix must divide the per-thread count");
  float2 v[PER][R];
  if (act) {
#pragma unroll
    for (int b = 0; b < PER; ++b) {
      const int j = t + b * T;
#pragma unroll
      for (int m = 0; m < R; ++m) v[b][m] = x(j + m * NB);
    }
  }
  __syncthreads();
  if (act) {
#pragma unroll
    for (int b = 0; b < PER; ++b) {
      const int j = t + b * T;
      const int k = j % NS;
      if (NS > 1) {
        float2 w[R];
        stage_twiddles<L, R, INV, POW>(k * (L / (NS * R)), w);
#pragma unroll
        for (int m = 1; m < R; ++m) v[b][m] = cmul(v[b][m], w[m]);
      }
      DFT<R, INV>::run(v[b]);
      const int base = (j - k) * R + k;
#pragma unroll
      for (int m = 0; m < R; ++m) x(base + m * NS) = v[b][m];
    }
  }
  __syncthreads();
}

template <int L, int T, bool INV, int NS, bool POW, class Lay>
__device__ __forceinline__ void run_stages(const Lay&, int, bool, RL<>) {}
template <int L, int T, bool INV, int NS, bool POW, class Lay, int R, int... Rest>
__device__ __forceinline__ void run_stages(const Lay& x, int t, bool act, RL<R, Rest...>) {
  stockham_stage<L, R, NS, T, INV, Lay, POW>(x, t, act);
  run_stages<L, T, INV, NS * R, POW>(x, t, act, RL<Rest...>{});
}

// In-place complex FFT of length L (unnormalised), natural order in and out, by the plan P;
// POW: twiddles from products of fewer table entries (stage_twiddles).
template <int L, bool INV, class Lay, class P = Plan<L>, bool POW = false>
__device__ __forceinline__ void fft_inplace(const Lay& x, int t, bool act) {
  if (INV) run_stages<L, P::T, true, 1, POW>(x, t, act, typename P::Inv{});
  else     run_stages<L, P::T, false, 1, POW>(x, t, act, typename P::Fwd{});
}

// ------------------------------------------------------------------------------ warp four-step
// A length-1024 transform held by one warp, 32 values per lane: index n = n1 + 32 n2 on input
// (lane n1 holds n2 = 0..31), k = k1 + 32 k2 on output (lane k1 holds k2 = 0..31), as
//   X[k1 + 32 k2] = sum_n1 w_1024^(n1 k1) w_32^(n1 k2) sum_n2 x[n1 + 32 n2] w_32^(n2 k1)
// (w = exp(-/+ 2 pi i / L)): a radix-32 DFT in registers, the twiddles w_1024^(n1 k1), one 32 x 32
// transpose through the warp's shared buffer T (32 rows of 33 values, so that both the row
// writes and the column reads are free of bank conflicts), and a second radix-32 DFT.  No block
// barrier: the warp's rows are independent of the other warps.  T must hold 1056 float2; the
// caller orders T's previous use before the call (the function starts with __syncwarp).
template <bool INV>
__device__ __forceinline__ void warp_fft1024(float2 (&v)[32], float2* T, int lane) {
  DFT<32, INV>::run(v);
  // twiddles w^(lane q), q = 1..31: entries q = 1..7 and 8, 16, 24 of the lane's table, the
  // others as w^(lane 8a) w^(lane b) (one further rounding; 10 table reads instead of 31)
  float2 wb[8], wa[4];
#pragma unroll
  for (int q = 1; q < 8; ++q) wb[q] = tw4<INV>(lane, q);
#pragma unroll
  for (int a = 1; a < 4; ++a) wa[a] = tw4<INV>(lane, 8 * a);
#pragma unroll
  for (int q = 1; q < 32; ++q) {
    const int a = q >> 3, b = q & 7;
    const float2 w = a == 0 ? wb[b] : (b == 0 ? wa[a] : cmul(wa[a], wb[b]));
    v[q] = cmul(v[q], w);
  }
  __syncwarp();
#pragma unroll
  for (int q = 0; q < 32; ++q) T[q * 33 + lane] = v[q];
  __syncwarp();
#pragma unroll
  for (int q = 0; q < 32; ++q) v[q] = T[lane * 33 + q];
  DFT<32, INV>::run(v);
}

}  // namespace sgp

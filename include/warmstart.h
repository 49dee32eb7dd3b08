/*
 * warmstart.h -- C ABI of the learned warm start: kernels of a small convolutional encoder-decoder
 * that maps a detected image g to a starting point f^(0) for SGP.  The paper has no counterpart:
 * its starting points are the ones of Sect. 3.1; SGP always refines the predicted f^(0) to the same
 * stopping rule (Sect. 3.3), so the network never replaces the method.
 *
 * Network (NHWC, batch B, 32 channels; bf16 activations and working weights, FP32 accumulation,
 * FP32 master weights and Adam state):
 *   x0 = (g - b)/s (1 channel, s per image)                 fp32
 *   a1 = relu(conv_in(x0))            1 -> 32               ws_conv_in
 *   a2 = relu(conv(a1))               32 -> 32              ws_conv32 mode 0
 *   p2 = avgpool2(a2)                                       ws_pool2
 *   a3 = relu(conv(p2)), a4 = relu(conv(a3))   half res     ws_conv32 mode 0
 *   s5 = up2(a4) + a2                                       ws_up2_add
 *   a5 = relu(conv(s5))                                     ws_conv32 mode 0
 *   z  = conv_out(a5)                 32 -> 1, linear       ws_conv_out
 *   f0 = s expm1(clamp(z + log(1 + max(x0, 0)), 0, 20))     ws_start
 * The network predicts a correction to the log-transformed data: training target
 * t = log(1 + max(f_SGP, 0)/s) - log(1 + max(x0, 0)), loss mean (z - t)^2 (ws_loss).
 *
 * Layouts: conv32 weights bf16 [co][tap][ci] (tap = 3 dy + dx), conv_in weights fp32 [co][tap],
 * conv_out weights fp32 [tap][ci]; activations bf16 [b][y][x][c]; every 3x3 convolution uses zero
 * ("same") padding.  ws_conv32 needs H % 16 == 0 and W % 8 == 0, ws_conv32_wgrad H % 8 == 0 and
 * W % 16 == 0, the pooling and upsampling calls even H and W.  All pointers are device pointers
 * owned by the caller; `stream` is a cudaStream_t.  Every call is asynchronous and returns 0, or 1 for
 * an invalid size, 4 for a CUDA launch error.  Gradient accumulators (dw, db, loss) are added to:
 * the caller zeroes them before a step.
 */
#ifndef SGP_WARMSTART_H
#define SGP_WARMSTART_H

#include <stddef.h>

#ifdef __cplusplus
extern "C" {
#endif

#if defined(__GNUC__)
#define WS_API __attribute__((visibility("default")))
#else
#define WS_API
#endif

/* 32 -> 32 3x3 convolution on the 5th-generation tensor cores (tcgen05.mma, bf16 operands staged in
 * shared memory, FP32 accumulators in tensor memory), persistent blocks over 16 x 8 pixel tiles.
 * mode 0: y = relu(conv + bias); 1: y = conv + bias; 2: y = conv * (mask > 0) (data gradient with the
 * ReLU mask of the layer below; pass the flipped weights of ws_flip_weights); 3: y = conv.
 * A wait for the tensor cores that exceeds its iteration limit sets the flag that ws_error reads. */
WS_API int ws_conv32(const void* x, const void* w, const float* bias, const void* mask, void* y, int B, int H, int W,
                     int mode, void* stream);
/* Reads and clears the device-side error flag of the warm-start kernels (1: a bounded wait for the
 * tensor cores gave up and the output of that call is undefined).  Synchronous. */
WS_API int ws_error(int* out);
/* dw[co][tap][ci] += sum_p dy[p][co] x[p + off(tap)][ci]  (x is the layer input) */
WS_API int ws_conv32_wgrad(const void* dy, const void* x, float* dw, int B, int H, int W, void* stream);
/* wt[ci][tap][co] = w[co][8 - tap][ci] */
WS_API int ws_flip_weights(const void* w, void* wt, void* stream);
/* input layer: y[p][co] = relu(sum_tap x[p + off] w[co][tap] + bias[co]), x fp32 (B, H, W) */
WS_API int ws_conv_in(const float* x, const float* w, const float* bias, void* y, int B, int H, int W, void* stream);
/* output layer: z[p] = sum_{tap, ci} x[p + off][ci] w[tap][ci] + bias[0] */
WS_API int ws_conv_out(const void* x, const float* w, const float* bias, float* z, int B, int H, int W, void* stream);
/* dx[q][ci] = (xin[q][ci] > 0) sum_tap dz[q - off(tap)] w[tap][ci] */
WS_API int ws_conv_out_dgrad(const float* dz, const float* w, const void* xin, void* dx, int B, int H, int W,
                             void* stream);
/* gradients of the small layers: mode 0 input layer (dy bf16 32 ch, x fp32), mode 1 output layer
 * (dy fp32 1 ch, x bf16 32 ch); dw and db are accumulated */
WS_API int ws_small_wgrad(const void* dy, const void* x, float* dw, float* db, int B, int H, int W, int mode,
                          void* stream);
/* db[c] += sum_p dy[p][c] (32 channels) */
WS_API int ws_bias_grad(const void* dy, float* db, int B, int H, int W, void* stream);
/* y (B, H/2, W/2, 32) = 2x2 average of x (B, H, W, 32) */
WS_API int ws_pool2(const void* x, void* y, int B, int H, int W, void* stream);
/* y (B, H, W, 32) = nearest-up(x (B, H/2, W/2, 32)) + skip */
WS_API int ws_up2_add(const void* x, const void* skip, void* y, int B, int H, int W, void* stream);
/* dz2 = (ds5 + pool^T(dp2)) * (a2 > 0) at full resolution */
WS_API int ws_junction_bwd(const void* ds5, const void* dp2, const void* a2, void* dz2, int B, int H, int W,
                           void* stream);
/* dz4 (half resolution) = up^T(ds5) * (a4 > 0) */
WS_API int ws_up2_bwd_mask(const void* ds5, const void* a4, void* dz4, int B, int H, int W, void* stream);
/* dz = 2 (z - t)/n, out[0] += sum (z - t)^2 */
WS_API int ws_loss(const float* z, const float* t, float* dz, double* out, size_t n, void* stream);
/* Adam step `step` (1-based) on n FP32 parameters */
WS_API int ws_adam(float* p, float* m, float* v, const float* g, int n, float lr, float b1, float b2, float eps,
                   int step, void* stream);
WS_API int ws_to_bf16(const float* x, void* y, int n, void* stream);
/* x = (g - b)/s and (if f != NULL) t = log(1 + max(f, 0)/s) - log(1 + max(x, 0)); b, s per image */
WS_API int ws_prep(const float* g, const float* f, const float* b, const float* s, float* x, float* t, int B,
                   size_t P, void* stream);
/* f0 = s expm1(clamp(z + log(1 + max(x, 0)), 0, 20)) */
WS_API int ws_start(const float* z, const float* x, const float* s, float* f0, int B, size_t P, void* stream);

/* s[b] = 1 + mean over the image of max(g - b, 0): the per-image input scale (B <= 1024; calls that
 * overlap on the GPU must not share the library's per-image accumulator, i.e. run them in order) */
WS_API int ws_scale(const float* g, const float* b, float* s, int B, size_t P, void* stream);
/* zero `bytes` bytes at p (gradient accumulators) */
WS_API int ws_zero(void* p, size_t bytes, void* stream);

#ifdef __cplusplus
}
#endif
#endif /* SGP_WARMSTART_H */

// Mosaic of boundary-corrected reconstructions (Sect. 4, second experiment; Table 2, Table 6):
// an H x W image is covered by ny x nx partially overlapping sub-domains; each is merged by zero
// padding into an EH x EW array (sub-image centred, mask M_S = 1 on it) and reconstructed with the
// boundary-effect correction of Sect. 2.4; the mosaic keeps a non-overlapping piece of each.
//
// Geometry along one axis of N pixels, n sub-domains of s pixels (the paper gives the example
// 256 -> 2 x 160 -> pieces of 128): sub-domain k = [w_k, w_k + s), w_k = floor(k (N - s)/(n - 1));
// piece k = [floor(k N / n), floor((k + 1) N / n)), which must lie inside sub-domain k.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

namespace sgp {

constexpr int kMosaicMax = 16;   // sub-domains per axis

struct MosaicGeom {
  int H, W, ny, nx, sy, sx, EH, EW, ey, ex;     // ey, ex: offset of the sub-image in the padded array
  int wy[kMosaicMax], wx[kMosaicMax];            // sub-domain starts
  int cy[kMosaicMax + 1], cx[kMosaicMax + 1];    // piece boundaries
};

// tiles[t][j] (t = ky * nx + kx, j < p views) = zero-padded sub-image of g[j]; masks[t] = M_S
__global__ void k_mosaic_split(const float* __restrict__ g, int p, MosaicGeom m, float* __restrict__ tiles,
                               uint8_t* __restrict__ masks) {
  const size_t E = size_t(m.EH) * m.EW, per_tile = E * p, total = per_tile * size_t(m.ny) * m.nx;
  for (size_t i = blockIdx.x * size_t(blockDim.x) + threadIdx.x; i < total; i += size_t(gridDim.x) * blockDim.x) {
    const int t = int(i / per_tile);
    const size_t r = i - size_t(t) * per_tile;
    const int j = int(r / E);
    const size_t e = r - size_t(j) * E;
    const int y = int(e / m.EW), x = int(e - size_t(y) * m.EW);
    const int yy = y - m.ey, xx = x - m.ex;
    const bool in = yy >= 0 && yy < m.sy && xx >= 0 && xx < m.sx;
    const int ky = t / m.nx, kx = t - ky * m.nx;
    tiles[i] = in ? g[(size_t(j) * m.H + (m.wy[ky] + yy)) * m.W + (m.wx[kx] + xx)] : 0.0f;
    if (j == 0) masks[size_t(t) * E + e] = in ? 1 : 0;
  }
}

// f[Y][X] = recs[t][Y - w_ky + ey][X - w_kx + ex] for the piece (ky, kx) that holds (Y, X)
__global__ void k_mosaic_stitch(const float* __restrict__ recs, MosaicGeom m, float* __restrict__ f) {
  const size_t total = size_t(m.H) * m.W, E = size_t(m.EH) * m.EW;
  for (size_t i = blockIdx.x * size_t(blockDim.x) + threadIdx.x; i < total; i += size_t(gridDim.x) * blockDim.x) {
    const int Y = int(i / m.W), X = int(i - size_t(Y) * m.W);
    int ky = 0, kx = 0;
    while (ky + 1 < m.ny && Y >= m.cy[ky + 1]) ++ky;
    while (kx + 1 < m.nx && X >= m.cx[kx + 1]) ++kx;
    const int t = ky * m.nx + kx;
    const int y = Y - m.wy[ky] + m.ey, x = X - m.wx[kx] + m.ex;
    f[i] = recs[size_t(t) * E + size_t(y) * m.EW + x];
  }
}

}  // namespace sgp

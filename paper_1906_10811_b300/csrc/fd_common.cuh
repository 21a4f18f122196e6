// fd_common.cuh -- padded field layout and stencil coefficients shared by all kernels.
//
// Every field of a context (u^n, u^{n-1}, and the acoustic coefficients A, C)
// lives in one padded layout:
//   3-D  [n0 + 2R][n1 + 2R][px]     axis 0 = z (slowest, streamed), axis 2 = x
//   2-D  [1]      [n1 + 2R][px]     (n0 = 1, no halo along axis 0)
// with a zero halo of R = space_order/2 cells around the interior (the zero
// values "outside the grid") and kHaloX floats before every interior row, so
// interior rows start on a 128-byte boundary; px is a multiple of 32 floats.
// The zero halo plays the part of the OPS dataset padding d_m/d_p (thesis
// §3.3.2, "Extracting relevant information about Functions").
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

namespace fdk {

constexpr int kMaxR = 8;     // space order up to 16
constexpr int kHaloX = 32;   // floats in front of each interior row (128 B)

enum Eq : int { kDiffusion = 0, kAcoustic = 1 };

struct Geom {
  int n0, n1, n2;    // interior nodes per axis (2-D: n0 = 1)
  int R;             // halo radius = space_order / 2
  int R0;            // halo along axis 0 (R in 3-D, 0 in 2-D)
  int px;            // row pitch in floats
  int py;            // rows per plane = n1 + 2R
  int64_t plane;     // px * py
  int64_t total;     // px * py * (n0 + 2 R0)
  int hold;          // diffusion: 1 = boundary nodes held (interior update), 0 = every node
};

__host__ __device__ inline int64_t gidx(const Geom &g, int z, int y, int x) {
  return ((int64_t)(z + g.R0) * g.py + (y + g.R)) * g.px + (x + kHaloX);
}

// Stencil weights, pre-divided by h_d² (and multiplied by ν dt for diffusion)
// on the host in double, rounded once to float: no divisions are left in the
// kernels (thesis §5.1.5: hoisting the divisions out of the generated kernel
// gave the GPU its 3-4x).
// The kernels evaluate L u = Σ_axes Σ_k w[axis][k] ((u_{+k} + u_{-k}) - 2u): the
// centre weight w_0 = -2 Σ_k w_k is implied, so the FP32 operator sums to zero
// exactly and leaves constants alone however the weights round.
struct Coef {
  float w[3][kMaxR + 1];  // w[axis][k] for k = 1..R; axis 0 unused in 2-D
  float2 wp[3][kMaxR + 1];  // the same weights as pairs (w, w) for packed FP32x2 arithmetic
  int iso2;               // 2-D with equal spacing: w[1] = w[2], one weight per offset
};

}  // namespace fdk

// lbf_mlp.cuh -- learned interface curvature: a 27-64-64-1 SiLU network on
// the canonically oriented 3x3x3 fill-level stencil, output y = 4 kappa
// (kappa as in Sec. 2.2 Eq. rhob).  BF16 weights and activations, FP32
// accumulation, on the fifth-generation tensor cores (lbf_tc.cuh):
// inference (the batched forward pass and the in-loop curvature) and
// training's forward and backward passes.
//
// Parameters, flat FP32 (6017): W1 (64x27 row-major), b1 (64), W2 (64x64),
// b2 (64), W3 (64), b3 (1).  Stencil index q = (dz+1)*9 + (dy+1)*3 + (dx+1).
// Canonical orientation: reflect the axes along which the Parker-Youngs
// normal (into the liquid) is negative, then order the axes by increasing
// normal component (ties keep the axis order).
#pragma once
#include <cuda_bf16.h>
#include <stdint.h>

namespace lbf {
namespace mlp {

constexpr int NP = 6017;
constexpr int OFF_W1 = 0, OFF_B1 = 1728, OFF_W2 = 1792, OFF_B2 = 5888, OFF_W3 = 5952, OFF_B3 = 6016;
constexpr float Y_SCALE = 4.f;

__device__ __forceinline__ uint32_t pack2(float lo, float hi) {
  const __nv_bfloat162 v = __floats2bfloat162_rn(lo, hi);
  return *reinterpret_cast<const uint32_t *>(&v);
}
// SiLU and its derivative with the fast exponential and quotient (their
// error, a few ulp, is far below the BF16 rounding the activations take)
__device__ __forceinline__ float silu(float z) { return __fdividef(z, 1.f + __expf(-z)); }
__device__ __forceinline__ float dsilu(float z) {
  const float s = __fdividef(1.f, 1.f + __expf(-z));
  return s * (1.f + z * (1.f - s));
}

// canonical source index of stencil position q for a normal (nx, ny, nz)
__device__ __forceinline__ void canonical_order(float nx, float ny, float nz, int (&order)[3], int (&sign)[3]) {
  const float an[3] = {fabsf(nx), fabsf(ny), fabsf(nz)};
  sign[0] = nx < 0.f ? -1 : 1;
  sign[1] = ny < 0.f ? -1 : 1;
  sign[2] = nz < 0.f ? -1 : 1;
  // stable sort of the axes by |n|
  int o0 = 0, o1 = 1, o2 = 2, tmp;
  if (an[o1] < an[o0]) { tmp = o0; o0 = o1; o1 = tmp; }
  if (an[o2] < an[o1]) {
    tmp = o1; o1 = o2; o2 = tmp;
    if (an[o1] < an[o0]) { tmp = o0; o0 = o1; o1 = tmp; }
  }
  order[0] = o0;
  order[1] = o1;
  order[2] = o2;
}
__device__ __forceinline__ int canonical_src(int q, const int (&order)[3], const int (&sign)[3]) {
  const int nw[3] = {q % 3 - 1, (q / 3) % 3 - 1, q / 9 - 1};
  int old[3];
  old[order[0]] = sign[order[0]] * nw[0];
  old[order[1]] = sign[order[1]] * nw[1];
  old[order[2]] = sign[order[2]] * nw[2];
  return (old[2] + 1) * 9 + (old[1] + 1) * 3 + (old[0] + 1);
}

// Parker-Youngs normal of a 27-value stencil (unnormalised, into liquid)
__device__ __forceinline__ void py_normal(const float *a, float &nx, float &ny, float &nz) {
  nx = ny = nz = 0.f;
#pragma unroll
  for (int q = 0; q < 27; ++q) {
    const int dx = q % 3 - 1, dy = (q / 3) % 3 - 1, dz = q / 9 - 1;
    const float wx = (dy == 0 ? 2.f : 1.f) * (dz == 0 ? 2.f : 1.f);
    const float wy = (dx == 0 ? 2.f : 1.f) * (dz == 0 ? 2.f : 1.f);
    const float wz = (dx == 0 ? 2.f : 1.f) * (dy == 0 ? 2.f : 1.f);
    nx += dx * wx * a[q];
    ny += dy * wy * a[q];
    nz += dz * wz * a[q];
  }
}

}  // namespace mlp
}  // namespace lbf

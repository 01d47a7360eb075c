// lbf_mlp.cuh -- learned interface curvature: a 27-64-64-1 SiLU network on
// the canonically oriented 3x3x3 fill-level stencil, output y = 4 kappa
// (kappa as in Sec. 2.2 Eq. rhob).  BF16 weights and activations, FP32
// accumulation.  Inference (the batched forward pass and the in-loop
// curvature) runs on the fifth-generation tensor cores (lbf_tc.cuh);
// training's forward and backward passes use the warp-level MMA below
// (mma.sync.m16n8k16, one warp computes 16 stencils at a time).
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
// shared-memory copy of the network: B operands with padded rows
constexpr int W1_LD = 40;  // 32 inputs (27 used) + pad, bf16
constexpr int W2_LD = 72;  // 64 + pad, bf16

// the network as the training kernels read it from shared memory
struct __align__(16) NetF {
  __nv_bfloat16 w1[64 * W1_LD];  // w1[n][k] = W1[n][k]
  __nv_bfloat16 w2[64 * W2_LD];  // w2[n][k] = W2[n][k]
  float b1[64], b2[64], w3[64], b3, pad[3];
};
// training adds the transpose of W2 for the backward pass
struct Smem {
  NetF f;
  __nv_bfloat16 w2t[64 * W2_LD];  // w2t[k][n] = W2[n][k]
};

__device__ __forceinline__ void load_netf(NetF &s, const float *theta) {
  for (int i = threadIdx.x; i < 64 * W1_LD; i += blockDim.x) {
    const int n = i / W1_LD, k = i % W1_LD;
    s.w1[i] = __float2bfloat16_rn(k < 27 ? theta[OFF_W1 + n * 27 + k] : 0.f);
  }
  for (int i = threadIdx.x; i < 64 * W2_LD; i += blockDim.x) {
    const int r = i / W2_LD, k = i % W2_LD;
    s.w2[i] = __float2bfloat16_rn(k < 64 ? theta[OFF_W2 + r * 64 + k] : 0.f);
  }
  for (int i = threadIdx.x; i < 64; i += blockDim.x) {
    s.b1[i] = theta[OFF_B1 + i];
    s.b2[i] = theta[OFF_B2 + i];
    s.w3[i] = theta[OFF_W3 + i];
  }
  if (threadIdx.x == 0) {
    s.b3 = theta[OFF_B3];
    s.pad[0] = s.pad[1] = s.pad[2] = 0.f;
  }
}

__device__ __forceinline__ void load_net(Smem &s, const float *theta) {
  load_netf(s.f, theta);
  for (int i = threadIdx.x; i < 64 * W2_LD; i += blockDim.x) {
    const int r = i / W2_LD, k = i % W2_LD;
    s.w2t[i] = __float2bfloat16_rn(k < 64 ? theta[OFF_W2 + k * 64 + r] : 0.f);
  }
}

__device__ __forceinline__ uint32_t pack2(float lo, float hi) {
  const __nv_bfloat162 v = __floats2bfloat162_rn(lo, hi);
  return *reinterpret_cast<const uint32_t *>(&v);
}
__device__ __forceinline__ uint32_t ld2(const __nv_bfloat16 *p) { return *reinterpret_cast<const uint32_t *>(p); }

// D = A (16x16, row) * B (16x8, col) + C, bf16 in, fp32 accumulate
__device__ __forceinline__ void mma16816(float (&d)[4], const uint32_t (&a)[4], uint32_t b0, uint32_t b1) {
  asm volatile(
      "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
      "{%0,%1,%2,%3};\n"
      : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
      : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b0), "r"(b1));
}

// SiLU and its derivative with the fast exponential and quotient (their
// error, a few ulp, is far below the BF16 rounding the activations take)
__device__ __forceinline__ float silu(float z) { return __fdividef(z, 1.f + __expf(-z)); }
__device__ __forceinline__ float dsilu(float z) {
  const float s = __fdividef(1.f, 1.f + __expf(-z));
  return s * (1.f + z * (1.f - s));
}

// Forward pass of 16 stencils held by one warp.  xs: the warp's 16x32
// input tile in shared memory (bf16, row = stencil, 27 used).  On return
// z1/z2 hold the pre-activations in accumulator layout (n-tile j: rows g
// and g+8, columns 8j + 2t, 8j + 2t + 1) and y the outputs of rows g, g+8
// (valid in the lanes with t == 0).
struct Fwd {
  float z1[8][4], z2[8][4];
  float y0, y1;
};

__device__ __forceinline__ void forward16(const NetF &s, const __nv_bfloat16 *xs, Fwd &F) {
  const int lane = threadIdx.x & 31, g = lane >> 2, t = lane & 3;
  // layer 1: 16x32 * 32x64
  uint32_t a[2][4];
#pragma unroll
  for (int kk = 0; kk < 2; ++kk) {
    a[kk][0] = ld2(xs + g * 32 + kk * 16 + 2 * t);
    a[kk][1] = ld2(xs + (g + 8) * 32 + kk * 16 + 2 * t);
    a[kk][2] = ld2(xs + g * 32 + kk * 16 + 8 + 2 * t);
    a[kk][3] = ld2(xs + (g + 8) * 32 + kk * 16 + 8 + 2 * t);
  }
#pragma unroll
  for (int j = 0; j < 8; ++j) {
    const float bl = s.b1[8 * j + 2 * t], bh = s.b1[8 * j + 2 * t + 1];
    F.z1[j][0] = bl;
    F.z1[j][1] = bh;
    F.z1[j][2] = bl;
    F.z1[j][3] = bh;
#pragma unroll
    for (int kk = 0; kk < 2; ++kk) {
      const __nv_bfloat16 *w = s.w1 + (8 * j + g) * W1_LD + kk * 16 + 2 * t;
      mma16816(F.z1[j], a[kk], ld2(w), ld2(w + 8));
    }
  }
  // layer 2: SiLU(z1) as the A operand (accumulator layout -> A layout)
  uint32_t h[4][4];
#pragma unroll
  for (int kc = 0; kc < 4; ++kc) {
    h[kc][0] = pack2(silu(F.z1[2 * kc][0]), silu(F.z1[2 * kc][1]));
    h[kc][1] = pack2(silu(F.z1[2 * kc][2]), silu(F.z1[2 * kc][3]));
    h[kc][2] = pack2(silu(F.z1[2 * kc + 1][0]), silu(F.z1[2 * kc + 1][1]));
    h[kc][3] = pack2(silu(F.z1[2 * kc + 1][2]), silu(F.z1[2 * kc + 1][3]));
  }
#pragma unroll
  for (int j = 0; j < 8; ++j) {
    const float bl = s.b2[8 * j + 2 * t], bh = s.b2[8 * j + 2 * t + 1];
    F.z2[j][0] = bl;
    F.z2[j][1] = bh;
    F.z2[j][2] = bl;
    F.z2[j][3] = bh;
#pragma unroll
    for (int kc = 0; kc < 4; ++kc) {
      const __nv_bfloat16 *w = s.w2 + (8 * j + g) * W2_LD + kc * 16 + 2 * t;
      mma16816(F.z2[j], h[kc], ld2(w), ld2(w + 8));
    }
  }
  // layer 3: dot with W3 (bf16-rounded activations, like the tensor path)
  float p0 = 0.f, p1 = 0.f;
#pragma unroll
  for (int j = 0; j < 8; ++j) {
    const float wl = s.w3[8 * j + 2 * t], wh = s.w3[8 * j + 2 * t + 1];
    p0 += __bfloat162float(__float2bfloat16_rn(silu(F.z2[j][0]))) * wl +
          __bfloat162float(__float2bfloat16_rn(silu(F.z2[j][1]))) * wh;
    p1 += __bfloat162float(__float2bfloat16_rn(silu(F.z2[j][2]))) * wl +
          __bfloat162float(__float2bfloat16_rn(silu(F.z2[j][3]))) * wh;
  }
  p0 += __shfl_xor_sync(0xffffffffu, p0, 1);
  p0 += __shfl_xor_sync(0xffffffffu, p0, 2);
  p1 += __shfl_xor_sync(0xffffffffu, p1, 1);
  p1 += __shfl_xor_sync(0xffffffffu, p1, 2);
  F.y0 = p0 + s.b3;
  F.y1 = p1 + s.b3;
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

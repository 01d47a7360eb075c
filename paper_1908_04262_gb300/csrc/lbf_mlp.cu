// lbf_mlp.cu -- learned curvature: synthetic training data (voxelised
// spheres and ellipsoids with analytic mean curvature), tensor-core forward
// and backward passes, Adam, and the host entry points of include/lbf.h.
#include <cuda_runtime.h>

#include <cmath>
#include <cstring>
#include <vector>

#include "../../include/lbf.h"
#include "lbf_mlp.cuh"
#include "lbf_tc.cuh"
#include "lbf_ops_api.h"

using namespace lbf;
using namespace lbf::mlp;

namespace {

int fail(int code, const char *msg) {
  set_last_error(msg);
  return code;
}
#define CKM(call)                                                     \
  do {                                                                \
    cudaError_t e_ = (call);                                          \
    if (e_ != cudaSuccess) return fail(LBF_ECUDA, cudaGetErrorString(e_)); \
  } while (0)

constexpr int WARPS = 4;  // warps per block of the network kernels

// inference: canonical stencils (n x 27 fp32) -> y = 4 kappa, on the
// fifth-generation tensor cores: tiles of 128 rows, each CTA (128 threads)
// walking tiles; a tile whose MMA did not complete within the wait bound
// (and every later tile of that CTA) gets NaN outputs
__global__ void __launch_bounds__(128) k_forward_tc(const float *theta, const float *x, int n, float *y) {
  extern __shared__ __align__(128) unsigned char tsm[];
  tc::Tile &t = *reinterpret_cast<tc::Tile *>(tsm);
  tc::pack_image(t.net, theta);
  tc::setup(t, nullptr);
  uint32_t phase = 0;
  bool failed = false;
  const int tiles = (n + tc::ROWS - 1) / tc::ROWS;
  for (int tile = blockIdx.x; tile < tiles; tile += gridDim.x) {
    const long long row0 = (long long)tile * tc::ROWS;
    const int rows = (int)min((long long)tc::ROWS, (long long)n - row0);
    const float *xt = x + row0 * 27;
    for (int e = threadIdx.x; e < tc::ROWS * 27; e += blockDim.x) {
      const int r = e / 27, k = e - 27 * r;
      tc::put_x(t, r, k, r < rows ? xt[e] : 0.f);
    }
    float yv = __int_as_float(0x7fc00000);
    if (!failed) failed = !tc::forward_tile<128>(t, phase, yv);
    if ((int)threadIdx.x < rows) y[row0 + threadIdx.x] = yv;
  }
  tc::teardown(t, phase, failed);
}

// per-warp staging of the backward pass
struct Stage {
  __nv_bfloat16 x[16 * 32];
  __nv_bfloat16 h1[16 * 64];
  __nv_bfloat16 d2[16 * 64];
  __nv_bfloat16 d1[16 * 64];
};

// gradient of L = (1/2n) sum (y - t)^2, accumulated into grad (fp32, global)
// and L into *loss; each block sums its tiles in shared memory first
// which rows of the data set a batch takes, and the augmentation: row r of
// the batch is data row (a (start + r) + b) mod ntot (a coprime to ntot: a
// cheap per-epoch shuffle); fill levels strictly inside (0, 1) get uniform
// noise of half-width `noise`, keyed by `key`
struct Batch {
  long long start, ntot;
  unsigned long long a, b, key;
  float noise;
};

__device__ __forceinline__ unsigned long long splitmix(unsigned long long x);

__global__ void __launch_bounds__(32 * WARPS) k_grad(const float *theta, const float *x, const float *tgt, int n,
                                                     Batch bt, float *grad, double *loss) {
  extern __shared__ __align__(16) unsigned char smraw[];
  Smem &s = *reinterpret_cast<Smem *>(smraw);
  float *gacc = reinterpret_cast<float *>(smraw + sizeof(Smem));
  Stage *st = reinterpret_cast<Stage *>(smraw + sizeof(Smem) + ((NP * 4 + 15) / 16) * 16);
  load_net(s, theta);
  for (int i = threadIdx.x; i < NP; i += blockDim.x) gacc[i] = 0.f;
  __syncthreads();
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5, g = lane >> 2, t = lane & 3;
  Stage &S = st[w];
  const float inv_n = 1.f / (float)n;
  const int tiles = (n + 15) / 16;
  double lsum = 0.0;
  for (int tile = blockIdx.x * WARPS + w; tile < tiles; tile += gridDim.x * WARPS) {
    for (int e = lane; e < 16 * 32; e += 32) {
      const int r = e / 32, k = e % 32, row = tile * 16 + r;
      float v = 0.f;
      if (k < 27 && row < n) {
        const long long src = (long long)((bt.a * (unsigned long long)(bt.start + row) + bt.b) %
                                          (unsigned long long)bt.ntot);
        v = x[(size_t)src * 27 + k];
        if (bt.noise > 0.f && v > 0.f && v < 1.f) {
          const unsigned long long h = splitmix(bt.key ^ splitmix((unsigned long long)src * 32ull + k));
          const float u = (float)(h >> 40) * (1.f / 16777216.f);
          v = fminf(fmaxf(v + bt.noise * (2.f * u - 1.f), 0.f), 1.f);
        }
      }
      S.x[e] = __float2bfloat16_rn(v);
    }
    __syncwarp();
    Fwd F;
    forward16(s.f, S.x, F);
    const int r0 = tile * 16 + g, r1 = r0 + 8;
    auto tg = [&](int row) {
      return tgt[(bt.a * (unsigned long long)(bt.start + row) + bt.b) % (unsigned long long)bt.ntot];
    };
    const float e0 = r0 < n ? F.y0 - tg(r0) : 0.f, e1 = r1 < n ? F.y1 - tg(r1) : 0.f;
    if (t == 0) lsum += 0.5 * ((double)e0 * e0 + (double)e1 * e1) * (double)inv_n;
    const float d30 = e0 * inv_n, d31 = e1 * inv_n;
    // output layer
    float gb3 = d30 + d31;
    // delta2 = d3 * W3 * SiLU'(z2); grads of W3 and b2 summed over the rows
#pragma unroll
    for (int j = 0; j < 8; ++j) {
#pragma unroll
      for (int c = 0; c < 2; ++c) {
        const int col = 8 * j + 2 * t + c;
        const float h20 = __bfloat162float(__float2bfloat16_rn(silu(F.z2[j][c])));
        const float h21 = __bfloat162float(__float2bfloat16_rn(silu(F.z2[j][2 + c])));
        float gw3 = d30 * h20 + d31 * h21;
        const float dd0 = d30 * s.f.w3[col] * dsilu(F.z2[j][c]);
        const float dd1 = d31 * s.f.w3[col] * dsilu(F.z2[j][2 + c]);
        float gb2 = dd0 + dd1;
        S.d2[g * 64 + col] = __float2bfloat16_rn(dd0);
        S.d2[(g + 8) * 64 + col] = __float2bfloat16_rn(dd1);
        S.h1[g * 64 + col] = __float2bfloat16_rn(silu(F.z1[j][c]));
        S.h1[(g + 8) * 64 + col] = __float2bfloat16_rn(silu(F.z1[j][2 + c]));
        // sum over the 8 row groups
        gw3 += __shfl_xor_sync(0xffffffffu, gw3, 4);
        gw3 += __shfl_xor_sync(0xffffffffu, gw3, 8);
        gw3 += __shfl_xor_sync(0xffffffffu, gw3, 16);
        gb2 += __shfl_xor_sync(0xffffffffu, gb2, 4);
        gb2 += __shfl_xor_sync(0xffffffffu, gb2, 8);
        gb2 += __shfl_xor_sync(0xffffffffu, gb2, 16);
        if (g == 0) {
          atomicAdd(gacc + OFF_W3 + col, gw3);
          atomicAdd(gacc + OFF_B2 + col, gb2);
        }
      }
    }
    gb3 += __shfl_xor_sync(0xffffffffu, gb3, 4);
    gb3 += __shfl_xor_sync(0xffffffffu, gb3, 8);
    gb3 += __shfl_xor_sync(0xffffffffu, gb3, 16);
    if (lane == 0) atomicAdd(gacc + OFF_B3, gb3);
    __syncwarp();
    // delta1 = (delta2 W2) * SiLU'(z1): A = delta2 (16 x 64), B[n][k] = W2[n][k]
    {
      uint32_t a[4][4];
#pragma unroll
      for (int kc = 0; kc < 4; ++kc) {
        a[kc][0] = ld2(S.d2 + g * 64 + kc * 16 + 2 * t);
        a[kc][1] = ld2(S.d2 + (g + 8) * 64 + kc * 16 + 2 * t);
        a[kc][2] = ld2(S.d2 + g * 64 + kc * 16 + 8 + 2 * t);
        a[kc][3] = ld2(S.d2 + (g + 8) * 64 + kc * 16 + 8 + 2 * t);
      }
#pragma unroll
      for (int j = 0; j < 8; ++j) {
        float acc[4] = {0.f, 0.f, 0.f, 0.f};
#pragma unroll
        for (int kc = 0; kc < 4; ++kc) {
          const __nv_bfloat16 *wv = s.w2t + (8 * j + g) * W2_LD + kc * 16 + 2 * t;
          mma16816(acc, a[kc], ld2(wv), ld2(wv + 8));
        }
#pragma unroll
        for (int c = 0; c < 2; ++c) {
          const int col = 8 * j + 2 * t + c;
          const float dd0 = acc[c] * dsilu(F.z1[j][c]);
          const float dd1 = acc[2 + c] * dsilu(F.z1[j][2 + c]);
          S.d1[g * 64 + col] = __float2bfloat16_rn(dd0);
          S.d1[(g + 8) * 64 + col] = __float2bfloat16_rn(dd1);
          float gb1 = dd0 + dd1;
          gb1 += __shfl_xor_sync(0xffffffffu, gb1, 4);
          gb1 += __shfl_xor_sync(0xffffffffu, gb1, 8);
          gb1 += __shfl_xor_sync(0xffffffffu, gb1, 16);
          if (g == 0) atomicAdd(gacc + OFF_B1 + col, gb1);
        }
      }
    }
    __syncwarp();
    // weight gradients: dW2[n][k] = sum_rows d2[row][n] h1[row][k] and
    // dW1[n][k] = sum_rows d1[row][n] x[row][k]; M = units, K = the 16 rows
#pragma unroll 1
    for (int mt = 0; mt < 4; ++mt) {
      uint32_t a2[4], a1[4];
      const int m0 = mt * 16 + g, m1 = m0 + 8;
      const int k0 = 2 * t, k1 = 2 * t + 8;
      auto pk = [](const __nv_bfloat16 *base, int ra, int rb, int col) {
        __nv_bfloat162 v;
        v.x = base[ra * 64 + col];
        v.y = base[rb * 64 + col];
        return *reinterpret_cast<uint32_t *>(&v);
      };
      a2[0] = pk(S.d2, k0, k0 + 1, m0);
      a2[1] = pk(S.d2, k0, k0 + 1, m1);
      a2[2] = pk(S.d2, k1, k1 + 1, m0);
      a2[3] = pk(S.d2, k1, k1 + 1, m1);
      a1[0] = pk(S.d1, k0, k0 + 1, m0);
      a1[1] = pk(S.d1, k0, k0 + 1, m1);
      a1[2] = pk(S.d1, k1, k1 + 1, m0);
      a1[3] = pk(S.d1, k1, k1 + 1, m1);
#pragma unroll
      for (int j = 0; j < 8; ++j) {
        float acc[4] = {0.f, 0.f, 0.f, 0.f};
        __nv_bfloat162 b0, b1;
        b0.x = S.h1[(2 * t) * 64 + 8 * j + g];
        b0.y = S.h1[(2 * t + 1) * 64 + 8 * j + g];
        b1.x = S.h1[(2 * t + 8) * 64 + 8 * j + g];
        b1.y = S.h1[(2 * t + 9) * 64 + 8 * j + g];
        mma16816(acc, a2, *reinterpret_cast<uint32_t *>(&b0), *reinterpret_cast<uint32_t *>(&b1));
        const int c0 = 8 * j + 2 * t;
        atomicAdd(gacc + OFF_W2 + m0 * 64 + c0, acc[0]);
        atomicAdd(gacc + OFF_W2 + m0 * 64 + c0 + 1, acc[1]);
        atomicAdd(gacc + OFF_W2 + m1 * 64 + c0, acc[2]);
        atomicAdd(gacc + OFF_W2 + m1 * 64 + c0 + 1, acc[3]);
      }
#pragma unroll
      for (int j = 0; j < 4; ++j) {
        float acc[4] = {0.f, 0.f, 0.f, 0.f};
        __nv_bfloat162 b0, b1;
        b0.x = S.x[(2 * t) * 32 + 8 * j + g];
        b0.y = S.x[(2 * t + 1) * 32 + 8 * j + g];
        b1.x = S.x[(2 * t + 8) * 32 + 8 * j + g];
        b1.y = S.x[(2 * t + 9) * 32 + 8 * j + g];
        mma16816(acc, a1, *reinterpret_cast<uint32_t *>(&b0), *reinterpret_cast<uint32_t *>(&b1));
        const int c0 = 8 * j + 2 * t;
        if (c0 < 27) {
          atomicAdd(gacc + OFF_W1 + m0 * 27 + c0, acc[0]);
          atomicAdd(gacc + OFF_W1 + m1 * 27 + c0, acc[2]);
        }
        if (c0 + 1 < 27) {
          atomicAdd(gacc + OFF_W1 + m0 * 27 + c0 + 1, acc[1]);
          atomicAdd(gacc + OFF_W1 + m1 * 27 + c0 + 1, acc[3]);
        }
      }
    }
    __syncwarp();
  }
  __syncthreads();
  for (int i = threadIdx.x; i < NP; i += blockDim.x)
    if (gacc[i] != 0.f) atomicAdd(grad + i, gacc[i]);
  lsum += __shfl_xor_sync(0xffffffffu, lsum, 4);
  lsum += __shfl_xor_sync(0xffffffffu, lsum, 8);
  lsum += __shfl_xor_sync(0xffffffffu, lsum, 16);
  if (lane == 0 && lsum != 0.0) atomicAdd(loss, lsum);
}

// Adam on the fp32 master parameters
__global__ void k_adam(float *theta, float *m, float *v, const float *grad, int step, float lr) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= NP) return;
  const float b1 = 0.9f, b2 = 0.999f, eps = 1e-8f;
  const float gi = grad[i];
  const float mi = b1 * m[i] + (1.f - b1) * gi;
  const float vi = b2 * v[i] + (1.f - b2) * gi * gi;
  m[i] = mi;
  v[i] = vi;
  const float mh = mi / (1.f - powf(b1, (float)step)), vh = vi / (1.f - powf(b2, (float)step));
  theta[i] -= lr * mh / (sqrtf(vh) + eps);
}

// ---------------------------------------------------------------------------
// synthetic stencils.  A sample is an ellipsoid {x : (x-c)^T A (x-c) < 1},
// A = R diag(1/a^2) R^T, gas or liquid inside, and the integer cell that
// contains a random point of its surface.  Parameters (20 doubles):
// c[3], a[3], R[9] row-major, gas_inside, cell[3], pad.

// SplitMix64 (Steele, Lea and Flood 2014) as a counter-based generator
__device__ __forceinline__ unsigned long long splitmix(unsigned long long x) {
  x += 0x9E3779B97F4A7C15ull;
  x = (x ^ (x >> 30)) * 0xBF58476D1CE4E5B9ull;
  x = (x ^ (x >> 27)) * 0x94D049BB133111EBull;
  return x ^ (x >> 31);
}
__device__ __forceinline__ double urand(unsigned long long seed, long long i, int k) {
  const unsigned long long h = splitmix(seed ^ splitmix((unsigned long long)i * 64ull + (unsigned long long)k));
  return (double)(h >> 11) * (1.0 / 9007199254740992.0);
}

__global__ void k_gen_params(unsigned long long seed, int n, double rmin, double rmax, double *par) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  double *P = par + (size_t)i * 20;
  const double R = exp(log(rmin) + urand(seed, i, 0) * (log(rmax) - log(rmin)));
  const bool ellipsoid = urand(seed, i, 1) < 0.5;
  for (int d = 0; d < 3; ++d) P[3 + d] = R * (ellipsoid ? 0.75 + 0.5 * urand(seed, i, 2 + d) : 1.0);
  // uniform random rotation from a unit quaternion (Shoemake)
  const double u1 = urand(seed, i, 5), u2 = urand(seed, i, 6), u3 = urand(seed, i, 7);
  const double qa = sqrt(1 - u1) * sin(6.283185307179586 * u2), qb = sqrt(1 - u1) * cos(6.283185307179586 * u2);
  const double qc = sqrt(u1) * sin(6.283185307179586 * u3), qd = sqrt(u1) * cos(6.283185307179586 * u3);
  // (w, x, y, z) = (qd, qa, qb, qc)
  const double W = qd, X = qa, Y = qb, Z = qc;
  double Rm[9] = {1 - 2 * (Y * Y + Z * Z), 2 * (X * Y - Z * W), 2 * (X * Z + Y * W),
                  2 * (X * Y + Z * W), 1 - 2 * (X * X + Z * Z), 2 * (Y * Z - X * W),
                  2 * (X * Z - Y * W), 2 * (Y * Z + X * W), 1 - 2 * (X * X + Y * Y)};
  for (int k = 0; k < 9; ++k) P[6 + k] = Rm[k];
  for (int d = 0; d < 3; ++d) P[d] = urand(seed, i, 8 + d);
  P[15] = urand(seed, i, 11) < 0.75 ? 1.0 : 0.0;
  // a random point of the surface: direction uniform on the sphere
  const double zz = 2 * urand(seed, i, 12) - 1, ph = 6.283185307179586 * urand(seed, i, 13);
  const double rr = sqrt(fmax(0.0, 1 - zz * zz));
  const double dv[3] = {rr * cos(ph), rr * sin(ph), zz};
  // t such that (t d)^T A (t d) = 1, A = R diag(1/a^2) R^T
  double q = 0;
  for (int k = 0; k < 3; ++k) {
    const double pk = Rm[0 * 3 + k] * dv[0] + Rm[1 * 3 + k] * dv[1] + Rm[2 * 3 + k] * dv[2];  // (R^T d)_k
    q += pk * pk / (P[3 + k] * P[3 + k]);
  }
  const double tt = 1 / sqrt(q);
  for (int d = 0; d < 3; ++d) P[16 + d] = floor(P[d] + tt * dv[d] + 0.5);
  P[19] = 0;
}

// fill levels (fraction of 6^3 sub-points that are liquid), curvature at the
// surface point reached from the cell centre by Newton steps along grad F,
// canonical orientation; writes x (27 fp32) and y = 4 kappa
__global__ void k_gen_stencils(const double *par, int n, float *x, float *y) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const double *P = par + (size_t)i * 20;
  double A[9];
  for (int r = 0; r < 3; ++r)
    for (int c = 0; c < 3; ++c) {
      double v = 0;
      for (int k = 0; k < 3; ++k) v += P[6 + r * 3 + k] * P[6 + c * 3 + k] / (P[3 + k] * P[3 + k]);
      A[r * 3 + c] = v;
    }
  const bool gas = P[15] > 0.5;
  float a[27];
  for (int q = 0; q < 27; ++q) {
    const double cx = P[16] + (q % 3 - 1) - P[0], cy = P[17] + ((q / 3) % 3 - 1) - P[1],
                 cz = P[18] + (q / 9 - 1) - P[2];
    int liq = 0;
    for (int kz = 0; kz < 6; ++kz)
      for (int ky = 0; ky < 6; ++ky)
        for (int kx = 0; kx < 6; ++kx) {
          const double dx = cx + (kx + 0.5) / 6 - 0.5, dy = cy + (ky + 0.5) / 6 - 0.5, dz = cz + (kz + 0.5) / 6 - 0.5;
          const double f = A[0] * dx * dx + A[4] * dy * dy + A[8] * dz * dz +
                           2 * (A[1] * dx * dy + A[2] * dx * dz + A[5] * dy * dz);
          const bool inside = f < 1.0;
          liq += (gas ? !inside : inside) ? 1 : 0;
        }
    a[q] = (float)((double)liq / 216.0);
  }
  double p[3] = {P[16] - P[0], P[17] - P[1], P[18] - P[2]};
  for (int it = 0; it < 8; ++it) {
    double gF[3];
    for (int r = 0; r < 3; ++r) gF[r] = 2 * (A[r * 3] * p[0] + A[r * 3 + 1] * p[1] + A[r * 3 + 2] * p[2]);
    const double F = 0.5 * (gF[0] * p[0] + gF[1] * p[1] + gF[2] * p[2]) - 1.0;
    const double g2 = gF[0] * gF[0] + gF[1] * gF[1] + gF[2] * gF[2];
    if (!(g2 > 0)) break;
    for (int r = 0; r < 3; ++r) p[r] -= F * gF[r] / g2;
  }
  double gF[3];
  for (int r = 0; r < 3; ++r) gF[r] = 2 * (A[r * 3] * p[0] + A[r * 3 + 1] * p[1] + A[r * 3 + 2] * p[2]);
  double gHg = 0;
  for (int r = 0; r < 3; ++r)
    for (int c = 0; c < 3; ++c) gHg += gF[r] * 2 * A[r * 3 + c] * gF[c];
  const double gn2 = gF[0] * gF[0] + gF[1] * gF[1] + gF[2] * gF[2], gn = sqrt(gn2);
  const double mean_out = (gHg - gn2 * 2 * (A[0] + A[4] + A[8])) / (2 * gn2 * gn);
  const double kappa = gas ? -mean_out : mean_out;
  float nx, ny, nz;
  py_normal(a, nx, ny, nz);
  int order[3], sign[3];
  canonical_order(nx, ny, nz, order, sign);
  for (int q = 0; q < 27; ++q) x[(size_t)i * 27 + q] = a[canonical_src(q, order, sign)];
  y[i] = (float)(Y_SCALE * kappa);
}

unsigned long long host_splitmix(unsigned long long x) {
  x += 0x9E3779B97F4A7C15ull;
  x = (x ^ (x >> 30)) * 0xBF58476D1CE4E5B9ull;
  x = (x ^ (x >> 27)) * 0x94D049BB133111EBull;
  return x ^ (x >> 31);
}
unsigned long long host_gcd(unsigned long long a, unsigned long long b) {
  while (b) {
    const unsigned long long t = a % b;
    a = b;
    b = t;
  }
  return a;
}

size_t grad_smem() { return sizeof(Smem) + ((NP * 4 + 15) / 16) * 16 + WARPS * sizeof(Stage); }

int grad_launch(const float *theta, const float *x, const float *t, int n, const Batch &bt, float *grad, double *loss,
                cudaStream_t st) {
  static bool attr = false;
  if (!attr) {
    CKM(cudaFuncSetAttribute(k_grad, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)grad_smem()));
    attr = true;
  }
  const int tiles = (n + 15) / 16;
  int blocks = (tiles + WARPS - 1) / WARPS;
  if (blocks > 304) blocks = 304;
  k_grad<<<blocks, 32 * WARPS, grad_smem(), st>>>(theta, x, t, n, bt, grad, loss);
  CKM(cudaGetLastError());
  return 0;
}

}  // namespace

namespace {
__global__ void k_pack_net(const float *theta, tc::Image *img) { tc::pack_image(*img, theta); }
}  // namespace

namespace lbf {
namespace mlp {
size_t image_bytes() { return sizeof(tc::Image); }
void pack_launch(const float *theta, void *img, cudaStream_t st) {
  k_pack_net<<<1, 256, 0, st>>>(theta, (tc::Image *)img);
}
// in-loop use by the simulation (declared in lbf_ops_api.h)
void forward_launch(const float *theta, const float *x, int n, float *y, cudaStream_t st) {
  const int tiles = (n + tc::ROWS - 1) / tc::ROWS;
  int dev = 0, sms = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  int blocks = tiles < sms ? tiles : sms;
  if (blocks < 1) blocks = 1;
  k_forward_tc<<<blocks, 128, sizeof(tc::Tile), st>>>(theta, x, n, y);
}
}  // namespace mlp
}  // namespace lbf

extern "C" {

int lbf_mlp_forward(const float *theta, const float *x, int n, float *y, void *stream) {
  if (!theta || !x || !y || n < 0) return fail(LBF_EINVAL, "bad arguments");
  if (n == 0) return 0;
  lbf::mlp::forward_launch(theta, x, n, y, (cudaStream_t)stream);
  CKM(cudaGetLastError());
  return 0;
}

int lbf_mlp_loss_grad(const float *theta, const float *x, const float *t, int n, float *grad, double *loss,
                      void *stream) {
  if (!theta || !x || !t || !grad || !loss || n <= 0) return fail(LBF_EINVAL, "bad arguments");
  cudaStream_t st = (cudaStream_t)stream;
  CKM(cudaMemsetAsync(grad, 0, sizeof(float) * NP, st));
  CKM(cudaMemsetAsync(loss, 0, sizeof(double), st));
  Batch bt{0, n, 1ull, 0ull, 0ull, 0.f};
  return grad_launch(theta, x, t, n, bt, grad, loss, st);
}

int lbf_mlp_generate(unsigned long long seed, int n, double rmin, double rmax, float *x, float *y, void *stream) {
  if (!x || !y || n < 0 || !(rmin > 0) || !(rmax >= rmin)) return fail(LBF_EINVAL, "bad arguments");
  if (n == 0) return 0;
  cudaStream_t st = (cudaStream_t)stream;
  double *par = nullptr;
  CKM(cudaMallocAsync((void **)&par, sizeof(double) * 20 * (size_t)n, st));
  k_gen_params<<<(n + 127) / 128, 128, 0, st>>>(seed, n, rmin, rmax, par);
  k_gen_stencils<<<(n + 127) / 128, 128, 0, st>>>(par, n, x, y);
  CKM(cudaGetLastError());
  CKM(cudaFreeAsync(par, st));
  return 0;
}

int lbf_mlp_stencils_from_params(const double *params, int n, float *x, float *y, void *stream) {
  if (!params || !x || !y || n <= 0) return fail(LBF_EINVAL, "bad arguments");
  cudaStream_t st = (cudaStream_t)stream;
  double *par = nullptr;
  CKM(cudaMallocAsync((void **)&par, sizeof(double) * 20 * (size_t)n, st));
  CKM(cudaMemcpyAsync(par, params, sizeof(double) * 20 * (size_t)n, cudaMemcpyHostToDevice, st));
  k_gen_stencils<<<(n + 127) / 128, 128, 0, st>>>(par, n, x, y);
  CKM(cudaGetLastError());
  CKM(cudaFreeAsync(par, st));
  CKM(cudaStreamSynchronize(st));
  return 0;
}

int lbf_mlp_train(const lbf_mlp_train_cfg *cfg, float *theta_io, float *loss_curve) {
  if (!cfg || !theta_io || cfg->n_samples < 0 || cfg->n_extra < 0 || cfg->batch < 16 || cfg->epochs < 1 ||
      !(cfg->noise >= 0.0) || (cfg->n_extra > 0 && (!cfg->x_extra || !cfg->y_extra)))
    return fail(LBF_EINVAL, "bad training configuration");
  cudaStream_t st = (cudaStream_t)cfg->stream;
  const long long n = (long long)cfg->n_samples + cfg->n_extra;
  const int B = cfg->batch;
  if (n < B) return fail(LBF_EINVAL, "fewer samples than one batch");
  float *x = nullptr, *y = nullptr, *theta = nullptr, *m = nullptr, *v = nullptr, *grad = nullptr;
  double *loss = nullptr;
  CKM(cudaMallocAsync((void **)&x, sizeof(float) * 27 * (size_t)n, st));
  CKM(cudaMallocAsync((void **)&y, sizeof(float) * (size_t)n, st));
  CKM(cudaMallocAsync((void **)&theta, sizeof(float) * NP, st));
  CKM(cudaMallocAsync((void **)&m, sizeof(float) * NP, st));
  CKM(cudaMallocAsync((void **)&v, sizeof(float) * NP, st));
  CKM(cudaMallocAsync((void **)&grad, sizeof(float) * NP, st));
  CKM(cudaMallocAsync((void **)&loss, sizeof(double) * (size_t)cfg->epochs, st));
  if (cfg->n_samples > 0) {
    int rc = lbf_mlp_generate(cfg->seed, cfg->n_samples, cfg->rmin, cfg->rmax, x, y, cfg->stream);
    if (rc) return rc;
  }
  if (cfg->n_extra > 0) {
    CKM(cudaMemcpyAsync(x + (size_t)cfg->n_samples * 27, cfg->x_extra, sizeof(float) * 27 * (size_t)cfg->n_extra,
                        cudaMemcpyDeviceToDevice, st));
    CKM(cudaMemcpyAsync(y + cfg->n_samples, cfg->y_extra, sizeof(float) * (size_t)cfg->n_extra,
                        cudaMemcpyDeviceToDevice, st));
  }
  CKM(cudaMemcpyAsync(theta, theta_io, sizeof(float) * NP, cudaMemcpyHostToDevice, st));
  CKM(cudaMemsetAsync(m, 0, sizeof(float) * NP, st));
  CKM(cudaMemsetAsync(v, 0, sizeof(float) * NP, st));
  CKM(cudaMemsetAsync(loss, 0, sizeof(double) * (size_t)cfg->epochs, st));
  int step = 0;
  const long long per_epoch = n / B;
  for (int ep = 0; ep < cfg->epochs; ++ep) {
    const float lr = (float)(cfg->lr * (ep >= cfg->epochs * 3 / 4 ? 0.1 : 1.0));
    // per-epoch affine shuffle: a odd-ish and coprime to n
    const unsigned long long h = host_splitmix(cfg->seed ^ host_splitmix(0xC0FFEEull + (unsigned long long)ep));
    unsigned long long a = (h % (unsigned long long)n) | 1ull;
    while (host_gcd(a, (unsigned long long)n) != 1ull) a += 2;
    const unsigned long long b = host_splitmix(h) % (unsigned long long)n;
    for (long long k = 0; k < per_epoch; ++k) {
      CKM(cudaMemsetAsync(grad, 0, sizeof(float) * NP, st));
      Batch bt{k * B, n, a % (unsigned long long)n, b, host_splitmix(h + (unsigned long long)k),
               (float)cfg->noise};
      int rc = grad_launch(theta, x, y, B, bt, grad, loss + ep, st);
      if (rc) return rc;
      k_adam<<<(NP + 255) / 256, 256, 0, st>>>(theta, m, v, grad, ++step, lr);
    }
    CKM(cudaGetLastError());
  }
  std::vector<double> lc(cfg->epochs);
  CKM(cudaMemcpyAsync(theta_io, theta, sizeof(float) * NP, cudaMemcpyDeviceToHost, st));
  CKM(cudaMemcpyAsync(lc.data(), loss, sizeof(double) * cfg->epochs, cudaMemcpyDeviceToHost, st));
  CKM(cudaStreamSynchronize(st));
  if (loss_curve)
    for (int ep = 0; ep < cfg->epochs; ++ep) loss_curve[ep] = (float)(lc[ep] / (double)per_epoch);
  CKM(cudaFreeAsync(x, st));
  CKM(cudaFreeAsync(y, st));
  CKM(cudaFreeAsync(theta, st));
  CKM(cudaFreeAsync(m, st));
  CKM(cudaFreeAsync(v, st));
  CKM(cudaFreeAsync(grad, st));
  CKM(cudaFreeAsync(loss, st));
  CKM(cudaStreamSynchronize(st));
  return 0;
}

}  // extern "C"

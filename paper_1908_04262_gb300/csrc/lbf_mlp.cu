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

// inference: canonical stencils (n x 27 fp32) -> y = 4 kappa, on the
// fifth-generation tensor cores: tiles of 128 rows, each CTA (128 threads)
// walking tiles; a tile whose MMA did not complete within the wait bound
// (and every later tile of that CTA) gets NaN outputs
__global__ void __launch_bounds__(128) k_forward_tc(const float *theta, const float *x, int n, float *y) {
  extern __shared__ __align__(128) unsigned char tsm[];
  tc::Tile &t = *reinterpret_cast<tc::Tile *>(tsm);
  tc::pack_image(t.net, theta);
  tc::setup(t, tc::TCOLS);
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

// The network as training reads it: the inference image plus W2^T (row i,
// K = j: the B operand of delta1 = delta2 W2), packed by Adam after every
// update so that each gradient CTA fetches it with two bulk copies.
struct __align__(128) TrainImage {
  tc::Image net;
  __nv_bfloat16 w2t[64 * 64];
};
static_assert(sizeof(TrainImage) % 16 == 0 && sizeof(tc::Image) % 16 == 0, "bulk copies move multiples of 16 bytes");

// parameter i (value v) into its places in the training image (the pads of
// W1 stay as the image was cleared)
__device__ __forceinline__ void place_param(TrainImage &m, int i, float v) {
  const __nv_bfloat16 b = __float2bfloat16_rn(v);
  if (i < OFF_B1) {
    const int r = i / 27, k = i - 27 * r;
    m.net.w1[tc::kofs(r, k, 32) / 2] = b;
  } else if (i < OFF_W2) {
    m.net.b1[i - OFF_B1] = v;
  } else if (i < OFF_B2) {
    const int q = i - OFF_W2, r = q >> 6, k = q & 63;
    m.net.w2[tc::kofs(r, k, 64) / 2] = b;
    m.w2t[tc::kofs(k, r, 64) / 2] = b;
  } else if (i < OFF_W3) {
    m.net.b2[i - OFF_B2] = v;
  } else if (i < OFF_B3) {
    m.net.w3[i - OFF_W3] = v;
  } else {
    m.net.b3 = v;
  }
}
__global__ void k_place_all(const float *theta, TrainImage *img) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < NP) place_param(*img, i, theta[i]);
}

// shared memory of a gradient CTA
struct __align__(128) GradSmem {
  tc::Tile t;                    // X (a1), H1 then BF16 H2 row-major (a2), the network
  __nv_bfloat16 w2t[64 * 64];    // W2^T
  __nv_bfloat16 ad2[128 * 64];   // delta2 (A of delta2 W2)
  __nv_bfloat16 ag[128 * 128];   // rows 0-63 delta2^T, 64-127 delta1^T; K = the tile's rows
  __nv_bfloat16 bg[112 * 128];   // rows 0-63 H1^T, 64-90 X^T, 96 ones, the rest zero
  float d3[128], le[128];        // delta3 and the loss of each row
  long long src[128];            // data row of each tile row
};
constexpr uint32_t GRAD_TCOLS = 512;  // Z1 0-63, Z2 64-127, delta2 W2 128-191, gradients 256-367

// Gradient of L = (1/2n) sum (y - t)^2 on the fifth-generation tensor
// cores: tiles of 128 rows, one row per thread in the epilogues.  Per tile:
//   Z1 = X W1^T, H1 = SiLU(Z1 + b1); Z2 = H1 W2^T, y = BF16(SiLU(Z2 + b2)) W3 + b3
//   delta3 = (y - t) / n, delta2 = delta3 W3 SiLU'(Z2 + b2)
//   delta1 = (delta2 W2) SiLU'(Z1 + b1)                    (MMA, K = 64)
//   [delta2^T; delta1^T] [H1^T; X^T; 1]^T accumulated over the tiles  (MMA,
//   K = 128 rows): its blocks are dW2, dW1, db2 and db1
// dW3, db3 and the loss are summed in shared memory per tile.  Everything
// is added into grad and *loss (global) once per CTA.  A timed-out wait
// adds NaN to *loss.
__global__ void __launch_bounds__(128) k_grad_tc(const TrainImage *img, const float *x, const float *tgt, int n,
                                                 Batch bt, float *grad, double *loss) {
  extern __shared__ __align__(128) unsigned char gsm[];
  GradSmem &s = *reinterpret_cast<GradSmem *>(gsm);
  tc::Tile &t = s.t;
  const int tid = threadIdx.x, w = tid >> 5;
  const int tiles = (n + tc::ROWS - 1) / tc::ROWS;
  for (int i = tid; i < 112 * 128; i += 128) {
    const int r = i >> 7, m = i & 127;
    s.bg[tc::kofs(r, m, 128) / 2] = __float2bfloat16_rn(r == 96 ? 1.f : 0.f);
  }
  tc::setup(t, GRAD_TCOLS, tc::Copy{&t.net, &img->net, (uint32_t)sizeof(tc::Image)},
            tc::Copy{s.w2t, img->w2t, (uint32_t)sizeof(img->w2t)});
  const uint32_t tm = t.tmem, lanes = (uint32_t)(32 * w) << 16;
  const float inv_n = 1.f / (float)n;
  uint32_t phase = 0;
  bool failed = false, net = false, any = false;
  for (int tile = blockIdx.x; tile < tiles && !failed; tile += gridDim.x) {
    const int row0 = tile * tc::ROWS, rows = min(tc::ROWS, n - row0);
    // the tile's data rows (thread = row), then X into a1 and X^T into bg
    float target = 0.f;
    if (tid < rows) {
      const long long src =
          (long long)((bt.a * (unsigned long long)(bt.start + row0 + tid) + bt.b) % (unsigned long long)bt.ntot);
      s.src[tid] = src;
      target = tgt[src];
    }
    __syncthreads();
#pragma unroll 9
    for (int c = 0; c < 27; ++c) {
      const int e = tid + 128 * c, r = e / 27, k = e - 27 * r;
      float v = 0.f;
      if (r < rows) {
        const long long src = s.src[r];
        v = x[(size_t)src * 27 + k];
        if (bt.noise > 0.f && v > 0.f && v < 1.f) {
          const unsigned long long h = splitmix(bt.key ^ splitmix((unsigned long long)src * 32ull + k));
          const float u = (float)(h >> 40) * (1.f / 16777216.f);
          v = fminf(fmaxf(v + bt.noise * (2.f * u - 1.f), 0.f), 1.f);
        }
      }
      const __nv_bfloat16 b = __float2bfloat16_rn(v);
      t.a1[tc::kofs(r, k, 32) / 2] = b;
      s.bg[tc::kofs(64 + k, r, 128) / 2] = b;
    }
    if (!net) {
      net = true;
      if (!tc::wait_net(t, phase)) {
        failed = true;
        break;
      }
    }
    // layer 1; H1 into a2 (row tid) and bg rows 0-63 (column tid)
    tc::to_tensor_cores();
    if (tid == 0) tc::issue(t, tm, t.a1, t.net.w1, 32, 64, 2, false);
    if (!tc::wait_mmas(t, phase)) {
      failed = true;
      break;
    }
#pragma unroll
    for (int c = 0; c < 4; ++c) {
      float z[16];
      tc::ld16(tm + lanes + 16 * c, z);
#pragma unroll
      for (int h = 0; h < 2; ++h) {
        uint4 q;
        uint32_t *qw = reinterpret_cast<uint32_t *>(&q);
#pragma unroll
        for (int e = 0; e < 4; ++e) {
          const int j = 16 * c + 8 * h + 2 * e;
          const __nv_bfloat162 hv =
              __floats2bfloat162_rn(silu(z[8 * h + 2 * e] + t.net.b1[j]), silu(z[8 * h + 2 * e + 1] + t.net.b1[j + 1]));
          qw[e] = *reinterpret_cast<const uint32_t *>(&hv);
          s.bg[tc::kofs(j, tid, 128) / 2] = hv.x;
          s.bg[tc::kofs(j + 1, tid, 128) / 2] = hv.y;
        }
        *reinterpret_cast<uint4 *>(reinterpret_cast<unsigned char *>(t.a2) + tc::kofs(tid, 16 * c + 8 * h, 64)) = q;
      }
    }
    // layer 2; y, delta3 and the loss of row tid; BF16 H2 into a2 (row-major)
    tc::to_tensor_cores();
    if (tid == 0) tc::issue(t, tm + 64, t.a2, t.net.w2, 64, 64, 4, false);
    if (!tc::wait_mmas(t, phase)) {
      failed = true;
      break;
    }
    float y = 0.f;
#pragma unroll
    for (int c = 0; c < 4; ++c) {
      float z[16];
      tc::ld16(tm + lanes + 64 + 16 * c, z);
#pragma unroll
      for (int e = 0; e < 16; e += 2) {
        const int j = 16 * c + e;
        const __nv_bfloat162 hv = __floats2bfloat162_rn(silu(z[e] + t.net.b2[j]), silu(z[e + 1] + t.net.b2[j + 1]));
        y += __bfloat162float(hv.x) * t.net.w3[j] + __bfloat162float(hv.y) * t.net.w3[j + 1];
        *reinterpret_cast<__nv_bfloat162 *>(t.a2 + tid * 64 + j) = hv;
      }
    }
    y += t.net.b3;
    const float err = tid < rows ? y - target : 0.f;
    const float d3 = err * inv_n;
    s.d3[tid] = d3;
    s.le[tid] = 0.5f * err * err * inv_n;
    // delta2 = delta3 W3 SiLU'(Z2 + b2): into ad2 (row tid) and ag rows 0-63
#pragma unroll
    for (int c = 0; c < 4; ++c) {
      float z[16];
      tc::ld16(tm + lanes + 64 + 16 * c, z);
#pragma unroll
      for (int h = 0; h < 2; ++h) {
        uint4 q;
        uint32_t *qw = reinterpret_cast<uint32_t *>(&q);
#pragma unroll
        for (int e = 0; e < 4; ++e) {
          const int j = 16 * c + 8 * h + 2 * e;
          const __nv_bfloat162 dv = __floats2bfloat162_rn(d3 * t.net.w3[j] * dsilu(z[8 * h + 2 * e] + t.net.b2[j]),
                                                          d3 * t.net.w3[j + 1] * dsilu(z[8 * h + 2 * e + 1] + t.net.b2[j + 1]));
          qw[e] = *reinterpret_cast<const uint32_t *>(&dv);
          s.ag[tc::kofs(j, tid, 128) / 2] = dv.x;
          s.ag[tc::kofs(j + 1, tid, 128) / 2] = dv.y;
        }
        *reinterpret_cast<uint4 *>(reinterpret_cast<unsigned char *>(s.ad2) + tc::kofs(tid, 16 * c + 8 * h, 64)) = q;
      }
    }
    // delta2 W2 on the tensor cores while the CTA sums dW3, db3 and the loss
    tc::to_tensor_cores();
    if (tid == 0) tc::issue(t, tm + 128, s.ad2, s.w2t, 64, 64, 4, false);
    if (tid < 64) {
      float g = 0.f;
      for (int m = 0; m < tc::ROWS; ++m) g += s.d3[m] * __bfloat162float(t.a2[m * 64 + tid]);
      atomicAdd(grad + OFF_W3 + tid, g);
    } else if (tid == 64) {
      float g = 0.f;
      for (int m = 0; m < tc::ROWS; ++m) g += s.d3[m];
      atomicAdd(grad + OFF_B3, g);
    } else if (tid == 96) {
      double l = 0.0;
      for (int m = 0; m < tc::ROWS; ++m) l += (double)s.le[m];
      atomicAdd(loss, l);
    }
    if (!tc::wait_mmas(t, phase)) {
      failed = true;
      break;
    }
    // delta1 = (delta2 W2) SiLU'(Z1 + b1): into ag rows 64-127
#pragma unroll
    for (int c = 0; c < 4; ++c) {
      float z[16], d[16];
      tc::ld16(tm + lanes + 16 * c, z);
      tc::ld16(tm + lanes + 128 + 16 * c, d);
#pragma unroll
      for (int e = 0; e < 16; ++e) {
        const int j = 16 * c + e;
        s.ag[tc::kofs(64 + j, tid, 128) / 2] = __float2bfloat16_rn(d[e] * dsilu(z[e] + t.net.b1[j]));
      }
    }
    // weight and bias gradients of the tile, accumulated in tensor memory
    tc::to_tensor_cores();
    if (tid == 0) tc::issue(t, tm + 256, s.ag, s.bg, 128, 112, 8, any);
    any = true;
    if (!tc::wait_mmas(t, phase)) {
      failed = true;
      break;
    }
  }
  if (failed) {
    if (tid == 0) atomicAdd(loss, (double)__int_as_float(0x7fc00000));
  } else if (any) {
    // row tid of the accumulated block product: rows 0-63 dW2 (columns
    // 0-63) and db2 (column 96), rows 64-127 dW1 (columns 64-90) and db1
    float z[16];
    tc::ld16(tm + lanes + 256 + 96, z);
    if (tid < 64) {
      atomicAdd(grad + OFF_B2 + tid, z[0]);
#pragma unroll
      for (int c = 0; c < 4; ++c) {
        tc::ld16(tm + lanes + 256 + 16 * c, z);
#pragma unroll
        for (int e = 0; e < 16; ++e) atomicAdd(grad + OFF_W2 + tid * 64 + 16 * c + e, z[e]);
      }
    } else {
      const int i = tid - 64;
      atomicAdd(grad + OFF_B1 + i, z[0]);
#pragma unroll
      for (int c = 0; c < 2; ++c) {
        tc::ld16(tm + lanes + 256 + 64 + 16 * c, z);
#pragma unroll
        for (int e = 0; e < 16; ++e)
          if (16 * c + e < 27) atomicAdd(grad + OFF_W1 + i * 27 + 16 * c + e, z[e]);
      }
    }
  }
  tc::teardown(t, phase, failed, GRAD_TCOLS);
}

// Adam on the fp32 master parameters; the updated parameter also goes into
// the training image
__global__ void k_adam(float *theta, float *m, float *v, const float *grad, int step, float lr, TrainImage *img) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= NP) return;
  const float b1 = 0.9f, b2 = 0.999f, eps = 1e-8f;
  const float gi = grad[i];
  const float mi = b1 * m[i] + (1.f - b1) * gi;
  const float vi = b2 * v[i] + (1.f - b2) * gi * gi;
  m[i] = mi;
  v[i] = vi;
  const float mh = mi / (1.f - powf(b1, (float)step)), vh = vi / (1.f - powf(b2, (float)step));
  const float th = theta[i] - lr * mh / (sqrtf(vh) + eps);
  theta[i] = th;
  place_param(*img, i, th);
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

// a cleared training image made from theta
int image_init(const float *theta, TrainImage *img, cudaStream_t st) {
  CKM(cudaMemsetAsync(img, 0, sizeof(TrainImage), st));
  k_place_all<<<(NP + 255) / 256, 256, 0, st>>>(theta, img);
  CKM(cudaGetLastError());
  return 0;
}

int grad_launch(const TrainImage *img, const float *x, const float *t, int n, const Batch &bt, float *grad,
                double *loss, cudaStream_t st) {
  int dev = 0;
  CKM(cudaGetDevice(&dev));
  static int attr_dev = -1;
  if (attr_dev != dev) {
    CKM(cudaFuncSetAttribute(k_grad_tc, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sizeof(GradSmem)));
    attr_dev = dev;
  }
  int sms = 0;
  CKM(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
  const int tiles = (n + tc::ROWS - 1) / tc::ROWS;
  const int blocks = tiles < sms ? tiles : sms;
  k_grad_tc<<<blocks, 128, sizeof(GradSmem), st>>>(img, x, t, n, bt, grad, loss);
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
  TrainImage *img = nullptr;
  CKM(cudaMallocAsync((void **)&img, sizeof(TrainImage), st));
  Batch bt{0, n, 1ull, 0ull, 0ull, 0.f};
  int rc = image_init(theta, img, st);
  if (!rc) rc = grad_launch(img, x, t, n, bt, grad, loss, st);
  CKM(cudaFreeAsync(img, st));
  return rc;
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
  TrainImage *img = nullptr;
  CKM(cudaMallocAsync((void **)&img, sizeof(TrainImage), st));
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
  {
    int rc = image_init(theta, img, st);
    if (rc) return rc;
  }
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
      int rc = grad_launch(img, x, y, B, bt, grad, loss + ep, st);
      if (rc) return rc;
      k_adam<<<(NP + 255) / 256, 256, 0, st>>>(theta, m, v, grad, ++step, lr, img);
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
  CKM(cudaFreeAsync(img, st));
  CKM(cudaStreamSynchronize(st));
  return 0;
}

}  // extern "C"

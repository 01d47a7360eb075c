// lbf_geom.cuh -- interface geometry for the next step: normals, PLIC
// offsets, curvature (Sec. 2.2 Eq. rhob) and disjoining pressure (Sec. 3.3,
// Appendix A Algorithm 1).  One thread per interface cell.
//
// Normal: gradient of the fill level over the 3^d stencil with face, edge and
// corner weights 4, 2, 1, normalised; it points into the liquid.
// PLIC: the plane n.p = s that leaves liquid fraction alpha on its +n side of
// the unit cell, inverted in closed form after Scardovelli and Zaleski (2000)
// (volume of a unit cube cut by a plane: piecewise polynomial in the
// plane constant; its quadratic branches are solved directly, its cubic
// branches by the trigonometric formula, then one Newton polish).
// Curvature: least-squares paraboloid through the PLIC points of the
// interface cells of the stencil (each cut with the centre normal) in a frame
// whose third axis is the normal (ridge-regularised normal equations);
// kappa = -(mean curvature), so a gas sphere
// has kappa = 1/R and a gas disk 1/(2R); limited to [-1, 1].
// Disjoining pressure: march from the cell centre along the normal, cell
// boundary by cell boundary (Algorithm 1, ties -- equal within a relative
// 1e-9, 1e-5 in single precision -- step diagonally), until an
// interface or gas cell of another bubble is met; d is the distance from this
// cell's plane to the other cell's plane along the ray (or to where the ray
// enters it when that plane does not face the ray); Pi = k_Pi (d_max - d)
// for d < d_max.
#pragma once
#include "lbf_common.cuh"

namespace lbf {

// 1 / sqrt(x): the correctly rounded quotient in double, the hardware
// reciprocal square root in single precision
__device__ __forceinline__ double rsqrt_r(double x) { return 1.0 / sqrt(x); }
__device__ __forceinline__ float rsqrt_r(float x) { return rsqrtf(x); }

// arccos for single precision: Abramowitz and Stegun 4.4.45,
// acos x = sqrt(1 - x) (a0 + a1 x + a2 x^2 + a3 x^3) on [0, 1] with absolute
// error below 6.7e-5, and acos(-x) = pi - acos x.  Only a starting value:
// the cubic's root taken from it is polished by Newton steps.
__device__ __forceinline__ float acos_as(float x) {
  const float ax = fabsf(x);
  const float v = sqrtf(1.f - ax) * (1.5707288f + ax * (-0.2121144f + ax * (0.0742610f + ax * -0.0187293f)));
  return x < 0.f ? 3.14159265358979f - v : v;
}

// real root of a^3 + b a^2 + c a + d = 0 closest to [lo, hi], polished
template <class R>
__device__ __forceinline__ R cubic_root_in(R b, R c, R d, R lo, R hi) {
  const R b3 = b / (R)3;
  const R P = c - b * b3;
  const R Qc = (R)2 * b3 * b3 * b3 - b3 * c + d;
  R best = (R)0.5 * (lo + hi), bestd = (R)1e30;
  auto consider = [&](R a) {
    const R dd = a < lo ? lo - a : (a > hi ? a - hi : (R)0);
    if (dd < bestd) {
      bestd = dd;
      best = a;
    }
  };
  if (P < (R)0) {
    const R r = (R)2 * sqrt(-P / (R)3);
    R arg = (R)3 * Qc / (P * r);
    arg = arg < (R)-1 ? (R)-1 : (arg > (R)1 ? (R)1 : arg);
    if constexpr (sizeof(R) == 4) {
      // the three cosines cos(th - 2 pi k / 3) from one sine and cosine
      const float th = acos_as(arg) * (1.f / 3.f);
      float sn, cs;
      __sincosf(th, &sn, &cs);
      const float h = 0.8660254037844386f * sn;
      consider(r * cs - b3);
      consider(r * (-0.5f * cs + h) - b3);
      consider(r * (-0.5f * cs - h) - b3);
    } else {
      const R th = acos(arg) / (R)3;
      const R twopi3 = (R)2.0943951023931954923;
      for (int k = 0; k < 3; ++k) consider(r * cos(th - twopi3 * (R)k) - b3);
    }
  } else {
    const R disc = Qc * Qc / (R)4 + P * P * P / (R)27;
    const R sq = sqrt(disc > (R)0 ? disc : (R)0);
    consider(cbrt(-Qc / (R)2 + sq) + cbrt(-Qc / (R)2 - sq) - b3);
  }
  R a = best < lo ? lo : (best > hi ? hi : best);
  for (int it = 0; it < 2; ++it) {
    const R fa = ((a + b) * a + c) * a + d;
    const R fp = ((R)3 * a + (R)2 * b) * a + c;
    if (fp != (R)0) {
      const R an = a - fa / fp;
      a = an < lo ? lo : (an > hi ? hi : an);
    }
  }
  return a;
}

// plane constant a in [0, 1/2] of the normalised problem: gas fraction V
// (<= 1/2) of the unit cube below m1 x + m2 y + m3 z = a, m sorted ascending,
// m1 + m2 + m3 = 1
template <class R>
__device__ __forceinline__ R plic_a3(R m1, R m2, R m3, R V) {
  if (m1 < (R)1e-12) {  // reduces to the 2D problem in (m2, m3)
    const R s = m2 + m3;
    const R n1 = m2 / s, n2 = m3 / s;
    const R V1 = n2 > (R)0 ? n1 / ((R)2 * n2) : (R)0;
    const R a = V < V1 ? sqrt((R)2 * n1 * n2 * V) : n2 * V + (R)0.5 * n1;
    return a * s;
  }
  const R m12 = m1 + m2;
  const R V1 = m1 * m1 / ((R)6 * m2 * m3);
  const R V2 = V1 + (m2 - m1) / ((R)2 * m3);
  if (V < V1) return cbrt((R)6 * m1 * m2 * m3 * V);
  if (V < V2) return (R)0.5 * m1 + sqrt((R)72 * m2 * m3 * V - (R)3 * m1 * m1) / (R)6;
  const R six = (R)6 * m1 * m2 * m3;
  if (m3 < m12) {
    const R V3 = (m3 * m3 * ((R)3 * m12 - m3) + m1 * m1 * (m1 - (R)3 * m3) + m2 * m2 * (m2 - (R)3 * m3)) / six;
    if (V < V3)
      return cubic_root_in<R>((R)-3 * m12, (R)3 * (m1 * m1 + m2 * m2),
                              -(m1 * m1 * m1 + m2 * m2 * m2 - six * V), m2, m3);
    const R S2 = m1 * m1 + m2 * m2 + m3 * m3, S3 = m1 * m1 * m1 + m2 * m2 * m2 + m3 * m3 * m3;
    return cubic_root_in<R>((R)-1.5, (R)1.5 * S2, -(S3 - six * V) / (R)2, m3, (R)0.5);
  }
  const R V3 = m12 / ((R)2 * m3);
  if (V < V3)
    return cubic_root_in<R>((R)-3 * m12, (R)3 * (m1 * m1 + m2 * m2),
                            -(m1 * m1 * m1 + m2 * m2 * m2 - six * V), m2, m12);
  return m3 * V + (R)0.5 * m12;
}

// PLIC inversion for one normal: the normalised, sorted components are
// computed once and reused for every fill level cut with that normal
template <int D, class R> struct Plic {
  R sum, m1, m2, m3;
  __device__ __forceinline__ Plic(R nx, R ny, R nz) {
    R a1 = fabs(nx), a2 = fabs(ny), a3 = D == 3 ? fabs(nz) : (R)0;
    sum = a1 + a2 + a3;
    const R inv = sum > (R)0 ? (R)1 / sum : (R)0;
    a1 *= inv;
    a2 *= inv;
    a3 *= inv;
    R t;
    if (a1 > a2) { t = a1; a1 = a2; a2 = t; }
    if (a2 > a3) { t = a2; a2 = a3; a3 = t; }
    if (a1 > a2) { t = a1; a1 = a2; a2 = t; }
    m1 = a1;
    m2 = a2;
    m3 = a3;
  }
  // offset s of the plane n.p = s leaving liquid fraction alpha on the +n
  // side of the cell [-1/2, 1/2]^d (out of line: inlining the several cuts of
  // a thread raised registers and was measured slower)
  __device__ __noinline__ R offset(R alpha) const {
    if (!(sum > (R)0)) return (R)0;
    if (alpha >= (R)1) return (R)-0.5 * sum;
    if (alpha <= (R)0) return (R)0.5 * sum;
    R V = (R)1 - alpha;
    const bool flip = V > (R)0.5;
    if (flip) V = (R)1 - V;
    R a = plic_a3<R>(m1, m2, m3, V);
    if (flip) a = (R)1 - a;
    return a * sum - (R)0.5 * sum;
  }
};

template <int D, class R>
__device__ __forceinline__ R plic_offset(R nx, R ny, R nz, R alpha) {
  return Plic<D, R>(nx, ny, nz).offset(alpha);
}

// Cholesky solve of the k x k symmetric positive definite system A x = b
// (the ridge keeps the least-squares normal matrix definite); the
// reciprocals of the factor's diagonal turn every division into a product
template <class R, int K>
__device__ __forceinline__ bool chol_solve(R (&A)[K][K], R (&b)[K], R (&x)[K]) {
  R il[K];
#pragma unroll
  for (int j = 0; j < K; ++j) {
    R d = A[j][j];
#pragma unroll
    for (int k = 0; k < j; ++k) d -= A[j][k] * A[j][k];
    if (!(d > (R)1e-9)) return false;
    il[j] = rsqrt_r(d);
#pragma unroll
    for (int i = j + 1; i < K; ++i) {
      R v = A[i][j];
#pragma unroll
      for (int k = 0; k < j; ++k) v -= A[i][k] * A[j][k];
      A[i][j] = v * il[j];
    }
  }
  R y[K];
#pragma unroll
  for (int i = 0; i < K; ++i) {
    R v = b[i];
#pragma unroll
    for (int k = 0; k < i; ++k) v -= A[i][k] * y[k];
    y[i] = v * il[i];
  }
#pragma unroll
  for (int i = K - 1; i >= 0; --i) {
    R v = y[i];
#pragma unroll
    for (int k = i + 1; k < K; ++k) v -= A[k][i] * x[k];
    x[i] = v * il[i];
  }
  return true;
}

// ridge added to the diagonal of the least-squares normal equations: point
// sets that cannot resolve every coefficient (next to walls, nearly
// axis-aligned planes) then give a smooth, bounded curvature
constexpr double kLsqRidge = 1e-3;

// sum over the G consecutive lanes of a group (G a power of two <= 32);
// every lane of the warp takes part
template <int G, class R> __device__ __forceinline__ R group_sum(R v) {
#pragma unroll
  for (int o = G / 2; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o, G);
  return v;
}

// GEO_LANES lanes per interface cell (32 / GEO_LANES cells per warp): lane t
// of a cell's group takes the stencil cells t, t + GEO_LANES, ... (27 in 3D,
// 9 in 2D), so the gradient, the PLIC cuts and the least-squares sums are
// spread over the group and reduced in log2(GEO_LANES) shuffles; the first
// lane of each group solves the normal equations and stores the results.
// Eight blocks of 128 threads per SM (64 registers, no spills) were measured
// faster than the six that 80 registers allow.
constexpr int GEO_LANES = 8;

template <int D, class R>
__global__ void __launch_bounds__(128, 8) k_geometry(Params p) {
  constexpr int K = D == 3 ? 5 : 2;
  constexpr int NS = D == 3 ? 27 : 9;
  constexpr int CTR = D == 3 ? 13 : 4;
  constexpr int G = GEO_LANES, CPW = 32 / G, PER = (NS + G - 1) / G;
  const int lane = threadIdx.x & 31, sub = lane / G, t = lane % G;
  const int warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int nwarps = (gridDim.x * blockDim.x) >> 5;
  const int cnt = *p.icount;
  const R *phi = (const R *)p.phi;
  R *kap = (R *)p.kappa, *nr = (R *)p.nrm, *ds = (R *)p.dst;
  // the lane of the group that holds the centre stencil cell
  constexpr int CT = CTR % G, CJ = CTR / G;
  for (int base = warp * CPW; base < cnt; base += nwarps * CPW) {
    const int k = base + sub;
    const bool valid = k < cnt;
    const long long n = valid ? p.ilist[k] : p.ilist[base];
    const Cell c = make_cell(p, n);
    R a[PER];
    int tm[PER];
#pragma unroll
    for (int j = 0; j < PER; ++j) {
      const int q = t + G * j;
      a[j] = 0;
      tm[j] = T_LIQ;
      if (q < NS) {
        const int dx = q % 3 - 1, dy = (q / 3) % 3 - 1, dz = D == 3 ? q / 9 - 1 : 0;
        const long long m = at(p, c, dx, dy, dz);
        // flag and fill level in one round of loads (the fill level of a
        // cell that is not interface is read and unused)
        const uint8_t fm = p.flags[m];
        const R v = phi[m];
        tm[j] = post_type(fm);  // may run while the conversion's marks are replaced
        if (tm[j] == T_LIQ) a[j] = 1;
        else if (tm[j] == T_IFC) a[j] = v < (R)0 ? (R)0 : (v > (R)1 ? (R)1 : v);
      }
    }
    const R ac = __shfl_sync(0xffffffffu, a[CJ], sub * G + CT);
    // Parker-Youngs weighted centred differences
    R gx = 0, gy = 0, gz = 0;
    bool act[PER];
#pragma unroll
    for (int j = 0; j < PER; ++j) {
      const int q = t + G * j;
      act[j] = false;
      if (q >= NS) continue;
      if (tm[j] == T_WALL) a[j] = ac;  // walls repeat the centre value
      act[j] = q != CTR && tm[j] == T_IFC && a[j] > (R)0 && a[j] < (R)1;
      const int dx = q % 3 - 1, dy = (q / 3) % 3 - 1, dz = D == 3 ? q / 9 - 1 : 0;
      const R wz = D == 3 ? (dz == 0 ? (R)2 : (R)1) : (R)1;
      gx += (R)dx * (dy == 0 ? (R)2 : (R)1) * wz * a[j];
      gy += (R)dy * (dx == 0 ? (R)2 : (R)1) * wz * a[j];
      if (D == 3) gz += (R)dz * (dx == 0 ? (R)2 : (R)1) * (dy == 0 ? (R)2 : (R)1) * a[j];
    }
    gx = group_sum<G, R>(gx);
    gy = group_sum<G, R>(gy);
    if (D == 3) gz = group_sum<G, R>(gz);
    const R gn = sqrt(gx * gx + gy * gy + gz * gz);
    const bool flat = !(gn > (R)1e-12);
    const R ign = flat ? (R)0 : (R)1 / gn;
    const R mx = gx * ign, my = gy * ign, mz = gz * ign;
    const Plic<D, R> plic(mx, my, mz);
    // every thread cuts its own stencil cells (and the centre's holder the centre)
    R sj[PER];
#pragma unroll
    for (int j = 0; j < PER; ++j) {
      const int q = t + G * j;
      sj[j] = (!flat && (act[j] || q == CTR)) ? plic.offset(q == CTR ? ac : a[j]) : (R)0;
    }
    const R s0 = __shfl_sync(0xffffffffu, sj[CJ], sub * G + CT);
    // local frame (t1, t2, m)
    R t1x, t1y, t1z, t2x = 0, t2y = 0, t2z = 0;
    if (D == 2) {
      t1x = -my; t1y = mx; t1z = 0;
    } else {
      const R ax = fabs(mx), ay = fabs(my), az = fabs(mz);
      const int kmin = ax <= ay ? (ax <= az ? 0 : 2) : (ay <= az ? 1 : 2);
      const R mk = kmin == 0 ? mx : (kmin == 1 ? my : mz);
      t1x = (kmin == 0 ? (R)1 : (R)0) - mk * mx;
      t1y = (kmin == 1 ? (R)1 : (R)0) - mk * my;
      t1z = (kmin == 2 ? (R)1 : (R)0) - mk * mz;
      const R l2 = t1x * t1x + t1y * t1y + t1z * t1z;
      const R l = l2 > (R)0 ? (R)1 / sqrt(l2) : (R)0;
      t1x *= l; t1y *= l; t1z *= l;
      t2x = my * t1z - mz * t1y;
      t2y = mz * t1x - mx * t1z;
      t2z = mx * t1y - my * t1x;
    }
    // this thread's share of the normal equations of the least-squares
    // paraboloid
    R NA[K][K], Nb[K], N1 = 0, b1 = 0;
#pragma unroll
    for (int i = 0; i < K; ++i) {
      Nb[i] = 0;
#pragma unroll
      for (int jj = 0; jj < K; ++jj) NA[i][jj] = 0;
    }
    int np = 0;
#pragma unroll
    for (int j = 0; j < PER; ++j) {
      if (!act[j]) continue;
      const int q = t + G * j;
      const int dx = q % 3 - 1, dy = (q / 3) % 3 - 1, dz = D == 3 ? q / 9 - 1 : 0;
      const R x = (R)dx * t1x + (R)dy * t1y + (R)dz * t1z;
      const R y = (R)dx * t2x + (R)dy * t2y + (R)dz * t2z;
      const R z = (R)dx * mx + (R)dy * my + (R)dz * mz + sj[j] - s0;
      R ph[K];
      if constexpr (D == 3) {
        ph[0] = x * x; ph[1] = y * y; ph[2] = x * y; ph[3] = x; ph[4] = y;
      } else {
        ph[0] = x * x; ph[1] = x;
      }
#pragma unroll
      for (int i = 0; i < K; ++i) {
#pragma unroll
        for (int jj = 0; jj <= i; ++jj) NA[i][jj] += ph[i] * ph[jj];
        Nb[i] += ph[i] * z;
      }
      const R r2 = x * x + y * y;
      N1 += r2 * r2;
      b1 += r2 * z;
      ++np;
    }
#pragma unroll
    for (int i = 0; i < K; ++i) {
#pragma unroll
      for (int jj = 0; jj <= i; ++jj) NA[i][jj] = group_sum<G, R>(NA[i][jj]);
      Nb[i] = group_sum<G, R>(Nb[i]);
    }
    N1 = group_sum<G, R>(N1);
    b1 = group_sum<G, R>(b1);
#pragma unroll
    for (int o = G / 2; o > 0; o >>= 1) np += __shfl_xor_sync(0xffffffffu, np, o, G);
    if (!valid || t != 0) continue;
    if (flat) {
      kap[n] = 0;
      ds[n] = 0;
      nr[n] = 0;
      nr[p.N + n] = 0;
      nr[2 * p.N + n] = 0;
      continue;
    }
#pragma unroll
    for (int i = 0; i < K; ++i) {
      NA[i][i] += (R)kLsqRidge;
#pragma unroll
      for (int jj = i + 1; jj < K; ++jj) NA[i][jj] = NA[jj][i];
    }
    R kv = 0;
    R beta[K];
    const bool full = np >= (D == 3 ? 5 : 2) && chol_solve<R, K>(NA, Nb, beta);
    if (full) {
      if constexpr (D == 3) {
        const R H = beta[3], I = beta[4];
        const R iq = rsqrt_r((R)1 + H * H + I * I);
        kv = -(((R)1 + I * I) * beta[0] - H * I * beta[2] + ((R)1 + H * H) * beta[1]) * (iq * iq * iq);
      } else {
        const R iq = rsqrt_r((R)1 + beta[1] * beta[1]);
        kv = -beta[0] * (iq * iq * iq);
      }
    } else if (np >= 1) {
      kv = (D == 3 ? (R)-2 : (R)-1) * (b1 / (N1 + (R)kLsqRidge));
    }
    kap[n] = kv < (R)-1 ? (R)-1 : (kv > (R)1 ? (R)1 : kv);
    nr[n] = mx;
    nr[p.N + n] = my;
    nr[2 * p.N + n] = mz;
    ds[n] = s0;
  }
}

// height-function curvature, the second method Sec. 2.2 names (switched on
// by cfg.kappa = 1): heights are the summed fill levels of 7-cell columns
// along the dominant axis of the cell's normal, 3 columns (2D) or 3 x 3
// (3D) around the cell; centred differences give the curvature of the
// height function, halved like the least-squares kappa (a gas disk 1/(2R),
// a gas sphere 1/R).  The summed liquid fraction makes the sign independent
// of the side the liquid is on.  It replaces the least-squares kappa
// wherever no column meets a wall, limited to [-1, 1].  One thread per
// interface cell, after k_geometry (it needs the normal).
template <int D, class R>
__global__ void __launch_bounds__(128) k_hf_kappa(Params p) {
  const int cnt = *p.icount;
  const R *phi = (const R *)p.phi, *nr = (const R *)p.nrm;
  R *kap = (R *)p.kappa;
  FOR_LIST(kk, cnt) {
    const long long n = p.ilist[kk];
    const R m[3] = {nr[n], nr[p.N + n], D == 3 ? nr[2 * p.N + n] : (R)0};
    if (m[0] == (R)0 && m[1] == (R)0 && m[2] == (R)0) continue;
    int d = 0;
#pragma unroll
    for (int q = 1; q < D; ++q)
      if (fabs(m[q]) > fabs(m[d])) d = q;
    const int a = d == 0 ? 1 : 0, b = 3 - d - a;
    const Cell c = make_cell(p, n);
    R ac = phi[n];
    ac = ac < (R)0 ? (R)0 : (ac > (R)1 ? (R)1 : ac);
    R h[3][3];
    bool wall = false;
#pragma unroll
    for (int j = -1; j <= 1; ++j)
#pragma unroll
      for (int i = -1; i <= 1; ++i) {
        R sum = 0;
        h[j + 1][i + 1] = 0;
        if (D == 2 && j != 0) continue;
        for (int k = -3; k <= 3; ++k) {
          int off[3] = {0, 0, 0};
          off[a] = i;
          off[b] = D == 2 ? 0 : j;
          off[d] = k;
          const long long y = at_far(p, c.x + off[0], c.y + off[1], c.z + off[2]);
          const int ty = post_type(p.flags[y]);
          R v;
          if (ty == T_WALL) {
            wall = true;
            v = ac;  // walls repeat the centre value
          } else if (ty == T_LIQ) {
            v = 1;
          } else if (ty == T_IFC) {
            v = phi[y];
            v = v < (R)0 ? (R)0 : (v > (R)1 ? (R)1 : v);
          } else {
            v = 0;
          }
          sum += v;
        }
        h[j + 1][i + 1] = sum;
      }
    if (wall) continue;
    R kv;
    if (D == 2) {
      const R ha = (R)0.5 * (h[1][2] - h[1][0]);
      const R haa = h[1][2] - (R)2 * h[1][1] + h[1][0];
      kv = haa / ((R)2 * pow((R)1 + ha * ha, (R)1.5));
    } else {
      const R ha = (R)0.5 * (h[1][2] - h[1][0]), hb = (R)0.5 * (h[2][1] - h[0][1]);
      const R haa = h[1][2] - (R)2 * h[1][1] + h[1][0], hbb = h[2][1] - (R)2 * h[1][1] + h[0][1];
      const R hab = (R)0.25 * (h[2][2] - h[0][2] - h[2][0] + h[0][0]);
      kv = (haa * ((R)1 + hb * hb) + hbb * ((R)1 + ha * ha) - (R)2 * hab * ha * hb) /
           ((R)2 * pow((R)1 + ha * ha + hb * hb, (R)1.5));
    }
    kap[n] = kv < (R)-1 ? (R)-1 : (kv > (R)1 ? (R)1 : kv);
  }
}

// lattice index of (x, y, z) a few cells outside the lattice at most, wrapped
__device__ __forceinline__ int wrap_near(const Params &p, int x, int y, int z) {
  while (x < 0) x += p.nx;
  while (x >= p.nx) x -= p.nx;
  while (y < 0) y += p.ny;
  while (y >= p.ny) y -= p.ny;
  while (z < 0) z += p.nz;
  while (z >= p.nz) z -= p.nz;
  return x + p.nx * (y + p.ny * z);
}

// The march visits cells fixed by the normal alone, so the cells of RAY_CHUNK
// consecutive boundary crossings are found first and their labels and flags
// loaded together; then the crossings are examined in order.
constexpr int RAY_CHUNK = 4;

template <int D, class R>
__global__ void k_disjoining(Params p) {
  const int cnt = *p.icount;
  R *Pi = (R *)p.Pi;
  const R *nr = (const R *)p.nrm, *ds = (const R *)p.dst;
  FOR_LIST(kk, cnt) {
    const long long n = p.ilist[kk];
    const int b = p.label_new[n];
    const R dir[3] = {nr[n], nr[p.N + n], nr[2 * p.N + n]};
    if (p.pf.k_pi == 0.f || b < 0 || (dir[0] == (R)0 && dir[1] == (R)0 && dir[2] == (R)0)) {
      Pi[n] = 0;
      continue;
    }
    const Cell c = make_cell(p, n);
    R tmax[3], tdel[3];
    int step[3], off[3] = {0, 0, 0};
    for (int d = 0; d < 3; ++d) {
      tmax[d] = dir[d] != (R)0 ? fabs((R)0.5 / dir[d]) : (R)INFINITY;
      tdel[d] = (R)2 * tmax[d];
      step[d] = dir[d] >= (R)0 ? 1 : -1;
    }
    R dist = -1;
    const R s0 = ds[n];
    // axes whose next boundary lies at the same ray parameter (within a
    // relative 1e-9, 1e-5 in single precision) are crossed together, so that
    // round-off in a normal with equal components cannot split a diagonal step
    const R tie = (R)1 + (R)(sizeof(R) == 4 ? 1e-5 : 1e-9);
    bool done = false;
    for (int it0 = 1; it0 <= p.ray_steps && !done; it0 += RAY_CHUNK) {
      const int nst = min(RAY_CHUNK, p.ray_steps - it0 + 1);
      int yy[RAY_CHUNK], ox[RAY_CHUNK], oy[RAY_CHUNK], oz[RAY_CHUNK];
      R tms[RAY_CHUNK];
#pragma unroll
      for (int j = 0; j < RAY_CHUNK; ++j) {
        yy[j] = (int)n;
        ox[j] = oy[j] = oz[j] = 0;
        tms[j] = 0;
        if (j >= nst) continue;
        const R tm = fmin(tmax[0], fmin(tmax[1], tmax[2]));
        for (int d = 0; d < 3; ++d)
          if (tmax[d] <= tm * tie) {
            tmax[d] += tdel[d];
            off[d] += step[d];
          }
        tms[j] = tm;
        ox[j] = off[0];
        oy[j] = off[1];
        oz[j] = off[2];
        yy[j] = wrap_near(p, c.x + off[0], c.y + off[1], c.z + off[2]);
      }
      int ly[RAY_CHUNK];
      uint8_t fy[RAY_CHUNK];
#pragma unroll
      for (int j = 0; j < RAY_CHUNK; ++j) {
        ly[j] = j < nst ? p.label_new[yy[j]] : b;
        fy[j] = j < nst ? p.flags[yy[j]] : (uint8_t)T_LIQ;
      }
#pragma unroll
      for (int j = 0; j < RAY_CHUNK; ++j) {
        if (done || j >= nst || ly[j] == b) continue;
        const int ty = post_type(fy[j]);
        if (ty == T_WALL) {
          done = true;
        } else if ((ty == T_IFC || ty == T_GAS) && ly[j] >= 0) {
          const int y = yy[j];
          const R ny0 = nr[y], ny1 = nr[p.N + y], ny2 = nr[2 * p.N + y];
          const R den = ny0 * dir[0] + ny1 * dir[1] + ny2 * dir[2];
          if (ty == T_IFC && den < (R)-1e-6) {
            const R ncy = ny0 * (R)ox[j] + ny1 * (R)oy[j] + ny2 * (R)oz[j];
            dist = (ds[y] + ncy) / den - s0;
          } else {
            dist = tms[j] - s0;
          }
          if (dist < (R)0) dist = 0;
          done = true;
        }
      }
    }
    Pi[n] = (dist >= (R)0 && dist < PV(R, d_max)) ? PV(R, k_pi) * (PV(R, d_max) - dist) : (R)0;
  }
}

}  // namespace lbf

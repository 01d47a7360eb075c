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
// boundary by cell boundary (Algorithm 1, ties step diagonally), until an
// interface or gas cell of another bubble is met; d is the distance from this
// cell's plane to the other cell's plane along the ray (or to where the ray
// enters it when that plane does not face the ray); Pi = k_Pi (d_max - d)
// for d < d_max.
#pragma once
#include "lbf_common.cuh"

namespace lbf {

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
    const R th = acos(arg) / (R)3;
    const R twopi3 = (R)2.0943951023931954923;
    for (int k = 0; k < 3; ++k) consider(r * cos(th - twopi3 * (R)k) - b3);
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

// offset s of the plane n.p = s (n unit) leaving liquid fraction alpha on
// the +n side of the cell [-1/2, 1/2]^d
template <int D, class R>
__device__ __forceinline__ R plic_offset(R nx, R ny, R nz, R alpha) {
  R a1 = fabs(nx), a2 = fabs(ny), a3 = D == 3 ? fabs(nz) : (R)0;
  const R sum = a1 + a2 + a3;
  if (!(sum > (R)0)) return (R)0;
  if (alpha >= (R)1) return (R)-0.5 * sum;
  if (alpha <= (R)0) return (R)0.5 * sum;
  a1 /= sum;
  a2 /= sum;
  a3 /= sum;
  // sort ascending
  R t;
  if (a1 > a2) { t = a1; a1 = a2; a2 = t; }
  if (a2 > a3) { t = a2; a2 = a3; a3 = t; }
  if (a1 > a2) { t = a1; a1 = a2; a2 = t; }
  R V = (R)1 - alpha;
  const bool flip = V > (R)0.5;
  if (flip) V = (R)1 - V;
  R a = plic_a3<R>(a1, a2, a3, V);
  if (flip) a = (R)1 - a;
  return a * sum - (R)0.5 * sum;
}

// k x k Gaussian elimination with partial pivoting (A, b destroyed)
template <class R, int K>
__device__ __forceinline__ bool solve_small(R (&A)[K][K], R (&b)[K], R (&x)[K]) {
#pragma unroll
  for (int i = 0; i < K; ++i) {
    int piv = i;
    R best = fabs(A[i][i]);
#pragma unroll
    for (int r = i + 1; r < K; ++r)
      if (fabs(A[r][i]) > best) {
        best = fabs(A[r][i]);
        piv = r;
      }
    if (best < (R)1e-9) return false;
    if (piv != i) {
#pragma unroll
      for (int j = 0; j < K; ++j) {
        const R tt = A[i][j];
        A[i][j] = A[piv][j];
        A[piv][j] = tt;
      }
      const R tt = b[i];
      b[i] = b[piv];
      b[piv] = tt;
    }
#pragma unroll
    for (int r = i + 1; r < K; ++r) {
      const R f = A[r][i] / A[i][i];
#pragma unroll
      for (int j = i; j < K; ++j) A[r][j] -= f * A[i][j];
      b[r] -= f * b[i];
    }
  }
#pragma unroll
  for (int i = K - 1; i >= 0; --i) {
    R acc = b[i];
#pragma unroll
    for (int j = i + 1; j < K; ++j) acc -= A[i][j] * x[j];
    x[i] = acc / A[i][i];
  }
  return true;
}

// ridge added to the diagonal of the least-squares normal equations: point
// sets that cannot resolve every coefficient (next to walls, nearly
// axis-aligned planes) then give a smooth, bounded curvature
constexpr double kLsqRidge = 1e-3;

template <int D, class R>
__global__ void __launch_bounds__(128) k_geometry(Params p) {
  const int cnt = *p.icount;
  FOR_LIST(kk, cnt) {
  const long long n = p.ilist[kk];
  const Cell c = make_cell(p, n);
  const R *phi = (const R *)p.phi;
  R *kap = (R *)p.kappa, *nr = (R *)p.nrm, *ds = (R *)p.dst;
  constexpr int ZR = D == 3 ? 1 : 0;
  R A[3][3][3];
  unsigned act = 0;
  const R ac = phi[n] < (R)0 ? (R)0 : (phi[n] > (R)1 ? (R)1 : phi[n]);
  for (int dz = -ZR; dz <= ZR; ++dz)
    for (int dy = -1; dy <= 1; ++dy)
      for (int dx = -1; dx <= 1; ++dx) {
        const long long m = at(p, c, dx, dy, dz);
        const int tm = ftype(p.flags[m]);
        R a;
        if (tm == T_LIQ) a = 1;
        else if (tm == T_GAS) a = 0;
        else if (tm == T_WALL) a = ac;
        else {
          a = phi[m];
          a = a < (R)0 ? (R)0 : (a > (R)1 ? (R)1 : a);
        }
        A[dz + 1][dy + 1][dx + 1] = a;
        if (tm == T_IFC && a > (R)0 && a < (R)1) act |= 1u << ((dz + 1) * 9 + (dy + 1) * 3 + dx + 1);
      }
  R gx = 0, gy = 0, gz = 0;
  for (int dz = -ZR; dz <= ZR; ++dz)
    for (int dy = -1; dy <= 1; ++dy)
      for (int dx = -1; dx <= 1; ++dx) {
        const R v = A[dz + 1][dy + 1][dx + 1];
        const R wx = (dy == 0 ? (R)2 : (R)1) * (D == 3 ? (dz == 0 ? (R)2 : (R)1) : (R)1);
        const R wy = (dx == 0 ? (R)2 : (R)1) * (D == 3 ? (dz == 0 ? (R)2 : (R)1) : (R)1);
        const R wz = (dx == 0 ? (R)2 : (R)1) * (dy == 0 ? (R)2 : (R)1);
        gx += (R)dx * wx * v;
        gy += (R)dy * wy * v;
        if (D == 3) gz += (R)dz * wz * v;
      }
  const R gn = sqrt(gx * gx + gy * gy + gz * gz);
  if (!(gn > (R)1e-12)) {
    kap[n] = 0;
    ds[n] = 0;
    nr[n] = 0;
    nr[p.N + n] = 0;
    nr[2 * p.N + n] = 0;
    continue;
  }
  const R mx = gx / gn, my = gy / gn, mz = gz / gn;
  const R s0 = plic_offset<D, R>(mx, my, mz, ac);
  nr[n] = mx;
  nr[p.N + n] = my;
  nr[2 * p.N + n] = mz;
  ds[n] = s0;
  // local frame
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
    const R l = sqrt(t1x * t1x + t1y * t1y + t1z * t1z);
    t1x /= l; t1y /= l; t1z /= l;
    t2x = my * t1z - mz * t1y;
    t2y = mz * t1x - mx * t1z;
    t2z = mx * t1y - my * t1x;
  }
  // normal equations of the least-squares fit
  constexpr int K = D == 3 ? 5 : 2;
  R NA[K][K], Nb[K], N1 = 0, b1 = 0;
  for (int i = 0; i < K; ++i) {
    Nb[i] = 0;
    for (int j = 0; j < K; ++j) NA[i][j] = 0;
  }
  int np = 0;
  for (int dz = -ZR; dz <= ZR; ++dz)
    for (int dy = -1; dy <= 1; ++dy)
      for (int dx = -1; dx <= 1; ++dx) {
        if (dx == 0 && dy == 0 && dz == 0) continue;
        if (!(act & (1u << ((dz + 1) * 9 + (dy + 1) * 3 + dx + 1)))) continue;
        const R sj = plic_offset<D, R>(mx, my, mz, A[dz + 1][dy + 1][dx + 1]);
        const R x = (R)dx * t1x + (R)dy * t1y + (R)dz * t1z;
        const R y = (R)dx * t2x + (R)dy * t2y + (R)dz * t2z;
        const R z = (R)dx * mx + (R)dy * my + (R)dz * mz + sj - s0;
        R ph[K];
        if constexpr (D == 3) {
          ph[0] = x * x; ph[1] = y * y; ph[2] = x * y; ph[3] = x; ph[4] = y;
        } else {
          ph[0] = x * x; ph[1] = x;
        }
#pragma unroll
        for (int i = 0; i < K; ++i) {
#pragma unroll
          for (int j = 0; j < K; ++j) NA[i][j] += ph[i] * ph[j];
          Nb[i] += ph[i] * z;
        }
        const R r2 = x * x + y * y;
        N1 += r2 * r2;
        b1 += r2 * z;
        ++np;
      }
  R kv = 0;
  R beta[K];
#pragma unroll
  for (int i = 0; i < K; ++i) NA[i][i] += (R)kLsqRidge;
  const bool full = np >= (D == 3 ? 5 : 2) && solve_small<R, K>(NA, Nb, beta);
  if (full) {
    if constexpr (D == 3) {
      const R H = beta[3], I = beta[4];
      kv = -(((R)1 + I * I) * beta[0] - H * I * beta[2] + ((R)1 + H * H) * beta[1]) /
           pow((R)1 + H * H + I * I, (R)1.5);
    } else {
      kv = -beta[0] / pow((R)1 + beta[1] * beta[1], (R)1.5);
    }
  } else if (np >= 1) {
    kv = (D == 3 ? (R)-2 : (R)-1) * (b1 / (N1 + (R)kLsqRidge));
  }
  kap[n] = kv < (R)-1 ? (R)-1 : (kv > (R)1 ? (R)1 : kv);
  }
}

template <int D, class R>
__global__ void k_disjoining(Params p) {
  const int cnt = *p.icount;
  FOR_LIST(kk, cnt) {
  const long long n = p.ilist[kk];
  R *Pi = (R *)p.Pi;
  const int b = p.label_new[n];
  const R *nr = (const R *)p.nrm, *ds = (const R *)p.dst;
  const R dir[3] = {nr[n], nr[p.N + n], nr[2 * p.N + n]};
  if (p.k_pi == 0.0 || b < 0 || (dir[0] == (R)0 && dir[1] == (R)0 && dir[2] == (R)0)) {
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
  for (int it = 1; it <= p.ray_steps; ++it) {
    const R tm = fmin(tmax[0], fmin(tmax[1], tmax[2]));
    for (int d = 0; d < 3; ++d)
      if (tmax[d] == tm) {
        tmax[d] += tdel[d];
        off[d] += step[d];
      }
    const long long y = at_far(p, c.x + off[0], c.y + off[1], c.z + off[2]);
    const int ly = p.label_new[y];
    if (ly == b) continue;
    const int ty = ftype(p.flags[y]);
    if (ty == T_WALL) break;
    if ((ty == T_IFC || ty == T_GAS) && ly >= 0) {
      const R ny0 = nr[y], ny1 = nr[p.N + y], ny2 = nr[2 * p.N + y];
      const R den = ny0 * dir[0] + ny1 * dir[1] + ny2 * dir[2];
      if (ty == T_IFC && den < (R)-1e-6) {
        const R ncy = ny0 * (R)off[0] + ny1 * (R)off[1] + ny2 * (R)off[2];
        dist = (ds[y] + ncy) / den - s0;
      } else {
        dist = tm - s0;
      }
      if (dist < (R)0) dist = 0;
      break;
    }
  }
  Pi[n] = (dist >= (R)0 && dist < (R)p.d_max) ? (R)p.k_pi * ((R)p.d_max - dist) : (R)0;
  }
}

}  // namespace lbf

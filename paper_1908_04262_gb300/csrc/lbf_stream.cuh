// lbf_stream.cuh -- the per-step lattice sweep.
//
// k_exchange (interface cells only) runs first: it reads the cell's own
// outgoing populations of the last step and the incoming ones from liquid
// and interface neighbours while no slot is being rewritten, and applies the
// mass exchange of Sec. 2.1 Eq. massexchange (Theta = 1 towards liquid,
// (alpha_x + alpha_nb)/2 towards interface, 0 towards gas and walls).  It
// also keeps the cell's last velocity u_I for the reconstruction.
//
// The sweep then streams in place (Sec. 2 Eq. streamingstep), bounces back
// at walls, relaxes with BGK plus Guo forcing (Sec. 2 Eq.
// collision/equilibrium) at a per-cell tau from the local shear rate
// (Sec. 2.3 Eq. tau/carreauTau) and advances the dissolved gas on D2Q5/D3Q7
// (Sec. 3.1 Eq. diffusion), in two kernels over disjoint sets of cells:
//   k_stream_liquid     every liquid cell (row grid); it needs nothing that
//                       the labelling, the bubble update, the geometry or
//                       the disjoining pressure of the last step produce
//   k_stream_interface  every interface cell of the step's list: it also
//                       rebuilds populations arriving from gas cells
//                       (Sec. 2.2 Eq. reconstruct with the gas density of
//                       Eq. rhob / rhobplusdisjoining), updates the fill
//                       level (Sec. 2.1 Eq. alpha), marks cells that fill or
//                       empty, applies Henry's law at gas links (Sec. 3.2
//                       Eq. henryslaw / reconstructdiffusion) and adds the
//                       cell's gas current (Sec. 3.1 Eq. gascurrent) to its
//                       bubble.
// In the AA pattern every cell reads and writes only its own set of slots,
// so the two kernels commute; the liquid one may run as soon as the mass
// exchange of its step has read the slots it rewrites.
#pragma once
#include "lbf_common.cuh"

namespace lbf {

template <class R> __device__ __forceinline__ R warp_sum_r(R v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

template <class R> struct Prec;
template <> struct Prec<double> { static constexpr double tol = 1e-13; static constexpr int iters = 60; };
template <> struct Prec<float> { static constexpr float tol = 2e-6f; static constexpr int iters = 24; };

// tau of the rheology model at shear rate gd, and d tau / d gd
template <class R> __device__ __forceinline__ R tau_model(const Params &p, R gd, R &dtau) {
  if (p.rheo == 1) {
    const R t = (R)3 * PV(R, rk) * pow(gd, PV(R, rn) - (R)1);
    dtau = t * (PV(R, rn) - (R)1) / gd;
    return (R)0.5 + t;
  }
  const R lg = pow(PV(R, rlam) * gd, PV(R, ra));
  const R base = (R)1 + lg;
  const R fac = pow(base, (PV(R, rn) - (R)1) / PV(R, ra));
  dtau = (R)(p.tau0 - p.tau_inf) * fac * (PV(R, rn) - (R)1) / base * lg / gd;
  return PV(R, tau_inf) + (R)(p.tau0 - p.tau_inf) * fac;
}

// Sec. 2.3: tau solves tau = tau_model(A / tau) (shear rate A / tau from the
// non-equilibrium stress), clamped to [tau_min, tau_max].
// Power law: with g = A / tau the equation reads g/2 + 3 k g^n = A; its root
// lies in [min(A, (A/6k)^(1/n)), min(2A, (A/3k)^(1/n))] (each term is below A
// at the lower end and at most A at the upper end), a bracket within a
// factor 2^(1/n); Newton inside it (monotone from the left for n < 1, from
// the right for n > 1).  Carreau-Yasuda: safeguarded Newton on tau.
template <class R> __device__ __forceinline__ R solve_tau(const Params &p, R A) {
  const R lo = PV(R, tau_min), hi = PV(R, tau_max);
  if (p.rheo == 1) {
    const R n = PV(R, rn), k3 = (R)3 * PV(R, rk);
    if (!(A > (R)0)) return n < (R)1 ? hi : lo;
    if (n == (R)1) {
      const R t = (R)0.5 + k3;
      return t < lo ? lo : (t > hi ? hi : t);
    }
    const R inv = (R)1 / n;
    R gl = fmin(A, pow(A / ((R)2 * k3), inv));
    R gu = fmin((R)2 * A, pow(A / k3, inv));
    if (!(gl > (R)0)) return n < (R)1 ? hi : lo;  // shear rate below range
    R g = n < (R)1 ? gl : gu;
    for (int it = 0; it < Prec<R>::iters; ++it) {
      const R gp = pow(g, n - (R)1);  // g^(n-1)
      const R fval = (R)0.5 * g + k3 * gp * g - A;
      const R fder = (R)0.5 + n * k3 * gp;
      R gn = g - fval / fder;
      if (!(gn >= gl && gn <= gu)) gn = (R)0.5 * (gl + gu);
      if (fval < (R)0) gl = g; else gu = g;
      const R step = gn - g;
      g = gn;
      if (fabs(step) <= Prec<R>::tol * g) break;
    }
    const R t = A / g;
    return t < lo ? lo : (t > hi ? hi : t);
  }
  R d;
  R l = lo, h = hi;
  if (!(h - tau_model<R>(p, A / h, d) > (R)0)) return h;
  if (!(l - tau_model<R>(p, A / l, d) < (R)0)) return l;
  // Newton from the upper end of the bracket, falling back to bisection
  // whenever a step leaves the bracket; h(t) = t - tau_model(A / t)
  R t = h;
  for (int it = 0; it < Prec<R>::iters; ++it) {
    R dm;
    const R hv = t - tau_model<R>(p, A / t, dm);
    if (hv > (R)0) h = t; else l = t;
    const R deriv = (R)1 + dm * A / (t * t);
    R tn = t - hv / deriv;
    if (!(tn > l && tn < h)) tn = (R)0.5 * (l + h);
    const R step = tn - t;
    t = tn;
    if (fabs(step) <= Prec<R>::tol * t) break;
  }
  return t;
}

// one warp per segment of interface cells, one lane per cell (loads along x
// coalesce like the lattice sweep's)
template <int D, class S, int PAR, bool WALLED = false>
__global__ void __launch_bounds__(128) k_exchange(Params p) {
  using R = typename ST<S>::R;
  constexpr int Q = Lat<D>::Q;
  const int lane = threadIdx.x & 31;
  const int warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int nwarps = (gridDim.x * blockDim.x) >> 5;
  const int cnt = *p.segcount;
  const S *f = (const S *)p.f;
  R *M = (R *)p.M;
  const R *phi = (const R *)p.phi;
  // the step's first kernel: the interface sweep lists marked cells afresh
  if (blockIdx.x == 0 && threadIdx.x == 0) *p.mcount = 0;
  for (int k = warp; k < cnt; k += nwarps) {
    Cell c;
    if (!(WALLED ? seg_cell_walled(p, p.seglist[k], lane, c) : seg_cell(p, p.seglist[k], lane, c))) continue;
    const int n = c.n;
    // types through the last conversion's marks: the exchange may run while
    // that conversion still writes the new types
    if (post_type(p.flags[n]) != T_IFC) continue;
    const R phn = phi[n];
    // every load issued at once (none waits for a neighbour's type; the
    // slots and fill levels of gas and wall neighbours are read and unused)
    R fo[Q], fin[Q], phm[Q];
    uint8_t fn[Q];
#pragma unroll
    for (int i = 0; i < Q; ++i) {
      fo[i] = ld(plane(f, p, dir_out<D>(i, PAR)), cell_out<D>(p, c, i, PAR), fshift<S, D>(p, i));
      if (i > 0) {
        const int m = nb<D>(p, c, i);
        fn[i] = p.flags[m];
        // arriving along opp(i) from m: the slot holding m's outgoing f_opp(i)
        fin[i] = ld(plane(f, p, dir_in<D>(opp(i), PAR)), cell_in<D>(p, c, opp(i), PAR), fshift<S, D>(p, opp(i)));
        phm[i] = phi[m];
      }
    }
    R rho = 0, jx = 0, jy = 0, jz = 0, dM = 0;
#pragma unroll
    for (int i = 0; i < Q; ++i) {
      rho += fo[i];
      jx += fo[i] * (R)Lat<D>::cx(i);
      jy += fo[i] * (R)Lat<D>::cy(i);
      jz += fo[i] * (R)Lat<D>::cz(i);
      if (i > 0) {
        const int tn = post_type(fn[i]);
        if (tn == T_LIQ || tn == T_IFC)
          dM += tn == T_LIQ ? fin[i] - fo[i] : (R)0.5 * (phn + phm[i]) * (fin[i] - fo[i]);
      }
    }
    R *uI = (R *)p.uI;
    const R irho = (R)1 / rho;
    uI[n] = (jx - (R)0.5 * rho * PV(R, ax)) * irho;
    uI[p.N + n] = (jy - (R)0.5 * rho * PV(R, ay)) * irho;
    uI[2 * p.N + n] = (jz - (R)0.5 * rho * PV(R, az)) * irho;
    M[n] = M[n] + dM;
  }
}

template <class R> struct SweepOcc;
template <> struct SweepOcc<double> { static constexpr int blocks = 3; };
template <> struct SweepOcc<float> { static constexpr int blocks = 8; };

// 1 / tau(A) of the single-precision forms: linear interpolation in ln A
// of a table built on the host by bisection (constant beyond its ends)
__device__ __forceinline__ float om_lookup(const Params &p, float A) {
  const float x = (__logf(fmaxf(A, 1e-30f)) - p.tab_lnA0) * p.tab_inv_dlnA;
  if (!(x > 0.f)) return __ldg(p.om_tab);
  if (x >= (float)(p.tab_n - 1)) return __ldg(p.om_tab + p.tab_n - 1);
  const int k = (int)x;
  const float fr = x - (float)k;
  const float a = __ldg(p.om_tab + k), b = __ldg(p.om_tab + k + 1);
  return a + fr * (b - a);
}
template <class R> __device__ __forceinline__ R model_om(const Params &p, R A) {
  if constexpr (sizeof(R) == 4)
    return om_lookup(p, A);
  else
    return (R)1 / solve_tau<R>(p, A);
}

// Sec. 2.3: local relaxation rate 1 / tau.  The non-equilibrium stress is the raw
// second moment minus its equilibrium value rho (u u + cs^2 I) (identical
// to sum e e (f - f_eq) for the second-order equilibrium).
template <int D, class R>
__device__ __forceinline__ R local_om(const Params &p, const R *fi, R rho, R irho, R ux, R uy, R uz) {
  if (p.rheo == 0) return PV(R, om);
  // opposite directions (i, i + 1) have the same e e: one sum per pair
  R mxx = 0, myy = 0, mzz = 0, mxy = 0, mxz = 0, myz = 0;
#pragma unroll
  for (int i = 1; i < Lat<D>::Q; i += 2) {
    const R s = fi[i] + fi[i + 1];
    const int ex = Lat<D>::cx(i), ey = Lat<D>::cy(i), ez = Lat<D>::cz(i);
    if (ex) mxx += s;
    if (ey) myy += s;
    if (ez) mzz += s;
    if (ex * ey > 0) mxy += s;
    if (ex * ey < 0) mxy -= s;
    if (ex * ez > 0) mxz += s;
    if (ex * ez < 0) mxz -= s;
    if (ey * ez > 0) myz += s;
    if (ey * ez < 0) myz -= s;
  }
  const R third = rho / (R)3;
  const R pxx = mxx - rho * ux * ux - third, pyy = myy - rho * uy * uy - third;
  const R pzz = D == 3 ? mzz - rho * uz * uz - third : (R)0;
  const R pxy = mxy - rho * ux * uy, pxz = mxz - rho * ux * uz, pyz = myz - rho * uy * uz;
  const R nrm2 = pxx * pxx + pyy * pyy + pzz * pzz + (R)2 * (pxy * pxy + pxz * pxz + pyz * pyz);
  // A = |Pi_neq| / (sqrt(2) rho c_s^2) with c_s^2 = 1/3
  return model_om<R>(p, sqrt(nrm2) * ((R)2.1213203435596424 * irho));
}

// The multiple-relaxation-time collision (Sec. 2 names it beside BGK and
// TRT) on the orthogonal moment basis of Lallemand and Luo (D2Q9) and
// d'Humieres et al. (D3Q19).  It is computed as the TRT collision (every
// even moment at the stress rate, every odd one at the energy-flux rate)
// plus a correction on each basis vector b whose rate s_b differs from its
// parity's TRT rate s_t:  f -= (s_b - s_t) (b.h / b.b) b  with
// h = f - f_eq + F/2 (F the Guo source), since both the relaxation and the
// source scaling (1 - s/2) act moment by moment.  The corrected vectors are
// the energy e and energy square eps (even), and in 3D the fourth-order
// anisotropic pi_xx, pi_ww (even) and the third-order m_x, m_y, m_z (odd).
template <int D> struct MrtBasis {
  static constexpr int NE = D == 3 ? 4 : 2;  // even vectors: e, eps[, pi_xx, pi_ww]
  static constexpr int NO = D == 3 ? 3 : 0;  // odd vectors: [m_x, m_y, m_z]
  // vector k (even ones first) at direction i
  __host__ __device__ static constexpr int val(int k, int i) {
    const int x = Lat<D>::cx(i), y = Lat<D>::cy(i), z = Lat<D>::cz(i);
    const int c2 = x * x + y * y + z * z;
    if (D == 2) return k == 0 ? 3 * c2 - 4 : (9 * c2 * c2 - 21 * c2 + 8) / 2;
    switch (k) {
      case 0: return 19 * c2 - 30;
      case 1: return (21 * c2 * c2 - 53 * c2 + 24) / 2;
      case 2: return (3 * c2 - 5) * (3 * x * x - c2);
      case 3: return (3 * c2 - 5) * (y * y - z * z);
      case 4: return (y * y - z * z) * x;
      case 5: return (z * z - x * x) * y;
      default: return (x * x - y * y) * z;
    }
  }
  __host__ __device__ static constexpr int norm2(int k) {
    int s = 0;
    for (int i = 0; i < Lat<D>::Q; ++i) s += val(k, i) * val(k, i);
    return s;
  }
};

// relaxation with Guo forcing of one cell (COLL 0 BGK, 1 two relaxation
// times, 2 multiple relaxation times), written to the outgoing slots
template <int D, class S, int PAR, int COLL>
__device__ __forceinline__ void relax_store(const Params &p, const Cell &c, long long n, S *f, const typename ST<S>::R *fi,
                                            typename ST<S>::R rho, typename ST<S>::R ux, typename ST<S>::R uy,
                                            typename ST<S>::R uz, typename ST<S>::R om) {
  using R = typename ST<S>::R;
  constexpr int Q = Lat<D>::Q;
  const R base = (R)1 - (ux * ux + uy * uy + uz * uz) * (R)1.5;
  if constexpr (COLL == 2) {
    using B = MrtBasis<D>;
    constexpr int NP = (Q - 1) / 2;
    const R tau = (R)1 / om;
    const R om_m = (R)1 / ((R)0.5 + PV(R, trt_magic) / (tau - (R)0.5));
    const R ax = p.has_force ? PV(R, ax) : (R)0, ay = p.has_force ? PV(R, ay) : (R)0,
            az = p.has_force ? PV(R, az) : (R)0;
    const R ua = ux * ax + uy * ay + uz * az;
    const R ge = ((R)1 - (R)0.5 * om) * rho, go = ((R)1 - (R)0.5 * om_m) * rho;
    // the TRT values (even part ev, odd part od of each pair) and h
    const R fe0 = (R)Lat<D>::w(0) * rho * base;
    const R F0 = (R)Lat<D>::w(0) * rho * (R)-3 * ua;
    R v0 = fi[0] - (fi[0] - fe0) * om + ((R)1 - (R)0.5 * om) * F0;
    const R h0 = fi[0] - fe0 + (R)0.5 * F0;
    R ev[NP], od[NP], he[NP], ho[NP];
#pragma unroll
    for (int j = 0; j < NP; ++j) {
      const int i = 2 * j + 1, k = i + 1;
      const R w = (R)Lat<D>::w(i);
      const R eu = (R)Lat<D>::cx(i) * ux + (R)Lat<D>::cy(i) * uy + (R)Lat<D>::cz(i) * uz;
      const R ea = (R)Lat<D>::cx(i) * ax + (R)Lat<D>::cy(i) * ay + (R)Lat<D>::cz(i) * az;
      const R fe_even = w * rho * (base + (R)4.5 * eu * eu), fe_odd = w * rho * (R)3 * eu;
      const R f_even = (R)0.5 * (fi[i] + fi[k]), f_odd = (R)0.5 * (fi[i] - fi[k]);
      const R Fe = w * ((R)9 * eu * ea - (R)3 * ua), Fo = w * (R)3 * ea;  // per unit rho
      ev[j] = f_even - (f_even - fe_even) * om + ge * Fe;
      od[j] = f_odd - (f_odd - fe_odd) * om_m + go * Fo;
      he[j] = f_even - fe_even + (R)0.5 * rho * Fe;
      ho[j] = f_odd - fe_odd + (R)0.5 * rho * Fo;
    }
    // rates of the corrected vectors: 0 in the configuration follows the
    // parity's TRT rate (no correction)
    const R se = PV(R, mrt_se) > (R)0 ? PV(R, mrt_se) : om;
    const R seps = PV(R, mrt_seps) > (R)0 ? PV(R, mrt_seps) : om;
    const R spi = PV(R, mrt_spi) > (R)0 ? PV(R, mrt_spi) : om;
    const R sm = PV(R, mrt_sm) > (R)0 ? PV(R, mrt_sm) : om_m;
    R cf[B::NE + B::NO];
#pragma unroll
    for (int k = 0; k < B::NE + B::NO; ++k) {
      const bool even = k < B::NE;
      // b.h: the rest direction and both members of each pair (an even
      // vector takes h_i + h_opp = 2 he, an odd one h_i - h_opp = 2 ho)
      R d = even ? (R)B::val(k, 0) * h0 : (R)0;
#pragma unroll
      for (int j = 0; j < NP; ++j) {
        const int i = 2 * j + 1;
        if (B::val(k, i) != 0) d += (R)(2 * B::val(k, i)) * (even ? he[j] : ho[j]);
      }
      const R s_b = k == 0 ? se : (k == 1 ? seps : (even ? spi : sm));
      const R s_t = even ? om : om_m;
      cf[k] = (s_b - s_t) * d * ((R)1 / (R)B::norm2(k));
    }
#pragma unroll
    for (int k = 0; k < B::NE; ++k) v0 -= cf[k] * (R)B::val(k, 0);
    st(plane(f, p, dir_out<D>(0, 1 - PAR)), cell_out<D>(p, c, 0, 1 - PAR), v0, fshift<S, D>(p, 0));
#pragma unroll
    for (int j = 0; j < NP; ++j) {
      const int i = 2 * j + 1, k = i + 1;
      R e_ = ev[j], o_ = od[j];
#pragma unroll
      for (int b = 0; b < B::NE + B::NO; ++b) {
        if (B::val(b, i) == 0) continue;
        if (b < B::NE)
          e_ -= cf[b] * (R)B::val(b, i);
        else
          o_ -= cf[b] * (R)B::val(b, i);
      }
      st(plane(f, p, dir_out<D>(i, 1 - PAR)), cell_out<D>(p, c, i, 1 - PAR), e_ + o_, fshift<S, D>(p, i));
      st(plane(f, p, dir_out<D>(k, 1 - PAR)), cell_out<D>(p, c, k, 1 - PAR), e_ - o_, fshift<S, D>(p, k));
    }
    return;
  }
  if constexpr (COLL == 1) {
    // two relaxation times: per pair (i, opp(i) = i + 1) the even part of
    // f - f_eq relaxes at om, the odd part at om_m with
    // (tau - 1/2)(tau_m - 1/2) = trt_magic; the Guo source
    // w_i rho [3 (e_i - u).a + 9 (e_i.u)(e_i.a)] splits alike (even part
    // w_i rho (9 (e.u)(e.a) - 3 u.a), odd part 3 w_i rho e.a), each scaled by
    // 1 - om/2 or 1 - om_m/2
    const R tau = (R)1 / om;
    const R om_m = (R)1 / ((R)0.5 + PV(R, trt_magic) / (tau - (R)0.5));
    const R ax = p.has_force ? PV(R, ax) : (R)0, ay = p.has_force ? PV(R, ay) : (R)0,
            az = p.has_force ? PV(R, az) : (R)0;
    const R ua = ux * ax + uy * ay + uz * az;
    const R ge = ((R)1 - (R)0.5 * om) * rho, go = ((R)1 - (R)0.5 * om_m) * rho;
    {
      const R fe = (R)Lat<D>::w(0) * rho * base;
      const R v = fi[0] - (fi[0] - fe) * om - (R)Lat<D>::w(0) * ge * (R)3 * ua;
      st(plane(f, p, dir_out<D>(0, 1 - PAR)), cell_out<D>(p, c, 0, 1 - PAR), v, fshift<S, D>(p, 0));
    }
#pragma unroll
    for (int i = 1; i < Q; i += 2) {
      const int k = i + 1;
      const R w = (R)Lat<D>::w(i);
      const R eu = (R)Lat<D>::cx(i) * ux + (R)Lat<D>::cy(i) * uy + (R)Lat<D>::cz(i) * uz;
      const R ea = (R)Lat<D>::cx(i) * ax + (R)Lat<D>::cy(i) * ay + (R)Lat<D>::cz(i) * az;
      const R fe_even = w * rho * (base + (R)4.5 * eu * eu), fe_odd = w * rho * (R)3 * eu;
      const R f_even = (R)0.5 * (fi[i] + fi[k]), f_odd = (R)0.5 * (fi[i] - fi[k]);
      const R even = f_even - (f_even - fe_even) * om + w * ge * ((R)9 * eu * ea - (R)3 * ua);
      const R odd = f_odd - (f_odd - fe_odd) * om_m + w * go * (R)3 * ea;
      st(plane(f, p, dir_out<D>(i, 1 - PAR)), cell_out<D>(p, c, i, 1 - PAR), even + odd, fshift<S, D>(p, i));
      st(plane(f, p, dir_out<D>(k, 1 - PAR)), cell_out<D>(p, c, k, 1 - PAR), even - odd, fshift<S, D>(p, k));
    }
    return;
  }
  if (p.has_force) {
    // Guo forcing: F_i = w_i rho [3 (e_i - u).a + 9 (e_i.u)(e_i.a)]
    const R ax = PV(R, ax), ay = PV(R, ay), az = PV(R, az);
    const R ua = ux * ax + uy * ay + uz * az;
    const R fr = ((R)1 - (R)0.5 * om) * rho;
#pragma unroll
    for (int i = 0; i < Q; ++i) {
      const R ex = (R)Lat<D>::cx(i), ey = (R)Lat<D>::cy(i), ez = (R)Lat<D>::cz(i);
      const R eu = ex * ux + ey * uy + ez * uz;
      const R ea = ex * ax + ey * ay + ez * az;
      const R fe = (R)Lat<D>::w(i) * rho * (base + eu * ((R)3 + eu * (R)4.5));
      const R F = (R)3 * (ea - ua) + (R)9 * eu * ea;
      st(plane(f, p, dir_out<D>(i, 1 - PAR)), cell_out<D>(p, c, i, 1 - PAR),
         fi[i] - (fi[i] - fe) * om + (R)Lat<D>::w(i) * fr * F, fshift<S, D>(p, i));
    }
  } else {
    // opposite directions (i, i + 1) share the even part w rho (base +
    // 4.5 (e.u)^2) of the equilibrium and differ in the sign of its odd part
    // 3 w rho e.u
    {
      const R fe = (R)Lat<D>::w(0) * rho * base;
      st(plane(f, p, dir_out<D>(0, 1 - PAR)), cell_out<D>(p, c, 0, 1 - PAR), fi[0] - (fi[0] - fe) * om, fshift<S, D>(p, 0));
    }
#pragma unroll
    for (int i = 1; i < Q; i += 2) {
      const int k = i + 1;
      const R eu = (R)Lat<D>::cx(i) * ux + (R)Lat<D>::cy(i) * uy + (R)Lat<D>::cz(i) * uz;
      const R wr = (R)Lat<D>::w(i) * rho;
      const R even = wr * (base + (R)4.5 * eu * eu), odd = (R)3 * wr * eu;
      st(plane(f, p, dir_out<D>(i, 1 - PAR)), cell_out<D>(p, c, i, 1 - PAR), fi[i] - (fi[i] - (even + odd)) * om, fshift<S, D>(p, i));
      st(plane(f, p, dir_out<D>(k, 1 - PAR)), cell_out<D>(p, c, k, 1 - PAR), fi[k] - (fi[k] - (even - odd)) * om, fshift<S, D>(p, k));
    }
  }
}

// a liquid cell: its lattice neighbours are liquid, interface or walls
// (liquid never touches gas); walls bounce back by reading the cell's own
// outgoing population from the wall cell's slot
template <int D, class S, int PAR, int COLL>
__device__ __forceinline__ void liquid_cell(const Params &p, const Cell &c, long long n, uint8_t fl, bool wallwarp) {
  using R = typename ST<S>::R;
  constexpr int Q = Lat<D>::Q, QA = Lat<D>::QA;
  S *f = (S *)p.f;
  S *g = (S *)p.g;
  const unsigned wallm = (fl & NEARWALL) ? p.wmask[n] : 0u;
  // wallwarp: some active lane of this warp is a near-wall cell (decided by
  // the caller with all lanes present).
  // Plain streaming loads; in a warp with near-wall cells every lane loads
  // plainly too (a wall direction's slot belongs to the wall cell: an
  // in-bounds read of a value this thread itself rewrites later) and the
  // near-wall lanes then replace their wall directions by bounce-back.  A
  // warp-uniform choice keeps the common path free of per-direction selects.
  R fi[Q];
  R gi[QA];
  if (!wallwarp) {
#pragma unroll
    for (int i = 0; i < Q; ++i) fi[i] = ld(plane(f, p, dir_in<D>(i, PAR)), cell_in<D>(p, c, i, PAR), fshift<S, D>(p, i));
#pragma unroll
    for (int i = 0; i < QA; ++i) gi[i] = ld(plane(g, p, dir_in<D>(i, PAR)), cell_in<D>(p, c, i, PAR), gshift<S, D>(p, i));
  } else {
#pragma unroll
    for (int i = 0; i < Q; ++i) fi[i] = ld(plane(f, p, dir_in<D>(i, PAR)), cell_in<D>(p, c, i, PAR), fshift<S, D>(p, i));
#pragma unroll
    for (int i = 0; i < QA; ++i) gi[i] = ld(plane(g, p, dir_in<D>(i, PAR)), cell_in<D>(p, c, i, PAR), gshift<S, D>(p, i));
    if (wallm) {
#pragma unroll
      for (int i = 1; i < Q; ++i)
        if ((wallm >> i) & 1u)
          fi[i] = ld(plane(f, p, dir_out<D>(opp(i), PAR)), cell_out<D>(p, c, opp(i), PAR), fshift<S, D>(p, opp(i)));
#pragma unroll
      for (int i = 1; i < QA; ++i)
        if ((wallm >> i) & 1u)
          gi[i] = ld(plane(g, p, dir_out<D>(opp(i), PAR)), cell_out<D>(p, c, opp(i), PAR), gshift<S, D>(p, opp(i)));
    }
  }
  if (wallm && (p.walls & 8)) {
    // moving walls of the +y face
#pragma unroll
    for (int i = 1; i < Q; ++i) {
      const bool top = Lat<D>::cy(i) > 0 ? c.y == 0 : (Lat<D>::cy(i) < 0 ? c.y == p.ny - 2 : c.y == p.ny - 1);
      if (((wallm >> i) & 1u) && top) {
        const R eu = (R)Lat<D>::cx(i) * PV(R, uwx) + (R)Lat<D>::cy(i) * PV(R, uwy) + (R)Lat<D>::cz(i) * PV(R, uwz);
        fi[i] += (R)2 * (R)Lat<D>::w(i) * PV(R, rho0) * eu * (R)3;
      }
    }
  }
  // density and momentum from the sums and differences of opposite pairs
  R rho = fi[0], jx = 0, jy = 0, jz = 0;
#pragma unroll
  for (int i = 1; i < Q; i += 2) {
    rho += fi[i] + fi[i + 1];
    const R d = fi[i] - fi[i + 1];
    if (Lat<D>::cx(i)) jx += Lat<D>::cx(i) > 0 ? d : -d;
    if (Lat<D>::cy(i)) jy += Lat<D>::cy(i) > 0 ? d : -d;
    if (Lat<D>::cz(i)) jz += Lat<D>::cz(i) > 0 ? d : -d;
  }
  const R irho = (R)1 / rho;
  const R ux = (jx + (R)0.5 * rho * PV(R, ax)) * irho;
  const R uy = (jy + (R)0.5 * rho * PV(R, ay)) * irho;
  const R uz = (jz + (R)0.5 * rho * PV(R, az)) * irho;
  relax_store<D, S, PAR, COLL>(p, c, n, f, fi, rho, ux, uy, uz, local_om<D, R>(p, fi, rho, irho, ux, uy, uz));
  R cg = 0;
#pragma unroll
  for (int i = 0; i < QA; ++i) cg += gi[i];
  const R omg = PV(R, omg);
#pragma unroll
  for (int i = 0; i < QA; ++i) {
    const R v = gi[i] + (geq<R, D>(i, cg, ux, uy, uz) - gi[i]) * omg + (R)Lat<D>::wa(i) * PV(R, q);
    st(plane(g, p, dir_out<D>(i, 1 - PAR)), cell_out<D>(p, c, i, 1 - PAR), v, gshift<S, D>(p, i));
  }
}

// the liquid cells of the lattice, one thread per cell along x rows; every
// warp takes the liquid path (interface cells are k_stream_interface's).
// A mark of the last step's conversion (its parity bit differs from PAR)
// stands for the type it gives, so that this sweep may start while that
// conversion still writes the new types; a mark of this step's interface
// sweep leaves the type as it is
// WALLED: walls close every face and hold no fluid (Params::walled), so
// the neighbour offsets are the same for every fluid cell (no periodic
// wrap): they are built from the lattice sizes alone, uniform across the
// warp, and the face cells that would need a wrap are walls, never swept.
template <int D, class S, int PAR, int COLL, bool WALLED = false>
__global__ void __launch_bounds__(128, SweepOcc<typename ST<S>::R>::blocks) k_stream_liquid(Params p) {
  Cell c;
  bool inr;
  if constexpr (WALLED) {
    const int x = blockIdx.x * blockDim.x + threadIdx.x, nx = p.nx, nxy = p.nx * p.ny;
    inr = x < nx;
    c.x = inr ? x : nx - 1;
    c.y = blockIdx.y;
    c.z = blockIdx.z;
    c.n = c.x + nx * c.y + nxy * c.z;
    c.dxm = -1;
    c.dxp = 1;
    c.dym = -nx;
    c.dyp = nx;
    c.dzm = -nxy;
    c.dzp = nxy;
  } else {
    inr = grid_cell(p, c);
  }
  const long long n = c.n;
  const uint8_t fl = inr ? p.flags[n] : (uint8_t)T_GAS;
  const bool last_mark = fmark(fl) && ((fl & MARKPAR) != 0) != (PAR != 0);
  const bool active = inr && (last_mark ? post_type(fl) : ftype(fl)) == T_LIQ;
  const bool wallwarp = __any_sync(0xffffffffu, active && (fl & NEARWALL));
  if (active) liquid_cell<D, S, PAR, COLL>(p, c, n, fl, wallwarp);
  if (p.pf.q != 0.f) {
    const unsigned b = __ballot_sync(0xffffffffu, active);
    if ((threadIdx.x & 31) == 0 && b) atomicAdd(p.fluid_updates, (unsigned long long)__popc(b));
  }
}

// an interface cell: streaming, bounce-back, reconstruction from gas
// neighbours, relaxation, fill level and marks, dissolved gas with Henry's
// law at gas links; returns the cell's gas current and its bubble label, and
// its conversion mark
template <int D, class S, int PAR, int COLL>
__device__ __forceinline__ int interface_cell(const Params &p, const Cell &c, long long n, uint8_t fl, double &flux,
                                              int &lab) {
  using R = typename ST<S>::R;
  constexpr int Q = Lat<D>::Q, QA = Lat<D>::QA;
  S *f = (S *)p.f;
  S *g = (S *)p.g;
  // The loads are issued in two rounds: first every neighbour's type and
  // label and every streamed population (f and g; those from gas and wall
  // neighbours are replaced below, an in-bounds read of a slot that is not
  // used), then what the kinds of the neighbours decide (the bubble
  // pressures, the cell's own outgoing populations towards gas and walls).
  unsigned gasm = 0, wallm = 0;  // bit i set when x - e_i is gas / a wall
  int lsrc[Q];                   // label of x - e_i
  R fi[Q];
  R gi[QA];
#pragma unroll
  for (int i = 0; i < Q; ++i) {
    if (i > 0) {
      const int s = src<D>(p, c, i);
      const int ts = ftype(p.flags[s]);
      gasm |= (ts == T_GAS ? 1u : 0u) << i;
      wallm |= (ts == T_WALL ? 1u : 0u) << i;
      lsrc[i] = p.label_old[s];
    }
    fi[i] = ld(plane(f, p, dir_in<D>(i, PAR)), cell_in<D>(p, c, i, PAR), fshift<S, D>(p, i));
  }
#pragma unroll
  for (int i = 0; i < QA; ++i) gi[i] = ld(plane(g, p, dir_in<D>(i, PAR)), cell_in<D>(p, c, i, PAR), gshift<S, D>(p, i));
  // the bubble pressure seen across each gas link (Eq. rhob), and the ADE
  // populations of gas and wall links (Henry's law, bounce-back)
  R pgs[Q];
#pragma unroll
  for (int i = 1; i < Q; ++i) pgs[i] = (gasm >> i & 1u) ? (lsrc[i] >= 0 ? (R)p.told.p[lsrc[i]] : PV(R, p0)) : (R)0;
  R gb[QA];
#pragma unroll
  for (int i = 1; i < QA; ++i)
    if ((gasm | wallm) >> i & 1u)
      gb[i] = ld(plane(g, p, dir_out<D>(opp(i), PAR)), cell_out<D>(p, c, opp(i), PAR), gshift<S, D>(p, opp(i)));
  if (gasm | wallm) {
    const R *uI = (const R *)p.uI;
    const R uIx = uI[n], uIy = uI[p.N + n], uIz = uI[2 * p.N + n];
    const R kap = ((const R *)p.kappa)[n], pi = ((const R *)p.Pi)[n];
#pragma unroll
    for (int i = 1; i < Q; ++i) {
      if (wallm >> i & 1u) {
        // half-way bounce-back: the cell's own outgoing population towards
        // the wall, reflected (the slot belongs to the wall cell)
        R v = ld(plane(f, p, dir_out<D>(opp(i), PAR)), cell_out<D>(p, c, opp(i), PAR), fshift<S, D>(p, opp(i)));
        const bool top = Lat<D>::cy(i) > 0 ? c.y == 0 : (Lat<D>::cy(i) < 0 ? c.y == p.ny - 2 : c.y == p.ny - 1);
        if ((p.walls & 8) && top) {
          const R eu = (R)Lat<D>::cx(i) * PV(R, uwx) + (R)Lat<D>::cy(i) * PV(R, uwy) + (R)Lat<D>::cz(i) * PV(R, uwz);
          v += (R)2 * (R)Lat<D>::w(i) * PV(R, rho0) * eu * (R)3;
        }
        fi[i] = v;
      } else if (gasm >> i & 1u) {
        // Sec. 2.2 Eq. reconstruct with rho_g of Eq. rhob / rhobplusdisjoining
        const R rg = (pgs[i] - (R)2 * PV(R, sigma) * kap - pi) * (R)3;
        const R fo = ld(plane(f, p, dir_out<D>(opp(i), PAR)), cell_out<D>(p, c, opp(i), PAR), fshift<S, D>(p, opp(i)));
        fi[i] = feq<R, D>(i, rg, uIx, uIy, uIz) + feq<R, D>(opp(i), rg, uIx, uIy, uIz) - fo;
      }
    }
  }
  // moments and Guo-shifted velocity
  R rho = 0, jx = 0, jy = 0, jz = 0;
#pragma unroll
  for (int i = 0; i < Q; ++i) {
    rho += fi[i];
    jx += fi[i] * (R)Lat<D>::cx(i);
    jy += fi[i] * (R)Lat<D>::cy(i);
    jz += fi[i] * (R)Lat<D>::cz(i);
  }
  const R irho = (R)1 / rho;
  const R ux = (jx + (R)0.5 * rho * PV(R, ax)) * irho;
  const R uy = (jy + (R)0.5 * rho * PV(R, ay)) * irho;
  const R uz = (jz + (R)0.5 * rho * PV(R, az)) * irho;
  relax_store<D, S, PAR, COLL>(p, c, n, f, fi, rho, ux, uy, uz, local_om<D, R>(p, fi, rho, irho, ux, uy, uz));

  R *phi = (R *)p.phi;
  const R Mn = ((const R *)p.M)[n];
  const R phin = Mn / rho;
  phi[n] = phin;
  int mk = MK_NONE;
  if (Mn > ((R)1 + PV(R, eps)) * rho)
    mk = MK_FILL;
  else if (Mn < -PV(R, eps) * rho)
    mk = MK_EMPTY;
  if (mk) p.flags[n] = (uint8_t)(fl | mark_bits(mk, PAR));

  // dissolved gas (Sec. 3.1-3.2)
  R cgas = 0, fl_gas = 0;
#pragma unroll
  for (int i = 0; i < QA; ++i) {
    if (i > 0 && (wallm >> i & 1u)) {
      gi[i] = gb[i];
    } else if (i > 0 && (gasm >> i & 1u)) {
      const R cH = PV(R, kH) * pgs[i];
      gi[i] = (R)2 * (R)Lat<D>::wa(i) * cH - gb[i];
      fl_gas += gb[i] - gi[i];
    }
    cgas += gi[i];
  }
  const R omg = PV(R, omg);
  R cout = 0;
#pragma unroll
  for (int i = 0; i < QA; ++i) {
    const R v = gi[i] + (geq<R, D>(i, cgas, ux, uy, uz) - gi[i]) * omg + (R)Lat<D>::wa(i) * PV(R, q);
    cout += v;
    st(plane(g, p, dir_out<D>(i, 1 - PAR)), cell_out<D>(p, c, i, 1 - PAR), v, gshift<S, D>(p, i));
  }
  // the moments of the post-collision populations (the collision keeps the
  // density; the Guo-shifted velocity is that of the outgoing populations):
  // a gas neighbour turning interface averages them
  {
    R *mo = (R *)p.mom;
    mo[n] = rho;
    mo[p.N + n] = ux;
    mo[2 * p.N + n] = uy;
    mo[3 * p.N + n] = uz;
    mo[4 * p.N + n] = cout;
  }
  // Sec. 3.1 Eq. gascurrent at the gas links: what the cell sends into the
  // gas minus what the Henry condition returns (only diffusive exchange
  // crosses there, so there is no advective part to deduct)
  flux = (double)fl_gas;
  lab = p.label_old[n];
  if (lab < 0) atomicAdd(p.led + 5, flux);
  return mk;
}

// the interface cells of the step, one warp per segment of the segment list
// and one lane per cell; cells that fill or empty are listed for the
// conversion.  Block 0 also resets the counters of the lists that the
// conversion fills.
template <int D, class S, int PAR, int COLL, bool WALLED = false>
__global__ void __launch_bounds__(128, 4) k_stream_interface(Params p) {
  __shared__ double wbuf[128];
  const int lane = threadIdx.x & 31;
  const int warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int nwarps = (gridDim.x * blockDim.x) >> 5;
  const int cnt = *p.segcount;
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    *p.ncount = 0;
    *p.segnext_count = 0;
    if (p.pf.q != 0.f) atomicAdd(p.fluid_updates, (unsigned long long)*p.icount);
  }
  for (int k = warp; k < cnt; k += nwarps) {
    const int seg = p.seglist[k];
    Cell c;
    const bool inr = WALLED ? seg_cell_walled(p, seg, lane, c) : seg_cell(p, seg, lane, c);
    const uint8_t fl = inr ? p.flags[c.n] : (uint8_t)T_GAS;
    double flux = 0.0;
    int lab = -1, mk = MK_NONE;
    if (ftype(fl) == T_IFC) mk = interface_cell<D, S, PAR, COLL>(p, c, c.n, fl, flux, lab);
    if (lane == 0) p.segflag[seg] = 0;  // free for the conversion's next list
    list_append(p.mlist, p.mcount, mk != MK_NONE, c.n);
    if (__any_sync(0xffffffffu, lab >= 0)) agg_add(p.told.dm, lab, flux, wbuf + (threadIdx.x & ~31));
  }
}

}  // namespace lbf

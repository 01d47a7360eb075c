/*
 * lbf_oracle.c -- plain, slow FP64 CPU oracle of the LBfoam free-surface
 * foaming step.  TEST INFRASTRUCTURE ONLY (see lbf_oracle.h): the product
 * path never loads it.
 *
 * Written for readability against the paper, not for speed: two-array
 * streaming, cell-by-cell loops in linear index order, breadth-first flood
 * fill for bubbles, bisection for every implicit quantity.  Compiled with
 * -ffp-contract=off so each expression rounds exactly as written.
 *
 * One step, in order (paper sections in brackets):
 *  1. stream + free-surface reconstruction + mass exchange + collision for
 *     every liquid/interface cell [Sec. 2, Eq. LBE/collision/equilibrium;
 *     Sec. 2.1 Eq. massexchange; Sec. 2.2 Eq. reconstruct/rhob; Sec. 3.3
 *     Eq. rhobplusdisjoining; Sec. 2.3 Eq. tau/carreauTau]
 *     and the D2Q5/D3Q7 advection-diffusion step with Henry's law and the
 *     per-interface-cell gas flux [Sec. 3.1 Eq. diffusion/gascurrent;
 *     Sec. 3.2 Eq. henryslaw/reconstructdiffusion]
 *  2. cell conversion with uniform excess-mass redistribution [Sec. 2.1]
 *  3. bubble labelling (flood fill), merge/split gas redistribution in
 *     proportion to volume, ideal-gas pressure [Sec. 3.5, Sec. 2.2 Eq. idealgas]
 *  4. interface normals, curvature, PLIC offsets and disjoining pressure by
 *     ray traversal for the next step [Sec. 2.2, Sec. 3.3, Appendix A]
 */
#include "lbf_oracle.h"

#include <math.h>
#include <stdlib.h>
#include <string.h>

enum { GAS = 0, LIQ = 1, IFC = 2, WALL = 3 };
enum { MK_NONE = 0, MK_FILL = 1, MK_EMPTY = 2, MK_GI = 3, MK_LI = 4 };
enum { ERR_CAPACITY = -6 };
static const double PI_ = 3.14159265358979323846;
static const double LSQ_RIDGE = 1e-3;

struct or_sim {
  or_config c;
  int dim, Q, QA;
  long N;
  int e[19][3];
  double w[19], wa[7], csa2;
  int opp[19];
  uint8_t *type, *mark;
  double *fc, *gc;           /* post-collision populations of the last step */
  double *M, *phi;           /* liquid mass and fill level                   */
  double *kappa, *Pi, *nrm, *dst;
  int32_t *label;            /* bubble index of gas/interface cells, else -1 */
  int nb;                    /* bubble table                                 */
  double *bm, *bV, *bp, *bdm;
  int32_t *bid, *batm;
  int64_t *broot;
  int next_id;
  double led[8];
  int err;
  double mrtM[19][19], mrtMi[19][19]; /* MRT moment basis and its inverse     */
  int mrtg[19];                       /* MRT group of each moment               */
};

/* ---------------------------------------------------------------------- */
/* velocity sets: Sec. 2 (D2Q9 and D3Q19 with the paper's weights); the    */
/* advection-diffusion sets D2Q5/D3Q7 are the first 5/7 vectors (Sec. 3.1) */

static void setup_lattice(or_sim *s) {
  static const int e2[9][2] = {{0, 0},  {1, 0},  {-1, 0}, {0, 1}, {0, -1},
                               {1, 1},  {-1, -1}, {1, -1}, {-1, 1}};
  static const int e3[19][3] = {
      {0, 0, 0},  {1, 0, 0},   {-1, 0, 0}, {0, 1, 0},   {0, -1, 0},
      {0, 0, 1},  {0, 0, -1},  {1, 1, 0},  {-1, -1, 0}, {1, 0, 1},
      {-1, 0, -1}, {0, 1, 1},  {0, -1, -1}, {1, -1, 0}, {-1, 1, 0},
      {1, 0, -1}, {-1, 0, 1},  {0, 1, -1}, {0, -1, 1}};
  int i;
  memset(s->e, 0, sizeof s->e);
  if (s->dim == 2) {
    s->Q = 9;
    s->QA = 5;
    for (i = 0; i < 9; ++i) {
      s->e[i][0] = e2[i][0];
      s->e[i][1] = e2[i][1];
      s->w[i] = i == 0 ? 4.0 / 9.0 : (i < 5 ? 1.0 / 9.0 : 1.0 / 36.0);
    }
    s->csa2 = 1.0 / 3.0;
    for (i = 0; i < 5; ++i) s->wa[i] = i == 0 ? 1.0 / 3.0 : 1.0 / 6.0;
  } else {
    s->Q = 19;
    s->QA = 7;
    for (i = 0; i < 19; ++i) {
      s->e[i][0] = e3[i][0];
      s->e[i][1] = e3[i][1];
      s->e[i][2] = e3[i][2];
      s->w[i] = i == 0 ? 1.0 / 3.0 : (i < 7 ? 1.0 / 18.0 : 1.0 / 36.0);
    }
    s->csa2 = 1.0 / 4.0;
    for (i = 0; i < 7; ++i) s->wa[i] = i == 0 ? 1.0 / 4.0 : 1.0 / 8.0;
  }
  for (i = 0; i < s->Q; ++i) s->opp[i] = i == 0 ? 0 : ((i & 1) ? i + 1 : i - 1);
}

/* ---------------------------------------------------------------------- */
/* multiple relaxation times (the collision variant Sec. 2 names besides    */
/* BGK): orthogonal polynomial moments of the velocity set, the basis of    */
/* Lallemand and Luo (2000) for D2Q9 and of d'Humieres et al. (2002) for    */
/* D3Q19.  The groups relax at s_e (energy), s_eps (energy square), s_q     */
/* (energy flux), s_nu = 1/tau (stress), s_pi (fourth-order anisotropic)    */
/* and s_m (third-order); density and momentum are conserved.               */

enum { MG_CONS = 0, MG_E = 1, MG_EPS = 2, MG_Q = 3, MG_NU = 4, MG_PI = 5, MG_M = 6 };

/* moment k of the basis at velocity (x, y, z); *g receives its group */
static double mrt_moment(int dim, int k, int x, int y, int z, int *g) {
  const double cx = x, cy = y, cz = z;
  const double c2 = cx * cx + cy * cy + cz * cz;
  if (dim == 2) {
    switch (k) {
      case 0: *g = MG_CONS; return 1.0;                                   /* rho  */
      case 1: *g = MG_E; return 3.0 * c2 - 4.0;                           /* e    */
      case 2: *g = MG_EPS; return (9.0 * c2 * c2 - 21.0 * c2 + 8.0) / 2.0; /* eps  */
      case 3: *g = MG_CONS; return cx;                                    /* j_x  */
      case 4: *g = MG_Q; return (3.0 * c2 - 5.0) * cx;                    /* q_x  */
      case 5: *g = MG_CONS; return cy;                                    /* j_y  */
      case 6: *g = MG_Q; return (3.0 * c2 - 5.0) * cy;                    /* q_y  */
      case 7: *g = MG_NU; return cx * cx - cy * cy;                       /* p_xx */
      default: *g = MG_NU; return cx * cy;                                /* p_xy */
    }
  }
  switch (k) {
    case 0: *g = MG_CONS; return 1.0;
    case 1: *g = MG_E; return 19.0 * c2 - 30.0;
    case 2: *g = MG_EPS; return (21.0 * c2 * c2 - 53.0 * c2 + 24.0) / 2.0;
    case 3: *g = MG_CONS; return cx;
    case 4: *g = MG_Q; return (5.0 * c2 - 9.0) * cx;
    case 5: *g = MG_CONS; return cy;
    case 6: *g = MG_Q; return (5.0 * c2 - 9.0) * cy;
    case 7: *g = MG_CONS; return cz;
    case 8: *g = MG_Q; return (5.0 * c2 - 9.0) * cz;
    case 9: *g = MG_NU; return 3.0 * cx * cx - c2;                        /* 3 p_xx  */
    case 10: *g = MG_PI; return (3.0 * c2 - 5.0) * (3.0 * cx * cx - c2); /* 3 pi_xx */
    case 11: *g = MG_NU; return cy * cy - cz * cz;                        /* p_ww    */
    case 12: *g = MG_PI; return (3.0 * c2 - 5.0) * (cy * cy - cz * cz);   /* pi_ww   */
    case 13: *g = MG_NU; return cx * cy;
    case 14: *g = MG_NU; return cy * cz;
    case 15: *g = MG_NU; return cx * cz;
    case 16: *g = MG_M; return (cy * cy - cz * cz) * cx;
    case 17: *g = MG_M; return (cz * cz - cx * cx) * cy;
    default: *g = MG_M; return (cx * cx - cy * cy) * cz;
  }
}

/* the basis matrix of the lattice and its inverse (Gauss-Jordan elimination
 * with partial pivoting) */
static void setup_mrt(or_sim *s) {
  const int Q = s->Q;
  double a[19][38];
  int i, k, r, col;
  for (k = 0; k < Q; ++k)
    for (i = 0; i < Q; ++i) s->mrtM[k][i] = mrt_moment(s->dim, k, s->e[i][0], s->e[i][1], s->e[i][2], &s->mrtg[k]);
  for (r = 0; r < Q; ++r)
    for (col = 0; col < 2 * Q; ++col) a[r][col] = col < Q ? s->mrtM[r][col] : (col - Q == r ? 1.0 : 0.0);
  for (col = 0; col < Q; ++col) {
    int piv = col;
    double t;
    for (r = col + 1; r < Q; ++r)
      if (fabs(a[r][col]) > fabs(a[piv][col])) piv = r;
    for (k = 0; k < 2 * Q; ++k) {
      t = a[col][k];
      a[col][k] = a[piv][k];
      a[piv][k] = t;
    }
    t = a[col][col];
    for (k = 0; k < 2 * Q; ++k) a[col][k] /= t;
    for (r = 0; r < Q; ++r) {
      if (r == col || a[r][col] == 0.0) continue;
      t = a[r][col];
      for (k = 0; k < 2 * Q; ++k) a[r][k] -= t * a[col][k];
    }
  }
  for (r = 0; r < Q; ++r)
    for (col = 0; col < Q; ++col) s->mrtMi[r][col] = a[r][Q + col];
}

int or_mrt_basis(int dim, double *M, int32_t *grp) {
  or_sim t;
  int i, k;
  memset(&t, 0, sizeof t);
  t.dim = dim == 2 ? 2 : 3;
  setup_lattice(&t);
  setup_mrt(&t);
  for (k = 0; k < t.Q; ++k) {
    grp[k] = t.mrtg[k];
    for (i = 0; i < t.Q; ++i) M[k * t.Q + i] = t.mrtM[k][i];
  }
  return t.Q;
}

static void coords(const or_sim *s, long n, long *x, long *y, long *z) {
  *x = n % s->c.nx;
  *y = (n / s->c.nx) % s->c.ny;
  *z = n / ((long)s->c.nx * s->c.ny);
}

/* index of the cell at offset (dx,dy,dz), periodic in every direction */
static long shift(const or_sim *s, long n, int dx, int dy, int dz) {
  long x, y, z, nx = s->c.nx, ny = s->c.ny, nz = s->c.nz;
  coords(s, n, &x, &y, &z);
  x = ((x + dx) % nx + nx) % nx;
  y = ((y + dy) % ny + ny) % ny;
  z = ((z + dz) % nz + nz) % nz;
  return x + nx * (y + ny * z);
}

static long nbr(const or_sim *s, long n, int i) {
  return shift(s, n, s->e[i][0], s->e[i][1], s->e[i][2]);
}
static long src(const or_sim *s, long n, int i) {
  return shift(s, n, -s->e[i][0], -s->e[i][1], -s->e[i][2]);
}

static double edot(const or_sim *s, int i, const double *u) {
  return s->e[i][0] * u[0] + s->e[i][1] * u[1] + s->e[i][2] * u[2];
}

/* Sec. 2 Eq. equilibrium, c_s^2 = 1/3 */
static double feq(const or_sim *s, int i, double rho, const double *u) {
  double eu = edot(s, i, u);
  double uu = u[0] * u[0] + u[1] * u[1] + u[2] * u[2];
  return s->w[i] * rho * (1.0 + eu / (1.0 / 3.0) + eu * eu / (2.0 / 9.0) - uu / (2.0 / 3.0));
}

/* Sec. 3.1 advection-diffusion equilibrium */
static double geq(const or_sim *s, int i, double c, const double *u) {
  return s->wa[i] * c * (1.0 + edot(s, i, u) / s->csa2);
}

/* ---------------------------------------------------------------------- */
/* Sec. 2.3: tau from the local strain rate.  The shear rate follows from   */
/* the non-equilibrium stress, gamma_dot = |Pi_neq| / (sqrt2 rho cs^2 tau); */
/* tau then solves tau = tau_model(gamma_dot(tau)), found by bisection.     */

static double tau_model(const or_sim *s, double gd) {
  const or_config *c = &s->c;
  if (c->rheo == 1) return 0.5 + 3.0 * c->rheo_k * pow(gd, c->rheo_n - 1.0);
  return c->tau_inf + (c->tau0 - c->tau_inf) *
                          pow(1.0 + pow(c->rheo_lambda * gd, c->rheo_a),
                              (c->rheo_n - 1.0) / c->rheo_a);
}

static double solve_tau(const or_sim *s, double A) {
  double lo = s->c.tau_min, hi = s->c.tau_max, mid;
  int it;
  if (s->c.rheo == 0) return s->c.tau;
  if (hi - tau_model(s, A / hi) <= 0.0) return hi;
  if (lo - tau_model(s, A / lo) >= 0.0) return lo;
  for (it = 0; it < 200; ++it) {
    mid = 0.5 * (lo + hi);
    if (mid - tau_model(s, A / mid) > 0.0)
      hi = mid;
    else
      lo = mid;
    if (hi - lo <= 1e-15 * hi) break;
  }
  return 0.5 * (lo + hi);
}

/* ---------------------------------------------------------------------- */

static int is_moving_wall(const or_sim *s, long n) {
  long x, y, z;
  if (!(s->c.walls & 8)) return 0;
  coords(s, n, &x, &y, &z);
  return y == s->c.ny - 1;
}

static double pop_sum(const double *p, int q) {
  double r = 0.0;
  int i;
  for (i = 0; i < q; ++i) r += p[i];
  return r;
}

static void velocity_of(const or_sim *s, const double *p, double rho, double *u) {
  double m[3] = {0.0, 0.0, 0.0};
  int i, d;
  for (i = 0; i < s->Q; ++i)
    for (d = 0; d < 3; ++d) m[d] += p[i] * s->e[i][d];
  for (d = 0; d < 3; ++d) u[d] = (m[d] - 0.5 * rho * s->c.accel[d]) / rho;
}

static double bubble_pressure(const or_sim *s, long gas_cell) {
  int b = s->label[gas_cell];
  return b >= 0 ? s->bp[b] : s->c.p0;
}

/* Step 1: stream, reconstruct, exchange mass, collide (flow and gas). */
static void stream_collide(or_sim *s) {
  const long N = s->N;
  const int Q = s->Q, QA = s->QA;
  const double *a = s->c.accel;
  const double taug = 0.5 + s->c.D / s->csa2; /* Sec. 3.1 Eq. diffusionconst */
  double *fcn = malloc(sizeof(double) * N * Q);
  double *gcn = malloc(sizeof(double) * N * QA);
  double *Mn = malloc(sizeof(double) * N);
  double *phin = malloc(sizeof(double) * N);
  long n;
  memcpy(fcn, s->fc, sizeof(double) * N * Q);
  memcpy(gcn, s->gc, sizeof(double) * N * QA);
  memcpy(Mn, s->M, sizeof(double) * N);
  memcpy(phin, s->phi, sizeof(double) * N);
  memset(s->mark, MK_NONE, N);

  for (n = 0; n < N; ++n) {
    const int t = s->type[n];
    const double *fo, *go;
    double f[19], g[7], uI[3], u[3], j[3], rho, rho_o, Mnew, tau, c, flux;
    int i, d;
    if (t != LIQ && t != IFC) continue;
    fo = s->fc + n * Q;
    go = s->gc + n * QA;
    rho_o = pop_sum(fo, Q);
    velocity_of(s, fo, rho_o, uI); /* u_I: the cell's velocity of the last step */

    /* streaming (Sec. 2 Eq. streamingstep) with bounce-back at walls and the
     * free-surface reconstruction (Sec. 2.2 Eq. reconstruct) from gas */
    f[0] = fo[0];
    for (i = 1; i < Q; ++i) {
      const long sidx = src(s, n, i);
      const int ts = s->type[sidx];
      if (ts == LIQ || ts == IFC) {
        f[i] = s->fc[sidx * Q + i];
      } else if (ts == WALL) {
        f[i] = fo[s->opp[i]];
        if (is_moving_wall(s, sidx))
          f[i] += 2.0 * s->w[i] * s->c.rho0 * edot(s, i, s->c.wall_u) / (1.0 / 3.0);
      } else {
        const double pg = bubble_pressure(s, sidx);
        const double rhog = (pg - 2.0 * s->c.sigma * s->kappa[n] - s->Pi[n]) / (1.0 / 3.0);
        f[i] = feq(s, i, rhog, uI) + feq(s, s->opp[i], rhog, uI) - fo[s->opp[i]];
      }
    }

    /* mass exchange (Sec. 2.1 Eq. massexchange, Theta weights) */
    Mnew = s->M[n];
    if (t == IFC) {
      for (i = 1; i < Q; ++i) {
        const long nb = nbr(s, n, i);
        const int tn = s->type[nb];
        const double dm = s->fc[nb * Q + s->opp[i]] - fo[i];
        if (tn == LIQ)
          Mnew += dm;
        else if (tn == IFC)
          Mnew += 0.5 * (s->phi[n] + s->phi[nb]) * dm;
      }
    }

    /* moments (Sec. 2 Eq. velocity), Guo-shifted velocity */
    rho = 0.0;
    j[0] = j[1] = j[2] = 0.0;
    for (i = 0; i < Q; ++i) {
      rho += f[i];
      for (d = 0; d < 3; ++d) j[d] += f[i] * s->e[i][d];
    }
    for (d = 0; d < 3; ++d) u[d] = (j[d] + 0.5 * rho * a[d]) / rho;

    /* relaxation time (Sec. 2.3) from the non-equilibrium stress */
    if (s->c.rheo != 0) {
      double P[3][3] = {{0}}, nrm2 = 0.0;
      int aa, bb;
      for (i = 0; i < Q; ++i) {
        const double fn = f[i] - feq(s, i, rho, u);
        for (aa = 0; aa < 3; ++aa)
          for (bb = 0; bb < 3; ++bb) P[aa][bb] += s->e[i][aa] * s->e[i][bb] * fn;
      }
      for (aa = 0; aa < 3; ++aa)
        for (bb = 0; bb < 3; ++bb) nrm2 += P[aa][bb] * P[aa][bb];
      tau = solve_tau(s, sqrt(nrm2) / (sqrt(2.0) * rho * (1.0 / 3.0)));
    } else {
      tau = s->c.tau;
    }

    if (s->c.collision == 1) {
      /* two relaxation times (the collision variant Sec. 2 names besides
         BGK): the parts of f - f_eq even under e -> -e relax at 1/tau, the
         odd parts at 1/tau_m with (tau - 1/2)(tau_m - 1/2) = trt_magic; the
         Guo source splits the same way, each part scaled by
         (1 - 1/(2 tau)) or (1 - 1/(2 tau_m)) */
      const double tau_m = 0.5 + s->c.trt_magic / (tau - 0.5);
      double fe[19], S[19];
      for (i = 0; i < Q; ++i) {
        fe[i] = feq(s, i, rho, u);
        S[i] = 0.0;
        for (d = 0; d < 3; ++d)
          S[i] += ((s->e[i][d] - u[d]) / (1.0 / 3.0) + edot(s, i, u) * s->e[i][d] / (1.0 / 9.0)) *
                  rho * a[d];
        S[i] *= s->w[i];
      }
      for (i = 0; i < Q; ++i) {
        const int k = s->opp[i];
        const double fe_even = 0.5 * (fe[i] + fe[k]), fe_odd = 0.5 * (fe[i] - fe[k]);
        const double f_even = 0.5 * (f[i] + f[k]), f_odd = 0.5 * (f[i] - f[k]);
        const double S_even = 0.5 * (S[i] + S[k]), S_odd = 0.5 * (S[i] - S[k]);
        fcn[n * Q + i] = f[i] - (f_even - fe_even) / tau - (f_odd - fe_odd) / tau_m +
                         (1.0 - 0.5 / tau) * S_even + (1.0 - 0.5 / tau_m) * S_odd;
      }
    } else if (s->c.collision == 2) {
      /* multiple relaxation times: m = M f, each moment relaxes towards the
         moment of f_eq at its group's rate, the Guo source enters moment by
         moment scaled by (1 - s_k/2); f = M^-1 m.  The stress moments take
         1/tau (the local tau of the rheology), the energy flux 1/tau_m of
         the TRT product trt_magic; density and momentum are conserved (their
         rate cancels against the source term, 1 is used) */
      const double tau_m = 0.5 + s->c.trt_magic / (tau - 0.5);
      const double *rr = s->c.mrt_rates;
      double rate[7], fe[19], S[19], ms[19];
      int k;
      rate[MG_CONS] = 1.0;
      rate[MG_NU] = 1.0 / tau;
      rate[MG_Q] = 1.0 / tau_m;
      rate[MG_E] = rr[0] > 0.0 ? rr[0] : 1.0 / tau;
      rate[MG_EPS] = rr[1] > 0.0 ? rr[1] : 1.0 / tau;
      rate[MG_PI] = rr[2] > 0.0 ? rr[2] : 1.0 / tau;
      rate[MG_M] = rr[3] > 0.0 ? rr[3] : 1.0 / tau_m;
      for (i = 0; i < Q; ++i) {
        fe[i] = feq(s, i, rho, u);
        S[i] = 0.0;
        for (d = 0; d < 3; ++d)
          S[i] += ((s->e[i][d] - u[d]) / (1.0 / 3.0) + edot(s, i, u) * s->e[i][d] / (1.0 / 9.0)) *
                  rho * a[d];
        S[i] *= s->w[i];
      }
      for (k = 0; k < Q; ++k) {
        double m = 0.0, me = 0.0, mS = 0.0;
        const double r = rate[s->mrtg[k]];
        for (i = 0; i < Q; ++i) {
          m += s->mrtM[k][i] * f[i];
          me += s->mrtM[k][i] * fe[i];
          mS += s->mrtM[k][i] * S[i];
        }
        ms[k] = m - r * (m - me) + (1.0 - 0.5 * r) * mS;
      }
      for (i = 0; i < Q; ++i) {
        double v = 0.0;
        for (k = 0; k < Q; ++k) v += s->mrtMi[i][k] * ms[k];
        fcn[n * Q + i] = v;
      }
    } else {
      /* BGK collision with Guo forcing (Sec. 2 Eq. collision) */
      for (i = 0; i < Q; ++i) {
        double F = 0.0;
        for (d = 0; d < 3; ++d)
          F += ((s->e[i][d] - u[d]) / (1.0 / 3.0) + edot(s, i, u) * s->e[i][d] / (1.0 / 9.0)) *
               rho * a[d];
        F *= (1.0 - 0.5 / tau) * s->w[i];
        fcn[n * Q + i] = f[i] - (f[i] - feq(s, i, rho, u)) / tau + F;
      }
    }

    if (t == IFC) {
      phin[n] = Mnew / rho; /* Sec. 2.1 Eq. alpha */
      Mn[n] = Mnew;
      if (Mnew > (1.0 + s->c.eps) * rho)
        s->mark[n] = MK_FILL;
      else if (Mnew < -s->c.eps * rho)
        s->mark[n] = MK_EMPTY;
    }

    /* advection-diffusion of dissolved gas (Sec. 3.1 Eq. diffusion) with
     * Henry's law at gas links (Sec. 3.2 Eq. henryslaw/reconstructdiffusion) */
    flux = 0.0;
    g[0] = go[0];
    for (i = 1; i < QA; ++i) {
      const long sidx = src(s, n, i);
      const int ts = s->type[sidx];
      if (ts == LIQ || ts == IFC) {
        g[i] = s->gc[sidx * QA + i];
      } else if (ts == WALL) {
        g[i] = go[s->opp[i]];
      } else {
        const double cH = s->c.kH * bubble_pressure(s, sidx);
        g[i] = geq(s, i, cH, uI) + geq(s, s->opp[i], cH, uI) - go[s->opp[i]];
        flux += go[s->opp[i]] - g[i];
      }
    }
    c = pop_sum(g, QA);
    for (i = 0; i < QA; ++i)
      gcn[n * QA + i] = g[i] + (geq(s, i, c, u) - g[i]) / taug + s->wa[i] * s->c.q;
    s->led[6] += s->c.q;

    /* gas flux into the cell's bubble (Sec. 3.1 Eq. gascurrent), measured
     * where it crosses the interface: at the gas links, what the cell sends
     * into the gas minus what the Henry condition returns.  Only the
     * diffusive exchange crosses there, so the advective part that the
     * equation's last term, -c (alpha(t) - alpha(t-1)), deducts from a
     * liquid-side measure is never in this sum and nothing is deducted;
     * with the cells that change between gas and interface carrying their
     * dissolved gas (convert), bubbles plus dissolved gas are conserved. */
    if (t == IFC) {
      const int b = s->label[n];
      if (b >= 0)
        s->bdm[b] += flux;
      else
        s->led[5] += flux;
    }
  }
  free(s->fc);
  free(s->gc);
  free(s->M);
  free(s->phi);
  s->fc = fcn;
  s->gc = gcn;
  s->M = Mn;
  s->phi = phin;
}

/* ---------------------------------------------------------------------- */
/* Step 2: cell conversion (Sec. 2.1).  Interface cells past the fill level  */
/* thresholds become liquid or gas; the surplus or shortage of mass goes in  */
/* equal parts to the neighbouring interface cells.                          */

static int post_type(const or_sim *s, long n) {
  switch (s->mark[n]) {
    case MK_FILL: return LIQ;
    case MK_EMPTY: return GAS;
    case MK_GI:
    case MK_LI: return IFC;
    default: return s->type[n];
  }
}

static void convert(or_sim *s) {
  const long N = s->N;
  const int Q = s->Q, QA = s->QA;
  double *ex = calloc(N, sizeof(double));
  long n;
  int i;

  /* a cell cannot empty next to a filling cell (filling wins) */
  for (n = 0; n < N; ++n) {
    if (s->mark[n] != MK_EMPTY) continue;
    for (i = 1; i < Q; ++i)
      if (s->mark[nbr(s, n, i)] == MK_FILL) {
        s->mark[n] = MK_NONE;
        break;
      }
  }
  /* gas next to a filling cell and liquid next to an emptying cell become
   * interface, so that liquid never touches gas */
  for (n = 0; n < N; ++n) {
    const int t = s->type[n];
    if (t != GAS && t != LIQ) continue;
    for (i = 1; i < Q; ++i) {
      const int m = s->mark[nbr(s, n, i)];
      if (t == GAS && m == MK_FILL) {
        s->mark[n] = MK_GI;
        break;
      }
      if (t == LIQ && m == MK_EMPTY) {
        s->mark[n] = MK_LI;
        break;
      }
    }
  }
  /* excess mass of converting cells, shared equally by the neighbours that
   * are interface cells after the conversion */
  for (n = 0; n < N; ++n) {
    const int m = s->mark[n];
    double rho, excess;
    int cnt = 0;
    if (m != MK_FILL && m != MK_EMPTY) continue;
    rho = pop_sum(s->fc + n * Q, Q);
    excess = m == MK_FILL ? s->M[n] - rho : s->M[n];
    for (i = 1; i < Q; ++i)
      if (post_type(s, nbr(s, n, i)) == IFC) ++cnt;
    if (cnt > 0)
      ex[n] = excess / cnt;
    else
      s->led[1] += excess;
    if (m == MK_EMPTY) { /* the cell's dissolved gas joins its bubble */
      const double cg = pop_sum(s->gc + n * QA, QA);
      if (s->label[n] >= 0)
        s->bdm[s->label[n]] += cg;
      else
        s->led[5] += cg;
    }
  }
  /* new interface cells from gas: equilibrium at the mean density, velocity
   * and concentration of their interface neighbours that are not emptying */
  for (n = 0; n < N; ++n) {
    double rs = 0.0, us[3] = {0.0, 0.0, 0.0}, cs = 0.0, u[3];
    int cnt = 0, d;
    if (s->mark[n] != MK_GI) continue;
    for (i = 1; i < Q; ++i) {
      const long nb = nbr(s, n, i);
      if (s->type[nb] == IFC && (s->mark[nb] == MK_NONE || s->mark[nb] == MK_FILL)) {
        const double r = pop_sum(s->fc + nb * Q, Q);
        double un[3];
        velocity_of(s, s->fc + nb * Q, r, un);
        rs += r;
        for (d = 0; d < 3; ++d) us[d] += un[d];
        cs += pop_sum(s->gc + nb * QA, QA);
        ++cnt;
      }
    }
    rs /= cnt;
    for (d = 0; d < 3; ++d) u[d] = us[d] / cnt;
    cs /= cnt;
    for (i = 0; i < Q; ++i) s->fc[n * Q + i] = feq(s, i, rs, u);
    for (i = 0; i < QA; ++i) s->gc[n * QA + i] = geq(s, i, cs, u);
    s->M[n] = 0.0;
    if (s->label[n] >= 0)
      s->bdm[s->label[n]] -= cs;
    else
      s->led[5] -= cs;
  }
  for (n = 0; n < N; ++n)
    if (s->mark[n] == MK_LI) s->M[n] = pop_sum(s->fc + n * Q, Q);

  /* interface cells collect the excess of converting neighbours */
  for (n = 0; n < N; ++n) {
    double recv = 0.0;
    int has = 0;
    if (post_type(s, n) != IFC) continue;
    for (i = 1; i < Q; ++i) {
      const long nb = nbr(s, n, i);
      if (s->mark[nb] == MK_FILL || s->mark[nb] == MK_EMPTY) {
        recv += ex[nb];
        has = 1;
      }
    }
    s->M[n] += recv;
    if (has || s->mark[n] == MK_GI || s->mark[n] == MK_LI)
      s->phi[n] = s->M[n] / pop_sum(s->fc + n * Q, Q);
  }
  for (n = 0; n < N; ++n) {
    const int pt = post_type(s, n);
    if (pt == LIQ) {
      s->phi[n] = 1.0;
      s->M[n] = 0.0;
    } else if (pt == GAS) {
      s->phi[n] = 0.0;
      s->M[n] = 0.0;
    }
    s->type[n] = (uint8_t)pt;
    s->mark[n] = MK_NONE;
  }
  free(ex);
}

/* ---------------------------------------------------------------------- */
/* Step 3: bubbles (Sec. 3.5).  Gas regions connected over lattice links    */
/* form bubbles, numbered by their smallest linear cell index; interface    */
/* cells join the bubble of their gas neighbour with the smallest number.   */
/* Gas content of bubbles that merged or split is redistributed in          */
/* proportion to volume; pressure follows the ideal-gas law (Eq. idealgas). */

static int uf_find(int *p, int a) {
  while (p[a] != a) a = p[a];
  return a;
}
static void uf_union(int *p, int a, int b) {
  a = uf_find(p, a);
  b = uf_find(p, b);
  if (a < b)
    p[b] = a;
  else if (b < a)
    p[a] = b;
}

static int top_layer(const or_sim *s) {
  const int up = s->dim - 1;
  const int n_up = up == 1 ? s->c.ny : s->c.nz;
  return n_up - 1 - ((s->c.walls >> (2 * up + 1)) & 1);
}

static int relabel(or_sim *s) {
  const long N = s->N;
  const int Q = s->Q, nbo = s->nb;
  int32_t *nl = malloc(sizeof(int32_t) * N);
  long *queue = malloc(sizeof(long) * N);
  int64_t *roots = NULL;
  int nc = 0, k, j, *par, *heir, *minid, *nold, *nnew, *atmg;
  double *V, *Mold, *Vnew, *nm, *np;
  int32_t *atm, *nid;
  long n;
  int i;

  for (n = 0; n < N; ++n) nl[n] = -1;
  for (n = 0; n < N; ++n) {
    long head = 0, tail = 0;
    if (s->type[n] != GAS || nl[n] >= 0) continue;
    roots = realloc(roots, sizeof(int64_t) * (nc + 1));
    roots[nc] = n; /* first cell met in index order is the smallest */
    nl[n] = nc;
    queue[tail++] = n;
    while (head < tail) {
      const long m = queue[head++];
      for (i = 1; i < Q; ++i) {
        const long nb = nbr(s, m, i);
        if (s->type[nb] == GAS && nl[nb] < 0) {
          nl[nb] = nc;
          queue[tail++] = nb;
        }
      }
    }
    ++nc;
  }
  free(queue);
  if (nc > s->c.bubble_capacity) {
    free(nl);
    free(roots);
    s->err = ERR_CAPACITY;
    return ERR_CAPACITY;
  }
  for (n = 0; n < N; ++n) {
    int best = -1;
    if (s->type[n] != IFC) continue;
    for (i = 1; i < Q; ++i) {
      const long nb = nbr(s, n, i);
      if (s->type[nb] == GAS && (best < 0 || nl[nb] < best)) best = nl[nb];
    }
    nl[n] = best;
  }

  /* volume V = gas cells + sum of (1 - alpha) over interface cells */
  V = calloc(nc + 1, sizeof(double));
  atm = calloc(nc + 1, sizeof(int32_t));
  for (n = 0; n < N; ++n) {
    if (nl[n] < 0) continue;
    if (s->type[n] == GAS) {
      long x, y, z;
      V[nl[n]] += 1.0;
      coords(s, n, &x, &y, &z);
      if (s->c.atmosphere && (s->dim == 2 ? y : z) == top_layer(s)) atm[nl[n]] = 1;
    } else {
      V[nl[n]] += 1.0 - s->phi[n];
    }
  }

  /* gas gained during the step belongs to the old bubbles */
  for (j = 0; j < nbo; ++j) {
    s->bm[j] += s->bdm[j];
    s->bdm[j] = 0.0;
  }

  /* groups of old and new bubbles that share cells */
  par = malloc(sizeof(int) * (nbo + nc + 1));
  for (k = 0; k < nbo + nc; ++k) par[k] = k;
  for (n = 0; n < N; ++n)
    if (s->label[n] >= 0 && nl[n] >= 0) uf_union(par, s->label[n], nbo + nl[n]);

  Mold = calloc(nbo + nc + 1, sizeof(double));
  Vnew = calloc(nbo + nc + 1, sizeof(double));
  nold = calloc(nbo + nc + 1, sizeof(int));
  nnew = calloc(nbo + nc + 1, sizeof(int));
  atmg = calloc(nbo + nc + 1, sizeof(int));
  heir = malloc(sizeof(int) * (nbo + nc + 1));
  minid = malloc(sizeof(int) * (nbo + nc + 1));
  for (k = 0; k < nbo + nc; ++k) {
    heir[k] = -1;
    minid[k] = -1;
  }
  for (j = 0; j < nbo; ++j) {
    const int g = uf_find(par, j);
    Mold[g] += s->bm[j];
    ++nold[g];
    if (minid[g] < 0 || s->bid[j] < minid[g]) minid[g] = s->bid[j];
  }
  for (k = 0; k < nc; ++k) {
    const int g = uf_find(par, nbo + k);
    Vnew[g] += V[k];
    ++nnew[g];
    if (atm[k]) atmg[g] = 1;
    if (heir[g] < 0 || V[k] > V[heir[g]]) heir[g] = k;
  }
  for (j = 0; j < nbo; ++j) { /* bubbles that vanished entirely */
    const int g = uf_find(par, j);
    if (nnew[g] == 0) s->led[5] += s->bm[j];
  }
  nm = malloc(sizeof(double) * (nc + 1));
  np = malloc(sizeof(double) * (nc + 1));
  nid = malloc(sizeof(int32_t) * (nc + 1));
  for (k = 0; k < nc; ++k) {
    const int g = uf_find(par, nbo + k);
    if (atmg[g]) {
      np[k] = s->c.p0;
      nm[k] = s->c.p0 * V[k] / s->c.RT;
    } else if (nold[g] == 0) { /* born: Laplace equilibrium with the ambient */
      const double Req = s->dim == 3 ? cbrt(3.0 * V[k] / (4.0 * PI_)) : sqrt(V[k] / PI_);
      np[k] = s->c.p0 + (s->dim - 1) * s->c.sigma / Req;
      nm[k] = np[k] * V[k] / s->c.RT;
      s->led[5] -= nm[k];
    } else {
      nm[k] = Mold[g] * V[k] / Vnew[g];
      np[k] = nm[k] * s->c.RT / V[k];
    }
    if (nold[g] > 0 && heir[g] == k)
      nid[k] = minid[g];
    else
      nid[k] = s->next_id++;
  }
  for (k = 0; k < nbo + nc; ++k) /* atmosphere groups exchange with outside */
    if (k == uf_find(par, k) && atmg[k]) {
      double mn = 0.0;
      int kk;
      for (kk = 0; kk < nc; ++kk)
        if (uf_find(par, nbo + kk) == k) mn += nm[kk];
      s->led[5] += Mold[k] - mn;
    }

  free(s->bm);
  free(s->bV);
  free(s->bp);
  free(s->bdm);
  free(s->bid);
  free(s->batm);
  free(s->broot);
  s->bm = nm;
  s->bp = np;
  s->bV = V;
  s->bid = nid;
  s->batm = atm;
  s->broot = roots ? roots : malloc(sizeof(int64_t));
  s->bdm = calloc(nc + 1, sizeof(double));
  s->nb = nc;
  free(s->label);
  s->label = nl;
  free(par);
  free(Mold);
  free(Vnew);
  free(nold);
  free(nnew);
  free(atmg);
  free(heir);
  free(minid);
  return 0;
}

/* ---------------------------------------------------------------------- */
/* PLIC (Sec. 3.3): the plane n.p = s through the cell [-1/2,1/2]^d with    */
/* liquid on the side n.p > s.  The gas fraction of the unit cube below     */
/* sum m_i x_i < a (m_i = |n_i|) equals the average, over the first         */
/* coordinate, of the same quantity one dimension lower.  Each average is   */
/* taken exactly: the integrand is a piecewise polynomial of degree < 2     */
/* (midpoint) or < 4 (two-point Gauss), split at its kinks.                 */

static double gas1(double b, double m) {
  double v;
  if (m <= 0.0) return b > 0.0 ? 1.0 : 0.0;
  v = b / m;
  return v < 0.0 ? 0.0 : (v > 1.0 ? 1.0 : v);
}

static int sorted_knots(double lo, double hi, const double *k, int nk, double *out) {
  int n = 0, i, j;
  out[n++] = lo;
  for (i = 0; i < nk; ++i)
    if (k[i] > lo && k[i] < hi) out[n++] = k[i];
  out[n++] = hi;
  for (i = 1; i < n; ++i)
    for (j = i; j > 0 && out[j] < out[j - 1]; --j) {
      const double t = out[j];
      out[j] = out[j - 1];
      out[j - 1] = t;
    }
  return n;
}

static double gas2(double b, double m2, double m3) {
  double kn[2], pts[4], sum = 0.0;
  int np, i;
  if (m2 <= 0.0) return gas1(b, m3);
  kn[0] = 0.0;
  kn[1] = m3;
  np = sorted_knots(b - m2, b, kn, 2, pts);
  if (!(pts[np - 1] > pts[0])) return gas1(b, m3); /* width lost to rounding */
  for (i = 0; i + 1 < np; ++i)
    sum += (pts[i + 1] - pts[i]) * gas1(0.5 * (pts[i] + pts[i + 1]), m3);
  return sum / (pts[np - 1] - pts[0]);
}

static double gas3(double a, double m1, double m2, double m3) {
  const double gl = 1.0 / sqrt(3.0);
  double kn[4], pts[6], sum = 0.0;
  int np, i;
  if (m1 <= 0.0) return gas2(a, m2, m3);
  kn[0] = 0.0;
  kn[1] = m2;
  kn[2] = m3;
  kn[3] = m2 + m3;
  np = sorted_knots(a - m1, a, kn, 4, pts);
  if (!(pts[np - 1] > pts[0])) return gas2(a, m2, m3); /* width lost to rounding */
  for (i = 0; i + 1 < np; ++i) {
    const double h = 0.5 * (pts[i + 1] - pts[i]), mid = 0.5 * (pts[i] + pts[i + 1]);
    sum += h * (gas2(mid - h * gl, m2, m3) + gas2(mid + h * gl, m2, m3));
  }
  return sum / (pts[np - 1] - pts[0]);
}

double or_plic_liquid_fraction(int dim, const double *n, double s) {
  const double m1 = fabs(n[0]), m2 = fabs(n[1]), m3 = dim == 3 ? fabs(n[2]) : 0.0;
  const double a = s + 0.5 * (m1 + m2 + m3);
  if (dim == 2) return 1.0 - gas2(a, m1, m2);
  return 1.0 - gas3(a, m1, m2, m3);
}

double or_plic_offset(int dim, const double *n, double alpha) {
  const double h = 0.5 * (fabs(n[0]) + fabs(n[1]) + (dim == 3 ? fabs(n[2]) : 0.0));
  double lo = -h, hi = h;
  int it;
  if (h <= 0.0) return 0.0;
  if (alpha >= 1.0) return -h;
  if (alpha <= 0.0) return h;
  for (it = 0; it < 200 && hi - lo > 1e-17; ++it) {
    const double mid = 0.5 * (lo + hi);
    if (or_plic_liquid_fraction(dim, n, mid) > alpha)
      lo = mid;
    else
      hi = mid;
  }
  return 0.5 * (lo + hi);
}

/* ---------------------------------------------------------------------- */
/* Step 4: geometry for the next step.                                       */
/* Normal (Sec. 3.3, used by PLIC and the ray): m = grad(alpha)/|grad alpha|, */
/* the gradient summed over the 2^d vertex blocks of the 3^d stencil (face,  */
/* edge and corner weights 4, 2, 1); m points into the liquid.               */
/* Curvature (Sec. 2.2 Eq. rhob): least-squares paraboloid through the PLIC */
/* points of the interface cells of the stencil, each cut with the centre    */
/* normal, in a frame whose third axis is m; kappa is minus the mean         */
/* curvature of that surface (a gas sphere has kappa = 1/R, a gas disk      */
/* 1/(2R)), limited to [-1, 1].                                              */

static double alpha_for_geometry(const or_sim *s, long n, long centre) {
  double a;
  if (s->type[n] == WALL) n = centre; /* walls repeat the centre value */
  if (s->type[n] == LIQ) return 1.0;
  if (s->type[n] == GAS) return 0.0;
  a = s->phi[n];
  return a < 0.0 ? 0.0 : (a > 1.0 ? 1.0 : a);
}

/* solve the k x k system A x = b (row-major, destroyed) by Gaussian
 * elimination with partial pivoting; returns 0 if a pivot is tiny */
static int solve_small(double *A, double *b, int k, double *x) {
  int i, j, r, piv;
  for (i = 0; i < k; ++i) {
    double best = fabs(A[i * k + i]);
    piv = i;
    for (r = i + 1; r < k; ++r)
      if (fabs(A[r * k + i]) > best) {
        best = fabs(A[r * k + i]);
        piv = r;
      }
    if (best < 1e-9) return 0;
    if (piv != i) {
      for (j = 0; j < k; ++j) {
        const double t = A[i * k + j];
        A[i * k + j] = A[piv * k + j];
        A[piv * k + j] = t;
      }
      {
        const double t = b[i];
        b[i] = b[piv];
        b[piv] = t;
      }
    }
    for (r = i + 1; r < k; ++r) {
      const double f = A[r * k + i] / A[i * k + i];
      for (j = i; j < k; ++j) A[r * k + j] -= f * A[i * k + j];
      b[r] -= f * b[i];
    }
  }
  for (i = k - 1; i >= 0; --i) {
    double acc = b[i];
    for (j = i + 1; j < k; ++j) acc -= A[i * k + j] * x[j];
    x[i] = acc / A[i * k + i];
  }
  return 1;
}

/* least-squares fit of z = sum_j beta_j phi_j(x, y), with a small ridge
 * term so that point sets that cannot resolve every coefficient (cells next
 * to walls, nearly axis-aligned planes) give a smooth, bounded answer */
static int lsq_fit(const double (*pts)[3], int np, int k, int kind, double *beta) {
  double A[25] = {0}, b[5] = {0}, ph[5];
  int p, i, j;
  for (p = 0; p < np; ++p) {
    const double x = pts[p][0], y = pts[p][1];
    if (kind == 3) { /* A x^2 + B y^2 + C xy + H x + I y */
      ph[0] = x * x; ph[1] = y * y; ph[2] = x * y; ph[3] = x; ph[4] = y;
    } else if (kind == 2) { /* A x^2 + H x */
      ph[0] = x * x; ph[1] = x;
    } else { /* A (x^2 + y^2) */
      ph[0] = x * x + y * y;
    }
    for (i = 0; i < k; ++i) {
      for (j = 0; j < k; ++j) A[i * k + j] += ph[i] * ph[j];
      b[i] += ph[i] * pts[p][2];
    }
  }
  for (i = 0; i < k; ++i) A[i * k + i] += LSQ_RIDGE;
  return solve_small(A, b, k, beta);
}

/* kappa of the least-squares surface through np points given in the local
 * frame (t1, t2, m) of the centre cell: 2D z = A x^2 + H x, kappa = minus
 * the curvature of that curve at 0; 3D z = A x^2 + B y^2 + C xy + H x + I y,
 * kappa = minus the mean curvature of that surface at 0 (one parameter
 * fits when there are too few points); limited to [-1, 1] */
static double kappa_from_points(int dim, const double (*pts)[3], int np) {
  double beta[5], kap = 0.0;
  if (dim == 2) {
    if (np >= 2 && lsq_fit(pts, np, 2, 2, beta))
      kap = -beta[0] / pow(1.0 + beta[1] * beta[1], 1.5);
    else if (np >= 1 && lsq_fit(pts, np, 1, 1, beta))
      kap = -beta[0];
  } else {
    if (np >= 5 && lsq_fit(pts, np, 5, 3, beta)) {
      const double H = beta[3], I = beta[4];
      kap = -((1.0 + I * I) * beta[0] - H * I * beta[2] + (1.0 + H * H) * beta[1]) /
            pow(1.0 + H * H + I * I, 1.5);
    } else if (np >= 1 && lsq_fit(pts, np, 1, 1, beta)) {
      kap = -2.0 * beta[0];
    }
  }
  return kap < -1.0 ? -1.0 : (kap > 1.0 ? 1.0 : kap);
}

/* test hook: the curvature of np (<= 27) points, x y z each */
double or_lsq_kappa(int dim, const double *pts, int np) {
  if (np < 0 || np > 27) return 0.0;
  return kappa_from_points(dim, (const double(*)[3])pts, np);
}

static void normals_curvature(or_sim *s) {
  const int dim = s->dim;
  long n;
  for (n = 0; n < s->N; ++n) {
    double A[3][3][3], g[3] = {0.0, 0.0, 0.0}, gn, m[3], t1[3], t2[3], pts[27][3];
    int act[3][3][3], dx, dy, dz, d, np = 0, kmin;
    s->kappa[n] = 0.0;
    s->dst[n] = 0.0;
    s->nrm[3 * n] = s->nrm[3 * n + 1] = s->nrm[3 * n + 2] = 0.0;
    if (s->type[n] != IFC) continue;
    for (dz = -1; dz <= 1; ++dz)
      for (dy = -1; dy <= 1; ++dy)
        for (dx = -1; dx <= 1; ++dx) {
          long y;
          double a = 0.0;
          act[dz + 1][dy + 1][dx + 1] = 0;
          if (dim == 2 && dz != 0) {
            A[dz + 1][dy + 1][dx + 1] = 0.0;
            continue;
          }
          y = shift(s, n, dx, dy, dz);
          a = alpha_for_geometry(s, y, n);
          A[dz + 1][dy + 1][dx + 1] = a;
          act[dz + 1][dy + 1][dx + 1] = s->type[y] == IFC && a > 0.0 && a < 1.0;
        }
    /* Parker-Youngs weighted centred differences */
    for (dz = -1; dz <= 1; ++dz)
      for (dy = -1; dy <= 1; ++dy)
        for (dx = -1; dx <= 1; ++dx) {
          const double v = A[dz + 1][dy + 1][dx + 1];
          if (dim == 2) {
            if (dz != 0) continue;
            g[0] += dx * (dy == 0 ? 2.0 : 1.0) * v;
            g[1] += dy * (dx == 0 ? 2.0 : 1.0) * v;
          } else {
            g[0] += dx * (dy == 0 ? 2.0 : 1.0) * (dz == 0 ? 2.0 : 1.0) * v;
            g[1] += dy * (dx == 0 ? 2.0 : 1.0) * (dz == 0 ? 2.0 : 1.0) * v;
            g[2] += dz * (dx == 0 ? 2.0 : 1.0) * (dy == 0 ? 2.0 : 1.0) * v;
          }
        }
    gn = sqrt(g[0] * g[0] + g[1] * g[1] + g[2] * g[2]);
    if (gn <= 1e-12) continue;
    for (d = 0; d < 3; ++d) m[d] = g[d] / gn;
    for (d = 0; d < 3; ++d) s->nrm[3 * n + d] = m[d];
    s->dst[n] = or_plic_offset(dim, m, A[1][1][1]);

    /* local frame (t1, t2, m) */
    if (dim == 2) {
      t1[0] = -m[1]; t1[1] = m[0]; t1[2] = 0.0;
      t2[0] = t2[1] = t2[2] = 0.0;
    } else {
      double e[3] = {0.0, 0.0, 0.0}, len;
      kmin = fabs(m[0]) <= fabs(m[1]) ? (fabs(m[0]) <= fabs(m[2]) ? 0 : 2) : (fabs(m[1]) <= fabs(m[2]) ? 1 : 2);
      e[kmin] = 1.0;
      for (d = 0; d < 3; ++d) t1[d] = e[d] - m[kmin] * m[d];
      len = sqrt(t1[0] * t1[0] + t1[1] * t1[1] + t1[2] * t1[2]);
      for (d = 0; d < 3; ++d) t1[d] /= len;
      t2[0] = m[1] * t1[2] - m[2] * t1[1];
      t2[1] = m[2] * t1[0] - m[0] * t1[2];
      t2[2] = m[0] * t1[1] - m[1] * t1[0];
    }
    /* PLIC points of the neighbouring interface cells, cut with m */
    for (dz = -1; dz <= 1; ++dz)
      for (dy = -1; dy <= 1; ++dy)
        for (dx = -1; dx <= 1; ++dx) {
          const double o[3] = {dx, dy, dz};
          double sj;
          if (dx == 0 && dy == 0 && dz == 0) continue;
          if (!act[dz + 1][dy + 1][dx + 1]) continue;
          sj = or_plic_offset(dim, m, A[dz + 1][dy + 1][dx + 1]);
          pts[np][0] = o[0] * t1[0] + o[1] * t1[1] + o[2] * t1[2];
          pts[np][1] = o[0] * t2[0] + o[1] * t2[1] + o[2] * t2[2];
          pts[np][2] = o[0] * m[0] + o[1] * m[1] + o[2] * m[2] + sj - s->dst[n];
          ++np;
        }
    s->kappa[n] = kappa_from_points(dim, (const double(*)[3])pts, np);
  }
}

/* Height-function curvature (see the header).  The heights are the
 * liquid lengths of the columns; a column of liquid above (or below) a
 * convex gas cap grows away from the cap's apex, so h'' > 0 gives kappa > 0
 * whichever side the liquid is on, and the curvature of the height
 * function is halved to the scale of the least-squares kappa. */
/* height-function curvature of interface cell n; returns 0 where it is
 * undefined (a zero normal, a wall in one of the columns) */
static int hf_kappa(const or_sim *s, long n, double *out) {
  const int dim = s->dim;
  const double *m = s->nrm + 3 * n;
  double h[3][3];
  int d = 0, a, b, i, j, k, wall = 0;
  if (m[0] == 0.0 && m[1] == 0.0 && m[2] == 0.0) return 0;
  for (k = 1; k < dim; ++k)
    if (fabs(m[k]) > fabs(m[d])) d = k;
  a = d == 0 ? 1 : 0;
  b = 3 - d - a;
  for (j = -1; j <= 1; ++j)
    for (i = -1; i <= 1; ++i) {
      double sum = 0.0;
      h[j + 1][i + 1] = 0.0;
      if (dim == 2 && j != 0) continue;
      for (k = -3; k <= 3; ++k) {
        int off[3] = {0, 0, 0};
        long y;
        off[a] = i;
        off[b] = dim == 2 ? 0 : j;
        off[d] = k;
        y = shift(s, n, off[0], off[1], off[2]);
        if (s->type[y] == WALL) wall = 1;
        sum += alpha_for_geometry(s, y, n);
      }
      h[j + 1][i + 1] = sum;
    }
  if (wall) return 0;
  if (dim == 2) {
    const double ha = 0.5 * (h[1][2] - h[1][0]);
    const double haa = h[1][2] - 2.0 * h[1][1] + h[1][0];
    *out = haa / (2.0 * pow(1.0 + ha * ha, 1.5));
  } else {
    const double ha = 0.5 * (h[1][2] - h[1][0]), hb = 0.5 * (h[2][1] - h[0][1]);
    const double haa = h[1][2] - 2.0 * h[1][1] + h[1][0], hbb = h[2][1] - 2.0 * h[1][1] + h[0][1];
    const double hab = 0.25 * (h[2][2] - h[0][2] - h[2][0] + h[0][0]);
    *out = (haa * (1.0 + hb * hb) + hbb * (1.0 + ha * ha) - 2.0 * hab * ha * hb) /
           (2.0 * pow(1.0 + ha * ha + hb * hb, 1.5));
  }
  return 1;
}

int or_hf_curvature(const or_sim *s, double *out) {
  long n;
  for (n = 0; n < s->N; ++n) {
    out[n] = 0.0;
    if (s->type[n] != IFC) continue;
    if (!hf_kappa(s, n, &out[n])) out[n] = NAN;
  }
  return 0;
}

/* Disjoining pressure (Sec. 3.3 Eq. for Pi) with the ray traversal of
 * Appendix A (Algorithm 1): march from the cell centre along the normal
 * into the liquid, cell boundary by cell boundary, until an interface or
 * gas cell of another bubble is met, a wall stops the ray, or the step
 * budget runs out.  The distance d runs from this cell's PLIC plane to the
 * other cell's PLIC plane along the ray (or to where the ray enters the
 * other cell when that cell has no plane facing the ray). */
static void disjoining(or_sim *s) {
  const int steps = (int)ceil(s->c.d_max) + 1;
  long n;
  for (n = 0; n < s->N; ++n) {
    const double *dir = s->nrm + 3 * n;
    double tmax[3], tdel[3], tent = 0.0, dist = -1.0;
    int step[3], off[3] = {0, 0, 0}, it, d;
    const int b = s->label[n];
    s->Pi[n] = 0.0;
    if (s->c.k_pi == 0.0 || s->type[n] != IFC || b < 0) continue;
    if (dir[0] == 0.0 && dir[1] == 0.0 && dir[2] == 0.0) continue;
    for (d = 0; d < 3; ++d) {
      tmax[d] = dir[d] != 0.0 ? fabs(0.5 / dir[d]) : INFINITY;
      tdel[d] = 2.0 * tmax[d];
      step[d] = dir[d] >= 0.0 ? 1 : -1;
    }
    for (it = 1; it <= steps; ++it) {
      const double tm = fmin(tmax[0], fmin(tmax[1], tmax[2]));
      long y;
      int ty;
      tent = tm;
      /* axes whose next boundary lies at the same ray parameter are crossed
       * together (a diagonal step); "the same" within a relative 1e-9, so
       * that round-off in a normal with equal components cannot turn one
       * diagonal step into two axis steps */
      for (d = 0; d < 3; ++d)
        if (tmax[d] <= tm * (1.0 + 1e-9)) {
          tmax[d] += tdel[d];
          off[d] += step[d];
        }
      y = shift(s, n, off[0], off[1], off[2]);
      ty = s->type[y];
      if (s->label[y] == b) continue;
      if (ty == WALL) break;
      if ((ty == IFC || ty == GAS) && s->label[y] >= 0) {
        const double *ny = s->nrm + 3 * y;
        const double den = ny[0] * dir[0] + ny[1] * dir[1] + ny[2] * dir[2];
        if (ty == IFC && den < -1e-6) {
          const double ncy = ny[0] * off[0] + ny[1] * off[1] + ny[2] * off[2];
          dist = (s->dst[y] + ncy) / den - s->dst[n];
        } else {
          dist = tent - s->dst[n];
        }
        if (dist < 0.0) dist = 0.0;
        break;
      }
    }
    if (dist >= 0.0 && dist < s->c.d_max) s->Pi[n] = s->c.k_pi * (s->c.d_max - dist);
  }
}

static void geometry(or_sim *s) {
  normals_curvature(s);
  if (s->c.kappa == 1) {
    /* the height-function curvature (the second method Sec. 2.2 names)
     * replaces the least-squares one wherever it is defined, limited to
     * [-1, 1] like it */
    long n;
    for (n = 0; n < s->N; ++n) {
      double k;
      if (s->type[n] == IFC && hf_kappa(s, n, &k)) s->kappa[n] = k < -1.0 ? -1.0 : (k > 1.0 ? 1.0 : k);
    }
  }
  disjoining(s);
}

/* ---------------------------------------------------------------------- */

static void alloc_fields(or_sim *s) {
  const long N = s->N;
  s->type = calloc(N, 1);
  s->mark = calloc(N, 1);
  s->fc = calloc(N * s->Q, sizeof(double));
  s->gc = calloc(N * s->QA, sizeof(double));
  s->M = calloc(N, sizeof(double));
  s->phi = calloc(N, sizeof(double));
  s->kappa = calloc(N, sizeof(double));
  s->Pi = calloc(N, sizeof(double));
  s->nrm = calloc(3 * N, sizeof(double));
  s->dst = calloc(N, sizeof(double));
  s->label = malloc(sizeof(int32_t) * N);
  for (long n = 0; n < N; ++n) s->label[n] = -1;
  s->bm = calloc(1, sizeof(double));
  s->bV = calloc(1, sizeof(double));
  s->bp = calloc(1, sizeof(double));
  s->bdm = calloc(1, sizeof(double));
  s->bid = calloc(1, sizeof(int32_t));
  s->batm = calloc(1, sizeof(int32_t));
  s->broot = calloc(1, sizeof(int64_t));
}

static int is_wall_cell(const or_sim *s, long n) {
  long x, y, z;
  const int w = s->c.walls;
  coords(s, n, &x, &y, &z);
  if ((w & 1) && x == 0) return 1;
  if ((w & 2) && x == s->c.nx - 1) return 1;
  if ((w & 4) && y == 0) return 1;
  if ((w & 8) && y == s->c.ny - 1) return 1;
  if (s->dim == 3 && (w & 16) && z == 0) return 1;
  if (s->dim == 3 && (w & 32) && z == s->c.nz - 1) return 1;
  return 0;
}

/* liquid next to gas becomes interface with alpha = 1 (keeps the invariant
 * that liquid and gas are always separated by interface cells) */
static void separate_liquid_from_gas(or_sim *s) {
  long n;
  int i;
  for (n = 0; n < s->N; ++n) {
    if (s->type[n] != LIQ) continue;
    for (i = 1; i < s->Q; ++i)
      if (s->type[nbr(s, n, i)] == GAS) {
        s->mark[n] = MK_LI;
        break;
      }
  }
  for (n = 0; n < s->N; ++n)
    if (s->mark[n] == MK_LI) {
      s->type[n] = IFC;
      s->phi[n] = 1.0;
      s->M[n] = pop_sum(s->fc + n * s->Q, s->Q);
      s->mark[n] = MK_NONE;
    }
}

static void forget_bubbles(or_sim *s) {
  long n;
  for (n = 0; n < s->N; ++n) s->label[n] = -1;
  s->nb = 0;
}

or_sim *or_create(const or_config *cfg) {
  or_sim *s = calloc(1, sizeof(or_sim));
  const double u0[3] = {0.0, 0.0, 0.0};
  long n;
  int i;
  s->c = *cfg;
  s->dim = cfg->nz == 1 ? 2 : 3;
  s->N = (long)cfg->nx * cfg->ny * cfg->nz;
  setup_lattice(s);
  setup_mrt(s);
  alloc_fields(s);
  for (n = 0; n < s->N; ++n) {
    long x, y, z;
    double a;
    coords(s, n, &x, &y, &z);
    if (is_wall_cell(s, n)) {
      s->type[n] = WALL;
      continue;
    }
    a = cfg->fill_height - ((s->dim == 2 ? y : z) - 0.5);
    a = a < 0.0 ? 0.0 : (a > 1.0 ? 1.0 : a);
    s->type[n] = a >= 1.0 ? LIQ : (a <= 0.0 ? GAS : IFC);
    s->phi[n] = a;
    if (s->type[n] != GAS) {
      for (i = 0; i < s->Q; ++i) s->fc[n * s->Q + i] = feq(s, i, cfg->rho0, u0);
      for (i = 0; i < s->QA; ++i) s->gc[n * s->QA + i] = geq(s, i, cfg->c0, u0);
      s->M[n] = s->type[n] == IFC ? a * cfg->rho0 : 0.0;
    }
  }
  separate_liquid_from_gas(s);
  forget_bubbles(s);
  relabel(s);
  geometry(s);
  return s;
}

void or_destroy(or_sim *s) {
  if (!s) return;
  free(s->type);
  free(s->mark);
  free(s->fc);
  free(s->gc);
  free(s->M);
  free(s->phi);
  free(s->kappa);
  free(s->Pi);
  free(s->nrm);
  free(s->dst);
  free(s->label);
  free(s->bm);
  free(s->bV);
  free(s->bp);
  free(s->bdm);
  free(s->bid);
  free(s->batm);
  free(s->broot);
  free(s);
}

int or_error(const or_sim *s) { return s->err; }

int or_set_cells(or_sim *s, const uint8_t *type, const double *rho, const double *u,
                 const double *alpha, const double *c) {
  long n;
  int i;
  for (n = 0; n < s->N; ++n) {
    const int t = type[n];
    s->type[n] = (uint8_t)t;
    s->M[n] = 0.0;
    s->phi[n] = t == LIQ ? 1.0 : (t == IFC ? alpha[n] : 0.0);
    for (i = 0; i < s->Q; ++i)
      s->fc[n * s->Q + i] = (t == LIQ || t == IFC) ? feq(s, i, rho[n], u + 3 * n) : 0.0;
    for (i = 0; i < s->QA; ++i)
      s->gc[n * s->QA + i] = (t == LIQ || t == IFC) ? geq(s, i, c[n], u + 3 * n) : 0.0;
    if (t == IFC) s->M[n] = alpha[n] * rho[n];
  }
  separate_liquid_from_gas(s);
  forget_bubbles(s);
  if (relabel(s)) return s->err;
  geometry(s);
  return 0;
}

/* Nucleation (Sec. 3.4): a gas sphere (disk in 2D) of radius R is carved
 * into liquid cells.  A cell's fill level is the fraction of its 4^d
 * sub-cell sample points outside the sphere. */
int or_nucleate(or_sim *s, int nn, const double *centres, const double *radii) {
  int k;
  for (k = 0; k < nn; ++k) {
    const double *c = centres + 3 * k, R = radii[k];
    const long x0 = (long)floor(c[0] - R - 1.0), x1 = (long)ceil(c[0] + R + 1.0);
    const long y0 = (long)floor(c[1] - R - 1.0), y1 = (long)ceil(c[1] + R + 1.0);
    const long z0 = s->dim == 3 ? (long)floor(c[2] - R - 1.0) : 0;
    const long z1 = s->dim == 3 ? (long)ceil(c[2] + R + 1.0) : 0;
    const int total = s->dim == 3 ? 64 : 16;
    long X, Y, Z;
    for (Z = z0; Z <= z1; ++Z)
      for (Y = y0; Y <= y1; ++Y)
        for (X = x0; X <= x1; ++X) {
          const long n = shift(s, 0, (int)X, (int)Y, (int)Z);
          int a, b, cc, nout = 0;
          double rho;
          if (s->type[n] != LIQ) continue;
          for (cc = 0; cc < (s->dim == 3 ? 4 : 1); ++cc)
            for (b = 0; b < 4; ++b)
              for (a = 0; a < 4; ++a) {
                const double px = X + (a + 0.5) / 4.0 - 0.5 - c[0];
                const double py = Y + (b + 0.5) / 4.0 - 0.5 - c[1];
                const double pz = s->dim == 3 ? Z + (cc + 0.5) / 4.0 - 0.5 - c[2] : 0.0;
                if (px * px + py * py + pz * pz >= R * R) ++nout;
              }
          if (nout == total) continue;
          rho = pop_sum(s->fc + n * s->Q, s->Q);
          if (nout == 0) {
            s->type[n] = GAS;
            s->phi[n] = 0.0;
            s->M[n] = 0.0;
            s->led[2] += rho;
            s->led[5] += pop_sum(s->gc + n * s->QA, s->QA);
          } else {
            const double al = (double)nout / total;
            s->type[n] = IFC;
            s->phi[n] = al;
            s->M[n] = al * rho;
            s->led[2] += rho - al * rho;
          }
        }
  }
  separate_liquid_from_gas(s);
  if (relabel(s)) return s->err;
  geometry(s);
  return 0;
}

/* test hooks: change cell types without touching the bubble table, then run
 * the labelling and merge/split redistribution alone */
int or_debug_set_types(or_sim *s, const uint8_t *type) {
  long n;
  for (n = 0; n < s->N; ++n) s->type[n] = type[n];
  return 0;
}
int or_debug_relabel(or_sim *s) { return relabel(s); }

int or_step(or_sim *s, int nsteps) {
  int k;
  for (k = 0; k < nsteps; ++k) {
    stream_collide(s);
    convert(s);
    if (relabel(s)) return s->err;
    geometry(s);
  }
  return 0;
}

/* ---------------------------------------------------------------------- */

int or_get(const or_sim *s, int field, double *out) {
  const int Q = s->Q, QA = s->QA;
  long n;
  int i;
  for (n = 0; n < s->N; ++n) {
    const int fl = s->type[n] == LIQ || s->type[n] == IFC;
    const double *p = s->fc + n * Q;
    switch (field) {
      case OR_RHO: out[n] = fl ? pop_sum(p, Q) : 0.0; break;
      case OR_U: {
        double u[3] = {0.0, 0.0, 0.0};
        if (fl) velocity_of(s, p, pop_sum(p, Q), u);
        out[3 * n] = u[0];
        out[3 * n + 1] = u[1];
        out[3 * n + 2] = u[2];
        break;
      }
      case OR_ALPHA: out[n] = s->phi[n]; break;
      case OR_MASS: out[n] = s->type[n] == IFC ? s->M[n] : (s->type[n] == LIQ ? pop_sum(p, Q) : 0.0); break;
      case OR_CONC: out[n] = fl ? pop_sum(s->gc + n * QA, QA) : 0.0; break;
      case OR_KAPPA: out[n] = s->kappa[n]; break;
      case OR_PI: out[n] = s->Pi[n]; break;
      case OR_NORMAL:
        for (i = 0; i < 3; ++i) out[3 * n + i] = s->nrm[3 * n + i];
        break;
      case OR_DSTAR: out[n] = s->dst[n]; break;
      case OR_FPOP:
        for (i = 0; i < Q; ++i) out[n * Q + i] = fl ? p[i] : 0.0;
        break;
      case OR_GPOP:
        for (i = 0; i < QA; ++i) out[n * QA + i] = fl ? s->gc[n * QA + i] : 0.0;
        break;
      default: return -1;
    }
  }
  return 0;
}

int or_get_type(const or_sim *s, uint8_t *out) {
  memcpy(out, s->type, s->N);
  return 0;
}

int or_get_label(const or_sim *s, int32_t *out) {
  memcpy(out, s->label, sizeof(int32_t) * s->N);
  return 0;
}

int or_num_bubbles(const or_sim *s) { return s->nb; }

int or_bubbles(const or_sim *s, int32_t *id, int64_t *root, double *vol, double *mass,
               double *pres, int32_t *atm) {
  int k;
  for (k = 0; k < s->nb; ++k) {
    id[k] = s->bid[k];
    root[k] = s->broot[k];
    vol[k] = s->bV[k];
    mass[k] = s->bm[k];
    pres[k] = s->bp[k];
    atm[k] = s->batm[k];
  }
  return s->nb;
}

int or_ledger(const or_sim *s, double *out) {
  long n;
  int i, k;
  for (i = 0; i < 8; ++i) out[i] = 0.0;
  for (n = 0; n < s->N; ++n) {
    if (s->type[n] == LIQ) out[0] += pop_sum(s->fc + n * s->Q, s->Q);
    if (s->type[n] == IFC) out[0] += s->M[n];
    if (s->type[n] == LIQ || s->type[n] == IFC) {
      out[3] += pop_sum(s->gc + n * s->QA, s->QA);
      for (i = 0; i < s->Q; ++i)
        if (!isfinite(s->fc[n * s->Q + i])) out[7] += 1.0;
    }
  }
  for (k = 0; k < s->nb; ++k) out[4] += s->bm[k];
  out[1] = s->led[1];
  out[2] = s->led[2];
  out[5] = s->led[5];
  out[6] = s->led[6];
  return 0;
}

/*
 * lbf_oracle.h -- plain, slow FP64 CPU oracle of the free-surface lattice
 * Boltzmann foaming step (LBfoam, arXiv 1908.04262).
 *
 * TEST INFRASTRUCTURE ONLY.  Only the test-suite, the smoke check and the
 * CPU-baseline leg of the benchmark may load this library.  It shares no
 * source, header, table or helper with the CUDA path.
 *
 * Every routine follows the paper's equations in the paper's order:
 *   Sec. 2 (LBE, BGK and the TRT and MRT variants it names, equilibrium,
 *           moments, bounce-back),
 *   Sec. 2.1 (VOF fill level, mass exchange, cell conversion),
 *   Sec. 2.2 (free-surface reconstruction, gas density, ideal-gas law),
 *   Sec. 2.3 (tau-nu relation, Carreau-Yasuda),
 *   Sec. 3.1-3.2 (D2Q5/D3Q7 advection-diffusion, gas flux, Henry's law),
 *   Sec. 3.3 (disjoining pressure, PLIC, Appendix A / Algorithm 1),
 *   Sec. 3.5 (per-iteration bubble labelling, merge/split redistribution).
 */
#ifndef LBF_ORACLE_H
#define LBF_ORACLE_H
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct {
  int nx, ny, nz;            /* nz == 1 selects D2Q9 + D2Q5, else D3Q19 + D3Q7 */
  double tau, rho0;          /* Newtonian relaxation time; reference density   */
  double accel[3];           /* body acceleration a (Guo forcing)               */
  int rheo;                  /* 0 Newtonian, 1 power law, 2 Carreau-Yasuda     */
  double rheo_n, rheo_k, rheo_lambda, rheo_a, tau0, tau_inf, tau_min, tau_max;
  double sigma, k_pi, d_max; /* surface tension gamma, disjoining slope, cutoff */
  double D, kH, RT, c0, q, p0;
  double fill_height;        /* liquid below this height along the up axis     */
  int walls;                 /* bit f of the face list -x,+x,-y,+y,-z,+z        */
  double wall_u[3];          /* velocity of the walls on the +y face            */
  int atmosphere;            /* 1: gas touching the top interior layer is at p0 */
  double eps;                /* conversion margin on alpha                      */
  int bubble_capacity;
  int collision;             /* 0 BGK, 1 two relaxation times (TRT), 2 multiple
                                relaxation times (MRT)                           */
  double trt_magic;          /* TRT: (tau - 1/2)(tau_minus - 1/2); MRT: the same
                                product fixes the energy-flux rate s_q           */
  int kappa;                 /* curvature in the step: 0 least squares, 1 height
                                function (least squares where it is undefined)  */
  double mrt_rates[4];       /* MRT: s_e, s_eps, s_pi, s_m; 0 takes 1/tau for the
                                first three and s_q for s_m                      */
} or_config;

typedef struct or_sim or_sim;

or_sim *or_create(const or_config *cfg);
void or_destroy(or_sim *s);
int or_error(const or_sim *s);

/* Replace the state: per-cell type (0 gas, 1 liquid, 2 interface, 3 wall),
 * density, velocity (3 per cell, x fastest inside a cell), fill level and
 * dissolved-gas concentration.  Populations are set to equilibrium. */
int or_set_cells(or_sim *s, const uint8_t *type, const double *rho,
                 const double *u, const double *alpha, const double *c);
int or_nucleate(or_sim *s, int n, const double *centres, const double *radii);
int or_step(or_sim *s, int nsteps);

/* field ids for or_get */
enum { OR_RHO = 0, OR_U = 1, OR_ALPHA = 2, OR_MASS = 3, OR_CONC = 4,
       OR_KAPPA = 5, OR_PI = 6, OR_NORMAL = 7, OR_DSTAR = 8, OR_FPOP = 9,
       OR_GPOP = 10 };
int or_get(const or_sim *s, int field, double *out);
int or_get_type(const or_sim *s, uint8_t *out);
int or_get_label(const or_sim *s, int32_t *out);
int or_num_bubbles(const or_sim *s);
/* per bubble: id, canonical label (min linear index), volume, gas mass,
 * pressure, atmosphere flag */
int or_bubbles(const or_sim *s, int32_t *id, int64_t *root, double *vol,
               double *mass, double *pres, int32_t *atm);
/* [0] lattice liquid mass, [1] unplaced excess, [2] liquid removed by
 * nucleation, [3] dissolved gas, [4] bubble gas, [5] gas exchanged with the
 * outside (atmosphere, collapse, birth, unlabelled cells), [6] gas added by
 * the source term, [7] non-finite population count */
int or_ledger(const or_sim *s, double *out8);

/* Height-function curvature of every interface cell (the second classical
 * curvature Sec. 2.2 names besides the smoothed gradient): columns of
 * 7 cells along the dominant axis of the cell's geometry normal, 3 (2D) or
 * 3 x 3 (3D) of them around the cell, summed fill levels as heights,
 * centred differences; same sign and scale as the least-squares kappa
 * (1/(2R) on a gas disk, 1/R on a gas sphere).  out[n] = 0 for other cells,
 * NaN where a column meets a wall or the normal is zero. */
int or_hf_curvature(const or_sim *s, double *out);

/* test hooks for the merge/split pins */
int or_debug_set_types(or_sim *s, const uint8_t *type);
int or_debug_relabel(or_sim *s);

/* geometry helpers exposed for pins */
double or_plic_liquid_fraction(int dim, const double *n, double s);
double or_plic_offset(int dim, const double *n, double alpha);
/* test hook: least-squares curvature of np (<= 27) points (x, y, z in the
 * local frame of a cell: tangents, then the normal into the liquid) */
double or_lsq_kappa(int dim, const double *pts, int np);

/* The moment basis of the MRT collision for the oracle's velocity order of
 * a 2D (D2Q9) or 3D (D3Q19) lattice: M receives Q x Q doubles (row k is
 * moment k evaluated at every velocity), grp Q group ids (0 conserved,
 * 1 energy e, 2 energy square eps, 3 energy flux q, 4 stress p, 5 pi,
 * 6 third-order m).  Returns Q. */
int or_mrt_basis(int dim, double *M, int32_t *grp);

#ifdef __cplusplus
}
#endif
#endif

/*
 * lbf.h -- C ABI of the GB300 (sm_103a) free-surface lattice Boltzmann
 * foaming step (LBfoam, arXiv 1908.04262).
 *
 * One lbf_sim owns one lattice on one GPU: populations of the flow
 * (D2Q9 / D3Q19, Sec. 2) and of the dissolved gas (D2Q5 / D3Q7, Sec. 3.1),
 * cell types and fill levels (Sec. 2.1), bubble labels and the bubble table
 * (Sec. 2.2 Eq. idealgas, Sec. 3.5), curvature and disjoining pressure
 * (Sec. 2.2 Eq. rhob, Sec. 3.3).  All device memory is owned by the library.
 *
 * Conventions shared by every entry point
 *  - Return value: 0 on success, a negative LBF_E* code on failure; the
 *    message of the last failure on the calling thread is lbf_last_error().
 *  - Cells are indexed n = x + nx*(y + ny*z); the up axis is y in 2D
 *    (nz == 1) and z in 3D.  Every face is periodic unless its bit is set in
 *    cfg.walls (bit 0 -x, 1 +x, 2 -y, 3 +y, 4 -z, 5 +z), which turns the
 *    outermost layer of that face into half-way bounce-back walls (Sec. 2).
 *  - Work is queued on cfg.stream (a cudaStream_t; NULL = the legacy default
 *    stream).  Calls that return host data synchronise that stream.
 *  - A lbf_sim is not thread-safe; distinct lbf_sim objects are independent.
 *  - Host pointers are plain pageable or pinned memory owned by the caller;
 *    device pointers must be on the lbf_sim's device and stay valid for the
 *    duration of the call (work on them is complete when the call returns).
 */
#ifndef LBF_H
#define LBF_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* error codes */
#define LBF_OK 0
#define LBF_EINVAL (-1)     /* bad argument or configuration                  */
#define LBF_ENOMEM (-2)     /* device allocation failed                       */
#define LBF_ECUDA (-3)      /* a CUDA runtime call failed                     */
#define LBF_ENOTCONV (-4)   /* union-find iteration cap reached               */
#define LBF_ENONFINITE (-5) /* a NaN or infinity given to lbf_set_cells, or
                               non-finite populations found by lbf_ledger   */
#define LBF_ECAPACITY (-6)  /* more bubbles than cfg.bubble_capacity          */

typedef struct lbf_sim lbf_sim;

/* population storage (the arithmetic type follows in brackets):
 * FP64 [f64], FP32 [f32], FP16S / BF16S: populations stored as f - w_i
 * (and g - w_i c0) in binary16 / bfloat16 [f32] */
typedef enum { LBF_FP64 = 0, LBF_FP32 = 1, LBF_FP16S = 2, LBF_BF16S = 3 } lbf_storage;
typedef enum { LBF_NEWTONIAN = 0, LBF_POWERLAW = 1, LBF_CARREAU_YASUDA = 2 } lbf_rheology;

typedef struct {
  int nx, ny, nz;           /* lattice; nz == 1 selects D2Q9 + D2Q5            */
  int storage;              /* lbf_storage                                      */
  double tau, rho0;         /* Newtonian relaxation time (Sec. 2.3 Eq. tau)     */
  double accel[3];          /* body acceleration (Guo forcing)                  */
  int rheo;                 /* lbf_rheology (Sec. 2.3)                           */
  double rheo_n, rheo_k;    /* power law: nu = k gamma_dot^(n-1)                */
  double rheo_lambda, rheo_a, tau0, tau_inf; /* Carreau-Yasuda, Eq. carreauTau */
  double tau_min, tau_max;  /* clamp of the local relaxation time               */
  double sigma;             /* surface tension gamma (Eq. rhob)                  */
  double k_pi, d_max;       /* disjoining pressure slope and range (Sec. 3.3)   */
  double D, kH, RT, c0, q, p0; /* diffusivity, Henry constant, gas constant x
                                  temperature, initial concentration, source,
                                  ambient pressure (Sec. 3.1-3.2)               */
  double fill_height;       /* initial liquid below this height (up axis)      */
  int walls;                /* bounce-back faces, see above                     */
  double wall_u[3];         /* velocity of the walls of the +y face             */
  int atmosphere;           /* 1: gas touching the top interior layer is held
                               at p0 (the headspace)                            */
  double eps;               /* conversion margin: fill when alpha > 1 + eps,
                               empty when alpha < -eps (Sec. 2.1)               */
  int bubble_capacity;      /* maximum number of bubbles (<= 16384)             */
  void *stream;             /* cudaStream_t used by every call                  */
  int collision;            /* 0 BGK (Sec. 2 Eq. collision); 1 two relaxation
                               times, a variant Sec. 2 names: the parts of
                               f - f_eq even under e -> -e relax at 1/tau, the
                               odd parts at 1/tau_m; 2 multiple relaxation
                               times, the other variant Sec. 2 names: the
                               moments of the orthogonal basis of Lallemand
                               and Luo (D2Q9) or d'Humieres et al. (D3Q19)
                               relax at their own rates, the stress at 1/tau,
                               the energy flux at 1/tau_m, the rest at
                               mrt_rates (the dissolved gas stays BGK)         */
  double trt_magic;         /* collision 1 and 2: (tau - 1/2)(tau_m - 1/2) > 0;
                               3/16 puts half-way bounce-back walls exactly
                               half-way for every tau                           */
  int kappa;                /* curvature of Eq. rhob: 0 least squares; 1 height
                               function, the second method Sec. 2.2 names
                               (summed fill levels of 7-cell columns along the
                               normal's dominant axis, 3 columns in 2D, 3 x 3
                               in 3D, centred differences; the least-squares
                               value stays where a column meets a wall)        */
  double mrt_rates[4];      /* collision 2: rates s_e (energy: bulk viscosity
                               (2/d)(1/s_e - 1/2)/3), s_eps (energy square),
                               s_pi (fourth-order anisotropic, 3D) and s_m
                               (third-order, 3D), each in [0, 2); 0 takes 1/tau
                               for the first three and 1/tau_m for s_m (all 0:
                               the TRT collision)                               */
} lbf_config;

/* one row of the bubble table */
typedef struct {
  int32_t id;        /* stable id: kept through growth; merges keep the
                        smallest id, the largest piece of a split keeps it  */
  int32_t atm;       /* 1 for the atmosphere (held at p0)                   */
  int64_t label;     /* canonical label: smallest linear index of its gas  */
  double volume;     /* gas cells + sum of (1 - alpha) of interface cells   */
  double gas_mass;   /* m_g (Eq. idealgas)                                  */
  double pressure;   /* p_g = m_g RT / V (Eq. idealgas)                     */
} lbf_bubble;

/* Sec. 2-3: allocate and initialise a lattice: liquid below fill_height
 * at rest (f = f_eq(rho0, 0), g = g_eq(c0, 0)), walls, headspace; labels
 * bubbles and computes the geometry.  *out receives the handle.
 * Errors: LBF_EINVAL (sizes <= 0, more than 2^31-1 cells, bad enums, tau or
 * tau_min <= 1/2, capacity outside [1, 16384], trt_magic <= 0 with
 * collision 1 or 2, an MRT rate outside [0, 2)), LBF_ENOMEM, LBF_ECUDA. */
int lbf_create(const lbf_config *cfg, lbf_sim **out);

/* Release every resource; NULL is ignored. */
void lbf_destroy(lbf_sim *s);

/* Sec. 3.4: nucleate n gas spheres (disks in 2D).  centres: host, n x 3
 * doubles (lattice coordinates, z ignored in 2D); radii: host, n doubles.
 * at_step: host, n step numbers at which each nucleus appears, or NULL for
 * "now".  Only liquid cells are carved; a cell's fill level is the fraction
 * of its 4^d sub-cell points outside the sphere.  A new bubble starts in
 * Laplace equilibrium, p = p0 + (d-1) sigma / R_eq.
 * Errors: LBF_EINVAL (n < 0, NULL arrays, radius <= 0, step in the past). */
int lbf_nucleate(lbf_sim *s, int n, const double *centres, const double *radii,
                 const long long *at_step);

/* Replace the state from host arrays of N cells: type (0 gas, 1 liquid,
 * 2 interface, 3 wall), rho, u (3 doubles per cell), alpha (fill level of
 * interface cells), c (dissolved gas).  Populations are set to equilibrium;
 * liquid touching gas becomes interface with alpha = 1; every bubble is
 * new (Laplace equilibrium).  The arrays are checked on the device before
 * they replace anything; a rejected call leaves the state as it was.
 * Errors: LBF_EINVAL (NULL arrays, a type outside 0..3, rho <= 0 in a liquid
 * or interface cell), LBF_ENONFINITE (a NaN or infinity in rho, u, alpha or
 * c), LBF_ECUDA. */
int lbf_set_cells(lbf_sim *s, const uint8_t *type, const double *rho, const double *u,
                  const double *alpha, const double *c);

/* Advance nsteps full steps: stream/collide/reconstruct/exchange/ADE
 * (Sec. 2, 2.1, 2.2, 3.1, 3.2), conversion (Sec. 2.1), labelling and bubble
 * update (Sec. 3.5, Eq. idealgas), curvature and disjoining pressure
 * (Sec. 2.2, 3.3); nuclei due in the interval are carved at their step.
 * Steps run as CUDA graphs of one, two or four steps; the first call (and
 * the first after lbf_mlp_attach or lbf_checkpoint_load) captures and
 * instantiates every graph shape for both parities before any step runs.
 * Synchronises at the end and returns the sticky device error, if any
 * (LBF_ECAPACITY, LBF_ENOTCONV; LBF_ECUDA when a wait of the learned
 * curvature on the tensor cores ran past its bound).  Errors: LBF_EINVAL
 * (nsteps < 0). */
int lbf_step(lbf_sim *s, int nsteps);

/* Copy the bubble table to host memory: out has room for capacity rows;
 * *count receives the number of bubbles (rows beyond capacity are dropped).
 * Synchronises.  Errors: LBF_EINVAL (NULL pointers, capacity < 0). */
int lbf_bubbles(lbf_sim *s, lbf_bubble *out, int capacity, int *count);

/* field bits for lbf_fields; dst[k] receives the k-th requested field in
 * bit order; vector fields (U, NORMAL) hold 3 values per cell (x fastest
 * inside the cell).  RHO, U, CONC are zero outside liquid and interface
 * cells; FLAGS and LABEL are int32 whatever dtype says. */
#define LBF_F_RHO (1u << 0)    /* density sum f (Sec. 2)                       */
#define LBF_F_U (1u << 1)      /* velocity, force-shifted (Sec. 2)             */
#define LBF_F_ALPHA (1u << 2)  /* fill level (Sec. 2.1 Eq. alpha)              */
#define LBF_F_MASS (1u << 3)   /* liquid mass M (rho in liquid cells)          */
#define LBF_F_FLAGS (1u << 4)  /* cell type 0..3                               */
#define LBF_F_CONC (1u << 5)   /* dissolved gas sum g (Sec. 3.1)               */
#define LBF_F_KAPPA (1u << 6)  /* curvature (Eq. rhob)                         */
#define LBF_F_LABEL (1u << 7)  /* bubble index into the table, or -1           */
#define LBF_F_PI (1u << 8)     /* disjoining pressure (Sec. 3.3)               */
#define LBF_F_NORMAL (1u << 9) /* interface normal, into the liquid            */
#define LBF_F_DSTAR (1u << 10) /* PLIC offset of the interface plane           */
/* Copy the requested fields.  dst_is_device: 1 if every dst[k] is device
 * memory, 0 for host memory (the call then synchronises; page-locked host
 * memory is written by one direct copy per field, pageable memory through
 * two page-locked chunks of the library's).  dtype: 0 float, 1 double for
 * the floating-point fields.  Errors: LBF_EINVAL. */
int lbf_fields(lbf_sim *s, unsigned mask, void *const *dst, int dst_is_device, int dtype);

/* FP64 ledgers (synchronises): [0] liquid mass on the lattice (sum of rho
 * over liquid cells + M over interface cells), [1] excess mass that found
 * no interface neighbour, [2] liquid removed by nucleation, [3] dissolved
 * gas, [4] gas in bubbles, [5] gas exchanged with the outside, [6] gas added
 * by the source term, [7] count of non-finite populations.
 * Returns LBF_ENONFINITE when [7] > 0. */
int lbf_ledger(lbf_sim *s, double *out8);

/* Checkpoint and resume (the paper has no counterpart; its Palabos base
 * writes checkpoints of its own).  A checkpoint holds every device array the
 * sim made at creation (populations, flags, masses, fill levels, geometry,
 * labels, union-find forest, bubble tables, lists, ledgers), the step count
 * and the nuclei still queued: loading it into a sim created with the same
 * configuration (and with the learned curvature attached alike) resumes the
 * run where it was saved.
 * lbf_checkpoint_bytes: *bytes = size of the checkpoint.
 * lbf_checkpoint_save: writes it to host memory dst (bytes >= that size);
 *   synchronises.  Errors: LBF_EINVAL, LBF_ECUDA.
 * lbf_checkpoint_load: restores from host memory src (bytes long);
 *   synchronises.  Errors: LBF_EINVAL (not a checkpoint, too short, another
 *   lattice or storage, the learned curvature attached differently or with
 *   other parameters -- the header holds a 64-bit FNV-1a hash of them),
 *   LBF_ECUDA. */
int lbf_checkpoint_bytes(lbf_sim *s, size_t *bytes);
int lbf_checkpoint_save(lbf_sim *s, void *dst, size_t bytes);
int lbf_checkpoint_load(lbf_sim *s, const void *src, size_t bytes);

/* Kernel timing for measurements: while enabled, lbf_step replays a second
 * CUDA graph of the same step in which every kernel group is bracketed by
 * CUDA event records on cfg.stream, and synchronises after each step to read
 * them.  lbf_timing_read sums the device time of every kernel group since
 * the last enable: out_ms[k] and out_launches[k] for k < nmax, in the order
 * of lbf_timing_name(k).  Returns the number of groups. */
int lbf_timing_enable(lbf_sim *s, int enable);
int lbf_timing_read(lbf_sim *s, double *out_ms, long long *out_launches, int nmax);
const char *lbf_timing_name(int k);

/* Counts of gas, liquid, interface and wall cells (synchronises). */
int lbf_cell_counts(lbf_sim *s, long long *out4);

/* Number of completed steps. */
long long lbf_step_count(const lbf_sim *s);


const char *lbf_last_error(void);

/* ------------------------------------------------------------------------
 * Learned interface curvature (not in the paper; replaces the least-squares
 * kappa of Sec. 2.2 Eq. rhob where it is inside its training range).
 * Network: canonical 3x3x3 fill-level stencil (27 values in [0,1], index
 * (dz+1)*9 + (dy+1)*3 + (dx+1); axes reflected so the interface normal is
 * non-negative, then ordered by increasing normal component) -> 64 -> 64 -> 1
 * with SiLU; output y = 4 kappa.  BF16 weights and activations, FP32
 * accumulation in tensor memory (tcgen05 MMAs on tiles of 128 rows).
 * Parameters theta: 6017 FP32 values, W1 (64x27 row-major), b1 (64), W2
 * (64x64), b2 (64), W3 (64), b3 (1).  Every wait of these kernels on the
 * tensor cores is bounded (about half a second); past the bound a kernel
 * frees its tensor memory and reports NaN in its outputs or loss.
 */
typedef struct {
  unsigned long long seed; /* counter-based generator seed                   */
  int n_samples;           /* synthetic stencils generated on the device     */
  int epochs, batch;       /* Adam epochs over the samples, mini-batch size  */
  double lr;               /* Adam learning rate (x0.1 for the last quarter) */
  double rmin, rmax;       /* radii, log-uniform; spheres and ellipsoids     */
  double noise;            /* augmentation: fill levels strictly inside (0,1)
                              get uniform noise of this half-width, clamped  */
  const float *x_extra;    /* device, n_extra x 27: further canonical stencils
                              (e.g. harvested by lbf_mlp_harvest), or NULL   */
  const float *y_extra;    /* device, n_extra targets y = 4 kappa            */
  int n_extra;
  void *stream;            /* cudaStream_t                                   */
} lbf_mlp_train_cfg;

/* y[i] for n canonical stencils x (device, n x 27 FP32); theta and y are
 * device pointers.  Asynchronous on `stream`; allocates nothing.
 * Errors: LBF_EINVAL. */
int lbf_mlp_forward(const float *theta, const float *x, int n, float *y, void *stream);
/* Loss 0.5 mean((y - t)^2) of n stencils x with targets t (all device) and
 * its gradient: grad (device, 6017 FP32) and *loss (device, one double) are
 * overwritten.  Asynchronous; takes a 21 KB packed copy of the network
 * from the stream's memory pool for the call.  Errors: LBF_EINVAL,
 * LBF_ECUDA. */
int lbf_mlp_loss_grad(const float *theta, const float *x, const float *t, int n, float *grad, double *loss,
                      void *stream);
/* n synthetic training pairs (canonical stencil, y = 4 kappa) into device
 * buffers x (n x 27) and y (n): voxelised spheres and ellipsoids (axes
 * 0.75-1.25 R, random rotation and sub-cell offset, 3/4 gas inside), R
 * log-uniform in [rmin, rmax], fill level = fraction of 6^3 sub-points in
 * the liquid, kappa = analytic mean curvature at the surface point nearest
 * the cell centre (positive for convex gas).  Errors: LBF_EINVAL, LBF_ECUDA. */
int lbf_mlp_generate(unsigned long long seed, int n, double rmin, double rmax, float *x, float *y, void *stream);
/* The same from explicit shape parameters (host, n x 20 doubles: centre[3],
 * axes[3], rotation[9] row-major, gas_inside, cell[3], unused); synchronises. */
int lbf_mlp_stencils_from_params(const double *params, int n, float *x, float *y, void *stream);
/* Train the network on the device (generation, forward/backward on the
 * tensor cores, Adam); theta_io (host, 6017) holds the start point and
 * receives the result; loss_curve (host, epochs floats, may be NULL)
 * receives the mean training loss of every epoch.  Synchronises. */
int lbf_mlp_train(const lbf_mlp_train_cfg *cfg, float *theta_io, float *loss_curve);
/* Training pairs from the current state of s (3D): the canonical stencil of
 * every interface cell (x: device, cap x 27 FP32) and the target
 * y = 4 / R_eq of the cell's bubble (y: device, cap FP32), R_eq =
 * (3 V / 4 pi)^(1/3) from the bubble's volume -- the curvature of a
 * relaxed, nearly spherical bubble.  Skipped: cells with a wall in the
 * stencil, a zero normal, no bubble or the atmosphere.  cells (device,
 * cap int32, may be NULL) receives each pair's linear cell index; the
 * order of the pairs is unspecified.  *count (host)
 * receives the number written (<= cap).  Synchronises.
 * Errors: LBF_EINVAL, LBF_ECUDA. */
int lbf_mlp_harvest(lbf_sim *s, float *x, float *y, int *cells, int cap, int *count);
/* Use the network for kappa in every following step of s (3D only): theta
 * host, copied; NULL returns to the least-squares curvature.  The network's
 * kappa replaces the least-squares value where |kappa_LSQ| lies in
 * [0.02, 0.55] and no wall is in the stencil.  Errors: LBF_EINVAL. */
int lbf_mlp_attach(lbf_sim *s, const float *theta);

/* Bubble labels of a cell-type field without allocating any memory.
 * The paper has no counterpart: this is a service for callers that cannot
 * call cudaMalloc (a framework whose caching allocator has reserved the
 * device, or a real-time loop where an allocation may stall).
 * type: device, N = nx*ny*nz bytes, cell types 0 gas, 1 liquid,
 * 2 interface, 3 wall (cells indexed as everywhere in this header; every
 * face periodic).  label: device, N int32 outputs -- gas cells get the
 * index of their bubble (bubbles = gas regions connected over D2Q9/D3Q19
 * links, numbered by their smallest cell index), interface cells the
 * smallest index among their gas neighbours, other cells -1; identical to
 * lbf_fields(LBF_F_LABEL) after lbf_set_cells with the same types.
 * count: device, one int32: the number of bubbles, or -1 if there were more
 * than 4096 of them or the union-find hit its iteration cap.
 * Work is queued on `stream` (a cudaStream_t) and the call returns without
 * waiting.  Scratch: one static device array per GPU, held from the first
 * call on that GPU until the process exits, for at most 1,048,576 cells
 * (and 65,536 tiles of 32x8x4 / 32x32 cells); larger lattices return
 * LBF_EINVAL.  Each call made outside stream capture looks the array's
 * address up with the calling thread's device current (so a device reset or
 * another context never leaves a stale address); make the first call on a
 * device before any stream capture (LBF_EINVAL otherwise).
 * Every call on a device shares the array: calls that overlap on the GPU
 * (other streams, other threads) race and must be serialised by the caller;
 * each call clears the counters it needs.  No cudaMalloc, cudaFree or
 * allocating library routine is called.
 * Errors: LBF_EINVAL (NULL buffers, bad extents, lattice too large),
 * LBF_ECUDA. */
int lbf_label_gas_noalloc(const uint8_t *type, int nx, int ny, int nz, int32_t *label, int32_t *count,
                          void *stream);

#ifdef __cplusplus
}
#endif
#endif

// lbf_common.cuh -- lattice definitions, storage codecs, the in-place AA
// population layout and the launch parameter block shared by every kernel of
// the GB300 free-surface foaming step.
//
// Populations are SoA, one plane of N cells per direction, updated in place
// with the AA access pattern: a step that starts from parity 0 reads and
// writes only the cell's own slots; a step that starts from parity 1 reads
// from and writes to the neighbours' slots.  Each (cell, direction) outgoing
// population owns exactly one slot in either parity, so no two threads write
// the same slot.
#pragma once

#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <stdint.h>

namespace lbf {

// cell types (bits 0-1 of the flag byte), conversion marks (bits 2-4), a
// static bit for cells with a wall among their lattice neighbours (bit 5)
// and the parity of the step that set the mark (bit 6): the liquid sweep of
// the next step starts before the last conversion has written the new types
// over its marks, and runs beside the interface sweep that marks cells for
// its own conversion; the parity tells the two kinds of mark apart
enum : int { T_GAS = 0, T_LIQ = 1, T_IFC = 2, T_WALL = 3 };
enum : int { MK_NONE = 0, MK_FILL = 1, MK_EMPTY = 2, MK_GI = 3, MK_LI = 4 };
constexpr uint8_t NEARWALL = 0x20;
constexpr uint8_t MARKPAR = 0x40;
__device__ __forceinline__ uint8_t mark_bits(int mk, int par) {
  return (uint8_t)((mk << 2) | (par ? MARKPAR : 0));
}
__device__ __forceinline__ int ftype(uint8_t f) { return f & 3; }
__device__ __forceinline__ int fmark(uint8_t f) { return (f >> 2) & 7; }

// fields of the export kernel (bit order of the public field mask)
enum : int { FLD_RHO = 0, FLD_U = 1, FLD_ALPHA = 2, FLD_MASS = 3, FLD_FLAGS = 4, FLD_CONC = 5,
             FLD_KAPPA = 6, FLD_LABEL = 7, FLD_PI = 8, FLD_NORMAL = 9, FLD_DSTAR = 10 };

// sticky device error bits
enum : int { ERR_CAPACITY = 1, ERR_NOTCONV = 2, ERR_HASH = 4 };

// ---------------------------------------------------------------------------
// velocity sets (Sec. 2: D2Q9 / D3Q19 with the paper's weights; Sec. 3.1:
// D2Q5 / D3Q7 are the first 5 / 7 vectors).  Opposite vectors are adjacent.

template <int D> struct Lat;
template <> struct Lat<2> {
  static constexpr int Q = 9, QA = 5;
  __host__ __device__ static constexpr int cx(int i) { return i == 1 || i == 5 || i == 7 ? 1 : (i == 2 || i == 6 || i == 8 ? -1 : 0); }
  __host__ __device__ static constexpr int cy(int i) { return i == 3 || i == 5 || i == 8 ? 1 : (i == 4 || i == 6 || i == 7 ? -1 : 0); }
  __host__ __device__ static constexpr int cz(int) { return 0; }
  __host__ __device__ static constexpr double w(int i) { return i == 0 ? 4.0 / 9.0 : (i < 5 ? 1.0 / 9.0 : 1.0 / 36.0); }
  __host__ __device__ static constexpr double wa(int i) { return i == 0 ? 1.0 / 3.0 : 1.0 / 6.0; }
  static constexpr double csa2 = 1.0 / 3.0;
};
template <> struct Lat<3> {
  static constexpr int Q = 19, QA = 7;
  __host__ __device__ static constexpr int cx(int i) {
    return (i == 1 || i == 7 || i == 9 || i == 13 || i == 15) ? 1 : ((i == 2 || i == 8 || i == 10 || i == 14 || i == 16) ? -1 : 0);
  }
  __host__ __device__ static constexpr int cy(int i) {
    return (i == 3 || i == 7 || i == 11 || i == 14 || i == 17) ? 1 : ((i == 4 || i == 8 || i == 12 || i == 13 || i == 18) ? -1 : 0);
  }
  __host__ __device__ static constexpr int cz(int i) {
    return (i == 5 || i == 9 || i == 11 || i == 16 || i == 18) ? 1 : ((i == 6 || i == 10 || i == 12 || i == 15 || i == 17) ? -1 : 0);
  }
  __host__ __device__ static constexpr double w(int i) { return i == 0 ? 1.0 / 3.0 : (i < 7 ? 1.0 / 18.0 : 1.0 / 36.0); }
  __host__ __device__ static constexpr double wa(int i) { return i == 0 ? 0.25 : 0.125; }
  static constexpr double csa2 = 0.25;
};
__host__ __device__ constexpr int opp(int i) { return i == 0 ? 0 : ((i & 1) ? i + 1 : i - 1); }

// ---------------------------------------------------------------------------
// storage codecs: the arithmetic type R and the shifted reduced-precision
// forms (stored value = population - shift, shift = w_i rho0 or wa_i c0)

template <class S> struct ST;
template <> struct ST<double> { using R = double; };
template <> struct ST<float> { using R = float; };
template <> struct ST<__half> { using R = float; };
template <> struct ST<__nv_bfloat16> { using R = float; };

__device__ __forceinline__ double ld(const double *p, size_t k, double) { return p[k]; }
__device__ __forceinline__ float ld(const float *p, size_t k, float) { return p[k]; }
__device__ __forceinline__ float ld(const __half *p, size_t k, float sh) { return __half2float(p[k]) + sh; }
__device__ __forceinline__ float ld(const __nv_bfloat16 *p, size_t k, float sh) { return __bfloat162float(p[k]) + sh; }
__device__ __forceinline__ void st(double *p, size_t k, double v, double) { p[k] = v; }
__device__ __forceinline__ void st(float *p, size_t k, float v, float) { p[k] = v; }
__device__ __forceinline__ void st(__half *p, size_t k, float v, float sh) { p[k] = __float2half_rn(v - sh); }
__device__ __forceinline__ void st(__nv_bfloat16 *p, size_t k, float v, float sh) { p[k] = __float2bfloat16_rn(v - sh); }
__device__ __forceinline__ double ld(const double *p, int k, double) { return p[k]; }
__device__ __forceinline__ float ld(const float *p, int k, float) { return p[k]; }
__device__ __forceinline__ float ld(const __half *p, int k, float sh) { return __half2float(p[k]) + sh; }
__device__ __forceinline__ float ld(const __nv_bfloat16 *p, int k, float sh) { return __bfloat162float(p[k]) + sh; }
__device__ __forceinline__ void st(double *p, int k, double v, double) { p[k] = v; }
__device__ __forceinline__ void st(float *p, int k, float v, float) { p[k] = v; }
__device__ __forceinline__ void st(__half *p, int k, float v, float sh) { p[k] = __float2half_rn(v - sh); }
__device__ __forceinline__ void st(__nv_bfloat16 *p, int k, float v, float sh) { p[k] = __float2bfloat16_rn(v - sh); }

// ---------------------------------------------------------------------------
// bubble table (one of two, swapped every step)

struct Table {
  double *m, *p, *V, *dm;  // gas mass, pressure, volume, gas gained this step
  int *id, *atm, *root;    // stable id, atmosphere flag, canonical label
  int *ng;                 // gas cells of the bubble (V = ng + interface shares)
  int *count;              // number of rows (device)
};

// everything a kernel may need; passed by value
struct Params {
  int nx, ny, nz, dim;
  long long N;
  void *f, *g;           // populations (storage type)
  uint8_t *flags;        // cell flags (conversion marks written in place)
  unsigned *wmask;       // per cell: bit i set when x - e_i is a wall (walls never move)
  int *ilist, *icount;   // interface cells at the start of the step
  int *inext, *inext_count;  // interface cells after the conversion
  int *nlist, *ncount;   // gas/liquid cells turning interface this step
  int *mlist, *mcount;   // interface cells the sweep marked to fill or empty this step
                         // (the count is kept per parity: see make_params)
  // 32-cell segments along x that hold interface cells (the interface
  // kernels run one warp per segment, one lane per cell)
  int *seglist, *segcount;       // at the start of the step
  int *segnext, *segnext_count;  // after the conversion
  int *segflag;                  // per segment: 1 while listed in segnext (the interface sweep clears it)
  int list_blocks;       // persistent grid size of the thread-per-cell list kernels
  int warp_blocks;       // ... of the warp-per-cell list kernels (full occupancy)
  void *M, *phi;         // liquid mass, fill level (arithmetic type)
  void *uI;              // 3N: velocity of interface cells from the last step
  void *kappa, *Pi, *nrm, *dst, *ex;
  // 5 planes: density, velocity (3) and dissolved gas of each interface
  // cell after its sweep (the moments of its post-collision populations), which a
  // gas cell turning interface averages over its neighbours
  void *mom;
  int *label_old, *label_new, *parent;
  int *lsize;            // size of each tile-local gas component, at its root
  uint8_t *tstat;        // per union-find tile: 0 no gas, 1 one gas component, 2 several
  int *troot;            // per tile with one component: its root cell
  Table told, tnew;
  int *roots, *nroots;
  unsigned long long *hash;
  int *hlist, *hcount;   // occupied hash slots, in insertion order
  int hash_size, cap;
  // K10 scratch (2*cap each)
  int *gpar, *gnold, *gnnew, *gatm, *gminid, *gheir;
  double *gmold, *gvnew;
  unsigned long long *gvmax;
  int *next_id;
  double *led;                   // 8 ledger accumulators
  unsigned long long *fluid_updates;
  int *err;
  // what the conversion of this step did to the gas cells: 0 nothing (the
  // forest of the last labelling is still exact), 1 added some only (the
  // components can only grow or merge: the touched tiles, marked in
  // tdirty, are redone), anything else removed some or the state was set
  // from outside (full labelling).  NULL means always full.
  int *gas_dirty;
  uint8_t *tdirty;  // per union-find tile: touched by added gas cells since the last forest update
  // set by the marking when an added gas cell could join two bubbles or
  // move a bubble's smallest cell index: the step then needs the full
  // labelling (else the labels of the last step, patched, are exact)
  int *lab_slow;
  // after steps labelled without the union-find: bit 0, gas cells were
  // added (the forest lags behind in the touched tiles, tdirty, which the
  // next union-find labelling redoes); bit 1, gas cells were removed (the
  // next union-find labelling rebuilds the forest)
  int *forest_stale;
  // 1 while this step labels by patching the last labels (set on the device
  // after the marking; the union-find kernels then return at once, and the
  // patch kernels do otherwise).  NULL means the union-find labelling.
  int *lab_fast;
  // 1 when the labels of the last step are not the labels of the step
  // before patched at that step's listed cells (a full labelling ran, or the
  // state was set from outside): the next patched labelling then starts
  // from a full copy instead of copying the listed cells
  int *lab_full;
  // root moves of a patched step: [0] the bubble whose root cell turns
  // interface (-1 none; one bubble per step), [1] set when some bubble's
  // root is lowered by an added gas cell
  int *rmv;
  int tile_blocks;  // grid of the tile loops of the union-find (two blocks per SM)
  // label of each current root cell (rank among the sorted roots, -1 past
  // the bubble capacity); read only at cells that are roots
  int *rlabel;
  // tabulated relaxation time tau(A) of the non-Newtonian models for the
  // single-precision forms, as the relaxation rate 1 / tau: om_tab[k] at
  // ln A = tab_lnA0 + k * tab_dlnA
  const float *om_tab;
  int tab_n;
  float tab_lnA0, tab_inv_dlnA;
  // physics, in double and as float copies (the single-precision kernels
  // must not touch the FP64 pipe)
  struct PF {
    float tau, rho0, ax, ay, az, rn, rk, rlam, ra, tau0, tau_inf, tau_min, tau_max;
    float sigma, k_pi, d_max, taug, kH, RT, c0, q, p0, eps, uwx, uwy, uwz, trt_magic, omg, om;
    float mrt_se, mrt_seps, mrt_spi, mrt_sm;
  } pf;
  double tau, rho0, ax, ay, az;
  int has_force, rheo;
  int coll;           // collision: 0 BGK, 1 two relaxation times, 2 multiple
  int kappa_hf;       // height-function curvature (else least squares)
  double trt_magic;   // (tau - 1/2)(tau_m - 1/2)
  // multiple relaxation times: rates of the energy, energy-square,
  // fourth-order anisotropic and third-order moments (0: the stress rate
  // 1/tau for the first three, the energy-flux rate for the last)
  double mrt_se, mrt_seps, mrt_spi, mrt_sm;
  double rn, rk, rlam, ra, tau0, tau_inf, tau_min, tau_max;
  double sigma, k_pi, d_max, taug, kH, RT, c0, q, p0, eps;
  double uwx, uwy, uwz;
  double omg;  // 1 / taug
  double om;   // 1 / tau (the Newtonian relaxation rate)
  int walls, atmosphere, top_layer, ray_steps;
  int par;  // parity of the step (of the populations when it starts)
  // 1 when walls close every face and no fluid cell lies in a face layer:
  // no fluid cell then needs a periodic wrap of its neighbours
  int walled;
};

// a physics parameter in the arithmetic type R
template <class R> __device__ __forceinline__ R pv(double d, float f) {
  if constexpr (sizeof(R) == 4)
    return f;
  else
    return d;
}
#define PV(R, name) pv<R>(p.name, p.pf.name)

// ---------------------------------------------------------------------------
// indexing.  Full-lattice kernels run on a (ceil(nx/B), ny, nz) grid of
// B-thread blocks along x, so a thread finds its cell without division; the
// six periodic neighbour offsets are kept as index deltas.

// Lattices hold fewer than 2^31 cells (checked at creation), so cell
// indices and offsets are 32-bit; only plane offsets (direction x N) are
// 64-bit.
struct Cell {
  int x, y, z;
  int n;
  int dxm, dxp;  // -1 / +1 along x, wrapped
  int dym, dyp;  // -nx / +nx along y, wrapped
  int dzm, dzp;  // -nx*ny / +nx*ny along z, wrapped
};

__device__ __forceinline__ Cell cell_at(const Params &p, int x, int y, int z) {
  Cell c;
  c.x = x; c.y = y; c.z = z;
  const int nx = p.nx, nxy = p.nx * p.ny;
  c.n = x + nx * y + nxy * z;
  c.dxm = x == 0 ? p.nx - 1 : -1;
  c.dxp = x == p.nx - 1 ? 1 - p.nx : 1;
  c.dym = y == 0 ? (p.ny - 1) * nx : -nx;
  c.dyp = y == p.ny - 1 ? -(p.ny - 1) * nx : nx;
  c.dzm = z == 0 ? (p.nz - 1) * nxy : -nxy;
  c.dzp = z == p.nz - 1 ? -(p.nz - 1) * nxy : nxy;
  return c;
}

// the thread's cell in a full-lattice launch; false for padding threads
__device__ __forceinline__ bool grid_cell(const Params &p, Cell &c) {
  const int x = blockIdx.x * blockDim.x + threadIdx.x;
  c = cell_at(p, x < p.nx ? x : p.nx - 1, blockIdx.y, blockIdx.z);
  return x < p.nx;
}

// segments of 32 cells along x: ceil(nx / 32) per row of the lattice
__device__ __forceinline__ int seg_of(const Params &p, int n) {
  const int row = n / p.nx;
  return row * ((p.nx + 31) >> 5) + ((n - row * p.nx) >> 5);
}
// the lane's cell of segment `seg`; false past the end of the row
__device__ __forceinline__ bool seg_cell(const Params &p, int seg, int lane, Cell &c) {
  const int nxb = (p.nx + 31) >> 5;
  const int row = seg / nxb;
  const int x = (seg - row * nxb) * 32 + lane;
  const int z = row / p.ny;
  c = cell_at(p, x < p.nx ? x : p.nx - 1, row - z * p.ny, z);
  return x < p.nx;
}

// the same on a walled lattice (Params::walled): no fluid cell needs a
// periodic wrap, so the neighbour offsets come from the lattice sizes alone
// (uniform across the warp; face cells, all walls, get unwrapped offsets
// they never use)
__device__ __forceinline__ bool seg_cell_walled(const Params &p, int seg, int lane, Cell &c) {
  const int nxb = (p.nx + 31) >> 5;
  const int row = seg / nxb;
  const int x = (seg - row * nxb) * 32 + lane;
  const int z = row / p.ny;
  const int nx = p.nx, nxy = p.nx * p.ny;
  c.x = x < nx ? x : nx - 1;
  c.y = row - z * p.ny;
  c.z = z;
  c.n = c.x + nx * c.y + nxy * c.z;
  c.dxm = -1;
  c.dxp = 1;
  c.dym = -nx;
  c.dyp = nx;
  c.dzm = -nxy;
  c.dzp = nxy;
  return x < nx;
}

// cell from a linear index (rare paths only: uses division)
__device__ __forceinline__ Cell make_cell(const Params &p, long long n) {
  // lattices hold fewer than 2^31 cells: 32-bit division suffices
  const unsigned nxy = (unsigned)p.nx * (unsigned)p.ny;
  const unsigned u = (unsigned)n;
  const unsigned z = u / nxy;
  const unsigned r = u - z * nxy;
  const unsigned y = r / (unsigned)p.nx;
  return cell_at(p, (int)(r - y * (unsigned)p.nx), (int)y, (int)z);
}

// cell at offset (dx,dy,dz) in {-1,0,1}^3
__device__ __forceinline__ int at(const Params &, const Cell &c, int dx, int dy, int dz) {
  return c.n + (dx < 0 ? c.dxm : (dx > 0 ? c.dxp : 0)) + (dy < 0 ? c.dym : (dy > 0 ? c.dyp : 0)) +
         (dz < 0 ? c.dzm : (dz > 0 ? c.dzp : 0));
}

// general periodic offset (any distance)
__device__ __forceinline__ long long at_far(const Params &p, int x, int y, int z) {
  x %= p.nx; if (x < 0) x += p.nx;
  y %= p.ny; if (y < 0) y += p.ny;
  z %= p.nz; if (z < 0) z += p.nz;
  return x + (long long)p.nx * (y + (long long)p.ny * z);
}

template <int D> __device__ __forceinline__ int nb(const Params &p, const Cell &c, int i) {
  return at(p, c, Lat<D>::cx(i), Lat<D>::cy(i), Lat<D>::cz(i));
}
template <int D> __device__ __forceinline__ int src(const Params &p, const Cell &c, int i) {
  return at(p, c, -Lat<D>::cx(i), -Lat<D>::cy(i), -Lat<D>::cz(i));
}

// AA slots.  Parity 0: slot (i, n) holds the population arriving at n along
// e_i.  Parity 1: slot (opp(i), n) holds n's own outgoing population along e_i.
template <int D> __device__ __forceinline__ size_t slot_out(const Params &p, const Cell &c, long long n, int i, int par) {
  return par == 0 ? (size_t)i * p.N + nb<D>(p, c, i) : (size_t)opp(i) * p.N + n;
}
template <int D> __device__ __forceinline__ size_t slot_in(const Params &p, const Cell &c, long long n, int i, int par) {
  return par == 0 ? (size_t)i * p.N + n : (size_t)opp(i) * p.N + src<D>(p, c, i);
}

// the same slots as (plane, cell): the plane pointer is uniform across the
// warp, so an access costs one 32-bit index and one wide multiply-add
template <class T> __device__ __forceinline__ T *plane(T *f, const Params &p, int dir) {
  return f + (size_t)dir * (size_t)p.N;
}
template <int D> __device__ __forceinline__ int dir_out(int i, int par) { return par == 0 ? i : opp(i); }
template <int D> __device__ __forceinline__ int cell_out(const Params &p, const Cell &c, int i, int par) {
  return par == 0 ? nb<D>(p, c, i) : c.n;
}
template <int D> __device__ __forceinline__ int dir_in(int i, int par) { return par == 0 ? i : opp(i); }
template <int D> __device__ __forceinline__ int cell_in(const Params &p, const Cell &c, int i, int par) {
  return par == 0 ? c.n : src<D>(p, c, i);
}

template <class R, int D> __device__ __forceinline__ R feq(int i, R rho, R ux, R uy, R uz) {
  const R eu = (R)Lat<D>::cx(i) * ux + (R)Lat<D>::cy(i) * uy + (R)Lat<D>::cz(i) * uz;
  const R uu = ux * ux + uy * uy + uz * uz;
  return (R)Lat<D>::w(i) * rho * ((R)1 + eu * (R)3 + eu * eu * (R)4.5 - uu * (R)1.5);
}

template <class R, int D> __device__ __forceinline__ R geq(int i, R c, R ux, R uy, R uz) {
  const R eu = (R)Lat<D>::cx(i) * ux + (R)Lat<D>::cy(i) * uy + (R)Lat<D>::cz(i) * uz;
  return (R)Lat<D>::wa(i) * c * ((R)1 + eu / (R)Lat<D>::csa2);
}

template <class S, int D> __device__ __forceinline__ typename ST<S>::R fshift(const Params &p, int i) {
  using R = typename ST<S>::R;
  return (R)Lat<D>::w(i) * PV(R, rho0);
}
template <class S, int D> __device__ __forceinline__ typename ST<S>::R gshift(const Params &p, int i) {
  using R = typename ST<S>::R;
  return (R)Lat<D>::wa(i) * PV(R, c0);
}

// lists of cells: grid-stride loop over n entries
#define FOR_LIST(k, count) for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < (count); k += gridDim.x * blockDim.x)

// append to a list with one atomic per warp
__device__ __forceinline__ void list_append(int *list, int *count, bool take, int value) {
  const unsigned m = __ballot_sync(__activemask(), take);
  if (!m) return;
  const int lane = threadIdx.x & 31;
  const int leader = __ffs(m) - 1;
  int base = 0;
  if (lane == leader) base = atomicAdd(count, __popc(m));
  base = __shfl_sync(__activemask(), base, leader);
  if (take) list[base + __popc(m & ((1u << lane) - 1u))] = value;
}

// post-conversion type from a flag byte carrying marks
enum : int { LABEL_SKIP = 0, LABEL_ADDED = 1, LABEL_FULL = 2 };
__device__ __forceinline__ int label_mode(const Params &p) {
  if (!p.gas_dirty || !p.tdirty) return LABEL_FULL;
  const int d = *p.gas_dirty;
  const int stale = p.forest_stale ? *p.forest_stale : 0;
  if (stale & 2) return LABEL_FULL;  // the forest still holds removed gas cells
  if (d == 0) return stale ? LABEL_ADDED : LABEL_SKIP;
  return d == 1 ? LABEL_ADDED : LABEL_FULL;
}
__device__ __forceinline__ bool gas_unchanged(const Params &p) { return label_mode(p) == LABEL_SKIP; }
__device__ __forceinline__ bool label_fast(const Params &p) { return p.lab_fast && *p.lab_fast; }

// linear block index and block count of any grid shape (loops over work
// items that take one block each)
__device__ __forceinline__ int block_id() { return blockIdx.x + gridDim.x * (blockIdx.y + gridDim.y * blockIdx.z); }
__device__ __forceinline__ int block_count() { return gridDim.x * gridDim.y * gridDim.z; }

// union-find tiles: 32 x-rows of 32 cells
template <int D> struct Tile;
template <> struct Tile<3> { static constexpr int TX = 32, TY = 8, TZ = 4; };
template <> struct Tile<2> { static constexpr int TX = 32, TY = 32, TZ = 1; };
template <int D> __device__ __forceinline__ int tile_of(const Params &p, const Cell &c) {
  const int ntx = (p.nx + Tile<D>::TX - 1) / Tile<D>::TX, nty = (p.ny + Tile<D>::TY - 1) / Tile<D>::TY;
  return c.x / Tile<D>::TX + ntx * (c.y / Tile<D>::TY + nty * (c.z / Tile<D>::TZ));
}

__device__ __forceinline__ int post_type(uint8_t f) {
  const int m = fmark(f);
  if (m == MK_FILL) return T_LIQ;
  if (m == MK_EMPTY) return T_GAS;
  if (m == MK_GI || m == MK_LI) return T_IFC;
  return ftype(f);
}

// warp-aggregated FP64 atomic add keyed by a bubble index: lanes holding the
// integer counts per key, one atomic per distinct key of the warp; must be
// reached by all 32 lanes; lanes with key < 0 contribute nothing
__device__ __forceinline__ void agg_count(int *base, int key, int v) {
  const int lane = threadIdx.x & 31;
  const unsigned peers = __match_any_sync(0xffffffffu, key);
  const int s = (int)__reduce_add_sync(peers, (unsigned)v);  // each key group sums its own lanes
  if (key >= 0 && lane == __ffs(peers) - 1 && s) atomicAdd(base + key, s);
}

// same key are summed in lane order by their lowest lane.  Must be reached by
// all 32 lanes of the warp; lanes with key < 0 contribute nothing.
__device__ __forceinline__ void agg_add(double *base, int key, double v, double *wbuf) {
  const int lane = threadIdx.x & 31;
  const unsigned peers = __match_any_sync(0xffffffffu, key);
  wbuf[lane] = v;
  __syncwarp();
  if (key >= 0 && lane == __ffs(peers) - 1) {
    double s = 0.0;
    unsigned m = peers;
    while (m) {
      const int l = __ffs(m) - 1;
      s += wbuf[l];
      m &= m - 1;
    }
    atomicAdd(base + key, s);
  }
  __syncwarp();
}

}  // namespace lbf

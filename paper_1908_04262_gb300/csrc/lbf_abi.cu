// lbf_abi.cu -- host runtime behind the C ABI of include/lbf.h: device
// state, the per-step launch sequence (captured once per AA parity into a
// CUDA graph), the nucleation queue, exports, ledgers and kernel timing.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <string>
#include <vector>

#include "../../include/lbf.h"
#include "lbf_ops_api.h"

using namespace lbf;

namespace {

thread_local std::string g_err;

int fail(int code, const std::string &msg) {
  g_err = msg;
  return code;
}

#define CK(call)                                                                         \
  do {                                                                                   \
    cudaError_t e_ = (call);                                                             \
    if (e_ != cudaSuccess) return fail(LBF_ECUDA, std::string(#call ": ") + cudaGetErrorString(e_)); \
  } while (0)

// kernel groups of one step, in launch order
enum { G_EXCHANGE = 0, G_LIQUID, G_IFACE, G_CONVERT, G_LABEL, G_BUBBLE, G_GEOMETRY, G_DISJOIN, G_COUNT };
const char *kGroupNames[G_COUNT] = {"exchange", "stream_liquid", "stream_interface", "convert",   "label",
                                    "bubble_update", "geometry", "disjoining"};

struct Nucleus {
  long long step;
  double c[3], r;
};

}  // namespace

struct lbf_sim {
  lbf_config cfg;
  int dim = 0, Q = 0, QA = 0;
  long long N = 0;
  size_t ssz = 0, rsz = 0;
  cudaStream_t st = nullptr;
  bool own_stream = false;
  cudaStream_t st2 = nullptr, st3 = nullptr, st4 = nullptr;  // further branches of the step graphs
  int prio_least = 0, prio_greatest = 0;      // stream priority range of the device
  std::vector<cudaGraphNode_t> low_nodes;      // kernels captured for the lowest priority
  cudaEvent_t fork[2] = {nullptr, nullptr}, join[2] = {nullptr, nullptr}, joinx = nullptr, joinex = nullptr,
              fin = nullptr, applied = nullptr, joink = nullptr, checked = nullptr,
              sfork = nullptr, synced = nullptr;
  Ops *ops = nullptr;
  std::vector<void *> allocs;
  std::vector<size_t> alloc_bytes;  // sizes of allocs, in order
  size_t n_state_allocs = 0;        // the arrays made at creation (the checkpoint)
  // device state
  void *f = nullptr, *g = nullptr;
  uint8_t *flags = nullptr;
  int *ilist[2] = {nullptr, nullptr}, *icount[2] = {nullptr, nullptr}, *nlist = nullptr, *ncount = nullptr;
  int *seglist[2] = {nullptr, nullptr}, *segcount[2] = {nullptr, nullptr}, *segflag = nullptr;
  int *mlist = nullptr, *mcount = nullptr;
  size_t nseg = 0;  // 32-cell segments along x: ceil(nx / 32) per row
  int list_blocks = 0, warp_blocks = 0;
  void *M = nullptr, *phi = nullptr, *uI = nullptr, *kappa = nullptr, *Pi = nullptr, *nrm = nullptr,
       *dst = nullptr, *ex = nullptr, *mom = nullptr;
  int *label[2] = {nullptr, nullptr}, *parent = nullptr, *roots = nullptr, *nroots = nullptr;
  int *lsize = nullptr;
  uint8_t *tstat = nullptr;
  int *troot = nullptr;
  unsigned long long *hash = nullptr;
  int *hlist = nullptr, *hcount = nullptr;
  int hash_size = 0, cap = 0;
  Table tab[2];
  int *gpar, *gnold, *gnnew, *gatm, *gminid, *gheir;
  double *gmold, *gvnew;
  unsigned long long *gvmax;
  int *next_id = nullptr;
  double *led = nullptr;
  unsigned long long *fluid_updates = nullptr;
  int *err = nullptr;
  int *gas_dirty = nullptr;
  int *lab_slow = nullptr;
  int *forest_stale = nullptr;
  int *lab_fast = nullptr;
  int *lab_full = nullptr;
  bool walled = false;  // walls close every face and no fluid cell lies in a face layer
  int *rmv = nullptr;
  int tile_blocks = 0;
  uint8_t *tdirty = nullptr;
  size_t ntiles_alloc = 0;
  unsigned *wmask = nullptr;
  int *rlabel = nullptr;
  unsigned char *bub_dev = nullptr;   // packed bubble rows: count (16 bytes), then lbf_bubble records
  unsigned char *bub_host = nullptr;  // pinned staging copy
  int *err_host = nullptr;            // pinned copy of the sticky error bits
  void *pin[2] = {nullptr, nullptr};  // pinned chunks for host copies of fields
  cudaEvent_t pin_ev[2] = {nullptr, nullptr};
  double *acc = nullptr;
  unsigned long long *counts = nullptr;
  void *staging = nullptr;
  float *om_tab = nullptr;
  void *mlp_theta = nullptr;   // packed network image when attached, else NULL
  float *mlp_buf = nullptr;    // owned copy of the parameters
  void *mlp_img = nullptr;     // owned packed image
  int *mlp_count = nullptr;    // harvest counter
  unsigned long long mlp_hash = 0;  // FNV-1a of the attached parameters (0: none)
  int tab_n = 0;
  float tab_lnA0 = 0.f, tab_inv_dlnA = 0.f;
  long long step = 0;
  cudaGraphExec_t graph[2] = {nullptr, nullptr};
  cudaGraphExec_t tgraph[2] = {nullptr, nullptr};  // with event records
  cudaGraphExec_t graph2[2] = {nullptr, nullptr};  // two steps from parity k
  cudaGraphExec_t graph4[2] = {nullptr, nullptr};  // four steps from parity k
  cudaEvent_t tev[2][2 * G_COUNT];
  bool tev_made = false;
  std::vector<Nucleus> queue;
  // timing
  bool timing = false;
  double t_ms[G_COUNT] = {0};
  long long t_n[G_COUNT] = {0};
};

namespace {

int dev_alloc(lbf_sim *s, void **p, size_t bytes) {
  if (bytes == 0) bytes = 16;
  cudaError_t e = cudaMalloc(p, bytes);
  if (e != cudaSuccess) return fail(LBF_ENOMEM, std::string("cudaMalloc: ") + cudaGetErrorString(e));
  s->allocs.push_back(*p);
  s->alloc_bytes.push_back(bytes);
  return 0;
}

template <class T> int dalloc(lbf_sim *s, T **p, size_t count) {
  return dev_alloc(s, (void **)p, count * sizeof(T));
}

// parameters for work at step `step`: par = population parity; labels,
// bubble tables and interface lists [par] are current, [1-par] are written
// during the step
Params make_params(lbf_sim *s, long long step) {
  const int par = (int)(step & 1);
  const lbf_config &c = s->cfg;
  Params p;
  memset(&p, 0, sizeof p);
  p.nx = c.nx; p.ny = c.ny; p.nz = c.nz; p.dim = s->dim; p.N = s->N;
  p.f = s->f; p.g = s->g;
  p.flags = s->flags;
  p.par = par;
  p.walled = s->walled ? 1 : 0;
  p.wmask = s->wmask;
  p.ilist = s->ilist[par];
  p.icount = s->icount[par];
  p.inext = s->ilist[1 - par];
  p.inext_count = s->icount[1 - par];
  p.seglist = s->seglist[par];
  p.segcount = s->segcount[par];
  p.segnext = s->seglist[1 - par];
  p.segnext_count = s->segcount[1 - par];
  p.segflag = s->segflag;
  p.mlist = s->mlist;
  // one counter per parity: the next step's mass exchange clears its own
  // while this step's labelling may still read this one
  p.mcount = s->mcount + par;
  p.nlist = s->nlist;
  p.ncount = s->ncount;
  p.list_blocks = s->list_blocks;
  p.warp_blocks = s->warp_blocks;
  p.M = s->M; p.phi = s->phi; p.uI = s->uI; p.kappa = s->kappa; p.Pi = s->Pi; p.nrm = s->nrm;
  p.dst = s->dst; p.ex = s->ex; p.mom = s->mom;
  p.label_old = s->label[par];
  p.label_new = s->label[1 - par];
  p.parent = s->parent;
  p.lsize = s->lsize;
  p.tstat = s->tstat;
  p.troot = s->troot;
  p.told = s->tab[par];
  p.tnew = s->tab[1 - par];
  p.roots = s->roots; p.nroots = s->nroots; p.hash = s->hash; p.hlist = s->hlist; p.hcount = s->hcount; p.hash_size = s->hash_size; p.cap = s->cap;
  p.gpar = s->gpar; p.gnold = s->gnold; p.gnnew = s->gnnew; p.gatm = s->gatm; p.gminid = s->gminid;
  p.gheir = s->gheir; p.gmold = s->gmold; p.gvnew = s->gvnew; p.gvmax = s->gvmax;
  p.next_id = s->next_id; p.led = s->led; p.fluid_updates = s->fluid_updates; p.err = s->err;
  p.gas_dirty = s->gas_dirty;
  p.lab_slow = s->lab_slow;
  p.forest_stale = s->forest_stale;
  p.lab_fast = s->lab_fast;
  p.lab_full = s->lab_full;
  p.rmv = s->rmv;
  p.tile_blocks = s->tile_blocks;
  p.tdirty = s->tdirty;
  p.rlabel = s->rlabel;
  p.om_tab = s->om_tab; p.tab_n = s->tab_n; p.tab_lnA0 = s->tab_lnA0; p.tab_inv_dlnA = s->tab_inv_dlnA;
  p.tau = c.tau; p.rho0 = c.rho0; p.ax = c.accel[0]; p.ay = c.accel[1]; p.az = c.accel[2];
  p.has_force = (c.accel[0] != 0.0 || c.accel[1] != 0.0 || c.accel[2] != 0.0);
  p.rheo = c.rheo; p.rn = c.rheo_n; p.rk = c.rheo_k; p.rlam = c.rheo_lambda; p.ra = c.rheo_a;
  p.tau0 = c.tau0; p.tau_inf = c.tau_inf; p.tau_min = c.tau_min; p.tau_max = c.tau_max;
  p.sigma = c.sigma; p.k_pi = c.k_pi; p.d_max = c.d_max;
  p.taug = 0.5 + c.D / (s->dim == 2 ? 1.0 / 3.0 : 0.25);
  p.kH = c.kH; p.RT = c.RT; p.c0 = c.c0; p.q = c.q; p.p0 = c.p0; p.eps = c.eps;
  p.uwx = c.wall_u[0]; p.uwy = c.wall_u[1]; p.uwz = c.wall_u[2];
  p.walls = c.walls; p.atmosphere = c.atmosphere;
  const int up = s->dim - 1;
  const int n_up = up == 1 ? c.ny : c.nz;
  p.top_layer = n_up - 1 - ((c.walls >> (2 * up + 1)) & 1);
  p.ray_steps = (int)std::ceil(c.d_max) + 1;
  p.coll = c.collision;
  p.mrt_se = c.mrt_rates[0]; p.mrt_seps = c.mrt_rates[1]; p.mrt_spi = c.mrt_rates[2]; p.mrt_sm = c.mrt_rates[3];
  p.kappa_hf = c.kappa == 1;
  p.trt_magic = c.trt_magic;
  p.omg = 1.0 / p.taug;
  p.om = 1.0 / p.tau;
  p.pf = {(float)p.tau, (float)p.rho0, (float)p.ax, (float)p.ay, (float)p.az, (float)p.rn, (float)p.rk,
          (float)p.rlam, (float)p.ra, (float)p.tau0, (float)p.tau_inf, (float)p.tau_min, (float)p.tau_max,
          (float)p.sigma, (float)p.k_pi, (float)p.d_max, (float)p.taug, (float)p.kH, (float)p.RT, (float)p.c0,
          (float)p.q, (float)p.p0, (float)p.eps, (float)p.uwx, (float)p.uwy, (float)p.uwz, (float)c.trt_magic,
          (float)p.omg, (float)p.om, (float)p.mrt_se, (float)p.mrt_seps, (float)p.mrt_spi, (float)p.mrt_sm};
  return p;
}

// labelling + bubble update + geometry outside the step (create, set_cells,
// nucleation): the results are copied back into the current buffers
int relabel_in_place(lbf_sim *s) {
  const int par = (int)(s->step & 1);
  Params p = make_params(s, s->step);
  CK(cudaMemsetAsync(s->segflag, 0, sizeof(int) * s->nseg, s->st));
  s->ops->build_ilist(p, s->st);
  CK(cudaMemsetAsync(p.inext_count, 0, sizeof(int), s->st));
  CK(cudaMemsetAsync(p.segnext_count, 0, sizeof(int), s->st));
  s->ops->label_prep(p, s->st);
  // the state was set from outside: label from scratch
  CK(cudaMemsetAsync(s->gas_dirty, 0xff, sizeof(int), s->st));
  CK(cudaMemsetAsync(s->lab_fast, 0, sizeof(int), s->st));
  // the next patched labelling starts from a full copy
  CK(cudaMemsetAsync(s->lab_full, 0xff, sizeof(int), s->st));
  s->ops->label(p, s->st);
  s->ops->bubble_update(p, s->st);
  const size_t cap = (size_t)s->cap;
  Table &a = s->tab[par], &b = s->tab[1 - par];
  CK(cudaMemcpyAsync(s->label[par], s->label[1 - par], sizeof(int) * s->N, cudaMemcpyDeviceToDevice, s->st));
  CK(cudaMemcpyAsync(a.m, b.m, sizeof(double) * cap, cudaMemcpyDeviceToDevice, s->st));
  CK(cudaMemcpyAsync(a.p, b.p, sizeof(double) * cap, cudaMemcpyDeviceToDevice, s->st));
  CK(cudaMemcpyAsync(a.V, b.V, sizeof(double) * cap, cudaMemcpyDeviceToDevice, s->st));
  CK(cudaMemcpyAsync(a.dm, b.dm, sizeof(double) * cap, cudaMemcpyDeviceToDevice, s->st));
  CK(cudaMemcpyAsync(a.id, b.id, sizeof(int) * cap, cudaMemcpyDeviceToDevice, s->st));
  CK(cudaMemcpyAsync(a.atm, b.atm, sizeof(int) * cap, cudaMemcpyDeviceToDevice, s->st));
  CK(cudaMemcpyAsync(a.root, b.root, sizeof(int) * cap, cudaMemcpyDeviceToDevice, s->st));
  CK(cudaMemcpyAsync(a.ng, b.ng, sizeof(int) * cap, cudaMemcpyDeviceToDevice, s->st));
  CK(cudaMemcpyAsync(a.count, b.count, sizeof(int), cudaMemcpyDeviceToDevice, s->st));
  p.label_new = s->label[par];
  s->ops->geometry(p, s->st);
  if (s->mlp_theta) s->ops->mlp_kappa(p, s->mlp_theta, s->st);
  s->ops->disjoining(p, s->st);
  // the next step accumulates into table [1-par] and counts roots afresh
  s->ops->label_prep(p, s->st);
  CK(cudaGetLastError());
  return 0;
}

int separate_and_relabel(lbf_sim *s) {
  const int par = (int)(s->step & 1);
  Params p = make_params(s, s->step);
  s->ops->separate(p, par, s->st);
  CK(cudaGetLastError());
  return relabel_in_place(s);
}

// the geometry of the next step works on the interface list and the final
// flags the conversion produced; it needs no labels
Params next_geometry_params(const Params &p) {
  Params pn = p;
  pn.ilist = p.inext;
  pn.icount = p.inext_count;
  return pn;
}

void enqueue_geometry(lbf_sim *s, const Params &pn, cudaStream_t st) {
  s->ops->geometry(pn, st);
  if (s->mlp_theta) s->ops->mlp_kappa(pn, s->mlp_theta, st);
}

// the kernel just captured on stream `st` takes the lowest priority in the
// instantiated graph (set_node_priorities)
void mark_low_priority(lbf_sim *s, cudaStream_t st) {
  cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
  const cudaGraphNode_t *deps = nullptr;
  size_t nd = 0;
  if (cudaStreamGetCaptureInfo(st, &cs, nullptr, nullptr, &deps, nullptr, &nd) == cudaSuccess &&
      cs == cudaStreamCaptureStatusActive)
    s->low_nodes.insert(s->low_nodes.end(), deps, deps + nd);
}

// the step's label sync on the fourth branch, beside its interface sweep
// (the marking waits for it: it reads the last step's interface list, whose
// buffer the excess collection refills)
void enqueue_label_sync(lbf_sim *s, const Params &p) {
  cudaEventRecord(s->sfork, s->st);
  cudaStreamWaitEvent(s->st4, s->sfork, 0);
  s->ops->label_sync(p, s->st4);
  cudaEventRecord(s->synced, s->st4);
}

// everything of a step after its interface sweep.  The marking runs first;
// then every cell's post-conversion type is known and the union-find passes
// start, beside the excess pass (which with `waitx` also waits for the
// step's liquid sweep on the third branch) and the geometry (second branch,
// the learned curvature after it); the pass that writes the new types over
// the marks runs before the geometry on the second branch, or, with the
// learned curvature attached (a longer second branch), on the third branch
// once the excess pass is done, so that the geometry starts at once (the
// labelling, the geometry, the learned curvature and the disjoining
// pressure read post-conversion types, marked or not; measured: the early
// geometry pays with the learned curvature and costs ~4 % without it, as it
// then only competes with the labelling); the relabelling
// waits for the excess pass (it reads the fill levels) and the bubble update
// follows it; the disjoining pressure (labels and the geometry's normals,
// not the curvature) runs on a fourth branch.  With `pnext`, the next
// step's mass exchange and then its liquid sweep (which need only what the
// conversion left) follow on the third branch, signalled by `joinex` and
// `joinx`.
void enqueue_after_sweep(lbf_sim *s, const Params &p, int par, bool waitx, const Params *pnext, int parnext) {
  const Params pn = next_geometry_params(p);
  cudaStreamWaitEvent(s->st, s->synced, 0);
  s->ops->convert_mark(p, s->st);
  cudaEventRecord(s->fork[0], s->st);
  // the labelling check reads the marks (and writes nothing the excess pass
  // reads): beside the excess pass, before the flag rewrite
  s->ops->label_check(p, s->st);
  cudaEventRecord(s->checked, s->st);
  cudaStreamWaitEvent(s->st2, s->fork[0], 0);
  if (waitx) cudaStreamWaitEvent(s->st2, s->joinx, 0);
  s->ops->convert_excess(p, par, s->st2);
  cudaEventRecord(s->applied, s->st2);
  const bool early_geometry = s->mlp_theta != nullptr;
  if (!early_geometry) {
    cudaStreamWaitEvent(s->st2, s->checked, 0);
    s->ops->convert_finalize(p, s->st2);
    cudaEventRecord(s->fin, s->st2);
  }
  s->ops->geometry(pn, s->st2);
  cudaEventRecord(s->join[0], s->st2);
  if (s->mlp_theta) s->ops->mlp_kappa(pn, s->mlp_theta, s->st2);
  cudaEventRecord(s->joink, s->st2);
  if (early_geometry) {
    cudaStreamWaitEvent(s->st3, s->applied, 0);
    cudaStreamWaitEvent(s->st3, s->checked, 0);
    s->ops->convert_finalize(p, s->st3);
    cudaEventRecord(s->fin, s->st3);
  }
  if (pnext) {
    // the next step's mass exchange reads the types through the marks: it
    // starts once the excess is collected, beside the flag rewrite
    if (!early_geometry) cudaStreamWaitEvent(s->st3, s->applied, 0);
    s->ops->exchange(*pnext, parnext, s->st3);
    cudaEventRecord(s->joinex, s->st3);
    s->ops->stream_liquid(*pnext, parnext, s->st3);
    // the lowest priority: the labelling's blocks go first
    mark_low_priority(s, s->st3);
    cudaEventRecord(s->joinx, s->st3);
  }
  // the labelling branch is chosen on the device after the marking (see
  // k_label_choose): the kernels of the branch not taken return at once
  s->ops->label_choose(p, s->st);
  s->ops->label_forest(p, s->st);
  cudaStreamWaitEvent(s->st, s->applied, 0);
  // the patch first: ready with the excess collection, it goes ahead of the
  // geometry's blocks (the relabelling of the other branch returns at once)
  s->ops->label_fast(p, s->st);
  s->ops->label_relabel(p, s->st);
  cudaEventRecord(s->fork[1], s->st);
  s->ops->bubble_update(p, s->st);
  s->ops->bubble_update_fast(p, s->st);
  cudaStreamWaitEvent(s->st4, s->fork[1], 0);
  cudaStreamWaitEvent(s->st4, s->join[0], 0);
  s->ops->disjoining(pn, s->st4);
  cudaEventRecord(s->join[1], s->st4);
  cudaStreamWaitEvent(s->st, s->join[1], 0);
  cudaStreamWaitEvent(s->st, s->joink, 0);
  cudaStreamWaitEvent(s->st, s->fin, 0);
}

// the launch sequence of one step; with `ev` every kernel group runs in
// order on the one stream, bracketed by event records (the timing graph)
void enqueue_step(lbf_sim *s, const Params &p, int par, cudaEvent_t *ev) {
  auto group = [&](int gidx, auto &&fn) {
    if (ev) cudaEventRecordWithFlags(ev[2 * gidx], s->st, cudaEventRecordExternal);
    fn();
    if (ev) cudaEventRecordWithFlags(ev[2 * gidx + 1], s->st, cudaEventRecordExternal);
  };
  if (!ev) {
    // the liquid sweep on the third branch beside the interface sweep (the
    // two commute); the excess pass waits for it
    s->ops->exchange(p, par, s->st);
    cudaEventRecord(s->joinex, s->st);
    cudaStreamWaitEvent(s->st3, s->joinex, 0);
    s->ops->stream_liquid(p, par, s->st3);
    cudaEventRecord(s->joinx, s->st3);
    enqueue_label_sync(s, p);
    s->ops->stream_interface(p, par, s->st);
    enqueue_after_sweep(s, p, par, true, nullptr, 0);
    return;
  }
  group(G_EXCHANGE, [&] { s->ops->exchange(p, par, s->st); });
  group(G_LIQUID, [&] { s->ops->stream_liquid(p, par, s->st); });
  group(G_IFACE, [&] {
    s->ops->label_sync(p, s->st);
    s->ops->stream_interface(p, par, s->st);
  });
  group(G_CONVERT, [&] {
    s->ops->convert_mark(p, s->st);
    s->ops->label_check(p, s->st);
    s->ops->convert_excess(p, par, s->st);
    s->ops->convert_finalize(p, s->st);
  });
  const Params pn = next_geometry_params(p);
  group(G_LABEL, [&] {
    s->ops->label_choose(p, s->st);
    s->ops->label(p, s->st);
    s->ops->label_fast(p, s->st);
  });
  group(G_BUBBLE, [&] {
    s->ops->bubble_update(p, s->st);
    s->ops->bubble_update_fast(p, s->st);
  });
  group(G_GEOMETRY, [&] { enqueue_geometry(s, pn, s->st); });
  group(G_DISJOIN, [&] { s->ops->disjoining(pn, s->st); });
}

// k consecutive steps in one graph (parities alternating from par): every
// step after the first has its mass exchange and its liquid sweep overlap the
// previous step's labelling, geometry, bubble update and disjoining pressure;
// its interface sweep waits for those and for its mass exchange, its
// conversion's excess pass for both sweeps
void enqueue_chain(lbf_sim *s, const Params *ps, int par, int k) {
  s->ops->exchange(ps[0], par, s->st);
  s->ops->stream_liquid(ps[0], par, s->st);
  for (int i = 0; i < k; ++i) {
    const int pi = (par + i) & 1;
    if (i > 0) cudaStreamWaitEvent(s->st, s->joinex, 0);
    enqueue_label_sync(s, ps[i]);
    s->ops->stream_interface(ps[i], pi, s->st);
    enqueue_after_sweep(s, ps[i], pi, i > 0, i + 1 < k ? &ps[i + 1] : nullptr, 1 - pi);
  }
}

// kernel node priorities of a captured chain: the overlapped liquid sweeps
// the least, every other kernel the greatest (the graph is instantiated to
// honour them)
int set_node_priorities(lbf_sim *s, cudaGraph_t gr) {
  size_t nn = 0;
  CK(cudaGraphGetNodes(gr, nullptr, &nn));
  std::vector<cudaGraphNode_t> nodes(nn);
  CK(cudaGraphGetNodes(gr, nodes.data(), &nn));
  for (size_t j = 0; j < nn; ++j) {
    cudaGraphNodeType t;
    CK(cudaGraphNodeGetType(nodes[j], &t));
    if (t != cudaGraphNodeTypeKernel) continue;
    const bool low = std::find(s->low_nodes.begin(), s->low_nodes.end(), nodes[j]) != s->low_nodes.end();
    cudaLaunchAttributeValue v;
    std::memset(&v, 0, sizeof(v));
    v.priority = low ? s->prio_least : s->prio_greatest;
    CK(cudaGraphKernelNodeSetAttribute(nodes[j], cudaLaunchAttributePriority, &v));
  }
  return 0;
}

int capture_chain(lbf_sim *s, const Params *ps, int par, int k, cudaGraphExec_t *out) {
  cudaGraph_t gr = nullptr;
  s->low_nodes.clear();
  CK(cudaStreamBeginCapture(s->st, cudaStreamCaptureModeThreadLocal));
  enqueue_chain(s, ps, par, k);
  CK(cudaStreamEndCapture(s->st, &gr));
  int rc = set_node_priorities(s, gr);
  s->low_nodes.clear();
  if (rc) {
    cudaGraphDestroy(gr);
    return rc;
  }
  cudaError_t e = cudaGraphInstantiate(out, gr, cudaGraphInstantiateFlagUseNodePriority);
  cudaGraphDestroy(gr);
  if (e != cudaSuccess) return fail(LBF_ECUDA, std::string("cudaGraphInstantiate: ") + cudaGetErrorString(e));
  return 0;
}

int capture(lbf_sim *s, const Params &p, int par, cudaEvent_t *ev, cudaGraphExec_t *out) {
  cudaGraph_t gr = nullptr;
  s->low_nodes.clear();
  CK(cudaStreamBeginCapture(s->st, cudaStreamCaptureModeThreadLocal));
  enqueue_step(s, p, par, ev);
  CK(cudaStreamEndCapture(s->st, &gr));
  int rc = set_node_priorities(s, gr);
  s->low_nodes.clear();
  if (rc) {
    cudaGraphDestroy(gr);
    return rc;
  }
  cudaError_t e = cudaGraphInstantiate(out, gr, cudaGraphInstantiateFlagUseNodePriority);
  cudaGraphDestroy(gr);
  if (e != cudaSuccess) return fail(LBF_ECUDA, std::string("cudaGraphInstantiate: ") + cudaGetErrorString(e));
  return 0;
}

int ensure_graph(lbf_sim *s, int k, int par);

int run_one_step(lbf_sim *s) {
  const int par = (int)(s->step & 1);
  Params p = make_params(s, s->step);
  if (s->timing) {
    if (!s->tev_made) {
      for (int k = 0; k < 2; ++k)
        for (int j = 0; j < 2 * G_COUNT; ++j) CK(cudaEventCreate(&s->tev[k][j]));
      s->tev_made = true;
    }
    if (!s->tgraph[par]) {
      int rc = capture(s, p, par, s->tev[par], &s->tgraph[par]);
      if (rc) return rc;
    }
    CK(cudaGraphLaunch(s->tgraph[par], s->st));
    CK(cudaStreamSynchronize(s->st));
    for (int gidx = 0; gidx < G_COUNT; ++gidx) {
      float ms = 0.f;
      CK(cudaEventElapsedTime(&ms, s->tev[par][2 * gidx], s->tev[par][2 * gidx + 1]));
      s->t_ms[gidx] += ms;
      s->t_n[gidx] += 1;
    }
    return 0;
  }
  int rc = ensure_graph(s, 1, par);
  if (rc) return rc;
  CK(cudaGraphLaunch(s->graph[par], s->st));
  return 0;
}

// the graph of k = 1, 2 or 4 steps starting at parity par, captured and
// instantiated if it does not exist yet (the parameters of a step depend on
// the step number only through its parity)
int ensure_graph(lbf_sim *s, int k, int par) {
  cudaGraphExec_t &g = k == 4 ? s->graph4[par] : (k == 2 ? s->graph2[par] : s->graph[par]);
  if (g) return 0;
  int rc;
  if (k == 1) {
    rc = capture(s, make_params(s, par), par, nullptr, &g);
  } else {
    Params ps[4];
    for (int i = 0; i < k; ++i) ps[i] = make_params(s, par + i);
    rc = capture_chain(s, ps, par, k, &g);
  }
  if (rc) return rc;
  // moved to the device now rather than at its first launch
  CK(cudaGraphUpload(g, s->st));
  return 0;
}

// every graph shape lbf_step launches, for both parities: made on the first
// step call (and again after the shapes were dropped) so that no later call
// pays for a capture or an instantiation in the middle of a run
int ensure_all_graphs(lbf_sim *s) {
  for (int k : {4, 2, 1})
    for (int par = 0; par < 2; ++par) {
      int rc = ensure_graph(s, k, par);
      if (rc) return rc;
    }
  return 0;
}

// k = 2 or 4 steps as one graph (graphs[k / 4][parity])
int run_steps(lbf_sim *s, int k) {
  const int par = (int)(s->step & 1);
  int rc = ensure_graph(s, k, par);
  if (rc) return rc;
  CK(cudaGraphLaunch(k == 4 ? s->graph4[par] : s->graph2[par], s->st));
  return 0;
}

bool nucleus_due(const lbf_sim *s, long long step) {
  for (const auto &nu : s->queue)
    if (nu.step <= step) return true;
  return false;
}

int carve_due_nuclei(lbf_sim *s) {
  bool any = false;
  const int par = (int)(s->step & 1);
  Params p = make_params(s, s->step);
  std::vector<Nucleus> keep;
  for (auto &nu : s->queue) {
    if (nu.step <= s->step) {
      s->ops->nucleate(p, par, nu.c, nu.r, s->st);
      any = true;
    } else {
      keep.push_back(nu);
    }
  }
  s->queue.swap(keep);
  if (!any) return 0;
  CK(cudaGetLastError());
  return separate_and_relabel(s);
}

// device -> caller's (possibly pageable) host memory through two pinned
// chunks: the copy of one chunk overlaps the host copy of the other
int copy_to_host(lbf_sim *s, void *dst, const void *src, size_t bytes) {
  // page-locked destination: one direct copy
  cudaPointerAttributes pa;
  if (cudaPointerGetAttributes(&pa, dst) == cudaSuccess && pa.type == cudaMemoryTypeHost) {
    CK(cudaMemcpyAsync(dst, src, bytes, cudaMemcpyDeviceToHost, s->st));
    CK(cudaStreamSynchronize(s->st));
    return 0;
  }
  cudaGetLastError();  // a pageable pointer is not an error
  constexpr size_t kChunk = size_t(4) << 20;
  if (!s->pin[0]) {
    for (int b = 0; b < 2; ++b) {
      CK(cudaMallocHost(&s->pin[b], kChunk));
      CK(cudaEventCreateWithFlags(&s->pin_ev[b], cudaEventDisableTiming));
    }
  }
  const unsigned char *sp = (const unsigned char *)src;
  unsigned char *dp = (unsigned char *)dst;
  size_t prev_off = 0, prev_len = 0;
  int b = 0;
  for (size_t off = 0; off < bytes; off += kChunk, b ^= 1) {
    const size_t len = std::min(kChunk, bytes - off);
    CK(cudaMemcpyAsync(s->pin[b], sp + off, len, cudaMemcpyDeviceToHost, s->st));
    CK(cudaEventRecord(s->pin_ev[b], s->st));
    if (prev_len) {
      CK(cudaEventSynchronize(s->pin_ev[b ^ 1]));
      std::memcpy(dp + prev_off, s->pin[b ^ 1], prev_len);
    }
    prev_off = off;
    prev_len = len;
  }
  if (prev_len) {
    CK(cudaEventSynchronize(s->pin_ev[b ^ 1]));
    std::memcpy(dp + prev_off, s->pin[b ^ 1], prev_len);
  }
  return 0;
}

int check_device_error(lbf_sim *s) {
  if (!s->err_host) CK(cudaMallocHost((void **)&s->err_host, sizeof(int)));
  CK(cudaMemcpyAsync(s->err_host, s->err, sizeof(int), cudaMemcpyDeviceToHost, s->st));
  CK(cudaStreamSynchronize(s->st));
  const int e = *s->err_host;
  if (e & ERR_CAPACITY) return fail(LBF_ECAPACITY, "more bubbles than bubble_capacity");
  if (e & ERR_NOTCONV) return fail(LBF_ENOTCONV, "union-find iteration cap reached");
  if (e & ERR_HASH) return fail(LBF_ECAPACITY, "bubble overlap table full");
  if (e & ERR_TC_WAIT) return fail(LBF_ECUDA, "learned curvature: a tensor-core wait ran past its bound");
  return 0;
}

// Sec. 2.3 on the host: tau of the rheology model at shear rate gd, and the
// relaxation time solving tau = tau_model(A / tau), clamped to
// [tau_min, tau_max] (bisection; used to tabulate tau(A))
double host_tau_model(const lbf_config &c, double gd) {
  if (c.rheo == 1) return 0.5 + 3.0 * c.rheo_k * std::pow(gd, c.rheo_n - 1.0);
  return c.tau_inf + (c.tau0 - c.tau_inf) * std::pow(1.0 + std::pow(c.rheo_lambda * gd, c.rheo_a), (c.rheo_n - 1.0) / c.rheo_a);
}
double host_solve_tau(const lbf_config &c, double A) {
  double lo = c.tau_min, hi = c.tau_max;
  if (!(hi - host_tau_model(c, A / hi) > 0.0)) return hi;
  if (!(lo - host_tau_model(c, A / lo) < 0.0)) return lo;
  for (int it = 0; it < 200 && hi - lo > 1e-15 * hi; ++it) {
    const double mid = 0.5 * (lo + hi);
    if (mid - host_tau_model(c, A / mid) > 0.0) hi = mid; else lo = mid;
  }
  return 0.5 * (lo + hi);
}

int build_tau_table(lbf_sim *s) {
  const lbf_config &c = s->cfg;
  if (c.rheo == 0 || c.storage == LBF_FP64) return 0;
  const int n = 8192;
  const double lnA0 = std::log(1e-14), lnA1 = std::log(1e2);
  const double dl = (lnA1 - lnA0) / (n - 1);
  std::vector<float> tab(n);
  for (int k = 0; k < n; ++k) tab[k] = (float)(1.0 / host_solve_tau(c, std::exp(lnA0 + k * dl)));
  int rc = dalloc(s, &s->om_tab, (size_t)n);
  if (rc) return rc;
  CK(cudaMemcpy(s->om_tab, tab.data(), sizeof(float) * n, cudaMemcpyHostToDevice));
  s->tab_n = n;
  s->tab_lnA0 = (float)lnA0;
  s->tab_inv_dlnA = (float)(1.0 / dl);
  return 0;
}

int validate(const lbf_config *c) {
  if (!c) return fail(LBF_EINVAL, "cfg is NULL");
  if (c->nx <= 0 || c->ny <= 0 || c->nz <= 0) return fail(LBF_EINVAL, "lattice sizes must be positive");
  if ((long long)c->nx * c->ny * c->nz > 2147483647LL) return fail(LBF_EINVAL, "more than 2^31-1 cells");
  if (c->nx < 3 || c->ny < 3 || (c->nz != 1 && c->nz < 3)) return fail(LBF_EINVAL, "each extent must be >= 3 (nz == 1 for 2D)");
  if (c->ny > 65535 || c->nz > 65535) return fail(LBF_EINVAL, "ny and nz must be <= 65535");
  if (c->storage < 0 || c->storage > 3) return fail(LBF_EINVAL, "bad storage");
  if (c->rheo < 0 || c->rheo > 2) return fail(LBF_EINVAL, "bad rheology");
  if (!(c->tau > 0.5)) return fail(LBF_EINVAL, "tau must exceed 1/2");
  if (c->rheo != 0 && !(c->tau_min > 0.5 && c->tau_max > c->tau_min)) return fail(LBF_EINVAL, "need 1/2 < tau_min < tau_max");
  if (!(c->D > 0.0)) return fail(LBF_EINVAL, "D must be positive");
  if (c->collision < 0 || c->collision > 2) return fail(LBF_EINVAL, "bad collision");
  if (c->collision >= 1 && !(c->trt_magic > 0.0)) return fail(LBF_EINVAL, "trt_magic must be positive");
  if (c->collision == 2)
    for (int k = 0; k < 4; ++k)
      if (!(c->mrt_rates[k] >= 0.0 && c->mrt_rates[k] < 2.0)) return fail(LBF_EINVAL, "mrt_rates must be in [0, 2)");
  if (c->kappa < 0 || c->kappa > 1) return fail(LBF_EINVAL, "bad curvature method");
  if (!(c->RT > 0.0) || !(c->rho0 > 0.0)) return fail(LBF_EINVAL, "RT and rho0 must be positive");
  if (c->bubble_capacity < 1 || c->bubble_capacity > 16384) return fail(LBF_EINVAL, "bubble_capacity must be in [1, 16384]");
  if (c->k_pi != 0.0 && !(c->d_max > 0.0 && c->d_max <= 64.0)) return fail(LBF_EINVAL, "d_max must be in (0, 64]");
  return 0;
}

}  // namespace

namespace lbf {
void set_last_error(const char *msg) { g_err = msg; }

// the bubble table as lbf_bubble rows after a 16-byte header holding the
// row count
__global__ void k_pack_bubbles(Table t, unsigned char *out, int rows) {
  const int nb = *t.count;
  if (blockIdx.x == 0 && threadIdx.x == 0) *reinterpret_cast<int *>(out) = nb;
  lbf_bubble *r = reinterpret_cast<lbf_bubble *>(out + 16);
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < rows && i < nb; i += gridDim.x * blockDim.x) {
    lbf_bubble b;
    b.id = t.id[i];
    b.atm = t.atm[i];
    b.label = t.root[i];
    b.volume = t.V[i];
    b.gas_mass = t.m[i];
    b.pressure = t.p[i];
    r[i] = b;
  }
}
void pack_bubbles_launch(const Table &t, unsigned char *out, int rows, cudaStream_t st) {
  const int blocks = rows > 0 ? (rows + 255) / 256 : 1;
  k_pack_bubbles<<<blocks, 256, 0, st>>>(t, out, rows);
}

// checks a staged lbf_set_cells input before it replaces the state: bit 0 a
// cell type outside 0..3, bit 1 a non-finite value, bit 2 a density that is
// not positive in a liquid or interface cell
__global__ void k_check_cells(const uint8_t *type, const double *rho, const double *u, const double *alpha,
                              const double *c, long long N, unsigned long long *bad) {
  unsigned long long b = 0;
  for (long long n = blockIdx.x * (long long)blockDim.x + threadIdx.x; n < N; n += (long long)gridDim.x * blockDim.x) {
    const int t = type[n];
    if (t > 3) b |= 1;
    const double v[6] = {rho[n], u[3 * n], u[3 * n + 1], u[3 * n + 2], alpha[n], c[n]};
    for (int k = 0; k < 6; ++k)
      if (!isfinite(v[k])) b |= 2;
    if ((t == 1 || t == 2) && !(rho[n] > 0.0)) b |= 4;
  }
  b = __reduce_or_sync(0xffffffffu, (unsigned)b);
  if (b && (threadIdx.x & 31) == 0) atomicOr(bad, b);
}
void check_cells_launch(const uint8_t *type, const double *rho, const double *u, const double *alpha,
                        const double *c, long long N, unsigned long long *bad, int blocks, cudaStream_t st) {
  k_check_cells<<<blocks, 256, 0, st>>>(type, rho, u, alpha, c, N, bad);
}
}  // namespace lbf

extern "C" {

const char *lbf_last_error(void) { return g_err.c_str(); }

void lbf_destroy(lbf_sim *s) {
  if (!s) return;
  if (s->st) cudaStreamSynchronize(s->st);
  for (int k = 0; k < 2; ++k) {
    if (s->graph[k]) cudaGraphExecDestroy(s->graph[k]);
    if (s->tgraph[k]) cudaGraphExecDestroy(s->tgraph[k]);
    if (s->graph2[k]) cudaGraphExecDestroy(s->graph2[k]);
    if (s->graph4[k]) cudaGraphExecDestroy(s->graph4[k]);
  }
  if (s->tev_made)
    for (int k = 0; k < 2; ++k)
      for (int j = 0; j < 2 * G_COUNT; ++j) cudaEventDestroy(s->tev[k][j]);
  for (void *p : s->allocs) cudaFree(p);
  for (int k = 0; k < 2; ++k) {
    if (s->fork[k]) cudaEventDestroy(s->fork[k]);
    if (s->join[k]) cudaEventDestroy(s->join[k]);
  }
  if (s->bub_host) cudaFreeHost(s->bub_host);
  if (s->err_host) cudaFreeHost(s->err_host);
  for (int b = 0; b < 2; ++b) {
    if (s->pin[b]) cudaFreeHost(s->pin[b]);
    if (s->pin_ev[b]) cudaEventDestroy(s->pin_ev[b]);
  }
  if (s->joinx) cudaEventDestroy(s->joinx);
  if (s->joinex) cudaEventDestroy(s->joinex);
  if (s->fin) cudaEventDestroy(s->fin);
  if (s->applied) cudaEventDestroy(s->applied);
  if (s->joink) cudaEventDestroy(s->joink);
  if (s->checked) cudaEventDestroy(s->checked);
  if (s->sfork) cudaEventDestroy(s->sfork);
  if (s->synced) cudaEventDestroy(s->synced);
  if (s->st2) cudaStreamDestroy(s->st2);
  if (s->st3) cudaStreamDestroy(s->st3);
  if (s->st4) cudaStreamDestroy(s->st4);
  if (s->own_stream && s->st) cudaStreamDestroy(s->st);
  delete s->ops;
  delete s;
}

static void drop_graphs(lbf_sim *s);

// walls on every face of the lattice (cfg.walls)
bool all_faces_walled(const lbf_sim *s) {
  const int need = s->dim == 3 ? 0x3F : 0xF;
  return (s->cfg.walls & need) == need;
}

// a liquid or interface cell in a face layer of the host type array
bool fluid_in_faces(const lbf_sim *s, const uint8_t *type) {
  const long long nx = s->cfg.nx, ny = s->cfg.ny, nz = s->dim == 3 ? s->cfg.nz : 1;
  auto fluid = [&](long long x, long long y, long long z) {
    const int t = type[x + nx * (y + ny * z)] & 3;
    return t == 1 || t == 2;
  };
  for (long long z = 0; z < nz; ++z)
    for (long long y = 0; y < ny; ++y) {
      const bool face_row = y == 0 || y == ny - 1 || (s->dim == 3 && (z == 0 || z == nz - 1));
      if (face_row) {
        for (long long x = 0; x < nx; ++x)
          if (fluid(x, y, z)) return true;
      } else if (fluid(0, y, z) || fluid(nx - 1, y, z)) {
        return true;
      }
    }
  return false;
}

int lbf_create(const lbf_config *cfg, lbf_sim **out) {
  if (!out) return fail(LBF_EINVAL, "out is NULL");
  *out = nullptr;
  int rc = validate(cfg);
  if (rc) return rc;
  lbf_sim *s = new lbf_sim();
  s->cfg = *cfg;
  s->dim = cfg->nz == 1 ? 2 : 3;
  s->Q = s->dim == 2 ? 9 : 19;
  s->QA = s->dim == 2 ? 5 : 7;
  s->N = (long long)cfg->nx * cfg->ny * cfg->nz;
  static const size_t ssz[4] = {8, 4, 2, 2};
  s->ssz = ssz[cfg->storage];
  s->rsz = cfg->storage == LBF_FP64 ? 8 : 4;
  switch (cfg->storage) {
    case LBF_FP64: s->ops = make_ops_f64(s->dim); break;
    case LBF_FP32: s->ops = make_ops_f32(s->dim); break;
    case LBF_FP16S: s->ops = make_ops_f16(s->dim); break;
    default: s->ops = make_ops_bf16(s->dim); break;
  }
  if (cfg->stream) {
    s->st = (cudaStream_t)cfg->stream;
  } else {
    cudaError_t e = cudaStreamCreateWithFlags(&s->st, cudaStreamNonBlocking);
    if (e != cudaSuccess) {
      delete s->ops;
      delete s;
      return fail(LBF_ECUDA, std::string("cudaStreamCreate: ") + cudaGetErrorString(e));
    }
    s->own_stream = true;
  }
  {
    cudaError_t e = cudaDeviceGetStreamPriorityRange(&s->prio_least, &s->prio_greatest);
    if (e == cudaSuccess) e = cudaStreamCreateWithPriority(&s->st2, cudaStreamNonBlocking, s->prio_greatest);
    if (e == cudaSuccess) e = cudaStreamCreateWithPriority(&s->st3, cudaStreamNonBlocking, s->prio_least);
    if (e == cudaSuccess) e = cudaStreamCreateWithPriority(&s->st4, cudaStreamNonBlocking, s->prio_greatest);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&s->joinx, cudaEventDisableTiming);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&s->joinex, cudaEventDisableTiming);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&s->fin, cudaEventDisableTiming);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&s->applied, cudaEventDisableTiming);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&s->joink, cudaEventDisableTiming);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&s->checked, cudaEventDisableTiming);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&s->sfork, cudaEventDisableTiming);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&s->synced, cudaEventDisableTiming);
    for (int k = 0; k < 2 && e == cudaSuccess; ++k) {
      e = cudaEventCreateWithFlags(&s->fork[k], cudaEventDisableTiming);
      if (e == cudaSuccess) e = cudaEventCreateWithFlags(&s->join[k], cudaEventDisableTiming);
    }
    if (e != cudaSuccess) {
      lbf_destroy(s);
      return fail(LBF_ECUDA, std::string("cudaStreamCreate: ") + cudaGetErrorString(e));
    }
  }
  const size_t N = (size_t)s->N;
  {
    int dev = 0, sms = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    s->list_blocks = 4 * (sms > 0 ? sms : 132);
    s->warp_blocks = 16 * (sms > 0 ? sms : 132);
    s->tile_blocks = 2 * (sms > 0 ? sms : 132);
  }
  s->cap = cfg->bubble_capacity;
  int hs = 1024;
  while (hs < 4 * s->cap) hs <<= 1;
  s->hash_size = hs;
#define AL(expr)       \
  do {                 \
    rc = (expr);       \
    if (rc) {          \
      lbf_destroy(s);  \
      return rc;       \
    }                  \
  } while (0)
  AL(dev_alloc(s, &s->f, N * s->Q * s->ssz));
  AL(dev_alloc(s, &s->g, N * s->QA * s->ssz));
  AL(dalloc(s, &s->flags, N));
  AL(dalloc(s, &s->ilist[0], N));
  AL(dalloc(s, &s->ilist[1], N));
  AL(dalloc(s, &s->icount[0], 1));
  AL(dalloc(s, &s->icount[1], 1));
  AL(dalloc(s, &s->nlist, N));
  s->nseg = (size_t)cfg->ny * cfg->nz * ((cfg->nx + 31) / 32);
  AL(dalloc(s, &s->seglist[0], s->nseg));
  AL(dalloc(s, &s->seglist[1], s->nseg));
  AL(dalloc(s, &s->segcount[0], 1));
  AL(dalloc(s, &s->segcount[1], 1));
  AL(dalloc(s, &s->segflag, s->nseg));
  AL(dalloc(s, &s->mlist, N));
  AL(dalloc(s, &s->mcount, 2));
  AL(dalloc(s, &s->ncount, 1));
  AL(dev_alloc(s, &s->M, N * s->rsz));
  AL(dev_alloc(s, &s->phi, N * s->rsz));
  AL(dev_alloc(s, &s->uI, 3 * N * s->rsz));
  AL(dev_alloc(s, &s->kappa, N * s->rsz));
  AL(dev_alloc(s, &s->Pi, N * s->rsz));
  AL(dev_alloc(s, &s->nrm, 3 * N * s->rsz));
  AL(dev_alloc(s, &s->dst, N * s->rsz));
  AL(dev_alloc(s, &s->ex, N * s->rsz));
  AL(dev_alloc(s, &s->mom, 5 * N * s->rsz));
  AL(dalloc(s, &s->label[0], N));
  AL(dalloc(s, &s->label[1], N));
  AL(dalloc(s, &s->parent, N));
  AL(dalloc(s, &s->lsize, N));
  {
    // union-find tiles: 32x8x4 in 3D, 32x32 in 2D
    const size_t tx = (cfg->nx + 31) / 32, ty = (cfg->ny + (s->dim == 3 ? 7 : 31)) / (s->dim == 3 ? 8 : 32),
                 tz = s->dim == 3 ? (cfg->nz + 3) / 4 : 1;
    AL(dalloc(s, &s->tstat, tx * ty * tz));
    AL(dalloc(s, &s->troot, tx * ty * tz));
    AL(dalloc(s, &s->tdirty, tx * ty * tz));
    s->ntiles_alloc = tx * ty * tz;
  }
  AL(dalloc(s, &s->roots, (size_t)s->cap));
  AL(dalloc(s, &s->nroots, 1));
  AL(dalloc(s, &s->hash, (size_t)hs));
  AL(dalloc(s, &s->hlist, (size_t)hs));
  AL(dalloc(s, &s->hcount, 1));
  for (int k = 0; k < 2; ++k) {
    Table &t = s->tab[k];
    AL(dalloc(s, &t.m, s->cap));
    AL(dalloc(s, &t.p, s->cap));
    AL(dalloc(s, &t.V, s->cap));
    AL(dalloc(s, &t.dm, s->cap));
    AL(dalloc(s, &t.id, s->cap));
    AL(dalloc(s, &t.atm, s->cap));
    AL(dalloc(s, &t.root, s->cap));
    AL(dalloc(s, &t.ng, s->cap));
    AL(dalloc(s, &t.count, 1));
  }
  const size_t G2 = 2 * (size_t)s->cap;
  AL(dalloc(s, &s->gpar, G2));
  AL(dalloc(s, &s->gnold, G2));
  AL(dalloc(s, &s->gnnew, G2));
  AL(dalloc(s, &s->gatm, G2));
  AL(dalloc(s, &s->gminid, G2));
  AL(dalloc(s, &s->gheir, G2));
  AL(dalloc(s, &s->gmold, G2));
  AL(dalloc(s, &s->gvnew, G2));
  AL(dalloc(s, &s->gvmax, G2));
  AL(dalloc(s, &s->next_id, 1));
  AL(dalloc(s, &s->led, 8));
  AL(dalloc(s, &s->fluid_updates, 1));
  AL(dalloc(s, &s->err, 1));
  AL(dalloc(s, &s->gas_dirty, 1));
  AL(dalloc(s, &s->lab_slow, 1));
  AL(dalloc(s, &s->forest_stale, 1));
  AL(dalloc(s, &s->lab_fast, 1));
  AL(dalloc(s, &s->lab_full, 1));
  AL(dalloc(s, &s->rmv, 2));
  AL(dalloc(s, &s->wmask, N));
  AL(dalloc(s, &s->rlabel, N));
  AL(dalloc(s, &s->acc, 4));
  AL(dalloc(s, &s->counts, 4));
#undef AL
  // zero everything that is read before being written
  auto zero = [&](void *p, size_t b) { return cudaMemsetAsync(p, 0, b, s->st); };
  cudaError_t e = cudaSuccess;
  e = e ? e : zero(s->f, N * s->Q * s->ssz);
  e = e ? e : zero(s->g, N * s->QA * s->ssz);
  e = e ? e : zero(s->kappa, N * s->rsz);
  e = e ? e : zero(s->Pi, N * s->rsz);
  e = e ? e : zero(s->uI, 3 * N * s->rsz);
  e = e ? e : zero(s->ex, N * s->rsz);
  e = e ? e : zero(s->mom, 5 * N * s->rsz);
  e = e ? e : cudaMemsetAsync(s->label[0], 0xff, sizeof(int) * N, s->st);
  e = e ? e : cudaMemsetAsync(s->label[1], 0xff, sizeof(int) * N, s->st);
  e = e ? e : cudaMemsetAsync(s->hash, 0xff, sizeof(unsigned long long) * hs, s->st);
  for (int k = 0; k < 2; ++k) {
    e = e ? e : zero(s->tab[k].count, sizeof(int));
    e = e ? e : zero(s->tab[k].dm, sizeof(double) * s->cap);
    e = e ? e : zero(s->tab[k].ng, sizeof(int) * s->cap);
  }
  e = e ? e : zero(s->next_id, sizeof(int));
  e = e ? e : zero(s->icount[0], sizeof(int));
  e = e ? e : zero(s->icount[1], sizeof(int));
  e = e ? e : zero(s->ncount, sizeof(int));
  e = e ? e : zero(s->segcount[0], sizeof(int));
  e = e ? e : zero(s->segcount[1], sizeof(int));
  e = e ? e : zero(s->segflag, sizeof(int) * s->nseg);
  e = e ? e : zero(s->mcount, 2 * sizeof(int));
  e = e ? e : zero(s->hcount, sizeof(int));
  e = e ? e : zero(s->led, 8 * sizeof(double));
  e = e ? e : zero(s->fluid_updates, sizeof(unsigned long long));
  e = e ? e : zero(s->err, sizeof(int));
  e = e ? e : zero(s->gas_dirty, sizeof(int));
  e = e ? e : zero(s->lab_slow, sizeof(int));
  e = e ? e : zero(s->forest_stale, sizeof(int));
  e = e ? e : zero(s->lab_fast, sizeof(int));
  e = e ? e : cudaMemsetAsync(s->lab_full, 0xff, sizeof(int), s->st);
  e = e ? e : cudaMemsetAsync(s->rmv, 0xff, sizeof(int), s->st);
  e = e ? e : cudaMemsetAsync(s->rmv + 1, 0, sizeof(int), s->st);
  e = e ? e : zero(s->tdirty, s->ntiles_alloc);
  if (e != cudaSuccess) {
    lbf_destroy(s);
    return fail(LBF_ECUDA, std::string("cudaMemsetAsync: ") + cudaGetErrorString(e));
  }
  rc = build_tau_table(s);
  if (rc) {
    std::string msg = g_err;
    lbf_destroy(s);
    return fail(rc, msg);
  }
  Params p = make_params(s, 0);
  s->walled = all_faces_walled(s);  // the fill makes every face layer a wall
  s->ops->init_fill(p, 0, cfg->fill_height, s->st);
  s->ops->nearwall(p, s->st);
  rc = separate_and_relabel(s);
  if (!rc) rc = check_device_error(s);
  if (rc) {
    std::string msg = g_err;
    lbf_destroy(s);
    return fail(rc, msg);
  }
  s->n_state_allocs = s->allocs.size();
  *out = s;
  return 0;
}

int lbf_nucleate(lbf_sim *s, int n, const double *centres, const double *radii, const long long *at_step) {
  if (!s || n < 0 || (n > 0 && (!centres || !radii))) return fail(LBF_EINVAL, "bad arguments");
  for (int k = 0; k < n; ++k) {
    if (!(radii[k] > 0.0)) return fail(LBF_EINVAL, "radius must be positive");
    if (at_step && at_step[k] < s->step) return fail(LBF_EINVAL, "nucleation step is in the past");
  }
  for (int k = 0; k < n; ++k) {
    Nucleus nu;
    nu.step = at_step ? at_step[k] : s->step;
    nu.c[0] = centres[3 * k];
    nu.c[1] = centres[3 * k + 1];
    nu.c[2] = s->dim == 3 ? centres[3 * k + 2] : 0.0;
    nu.r = radii[k];
    s->queue.push_back(nu);
  }
  std::stable_sort(s->queue.begin(), s->queue.end(),
                   [](const Nucleus &a, const Nucleus &b) { return a.step < b.step; });
  int rc = carve_due_nuclei(s);
  if (rc) return rc;
  return check_device_error(s);
}

int lbf_set_cells(lbf_sim *s, const uint8_t *type, const double *rho, const double *u, const double *alpha,
                  const double *c) {
  if (!s || !type || !rho || !u || !alpha || !c) return fail(LBF_EINVAL, "NULL argument");
  const size_t N = (size_t)s->N;
  void *buf = nullptr;
  const size_t bytes = N + N * 8 * 6 + 64;
  CK(cudaMallocAsync(&buf, bytes, s->st));
  uint8_t *dt = (uint8_t *)buf;
  double *drho = (double *)((char *)buf + ((N + 15) / 16) * 16);
  double *du = drho + N, *da = du + 3 * N, *dc = da + N;
  CK(cudaMemcpyAsync(dt, type, N, cudaMemcpyHostToDevice, s->st));
  CK(cudaMemcpyAsync(drho, rho, 8 * N, cudaMemcpyHostToDevice, s->st));
  CK(cudaMemcpyAsync(du, u, 24 * N, cudaMemcpyHostToDevice, s->st));
  CK(cudaMemcpyAsync(da, alpha, 8 * N, cudaMemcpyHostToDevice, s->st));
  CK(cudaMemcpyAsync(dc, c, 8 * N, cudaMemcpyHostToDevice, s->st));
  // the input is checked before it replaces anything: a rejected call leaves
  // the state as it was
  CK(cudaMemsetAsync(s->counts, 0, sizeof(unsigned long long), s->st));
  lbf::check_cells_launch(dt, drho, du, da, dc, s->N, s->counts, s->list_blocks, s->st);
  CK(cudaGetLastError());
  unsigned long long bad = 0;
  CK(cudaMemcpyAsync(&bad, s->counts, sizeof bad, cudaMemcpyDeviceToHost, s->st));
  CK(cudaStreamSynchronize(s->st));
  if (bad) {
    CK(cudaFreeAsync(buf, s->st));
    CK(cudaStreamSynchronize(s->st));
    if (bad & 2) return fail(LBF_ENONFINITE, "non-finite value in the cell arrays");
    if (bad & 1) return fail(LBF_EINVAL, "cell type outside 0..3");
    return fail(LBF_EINVAL, "density not positive in a liquid or interface cell");
  }
  // the walled sweep needs fluid-free face layers; the step graphs change
  // shape when that changes
  const bool walled = all_faces_walled(s) && !fluid_in_faces(s, type);
  if (walled != s->walled) {
    s->walled = walled;
    drop_graphs(s);
  }
  const int par = (int)(s->step & 1);
  Params p = make_params(s, s->step);
  s->ops->init_cells(p, par, dt, drho, du, da, dc, s->st);
  s->ops->nearwall(p, s->st);
  CK(cudaFreeAsync(buf, s->st));
  CK(cudaMemsetAsync(s->label[par], 0xff, sizeof(int) * N, s->st));
  CK(cudaMemsetAsync(s->tab[par].count, 0, sizeof(int), s->st));
  int rc = separate_and_relabel(s);
  if (rc) return rc;
  return check_device_error(s);
}

int lbf_step(lbf_sim *s, int nsteps) {
  if (!s || nsteps < 0) return fail(LBF_EINVAL, "bad arguments");
  if (nsteps > 0 && !s->timing) {
    int rc = ensure_all_graphs(s);
    if (rc) return rc;
  }
  for (int k = 0; k < nsteps;) {
    int rc = carve_due_nuclei(s);
    if (rc) return rc;
    int chain = 1;
    if (!s->timing && k + 3 < nsteps && !nucleus_due(s, s->step + 3))
      chain = 4;
    else if (!s->timing && k + 1 < nsteps && !nucleus_due(s, s->step + 1))
      chain = 2;
    if (chain > 1) {
      rc = run_steps(s, chain);
      if (rc) return rc;
      s->step += chain;
      k += chain;
    } else {
      rc = run_one_step(s);
      if (rc) return rc;
      ++s->step;
      ++k;
    }
  }
  return check_device_error(s);
}

long long lbf_step_count(const lbf_sim *s) { return s ? s->step : -1; }


int lbf_mlp_harvest(lbf_sim *s, float *x, float *y, int *cells, int cap, int *count) {
  if (!s || !x || !y || cap < 0 || !count) return fail(LBF_EINVAL, "bad arguments");
  if (s->dim != 3) return fail(LBF_EINVAL, "the learned curvature is three-dimensional");
  if (!s->mlp_count) {
    int rc = dalloc(s, &s->mlp_count, 1);
    if (rc) return rc;
  }
  Params p = make_params(s, s->step);
  CK(cudaMemsetAsync(s->mlp_count, 0, sizeof(int), s->st));
  s->ops->mlp_harvest(p, x, y, cells, cap, s->mlp_count, s->st);
  CK(cudaGetLastError());
  int h = 0;
  CK(cudaMemcpyAsync(&h, s->mlp_count, sizeof(int), cudaMemcpyDeviceToHost, s->st));
  CK(cudaStreamSynchronize(s->st));
  *count = h < cap ? h : cap;
  return 0;
}

// the captured step graphs, rebuilt on the next step
static void drop_graphs(lbf_sim *s) {
  for (int k = 0; k < 2; ++k) {
    if (s->graph[k]) cudaGraphExecDestroy(s->graph[k]);
    if (s->tgraph[k]) cudaGraphExecDestroy(s->tgraph[k]);
    if (s->graph2[k]) cudaGraphExecDestroy(s->graph2[k]);
    if (s->graph4[k]) cudaGraphExecDestroy(s->graph4[k]);
    s->graph[k] = s->tgraph[k] = s->graph2[k] = s->graph4[k] = nullptr;
  }
}

int lbf_mlp_attach(lbf_sim *s, const float *theta) {
  if (!s) return fail(LBF_EINVAL, "NULL sim");
  if (theta && s->dim != 3) return fail(LBF_EINVAL, "the learned curvature is three-dimensional");
  if (theta) {
    if (!s->mlp_buf) {
      int rc = dalloc(s, &s->mlp_buf, 6017);
      if (rc) return rc;
    }
    if (!s->mlp_img) {
      int rc = dev_alloc(s, &s->mlp_img, lbf::mlp::image_bytes());
      if (rc) return rc;
    }
    CK(cudaMemcpyAsync(s->mlp_buf, theta, sizeof(float) * 6017, cudaMemcpyHostToDevice, s->st));
    // 64-bit FNV-1a of the parameter bytes: identifies the network in checkpoints
    unsigned long long h = 0xcbf29ce484222325ull;
    const unsigned char *tb = (const unsigned char *)theta;
    for (size_t k = 0; k < sizeof(float) * 6017; ++k) h = (h ^ tb[k]) * 0x100000001b3ull;
    s->mlp_hash = h ? h : 1;
    lbf::mlp::pack_launch(s->mlp_buf, s->mlp_img, s->st);
    CK(cudaGetLastError());
    CK(cudaStreamSynchronize(s->st));
    s->mlp_theta = s->mlp_img;
  } else {
    s->mlp_theta = nullptr;  // the buffer stays owned by the sim until destroy
    s->mlp_hash = 0;
  }
  // the step graphs change shape
  drop_graphs(s);
  return 0;
}

// ---------------------------------------------------------------------------
// checkpoint: every device array made at creation, the step count and the
// queued nuclei, after a header; restored into a sim of the same layout

namespace {
struct CkptHeader {
  unsigned long long magic;
  long long step, n_arrays, n_queue;
  int mlp_attached, dim;
  unsigned long long mlp_hash;  // FNV-1a of the attached network's parameters, 0 if none
  int walled, pad;              // the saved state's face layers hold no fluid
};
constexpr unsigned long long kCkptMagic = 0x3354504b4346424cull;  // "LBFCKPT3"

size_t ckpt_bytes(const lbf_sim *s) {
  size_t b = sizeof(CkptHeader) + s->n_state_allocs * sizeof(unsigned long long) + s->queue.size() * sizeof(Nucleus);
  for (size_t k = 0; k < s->n_state_allocs; ++k) b += s->alloc_bytes[k];
  return b;
}
}  // namespace

int lbf_checkpoint_bytes(lbf_sim *s, size_t *bytes) {
  if (!s || !bytes) return fail(LBF_EINVAL, "NULL argument");
  *bytes = ckpt_bytes(s);
  return 0;
}

int lbf_checkpoint_save(lbf_sim *s, void *dst, size_t bytes) {
  if (!s || !dst) return fail(LBF_EINVAL, "NULL argument");
  if (bytes < ckpt_bytes(s)) return fail(LBF_EINVAL, "buffer smaller than lbf_checkpoint_bytes");
  CK(cudaStreamSynchronize(s->st));
  unsigned char *o = (unsigned char *)dst;
  CkptHeader h;
  std::memset(&h, 0, sizeof h);
  h.magic = kCkptMagic;
  h.step = s->step;
  h.n_arrays = (long long)s->n_state_allocs;
  h.n_queue = (long long)s->queue.size();
  h.mlp_attached = s->mlp_theta != nullptr;
  h.dim = s->dim;
  h.mlp_hash = s->mlp_theta ? s->mlp_hash : 0;
  h.walled = s->walled ? 1 : 0;
  std::memcpy(o, &h, sizeof h);
  o += sizeof h;
  for (size_t k = 0; k < s->n_state_allocs; ++k) {
    const unsigned long long b = s->alloc_bytes[k];
    std::memcpy(o, &b, sizeof b);
    o += sizeof b;
  }
  if (!s->queue.empty()) std::memcpy(o, s->queue.data(), s->queue.size() * sizeof(Nucleus));
  o += s->queue.size() * sizeof(Nucleus);
  for (size_t k = 0; k < s->n_state_allocs; ++k) {
    CK(cudaMemcpyAsync(o, s->allocs[k], s->alloc_bytes[k], cudaMemcpyDeviceToHost, s->st));
    o += s->alloc_bytes[k];
  }
  CK(cudaStreamSynchronize(s->st));
  return 0;
}

int lbf_checkpoint_load(lbf_sim *s, const void *src, size_t bytes) {
  if (!s || !src) return fail(LBF_EINVAL, "NULL argument");
  const unsigned char *i = (const unsigned char *)src;
  CkptHeader h;
  if (bytes < sizeof h) return fail(LBF_EINVAL, "checkpoint too short");
  std::memcpy(&h, i, sizeof h);
  i += sizeof h;
  if (h.magic != kCkptMagic) return fail(LBF_EINVAL, "not a checkpoint");
  if (h.dim != s->dim || h.n_arrays != (long long)s->n_state_allocs || h.n_queue < 0)
    return fail(LBF_EINVAL, "checkpoint of a sim with another layout");
  if ((h.mlp_attached != 0) != (s->mlp_theta != nullptr))
    return fail(LBF_EINVAL, "attach the learned curvature alike before loading");
  if (h.mlp_attached && h.mlp_hash != s->mlp_hash)
    return fail(LBF_EINVAL, "checkpoint saved with another learned-curvature network");
  // the size table must lie inside the buffer before it is read
  const size_t table = s->n_state_allocs * sizeof(unsigned long long);
  if (bytes - sizeof h < table) return fail(LBF_EINVAL, "checkpoint too short");
  size_t arrays = 0;
  for (size_t k = 0; k < s->n_state_allocs; ++k) {
    unsigned long long b;
    std::memcpy(&b, i + k * sizeof b, sizeof b);
    if (b != s->alloc_bytes[k]) return fail(LBF_EINVAL, "checkpoint of a sim with another layout");
    arrays += b;
  }
  i += table;
  // what is left after the header, the table and the arrays bounds the queue
  const size_t rest = bytes - sizeof h - table;
  if (rest < arrays || (unsigned long long)h.n_queue > (rest - arrays) / sizeof(Nucleus))
    return fail(LBF_EINVAL, "checkpoint too short");
  std::vector<Nucleus> q((size_t)h.n_queue);
  if (h.n_queue) std::memcpy(q.data(), i, q.size() * sizeof(Nucleus));
  i += q.size() * sizeof(Nucleus);
  // ordered on the sim's stream (which does not synchronise with the legacy
  // stream) and complete before the call returns
  for (size_t k = 0; k < s->n_state_allocs; ++k) {
    CK(cudaMemcpyAsync(s->allocs[k], i, s->alloc_bytes[k], cudaMemcpyHostToDevice, s->st));
    i += s->alloc_bytes[k];
  }
  CK(cudaStreamSynchronize(s->st));
  s->step = h.step;
  s->walled = h.walled != 0 && all_faces_walled(s);
  s->queue.swap(q);
  drop_graphs(s);
  return 0;
}

int lbf_bubbles(lbf_sim *s, lbf_bubble *out, int capacity, int *count) {
  if (!s || !count || capacity < 0 || (capacity > 0 && !out)) return fail(LBF_EINVAL, "bad arguments");
  // rows packed on the device, then one copy into pinned staging memory
  const int rows = std::min(capacity, s->cap);
  const size_t bytes = 16 + sizeof(lbf_bubble) * (size_t)rows;
  if (!s->bub_dev) {
    int rc = dev_alloc(s, (void **)&s->bub_dev, 16 + sizeof(lbf_bubble) * (size_t)s->cap);
    if (rc) return rc;
    CK(cudaMallocHost((void **)&s->bub_host, 16 + sizeof(lbf_bubble) * (size_t)s->cap));
  }
  lbf::pack_bubbles_launch(s->tab[s->step & 1], s->bub_dev, rows, s->st);
  CK(cudaGetLastError());
  // the header and the first rows in one copy; the rest only when present
  constexpr int kFirst = 64;
  const size_t first = std::min(bytes, 16 + sizeof(lbf_bubble) * (size_t)kFirst);
  CK(cudaMemcpyAsync(s->bub_host, s->bub_dev, first, cudaMemcpyDeviceToHost, s->st));
  CK(cudaStreamSynchronize(s->st));
  int nb = 0;
  std::memcpy(&nb, s->bub_host, sizeof(int));
  *count = nb;
  const int k = std::min(nb, rows);
  if (k > kFirst) {
    const size_t off = 16 + sizeof(lbf_bubble) * (size_t)kFirst;
    CK(cudaMemcpyAsync(s->bub_host + off, s->bub_dev + off, sizeof(lbf_bubble) * (size_t)(k - kFirst),
                       cudaMemcpyDeviceToHost, s->st));
    CK(cudaStreamSynchronize(s->st));
  }
  if (k > 0) std::memcpy(out, s->bub_host + 16, sizeof(lbf_bubble) * (size_t)k);
  return 0;
}

int lbf_fields(lbf_sim *s, unsigned mask, void *const *dst, int dst_is_device, int dtype) {
  if (!s || !dst || (dtype != 0 && dtype != 1)) return fail(LBF_EINVAL, "bad arguments");
  if (mask >> 11) return fail(LBF_EINVAL, "unknown field bit");
  const int par = (int)(s->step & 1);
  Params p = make_params(s, s->step);
  p.label_new = s->label[par];
  const size_t N = (size_t)s->N;
  int k = 0;
  for (int bit = 0; bit < 11; ++bit) {
    if (!(mask & (1u << bit))) continue;
    void *out = dst[k++];
    if (!out) return fail(LBF_EINVAL, "NULL destination");
    const bool is_int = bit == FLD_FLAGS || bit == FLD_LABEL;
    const int width = (bit == FLD_U || bit == FLD_NORMAL) ? 3 : 1;
    const size_t bytes = N * width * (is_int ? 4 : (dtype ? 8 : 4));
    if (dst_is_device) {
      s->ops->field(p, par, bit, out, dtype, s->st);
      CK(cudaGetLastError());
    } else {
      if (!s->staging) {
        int rc = dev_alloc(s, &s->staging, N * 3 * 8);
        if (rc) return rc;
      }
      s->ops->field(p, par, bit, s->staging, dtype, s->st);
      CK(cudaGetLastError());
      int rc = copy_to_host(s, out, s->staging, bytes);
      if (rc) return rc;
    }
  }
  return 0;
}

static int run_ledger(lbf_sim *s, double *acc3, unsigned long long *cnt4) {
  const int par = (int)(s->step & 1);
  Params p = make_params(s, s->step);
  CK(cudaMemsetAsync(s->acc, 0, 4 * sizeof(double), s->st));
  CK(cudaMemsetAsync(s->counts, 0, 4 * sizeof(unsigned long long), s->st));
  s->ops->ledger(p, par, s->acc, s->counts, s->st);
  CK(cudaGetLastError());
  CK(cudaMemcpyAsync(acc3, s->acc, 3 * sizeof(double), cudaMemcpyDeviceToHost, s->st));
  CK(cudaMemcpyAsync(cnt4, s->counts, 4 * sizeof(unsigned long long), cudaMemcpyDeviceToHost, s->st));
  CK(cudaStreamSynchronize(s->st));
  return 0;
}

int lbf_ledger(lbf_sim *s, double *out) {
  if (!s || !out) return fail(LBF_EINVAL, "bad arguments");
  double acc[3];
  unsigned long long cnt[4];
  int rc = run_ledger(s, acc, cnt);
  if (rc) return rc;
  double led[8];
  unsigned long long upd = 0;
  CK(cudaMemcpyAsync(led, s->led, sizeof led, cudaMemcpyDeviceToHost, s->st));
  CK(cudaMemcpyAsync(&upd, s->fluid_updates, sizeof upd, cudaMemcpyDeviceToHost, s->st));
  const Table &t = s->tab[s->step & 1];
  int nb = 0;
  CK(cudaMemcpyAsync(&nb, t.count, sizeof(int), cudaMemcpyDeviceToHost, s->st));
  CK(cudaStreamSynchronize(s->st));
  double gas = 0.0;
  if (nb > 0) {
    std::vector<double> m(nb);
    CK(cudaMemcpyAsync(m.data(), t.m, sizeof(double) * nb, cudaMemcpyDeviceToHost, s->st));
    CK(cudaStreamSynchronize(s->st));
    for (double v : m) gas += v;
  }
  out[0] = acc[0];
  out[1] = led[1];
  out[2] = led[2];
  out[3] = acc[1];
  out[4] = gas;
  out[5] = led[5];
  out[6] = s->cfg.q * (double)upd;
  out[7] = acc[2];
  if (acc[2] > 0.0) return fail(LBF_ENONFINITE, "non-finite populations");
  return 0;
}

int lbf_cell_counts(lbf_sim *s, long long *out4) {
  if (!s || !out4) return fail(LBF_EINVAL, "bad arguments");
  double acc[3];
  unsigned long long cnt[4];
  int rc = run_ledger(s, acc, cnt);
  if (rc) return rc;
  for (int k = 0; k < 4; ++k) out4[k] = (long long)cnt[k];
  return 0;
}

int lbf_timing_enable(lbf_sim *s, int enable) {
  if (!s) return fail(LBF_EINVAL, "NULL sim");
  s->timing = enable != 0;
  for (int k = 0; k < G_COUNT; ++k) {
    s->t_ms[k] = 0.0;
    s->t_n[k] = 0;
  }
  return 0;
}

int lbf_timing_read(lbf_sim *s, double *out_ms, long long *out_launches, int nmax) {
  if (!s) return fail(LBF_EINVAL, "NULL sim");
  for (int k = 0; k < G_COUNT && k < nmax; ++k) {
    if (out_ms) out_ms[k] = s->t_ms[k];
    if (out_launches) out_launches[k] = s->t_n[k];
  }
  return G_COUNT;
}

const char *lbf_timing_name(int k) { return (k >= 0 && k < G_COUNT) ? kGroupNames[k] : ""; }

}  // extern "C"

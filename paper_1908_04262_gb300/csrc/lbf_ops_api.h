// lbf_ops_api.h -- the launch interface seen by the host runtime: one Ops
// object per (lattice, storage) pair, created by the factory of the
// translation unit that holds that storage type's kernels.
#pragma once
#include <cuda_runtime.h>

#include "lbf_common.cuh"

namespace lbf {

// a further sticky device error bit beside those of lbf_common.cuh: a wait
// of the learned curvature on the tensor cores (MMA completion or the
// network's bulk copy) ran past its bound
constexpr int ERR_TC_WAIT = 8;

struct Ops {
  virtual ~Ops() {}
  virtual void init_fill(const Params &p, int par, double h, cudaStream_t s) = 0;
  virtual void init_cells(const Params &p, int par, const uint8_t *t, const double *rho, const double *u,
                          const double *a, const double *c, cudaStream_t s) = 0;
  virtual void separate(const Params &p, int par, cudaStream_t s) = 0;
  virtual void nearwall(const Params &p, cudaStream_t s) = 0;
  virtual void nucleate(const Params &p, int par, const double *c, double R, cudaStream_t s) = 0;
  // step pieces (par = parity of the populations when the step starts)
  virtual void exchange(const Params &p, int par, cudaStream_t s) = 0;
  virtual void build_ilist(const Params &p, cudaStream_t s) = 0;
  // the sweep: liquid cells, then interface cells (the two commute)
  virtual void stream_liquid(const Params &p, int par, cudaStream_t s) = 0;
  virtual void stream_interface(const Params &p, int par, cudaStream_t s) = 0;
  // conversion: marks (after which every cell's post-conversion type is
  // known), excess and its collection, and the pass that writes the new
  // types over the marks
  virtual void convert_mark(const Params &p, cudaStream_t s) = 0;
  virtual void convert_excess(const Params &p, int par, cudaStream_t s) = 0;
  virtual void convert_finalize(const Params &p, cudaStream_t s) = 0;
  void convert(const Params &p, int par, cudaStream_t s) {
    convert_mark(p, s);
    convert_excess(p, par, s);
  }
  // labelling: the union-find forest and sorted roots (post-conversion types
  // only), then the relabelling (which also reads the fill levels)
  virtual void label_forest(const Params &p, cudaStream_t s) = 0;
  virtual void label_relabel(const Params &p, cudaStream_t s) = 0;
  void label(const Params &p, cudaStream_t s) {
    label_forest(p, s);
    label_relabel(p, s);
  }
  virtual void label_prep(const Params &p, cudaStream_t s) = 0;
  virtual void bubble_update(const Params &p, cudaStream_t s) = 0;
  // a step whose added gas cells keep every bubble's cells, number and root
  // (decided on the device after the marking, label_choose) patches the
  // labels of the last step (label_fast) and updates one-to-one bubble
  // groups (bubble_update_fast); the union-find kernels, the relabelling and
  // the general bubble update return at once in such a step, the patch
  // kernels in every other
  virtual void label_check(const Params &p, cudaStream_t s) = 0;  // after the marking
  virtual void label_choose(const Params &p, cudaStream_t s) = 0;
  // at the start of the step, before the marking: label_new brought up to
  // the last labels (see k_label_sync); label_fast then writes the patch
  virtual void label_sync(const Params &p, cudaStream_t s) = 0;
  virtual void label_fast(const Params &p, cudaStream_t s) = 0;
  virtual void bubble_update_fast(const Params &p, cudaStream_t s) = 0;
  virtual void geometry(const Params &p, cudaStream_t s) = 0;
  virtual void disjoining(const Params &p, cudaStream_t s) = 0;
  virtual void mlp_kappa(const Params &p, const void *img, cudaStream_t s) = 0;
  virtual void mlp_harvest(const Params &p, float *x, float *y, int *cells, int cap, int *count, cudaStream_t s) = 0;
  // export
  virtual void field(const Params &p, int par, int which, void *out, int dtype, cudaStream_t s) = 0;
  virtual void ledger(const Params &p, int par, double *acc, unsigned long long *counts, cudaStream_t s) = 0;
};

// message returned by lbf_last_error() on the calling thread
void set_last_error(const char *msg);

namespace mlp {
// bytes of the packed BF16 image of the network parameters, and the launch
// that builds it from the 6017 FP32 parameters (both device pointers)
size_t image_bytes();
void pack_launch(const float *theta, void *img, cudaStream_t st);
}  // namespace mlp

// defined in one translation unit per storage type
Ops *make_ops_f64(int dim);
Ops *make_ops_f32(int dim);
Ops *make_ops_f16(int dim);
Ops *make_ops_bf16(int dim);

}  // namespace lbf

// lbf_ops.cuh -- launch layer: one Ops object per (lattice, storage) pair
// turns the host runtime's requests into kernel launches on a stream.
#pragma once
#include <cuda_runtime.h>

#include "lbf_common.cuh"
#include "lbf_ops_api.h"
#include "lbf_convert.cuh"
#include "lbf_geom.cuh"
#include "lbf_label.cuh"
#include "lbf_mlp_kappa.cuh"
#include "lbf_stream.cuh"

namespace lbf {

inline unsigned blocks_for(long long n, int b) { return (unsigned)((n + b - 1) / b); }

// full-lattice launches: blocks of B threads along x, one block row per (y, z)
inline int row_block(const Params &p) { return p.nx >= 96 ? 128 : (p.nx > 32 ? 64 : 32); }
inline dim3 row_grid(const Params &p) {
  const int b = row_block(p);
  return dim3((unsigned)((p.nx + b - 1) / b), (unsigned)p.ny, (unsigned)p.nz);
}

template <int D, class S>
struct OpsImpl final : Ops {
  using R = typename ST<S>::R;
  static constexpr int B = 256;

  // the root sort holds up to 16384 roots (64 KB) in shared memory
  OpsImpl() { cudaFuncSetAttribute(k_sort_roots, cudaFuncAttributeMaxDynamicSharedMemorySize, 16384 * (int)sizeof(int)); }

  void init_fill(const Params &p, int par, double h, cudaStream_t s) override {
    k_init_fill<D, S><<<row_grid(p), row_block(p), 0, s>>>(p, par, h);
  }
  void init_cells(const Params &p, int par, const uint8_t *t, const double *rho, const double *u,
                  const double *a, const double *c, cudaStream_t s) override {
    k_init_cells<D, S><<<row_grid(p), row_block(p), 0, s>>>(p, par, t, rho, u, a, c);
  }
  void separate(const Params &p, int par, cudaStream_t s) override {
    k_separate_mark<D><<<row_grid(p), row_block(p), 0, s>>>(p);
    k_separate_apply<D, S><<<row_grid(p), row_block(p), 0, s>>>(p, par);
  }
  void nearwall(const Params &p, cudaStream_t s) override { k_nearwall<D><<<row_grid(p), row_block(p), 0, s>>>(p); }
  void nucleate(const Params &p, int par, const double *c, double R0, cudaStream_t s) override {
    const int x0 = (int)floor(c[0] - R0 - 1.0), x1 = (int)ceil(c[0] + R0 + 1.0);
    const int y0 = (int)floor(c[1] - R0 - 1.0), y1 = (int)ceil(c[1] + R0 + 1.0);
    const int z0 = D == 3 ? (int)floor(c[2] - R0 - 1.0) : 0, z1 = D == 3 ? (int)ceil(c[2] + R0 + 1.0) : 0;
    const int bx = x1 - x0 + 1, by = y1 - y0 + 1, bz = z1 - z0 + 1;
    const long long cnt = (long long)bx * by * bz;
    k_nucleate<D, S><<<blocks_for(cnt, B), B, 0, s>>>(p, par, c[0], c[1], D == 3 ? c[2] : 0.0, R0, x0, y0,
                                                        z0, bx, by, bz);
  }
  void exchange(const Params &p, int par, cudaStream_t s) override {
    if (p.walled)
      par ? k_exchange<D, S, 1, true><<<p.warp_blocks, 128, 0, s>>>(p) : k_exchange<D, S, 0, true><<<p.warp_blocks, 128, 0, s>>>(p);
    else
      par ? k_exchange<D, S, 1><<<p.warp_blocks, 128, 0, s>>>(p) : k_exchange<D, S, 0><<<p.warp_blocks, 128, 0, s>>>(p);
  }
  void build_ilist(const Params &p, cudaStream_t s) override {
    cudaMemsetAsync(p.icount, 0, sizeof(int), s);
    cudaMemsetAsync(p.segcount, 0, sizeof(int), s);
    k_build_ilist<<<row_grid(p), row_block(p), 0, s>>>(p);
  }
  // (the collision model is a template parameter: the BGK sweep keeps its
  // registers)
  void stream_liquid(const Params &p, int par, cudaStream_t s) override {
    const dim3 g = row_grid(p);
    const int b = row_block(p);
    if (p.coll == 2)
      par ? k_stream_liquid<D, S, 1, 2><<<g, b, 0, s>>>(p) : k_stream_liquid<D, S, 0, 2><<<g, b, 0, s>>>(p);
    else if (p.coll == 1)
      par ? k_stream_liquid<D, S, 1, 1><<<g, b, 0, s>>>(p) : k_stream_liquid<D, S, 0, 1><<<g, b, 0, s>>>(p);
    else if (p.walled)
      par ? k_stream_liquid<D, S, 1, 0, true><<<g, b, 0, s>>>(p)
          : k_stream_liquid<D, S, 0, 0, true><<<g, b, 0, s>>>(p);
    else
      par ? k_stream_liquid<D, S, 1, 0><<<g, b, 0, s>>>(p) : k_stream_liquid<D, S, 0, 0><<<g, b, 0, s>>>(p);
  }
  void stream_interface(const Params &p, int par, cudaStream_t s) override {
    const int g = p.list_blocks;
    if (p.coll == 2)
      par ? k_stream_interface<D, S, 1, 2><<<g, 128, 0, s>>>(p) : k_stream_interface<D, S, 0, 2><<<g, 128, 0, s>>>(p);
    else if (p.coll == 1)
      par ? k_stream_interface<D, S, 1, 1><<<g, 128, 0, s>>>(p) : k_stream_interface<D, S, 0, 1><<<g, 128, 0, s>>>(p);
    else if (p.walled)
      par ? k_stream_interface<D, S, 1, 0, true><<<g, 128, 0, s>>>(p)
          : k_stream_interface<D, S, 0, 0, true><<<g, 128, 0, s>>>(p);
    else
      par ? k_stream_interface<D, S, 1, 0><<<g, 128, 0, s>>>(p)
          : k_stream_interface<D, S, 0, 0><<<g, 128, 0, s>>>(p);
  }
  void convert_mark(const Params &p, cudaStream_t s) override { k_conv_mark<D><<<p.list_blocks, 128, 0, s>>>(p); }
  void convert_excess(const Params &p, int par, cudaStream_t s) override {
    const int post = 1 - par;
    k_conv_compute<D, S><<<p.list_blocks, 128, 0, s>>>(p, post);
    k_conv_apply<D, S><<<p.list_blocks, 128, 0, s>>>(p, post);
  }
  void convert_finalize(const Params &p, cudaStream_t s) override {
    k_conv_finalize<D><<<p.list_blocks, 128, 0, s>>>(p);
  }
  void label_prep(const Params &p, cudaStream_t s) override {
    k_label_prep<<<blocks_for(p.cap, B), B, 0, s>>>(p);
  }
  void label_forest(const Params &p, cudaStream_t s) override {
    const dim3 tg((unsigned)((p.nx + Tile<D>::TX - 1) / Tile<D>::TX), (unsigned)((p.ny + Tile<D>::TY - 1) / Tile<D>::TY),
                  (unsigned)((p.nz + Tile<D>::TZ - 1) / Tile<D>::TZ));
    // tile loops on a grid of two blocks per SM (a block of the
    // graph's patch steps then costs one short wave)
    const unsigned ntiles = tg.x * tg.y * tg.z;
    const unsigned g = p.tile_blocks > 0 && (unsigned)p.tile_blocks < ntiles ? (unsigned)p.tile_blocks : ntiles;
    k_uf_local<D><<<g, TILE_THREADS, 0, s>>>(p);
    k_uf_merge<D><<<g, TILE_THREADS, 0, s>>>(p);
    k_uf_compress<D><<<g, TILE_THREADS, 0, s>>>(p);
    int P = 1;
    while (P < p.cap) P <<= 1;
    k_sort_roots<<<1, 1024, P * sizeof(int), s>>>(p);
  }
  void label_relabel(const Params &p, cudaStream_t s) override {
    // row blocks walked by a grid of 16 blocks per SM
    const unsigned nrb = row_grid(p).x * (unsigned)p.ny * (unsigned)p.nz;
    const unsigned g = (unsigned)p.warp_blocks < nrb ? (unsigned)p.warp_blocks : nrb;
    k_relabel<D, R><<<g, row_block(p), 0, s>>>(p);
  }
  void bubble_update(const Params &p, cudaStream_t s) override { k_bubble_update<<<1, 1024, 0, s>>>(p); }
  void label_check(const Params &p, cudaStream_t s) override {
    k_label_check<D><<<p.list_blocks, 128, 0, s>>>(p);
    k_root_scan<<<1, 1024, 0, s>>>(p);
  }
  void label_choose(const Params &p, cudaStream_t s) override { k_label_choose<<<1, 1, 0, s>>>(p); }
  void label_sync(const Params &p, cudaStream_t s) override { k_label_sync<<<p.list_blocks, 128, 0, s>>>(p); }
  void label_fast(const Params &p, cudaStream_t s) override {
    k_label_fast<D, R><<<p.list_blocks, 128, 0, s>>>(p);
  }
  void bubble_update_fast(const Params &p, cudaStream_t s) override {
    const unsigned g = blocks_for(p.cap, 128);
    k_bubble_update_fast<<<g < (unsigned)p.list_blocks ? g : (unsigned)p.list_blocks, 128, 0, s>>>(p);
  }
  void geometry(const Params &p, cudaStream_t s) override {
    k_geometry<D, R><<<p.warp_blocks, 128, 0, s>>>(p);
    if (p.kappa_hf) k_hf_kappa<D, R><<<p.list_blocks, 128, 0, s>>>(p);
  }
  void mlp_kappa(const Params &p, const void *img, cudaStream_t s) override {
    // up to two CTAs of 128 cells per SM (list_blocks holds 4 per SM);
    // each holds 128 of the SM's 512 tensor-memory columns, and no more
    // than four fit on an SM by their shared memory
    if (D == 3)
      k_mlp_kappa<D, R><<<p.list_blocks / 2, MLP_THREADS, sizeof(tc::Tile), s>>>(p, (const tc::Image *)img);
  }
  void mlp_harvest(const Params &p, float *x, float *y, int *cells, int cap, int *count, cudaStream_t s) override {
    if (D == 3) k_mlp_harvest<D, R><<<p.warp_blocks, 128, 0, s>>>(p, x, y, cells, cap, count);
  }
  void disjoining(const Params &p, cudaStream_t s) override {
    k_disjoining<D, R><<<p.list_blocks, 128, 0, s>>>(p);
  }
  void field(const Params &p, int par, int which, void *out, int dtype, cudaStream_t s) override {
    k_fields<D, S><<<row_grid(p), row_block(p), 0, s>>>(p, par, which, out, dtype);
  }
  void ledger(const Params &p, int par, double *acc, unsigned long long *counts, cudaStream_t s) override {
    k_ledger<D, S><<<row_grid(p), row_block(p), 0, s>>>(p, par, acc, counts);
  }
};

}  // namespace lbf

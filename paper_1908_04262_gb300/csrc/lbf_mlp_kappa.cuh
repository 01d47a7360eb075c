// lbf_mlp_kappa.cuh -- in-loop learned curvature kernel (3D): the network of
// lbf_mlp.cuh applied to the interface list after the least-squares
// geometry pass.
#pragma once
#include "lbf_common.cuh"
#include "lbf_mlp.cuh"
#include "lbf_ops_api.h"
#include "lbf_tc.cuh"

namespace lbf {

// In-loop learned curvature (3D): tiles of 128 interface cells of the
// list, one CTA of 256 threads per tile at a time.  The network's packed
// image (img) arrives by one bulk copy while the first tile is gathered;
// warp w gathers the stencils of rows 16w .. 16w + 15 (turned into the
// canonical orientation of each cell's geometry normal) into the operand
// tile of the tensor cores, and thread r < 128 writes the curvature of row
// r.  The least-squares curvature stays where the network is outside its
// training range (|kappa| outside [0.02, 0.55], i.e. radii beyond [1.8, 50]
// cells) or the stencil touches a wall, and everywhere once a wait has not
// completed within its bound (which also sets ERR_TC_WAIT: lbf_step then
// fails with LBF_ECUDA).
constexpr int MLP_THREADS = 256;
template <int D, class R>
__global__ void __launch_bounds__(MLP_THREADS) k_mlp_kappa(Params p, const tc::Image *img) {
  if constexpr (D == 3) {
    extern __shared__ __align__(128) unsigned char tsm[];
    tc::Tile &t = *reinterpret_cast<tc::Tile *>(tsm);
    __shared__ Cell cs[tc::ROWS];
    __shared__ int ord[tc::ROWS][3], sgn[tc::ROWS][3], use[tc::ROWS];
    const int cnt = *p.icount;
    const int tiles = (cnt + tc::ROWS - 1) / tc::ROWS;
    if ((int)blockIdx.x >= tiles) return;  // uniform over the CTA: no tensor memory taken
    tc::setup(t, img);
    const int tid = threadIdx.x, lane = tid & 31, w = tid >> 5;
    const R *phi = (const R *)p.phi, *nr = (const R *)p.nrm;
    R *kap = (R *)p.kappa;
    uint32_t phase = 0;
    bool failed = false, net = false;
    for (int tile = blockIdx.x; tile < tiles && !failed; tile += gridDim.x) {
      if (tid < tc::ROWS) {
        const int k = tile * tc::ROWS + tid;
        int ok = 0;
        Cell c;
        c.n = -1;
        if (k < cnt) {
          c = make_cell(p, p.ilist[k]);
          const float mx = (float)nr[c.n], my = (float)nr[p.N + c.n], mz = (float)nr[2 * p.N + c.n];
          const float ka = fabsf((float)kap[c.n]);
          ok = (mx != 0.f || my != 0.f || mz != 0.f) && ka >= 0.02f && ka <= 0.55f;
          mlp::canonical_order(mx, my, mz, ord[tid], sgn[tid]);
        }
        cs[tid] = c;
        use[tid] = ok;
      }
      __syncthreads();
      // lane q gathers stencil position q of the warp's 16 rows: every flag
      // and fill level is loaded before any is used
      const int r0 = 16 * w;
      uint8_t fr[16];
      R pr[16];
#pragma unroll
      for (int r = 0; r < 16; ++r) {
        const Cell &c = cs[r0 + r];
        fr[r] = (uint8_t)T_GAS;
        pr[r] = (R)0;
        if (c.n >= 0 && lane < 27 && use[r0 + r]) {
          const int src = mlp::canonical_src(lane, ord[r0 + r], sgn[r0 + r]);
          const int m = at(p, c, src % 3 - 1, (src / 3) % 3 - 1, src / 9 - 1);
          fr[r] = p.flags[m];  // read as post-conversion types below
          pr[r] = phi[m];
        }
      }
      __syncwarp();
#pragma unroll
      for (int r = 0; r < 16; ++r) {
        float a = 0.f;
        const int tm = post_type(fr[r]);
        if (tm == T_LIQ) a = 1.f;
        else if (tm == T_IFC) a = fminf(fmaxf((float)pr[r], 0.f), 1.f);
        else if (tm == T_WALL && lane < 27) use[r0 + r] = 0;
        if (lane < 27) tc::put_x(t, r0 + r, lane, a);
      }
      if (!net) {
        net = true;
        if (!tc::wait_net(t, phase)) {
          failed = true;
          break;
        }
      }
      float yv = 0.f;
      failed = !tc::forward_tile<MLP_THREADS>(t, phase, yv);
      if (tid < tc::ROWS) {
        const int n0 = cs[tid].n;
        if (!failed && n0 >= 0 && use[tid]) kap[n0] = (R)fminf(fmaxf(yv / mlp::Y_SCALE, -1.f), 1.f);
      }
      __syncthreads();
    }
    if (failed && tid == 0) atomicOr(p.err, ERR_TC_WAIT);
    tc::teardown(t, phase, failed);
  }
}

}  // namespace lbf

namespace lbf {

// Canonical stencils of the current interface cells (training data taken
// from the method's own runs) with the target y = 4 / R_eq of the cell's
// bubble, R_eq = (3 V / 4 pi)^(1/3) from the bubble's current volume: one
// warp per cell, lane q gathers stencil position q.  Skipped: cells with a
// wall in the stencil, a zero normal, no bubble, or the atmosphere.
template <int D, class R>
__global__ void __launch_bounds__(128) k_mlp_harvest(Params p, float *x, float *y, int *cells, int cap, int *count) {
  if constexpr (D == 3) {
    const int lane = threadIdx.x & 31;
    const int warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int nwarps = (gridDim.x * blockDim.x) >> 5;
    const int cnt = *p.icount;
    const int nb = *p.told.count;
    const R *phi = (const R *)p.phi, *nr = (const R *)p.nrm;
    for (int k = warp; k < cnt; k += nwarps) {
      const long long n = p.ilist[k];
      const int b = p.label_old[n];
      if (b < 0 || b >= nb || p.told.atm[b]) continue;
      const double V = p.told.V[b];
      if (!(V > 0.0)) continue;
      const float mx = (float)nr[n], my = (float)nr[p.N + n], mz = (float)nr[2 * p.N + n];
      if (mx == 0.f && my == 0.f && mz == 0.f) continue;
      int ord[3], sgn[3];
      mlp::canonical_order(mx, my, mz, ord, sgn);
      float a = 0.f;
      bool wall = false;
      if (lane < 27) {
        const int src = mlp::canonical_src(lane, ord, sgn);
        const Cell c = make_cell(p, n);
        const long long m = at(p, c, src % 3 - 1, (src / 3) % 3 - 1, src / 9 - 1);
        const int tm = ftype(p.flags[m]);
        if (tm == T_LIQ) a = 1.f;
        else if (tm == T_IFC) a = fminf(fmaxf((float)phi[m], 0.f), 1.f);
        else if (tm == T_WALL) wall = true;
      }
      if (__any_sync(0xffffffffu, wall)) continue;
      int slot = 0;
      if (lane == 0) slot = atomicAdd(count, 1);
      slot = __shfl_sync(0xffffffffu, slot, 0);
      if (slot < cap) {
        if (lane < 27) x[(size_t)slot * 27 + lane] = a;
        if (lane == 0) y[slot] = (float)(mlp::Y_SCALE / cbrt(3.0 * V / (4.0 * 3.141592653589793)));
        if (lane == 0 && cells) cells[slot] = (int)n;
      }
    }
  }
}

}  // namespace lbf

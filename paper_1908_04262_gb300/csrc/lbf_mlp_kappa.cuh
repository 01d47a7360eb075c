// lbf_mlp_kappa.cuh -- in-loop learned curvature kernel (3D): the network of
// lbf_mlp.cuh applied to the interface list after the least-squares
// geometry pass.
#pragma once
#include "lbf_common.cuh"
#include "lbf_mlp.cuh"

namespace lbf {

// In-loop learned curvature (3D): one warp per 16 interface cells of the
// list; every cell's stencil is gathered, turned into the canonical
// orientation of its geometry normal and fed to the network (img: the
// packed BF16 image of the parameters).  The least-squares curvature stays
// where the network is outside its training range (|kappa| outside
// [0.02, 0.55], i.e. radii beyond [1.8, 50] cells) or the stencil touches a
// wall.
constexpr int MLP_WARPS = 8;
template <int D, class R>
__global__ void __launch_bounds__(32 * MLP_WARPS) k_mlp_kappa(Params p, const mlp::NetF *img) {
  if constexpr (D == 3) {
    __shared__ mlp::NetF s;
    __shared__ __nv_bfloat16 xs[MLP_WARPS][16 * 32];
    __shared__ Cell cs[MLP_WARPS][16];
    __shared__ int ord[MLP_WARPS][16][3], sgn[MLP_WARPS][16][3], use[MLP_WARPS][16];
    mlp::copy_netf(s, img);
    __syncthreads();
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5, g = lane >> 2, t = lane & 3;
    const int cnt = *p.icount;
    const int tiles = (cnt + 15) / 16;
    const R *phi = (const R *)p.phi, *nr = (const R *)p.nrm;
    R *kap = (R *)p.kappa;
    for (int tile = blockIdx.x * MLP_WARPS + w; tile < tiles; tile += gridDim.x * MLP_WARPS) {
      if (lane < 16) {
        const int k = tile * 16 + lane;
        int ok = 0;
        Cell c;
        c.n = -1;
        if (k < cnt) {
          c = make_cell(p, p.ilist[k]);
          const float mx = (float)nr[c.n], my = (float)nr[p.N + c.n], mz = (float)nr[2 * p.N + c.n];
          const float ka = fabsf((float)kap[c.n]);
          ok = (mx != 0.f || my != 0.f || mz != 0.f) && ka >= 0.02f && ka <= 0.55f;
          mlp::canonical_order(mx, my, mz, ord[w][lane], sgn[w][lane]);
        }
        cs[w][lane] = c;
        use[w][lane] = ok;
      }
      __syncwarp();
      // lane q gathers stencil position q of the 16 cells: every flag and
      // fill level is loaded before any is used (one round trip, not 16)
      uint8_t fr[16];
      R pr[16];
#pragma unroll
      for (int r = 0; r < 16; ++r) {
        const Cell &c = cs[w][r];
        fr[r] = (uint8_t)T_GAS;
        pr[r] = (R)0;
        if (c.n >= 0 && lane < 27 && use[w][r]) {
          const int src = mlp::canonical_src(lane, ord[w][r], sgn[w][r]);
          const int m = at(p, c, src % 3 - 1, (src / 3) % 3 - 1, src / 9 - 1);
          fr[r] = p.flags[m];  // read as post-conversion types below
          pr[r] = phi[m];
        }
      }
#pragma unroll
      for (int r = 0; r < 16; ++r) {
        float a = 0.f;
        const int tm = post_type(fr[r]);
        if (tm == T_LIQ) a = 1.f;
        else if (tm == T_IFC) a = fminf(fmaxf((float)pr[r], 0.f), 1.f);
        else if (tm == T_WALL) use[w][r] = 0;
        xs[w][r * 32 + lane] = __float2bfloat16_rn(a);
      }
      __syncwarp();
      mlp::Fwd F;
      mlp::forward16(s, xs[w], F);
      if (t == 0) {
        const int n0 = cs[w][g].n, n1 = cs[w][g + 8].n;
        if (n0 >= 0 && use[w][g]) kap[n0] = (R)fminf(fmaxf(F.y0 / mlp::Y_SCALE, -1.f), 1.f);
        if (n1 >= 0 && use[w][g + 8]) kap[n1] = (R)fminf(fmaxf(F.y1 / mlp::Y_SCALE, -1.f), 1.f);
      }
      __syncwarp();
    }
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

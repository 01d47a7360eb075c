// lbf_mlp_kappa.cuh -- in-loop learned curvature kernel (3D): the network of
// lbf_mlp.cuh applied to the interface list after the least-squares
// geometry pass.
#pragma once
#include "lbf_common.cuh"
#include "lbf_mlp.cuh"

namespace lbf {

// In-loop learned curvature (3D): one warp per 16 interface cells of the
// list; every cell's stencil is gathered, turned into the canonical
// orientation of its geometry normal and fed to the network.  The
// least-squares curvature stays where the network is outside its training
// range (|kappa| outside [0.02, 0.55], i.e. radii beyond [1.8, 50] cells) or
// the stencil touches a wall.
template <int D, class R>
__global__ void __launch_bounds__(128) k_mlp_kappa(Params p, const float *theta) {
  if constexpr (D == 3) {
    __shared__ mlp::Smem s;
    __shared__ __nv_bfloat16 xs[4][16 * 32];
    __shared__ long long cn[4][16];
    __shared__ int ord[4][16][3], sgn[4][16][3], use[4][16];
    mlp::load_net(s, theta);
    __syncthreads();
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5, g = lane >> 2, t = lane & 3;
    const int cnt = *p.icount;
    const int tiles = (cnt + 15) / 16;
    const R *phi = (const R *)p.phi, *nr = (const R *)p.nrm;
    R *kap = (R *)p.kappa;
    for (int tile = blockIdx.x * 4 + w; tile < tiles; tile += gridDim.x * 4) {
      if (lane < 16) {
        const int k = tile * 16 + lane;
        long long n = -1;
        int ok = 0;
        if (k < cnt) {
          n = p.ilist[k];
          const float mx = (float)nr[n], my = (float)nr[p.N + n], mz = (float)nr[2 * p.N + n];
          const float ka = fabsf((float)kap[n]);
          ok = (mx != 0.f || my != 0.f || mz != 0.f) && ka >= 0.02f && ka <= 0.55f;
          mlp::canonical_order(mx, my, mz, ord[w][lane], sgn[w][lane]);
        }
        cn[w][lane] = n;
        use[w][lane] = ok;
      }
      __syncwarp();
      for (int e = lane; e < 16 * 32; e += 32) {
        const int r = e >> 5, q = e & 31;
        const long long n = cn[w][r];
        float a = 0.f;
        if (n >= 0 && q < 27) {
          const int src = mlp::canonical_src(q, ord[w][r], sgn[w][r]);
          const Cell c = make_cell(p, n);
          const long long m = at(p, c, src % 3 - 1, (src / 3) % 3 - 1, src / 9 - 1);
          const int tm = ftype(p.flags[m]);
          if (tm == T_LIQ) a = 1.f;
          else if (tm == T_IFC) a = fminf(fmaxf((float)phi[m], 0.f), 1.f);
          else if (tm == T_WALL) use[w][r] = 0;
        }
        xs[w][e] = __float2bfloat16_rn(a);
      }
      __syncwarp();
      mlp::Fwd F;
      mlp::forward16(s, xs[w], F);
      if (t == 0) {
        const long long n0 = cn[w][g], n1 = cn[w][g + 8];
        if (n0 >= 0 && use[w][g]) kap[n0] = (R)(F.y0 / mlp::Y_SCALE);
        if (n1 >= 0 && use[w][g + 8]) kap[n1] = (R)(F.y1 / mlp::Y_SCALE);
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

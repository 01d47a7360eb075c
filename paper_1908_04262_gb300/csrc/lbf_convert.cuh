// lbf_convert.cuh -- cell conversion with excess-mass redistribution
// (Sec. 2.1), lattice initialisation, nucleation (Sec. 3.4), field export and
// the FP64 ledgers.  All kernels run one thread per cell.
//
// Conversion (after the sweep has marked interface cells whose fill level
// left [-eps, 1+eps] and listed them):
//   k_conv_mark       an emptying cell next to a filling cell stays interface;
//                     gas next to a filling cell and liquid next to an
//                     emptying cell become interface (liquid never meets gas)
//   k_conv_compute    excess mass of converting cells, split equally over the
//                     neighbours that are interface afterwards; new interface
//                     cells from gas start at the mean equilibrium of their
//                     interface neighbours; dissolved gas moves between the
//                     liquid and the cell's bubble
//   k_conv_apply      interface cells collect the excess and refresh alpha;
//                     the interface cells of the next step and their
//                     segments are listed
//   k_conv_finalize   the new types replace the marks
// The first two and the last walk the marked cells and the new interface
// cells only; k_conv_apply walks the step's interface cells and the new
// interface cells.
#pragma once
#include "lbf_common.cuh"

namespace lbf {

template <int D, class S>
__device__ __forceinline__ typename ST<S>::R sum_out_f(const Params &p, const Cell &c, long long n, int par,
                                                       typename ST<S>::R *u) {
  using R = typename ST<S>::R;
  const S *f = (const S *)p.f;
  R rho = 0, jx = 0, jy = 0, jz = 0;
#pragma unroll
  for (int i = 0; i < Lat<D>::Q; ++i) {
    const R v = ld(f, slot_out<D>(p, c, n, i, par), fshift<S, D>(p, i));
    rho += v;
    jx += v * (R)Lat<D>::cx(i);
    jy += v * (R)Lat<D>::cy(i);
    jz += v * (R)Lat<D>::cz(i);
  }
  if (u) {
    u[0] = (jx - (R)0.5 * rho * PV(R, ax)) / rho;
    u[1] = (jy - (R)0.5 * rho * PV(R, ay)) / rho;
    u[2] = (jz - (R)0.5 * rho * PV(R, az)) / rho;
  }
  return rho;
}

template <int D, class S>
__device__ __forceinline__ typename ST<S>::R sum_out_g(const Params &p, const Cell &c, long long n, int par) {
  using R = typename ST<S>::R;
  const S *g = (const S *)p.g;
  R s = 0;
#pragma unroll
  for (int i = 0; i < Lat<D>::QA; ++i) s += ld(g, slot_out<D>(p, c, n, i, par), gshift<S, D>(p, i));
  return s;
}

template <int D, class S>
__device__ __forceinline__ void write_equilibrium(const Params &p, const Cell &c, long long n, int par,
                                                  typename ST<S>::R rho, const typename ST<S>::R *u,
                                                  typename ST<S>::R conc) {
  using R = typename ST<S>::R;
  S *f = (S *)p.f;
  S *g = (S *)p.g;
#pragma unroll
  for (int i = 0; i < Lat<D>::Q; ++i)
    st(f, slot_out<D>(p, c, n, i, par), feq<R, D>(i, rho, u[0], u[1], u[2]), fshift<S, D>(p, i));
#pragma unroll
  for (int i = 0; i < Lat<D>::QA; ++i)
    st(g, slot_out<D>(p, c, n, i, par), geq<R, D>(i, conc, u[0], u[1], u[2]), gshift<S, D>(p, i));
}

// all conversion kernels walk the interface list of the step (every cell
// that can fill or empty) and the list of cells they turn into interface;
// persistent grids, one thread per listed cell

// passes over a short list: entry base + k sits on thread k / gridDim.x of
// block k % gridDim.x, so that a few hundred entries occupy one thread in as
// many blocks (and SMs) instead of whole warps of a few
__device__ __forceinline__ int spread_index(int base) {
  return base + (int)threadIdx.x * (int)gridDim.x + (int)blockIdx.x;
}

// set a conversion mark on a neighbour's flag byte; true for the first writer
__device__ __forceinline__ bool mark_byte(uint8_t *flags, long long m, int mk, int par) {
  const uintptr_t a = (uintptr_t)(flags + m);
  unsigned *word = (unsigned *)(a & ~(uintptr_t)3);
  const int sh = (int)(a & 3) * 8;
  const unsigned old = atomicOr(word, (unsigned)mark_bits(mk, par) << sh);
  return ((old >> sh) & (7u << 2)) == 0;
}

// An emptying cell next to a filling cell stays interface (filling wins);
// gas next to a filling cell and liquid next to a (still) emptying cell
// become interface, so that liquid never meets gas.  The first marker lists
// the new interface cell.  Filling marks are final when this runs, so an
// emptying cell decides its own fate without waiting for other threads.
// The neighbours' flags are loaded up front, the claims issued together and
// the new interface cells of a warp appended with one atomic.
template <int D>
__global__ void __launch_bounds__(128) k_conv_mark(Params p) {
  constexpr int Q = Lat<D>::Q;
  const int lane = threadIdx.x & 31;
  const int cnt = *p.mcount;
  // the next interface list is collected afresh (its buffer held the last
  // step's list until the label sync of this step read it)
  if (blockIdx.x == 0 && threadIdx.x == 0) *p.inext_count = 0;
  for (int base = 0; base < cnt; base += gridDim.x * blockDim.x) {
    const int k = spread_index(base);
    int mk = MK_NONE;
    int n = 0;
    if (k < cnt) {
      n = p.mlist[k];
      mk = fmark(p.flags[n]);
    }
    unsigned claimed = 0;  // bit i: neighbour x + e_i turned interface by this cell
    Cell c;
    if (mk == MK_FILL || mk == MK_EMPTY) {
      c = make_cell(p, n);
      uint8_t fn[Q];
#pragma unroll
      for (int i = 1; i < Q; ++i) fn[i] = p.flags[nb<D>(p, c, i)];
      bool stay = false;
      if (mk == MK_EMPTY) {
#pragma unroll
        for (int i = 1; i < Q; ++i) stay |= fmark(fn[i]) == MK_FILL;
      }
      if (stay) {
        // clear the emptying mark (mark bits only; other threads read the
        // type bits of this byte)
        const uintptr_t a = (uintptr_t)(p.flags + n);
        atomicAnd((unsigned *)(a & ~(uintptr_t)3), ~((unsigned)mark_bits(7, 1) << ((int)(a & 3) * 8)));
      } else {
        const int want = mk == MK_FILL ? T_GAS : T_LIQ;
        const int put = mk == MK_FILL ? MK_GI : MK_LI;
#pragma unroll
        for (int i = 1; i < Q; ++i)
          if (ftype(fn[i]) == want && mark_byte(p.flags, nb<D>(p, c, i), put, p.par)) claimed |= 1u << i;
        if (p.gas_dirty) {
          if (mk == MK_EMPTY) {  // this cell turns gas
            atomicOr(p.gas_dirty, 1);
            if (p.tdirty) p.tdirty[tile_of<D>(p, c)] = 1;
          }
          if (put == MK_GI && claimed) atomicOr(p.gas_dirty, 2);  // gas cells turn interface
        }
      }
    }
    // warp-aggregated append of the claimed neighbours
    const int mine = __popc(claimed);
    int incl = mine;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const int v = __shfl_up_sync(0xffffffffu, incl, o);
      if (lane >= o) incl += v;
    }
    const int total = __shfl_sync(0xffffffffu, incl, 31);
    if (total == 0) continue;
    int at = 0;
    if (lane == 31) at = atomicAdd(p.ncount, total);
    at = __shfl_sync(0xffffffffu, at, 31) + incl - mine;
    while (claimed) {
      const int i = __ffs(claimed) - 1;
      claimed &= claimed - 1;
      p.nlist[at++] = nb<D>(p, c, i);
    }
  }
}

// cell k of the marked list followed by the new-interface list
__device__ __forceinline__ long long list_cell(const Params &p, int k, int nm) {
  return k < nm ? p.mlist[k] : p.nlist[k - nm];
}

// An added gas cell (an emptied interface cell) keeps the bubble structure
// of the last labelling when it carries a bubble label L (the smallest of
// its gas neighbours' as an interface cell), every gas neighbour after the
// conversion carries L (it joins no other bubble) and one of them is a gas
// cell of the last step that stays gas (it is joined to its bubble).  Below
// the bubble's root it becomes the new root (the patch takes the minimum);
// the labels, ranks of the roots, stay as they are while it lies above the
// root of bubble L - 1.
template <int D>
__device__ __forceinline__ bool addition_keeps_bubble(const Params &p, const Cell &c, int n) {
  const int L = p.label_old[n];
  // the neighbours' flags and labels in one round of loads
  uint8_t fn[Lat<D>::Q];
  int ln[Lat<D>::Q];
#pragma unroll
  for (int i = 1; i < Lat<D>::Q; ++i) {
    const int m = nb<D>(p, c, i);
    fn[i] = p.flags[m];
    ln[i] = p.label_old[m];
  }
  if (L < 0 || (n < p.told.root[L] && L > 0 && n < p.told.root[L - 1])) return false;
  if (n < p.told.root[L]) p.rmv[1] = 1;
  bool anchored = false;
#pragma unroll
  for (int i = 1; i < Lat<D>::Q; ++i) {
    if (post_type(fn[i]) != T_GAS) continue;
    if (ln[i] != L) return false;
    if (ftype(fn[i]) == T_GAS) anchored = true;  // gas before, and no mark turns it interface
  }
  return anchored;
}

// A gas cell turning interface (a filling neighbour claimed it) keeps the
// bubble structure of the last labelling when it is not in the top layer
// (the headspace flag), its gas neighbours after the
// conversion stay connected to one another inside its own 3^d neighbourhood
// (over D2Q9 / D3Q19 links between neighbourhood cells), and it shares a
// gas neighbour with every linked cell that turns interface with it.  Then
// any path of gas cells through a run of such cells can go round them
// (from one shared neighbour to the next), so no bubble splits or vanishes.
template <int D>
__device__ __forceinline__ bool cube_link(int a, int b) {
  const int ddx = abs(a % 3 - b % 3), ddy = abs((a / 3) % 3 - (b / 3) % 3), ddz = D == 3 ? abs(a / 9 - b / 9) : 0;
  return a != b && ddx <= 1 && ddy <= 1 && ddz <= 1 && (D == 2 || ddx + ddy + ddz <= 2);
}
template <int D>
__device__ __forceinline__ bool removal_keeps_bubble(const Params &p, const Cell &c, int n) {
  constexpr int NS = D == 3 ? 27 : 9, CTR = D == 3 ? 13 : 4;
  const int L = p.label_old[n];
  if (L < 0) return false;
  if (n == p.told.root[L]) {
    // the root moves up: k_root_scan finds the new one (one bubble per step)
    const int prev = atomicCAS(p.rmv, -1, L);
    if (prev != -1 && prev != L) return false;
  }
  if (p.atmosphere && (D == 2 ? c.y : c.z) == p.top_layer) return false;
  unsigned gas = 0, link = 0, gone = 0;  // bit k: stencil cell k is gas after the conversion /
                                         // a gas neighbour of the centre / linked and turning interface
#pragma unroll
  for (int k = 0; k < NS; ++k) {
    if (k == CTR) continue;
    const int dx = k % 3 - 1, dy = (k / 3) % 3 - 1, dz = D == 3 ? k / 9 - 1 : 0;
    const uint8_t f = p.flags[at(p, c, dx, dy, dz)];
    const bool centre_link = cube_link<D>(k, CTR);
    if (centre_link && ftype(f) == T_GAS && fmark(f) == MK_GI) gone |= 1u << k;
    if (post_type(f) == T_GAS) {
      gas |= 1u << k;
      if (centre_link) link |= 1u << k;
    }
  }
  if (!link) return false;  // it was a bubble of its own
  // a shared gas neighbour with every linked cell turning interface
  for (unsigned g = gone; g; g &= g - 1) {
    const int b = __ffs(g) - 1;
    bool shared = false;
    for (unsigned q = link; q; q &= q - 1) shared |= cube_link<D>(__ffs(q) - 1, b);
    if (!shared) return false;
  }
  // flood fill over the gas cells of the neighbourhood from one linked cell
  unsigned reach = link & (~link + 1u), grown = 0;
  while (reach != grown) {
    grown = reach;
    for (unsigned r = reach; r; r &= r - 1) {
      const int a = __ffs(r) - 1;
      for (unsigned q = gas & ~reach; q; q &= q - 1) {
        const int b = __ffs(q) - 1;
        if (cube_link<D>(a, b)) reach |= 1u << b;
      }
    }
  }
  return (link & ~reach) == 0;
}

// After the labelling check, when a bubble's root cell turns interface: its
// new root is the smallest cell after the old one that is gas after the
// conversion and carries the bubble's label (a gas cell that stays, or an
// emptied interface cell of the bubble).  One block scans forward 8 cells
// per thread at a time, at most four times; the labels (ranks of the roots)
// stay valid when the new root lies below the next bubble's and no root was
// lowered in the same step, otherwise (or when the scan gives up) the step
// takes the full labelling.
static __global__ void __launch_bounds__(1024) k_root_scan(Params p) {
  __shared__ int L, found;
  if (threadIdx.x == 0) {
    L = p.rmv[0];
    found = 0x7fffffff;
  }
  __syncthreads();
  if (L < 0) {
    if (threadIdx.x == 0) p.rmv[1] = 0;
    return;
  }
  const long long r0 = (long long)p.told.root[L] + 1;
  for (int it = 0; it < 4; ++it) {
    const long long base = r0 + (long long)it * (8 * 1024) + 8 * (long long)threadIdx.x;
#pragma unroll
    for (int j = 0; j < 8; ++j) {
      const long long n = base + j;
      if (n < p.N && post_type(p.flags[n]) == T_GAS && p.label_old[n] == L) atomicMin(&found, (int)n);
    }
    __syncthreads();
    const bool done = found != 0x7fffffff;
    __syncthreads();
    if (done) break;
  }
  if (threadIdx.x == 0) {
    const int nb = *p.told.count;
    if (found == 0x7fffffff || p.rmv[1] || (L + 1 < nb && found > p.told.root[L + 1]))
      atomicOr(p.lab_slow, 1);
    else
      p.tnew.root[L] = found;
    p.rmv[0] = -1;
    p.rmv[1] = 0;
  }
}

// after the marking (every mark final): the emptied cells are on the marked
// list, the gas cells turned interface on the new-interface list; any of
// them that could join, split, empty or re-root a bubble vetoes the patched
// labelling of this step (lab_slow)
template <int D>
__global__ void __launch_bounds__(128) k_label_check(Params p) {
  const int nm = *p.mcount, total = nm + *p.ncount;
  for (int base = 0; base < total; base += gridDim.x * blockDim.x) {
    const int k = spread_index(base);
    if (k >= total) continue;
    const int n = (int)list_cell(p, k, nm);
    const uint8_t f = p.flags[n];
    bool ok = true;
    if (k < nm) {
      if (post_type(f) == T_GAS) ok = addition_keeps_bubble<D>(p, make_cell(p, n), n);
    } else if (ftype(f) == T_GAS) {  // (liquid turning interface changes no bubble)
      ok = removal_keeps_bubble<D>(p, make_cell(p, n), n);
    }
    if (!ok) atomicOr(p.lab_slow, 1);
  }
}

// par: parity of the populations after the sweep
template <int D, class S>
__global__ void __launch_bounds__(128) k_conv_compute(Params p, int par) {
  using R = typename ST<S>::R;
  __shared__ double wbuf[128];
  const int ni = *p.mcount, total = ni + *p.ncount;
  for (int base = 0; base < total; base += gridDim.x * blockDim.x) {
    const int k = spread_index(base);
    double dmv = 0.0;
    int lab = -1;
    if (k < total) {
      const long long n = list_cell(p, k, ni);
      const uint8_t fl = p.flags[n];
      const int mk = fmark(fl);
      if (mk != MK_NONE) {
        const Cell c = make_cell(p, n);
        R *M = (R *)p.M;
        if (mk == MK_FILL || mk == MK_EMPTY) {
          const R rho = sum_out_f<D, S>(p, c, n, par, nullptr);
          const R excess = mk == MK_FILL ? M[n] - rho : M[n];
          int cnt = 0;
#pragma unroll
          for (int i = 1; i < Lat<D>::Q; ++i) cnt += post_type(p.flags[nb<D>(p, c, i)]) == T_IFC;
          R *ex = (R *)p.ex;
          if (cnt > 0)
            ex[n] = excess / (R)cnt;
          else
            atomicAdd(p.led + 1, (double)excess);
          if (mk == MK_EMPTY) {
            const double cg = (double)sum_out_g<D, S>(p, c, n, par);
            lab = p.label_old[n];
            if (lab >= 0)
              dmv = cg;
            else
              atomicAdd(p.led + 5, cg);
          }
        } else if (mk == MK_GI) {
          // the mean density, velocity and dissolved gas of the interface
          // neighbours that do not empty, as their sweeps left them
          R rs = 0, us[3] = {0, 0, 0}, cs = 0;
          int cnt = 0;
          const R *mo = (const R *)p.mom;
          uint8_t fn[Lat<D>::Q];
          int mn[Lat<D>::Q];
#pragma unroll
          for (int i = 1; i < Lat<D>::Q; ++i) {
            mn[i] = nb<D>(p, c, i);
            fn[i] = p.flags[mn[i]];
          }
#pragma unroll
          for (int i = 1; i < Lat<D>::Q; ++i) {
            const uint8_t fm = fn[i];
            if (ftype(fm) == T_IFC && (fmark(fm) == MK_NONE || fmark(fm) == MK_FILL)) {
              const int m = mn[i];
              rs += mo[m];
              us[0] += mo[p.N + m];
              us[1] += mo[2 * p.N + m];
              us[2] += mo[3 * p.N + m];
              cs += mo[4 * p.N + m];
              ++cnt;
            }
          }
          const R inv = (R)cnt;
          rs /= inv;
          us[0] /= inv;
          us[1] /= inv;
          us[2] /= inv;
          cs /= inv;
          write_equilibrium<D, S>(p, c, n, par, rs, us, cs);
          M[n] = 0;
          lab = p.label_old[n];
          if (lab >= 0)
            dmv = -(double)cs;
          else
            atomicAdd(p.led + 5, -(double)cs);
        } else if (mk == MK_LI) {
          M[n] = sum_out_f<D, S>(p, c, n, par, nullptr);
        }
      }
    }
    if (__any_sync(0xffffffffu, lab >= 0)) agg_add(p.told.dm, lab, dmv, wbuf + (threadIdx.x & ~31));
  }
}

// one cell of k_conv_apply: an interface cell after the conversion collects
// the excess of its converting neighbours and refreshes its fill level
// (new interface cells always do); filled and emptied cells take alpha 1 / 0.
// True when the cell is interface after the conversion.
template <int D, class S>
__device__ __forceinline__ bool apply_cell(const Params &p, const Cell &c, int n, uint8_t fl, int par) {
  using R = typename ST<S>::R;
  const int pt = post_type(fl);
  const int mk = fmark(fl);
  if (pt == T_IFC) {
    const R *ex = (const R *)p.ex;
    R *M = (R *)p.M;
    R recv = 0;
    bool has = false;
    // the neighbours' flags and excess shares in one round of loads (the
    // share of a neighbour that does not convert is read and unused)
    uint8_t fn[Lat<D>::Q];
    R en[Lat<D>::Q];
#pragma unroll
    for (int i = 1; i < Lat<D>::Q; ++i) {
      const int m = nb<D>(p, c, i);
      fn[i] = p.flags[m];
      en[i] = ex[m];
    }
#pragma unroll
    for (int i = 1; i < Lat<D>::Q; ++i) {
      const int fm = fmark(fn[i]);
      if (fm == MK_FILL || fm == MK_EMPTY) {
        recv += en[i];
        has = true;
      }
    }
    if (has || mk == MK_GI || mk == MK_LI) {
      const R Mv = M[n] + recv;
      M[n] = Mv;
      ((R *)p.phi)[n] = Mv / sum_out_f<D, S>(p, c, n, par, nullptr);
    }
  } else if (mk == MK_FILL) {
    ((R *)p.phi)[n] = 1;
    ((R *)p.M)[n] = 0;
  } else if (mk == MK_EMPTY) {
    ((R *)p.phi)[n] = 0;
    ((R *)p.M)[n] = 0;
  }
  return pt == T_IFC;
}

// list a segment of the next step once (the interface sweep clears the flag)
__device__ __forceinline__ void claim_segment(const Params &p, bool take, int seg) {
  bool first = false;
  if (take) first = atomicExch(p.segflag + seg, 1) == 0;
  list_append(p.segnext, p.segnext_count, first, seg);
}

// the excess collection over the step's interface cells and the new
// interface cells (one thread each); lists the next step's interface cells
// and their segments.  Marks stay in the flags until k_conv_finalize:
// neighbours' marks are read here.
template <int D, class S>
__global__ void __launch_bounds__(128) k_conv_apply(Params p, int par) {
  const int lane = threadIdx.x & 31;
  const int ni = *p.icount, total = ni + *p.ncount;
  for (int base = blockIdx.x * blockDim.x; base < total; base += gridDim.x * blockDim.x) {
    const int k = base + threadIdx.x;
    bool take = false;
    int n = 0;
    if (k < total) {
      n = k < ni ? p.ilist[k] : p.nlist[k - ni];
      take = apply_cell<D, S>(p, make_cell(p, n), n, p.flags[n], par);
    }
    list_append(p.inext, p.inext_count, take, n);
    // one claim per distinct segment of the warp
    const int seg = take ? seg_of(p, n) : -1;
    const unsigned peers = __match_any_sync(0xffffffffu, seg);
    claim_segment(p, take && lane == __ffs(peers) - 1, seg);
  }
}

// the conversion's new types replace the marks (every marked cell is on the
// marked list or on the new-interface list); a separate pass because
// k_conv_apply reads the marks of neighbouring cells
template <int D>
__global__ void k_conv_finalize(Params p) {
  const int nm = *p.mcount, total = nm + *p.ncount;
  for (int base = 0; base < total; base += gridDim.x * blockDim.x) {
    const int k = spread_index(base);
    if (k >= total) continue;
    const int n = (int)list_cell(p, k, nm);
    const uint8_t fl = p.flags[n];
    if (fmark(fl)) p.flags[n] = (uint8_t)(post_type(fl) | (fl & NEARWALL));
  }
}

// list every interface cell and its segment (initialisation paths; blocks
// are whole multiples of 32 cells along x, so a warp is one segment)
static __global__ void k_build_ilist(Params p) {
  Cell c;
  const bool inr = grid_cell(p, c);
  const bool take = inr && ftype(p.flags[c.n]) == T_IFC;
  list_append(p.ilist, p.icount, take, (int)c.n);
  const bool any = __any_sync(0xffffffffu, take);
  list_append(p.seglist, p.segcount, any && (threadIdx.x & 31) == 0, seg_of(p, c.n));
}

// ---------------------------------------------------------------------------
// initialisation

template <int D> __device__ __forceinline__ bool is_wall_cell(const Params &p, const Cell &c) {
  const int w = p.walls;
  if ((w & 1) && c.x == 0) return true;
  if ((w & 2) && c.x == p.nx - 1) return true;
  if ((w & 4) && c.y == 0) return true;
  if ((w & 8) && c.y == p.ny - 1) return true;
  if (D == 3 && (w & 16) && c.z == 0) return true;
  if (D == 3 && (w & 32) && c.z == p.nz - 1) return true;
  return false;
}

// liquid below fill_height at rest, walls, gas above
template <int D, class S>
__global__ void k_init_fill(Params p, int par, double fill_height) {
  using R = typename ST<S>::R;
  Cell c;
  if (!grid_cell(p, c)) return;
  const long long n = c.n;
  R *M = (R *)p.M, *phi = (R *)p.phi;
  if (is_wall_cell<D>(p, c)) {
    p.flags[n] = T_WALL;
    phi[n] = 0;
    M[n] = 0;
    return;
  }
  const double h = D == 2 ? c.y : c.z;
  double a = fill_height - (h - 0.5);
  a = a < 0.0 ? 0.0 : (a > 1.0 ? 1.0 : a);
  const int t = a >= 1.0 ? T_LIQ : (a <= 0.0 ? T_GAS : T_IFC);
  p.flags[n] = (uint8_t)t;
  phi[n] = (R)a;
  M[n] = 0;
  if (t != T_GAS) {
    const R u[3] = {0, 0, 0};
    write_equilibrium<D, S>(p, c, n, par, PV(R, rho0), u, PV(R, c0));
    if (t == T_IFC) M[n] = (R)a * PV(R, rho0);
  }
}

// state from per-cell arrays (already on the device)
template <int D, class S>
__global__ void k_init_cells(Params p, int par, const uint8_t *type, const double *rho, const double *u,
                             const double *alpha, const double *conc) {
  using R = typename ST<S>::R;
  Cell c;
  if (!grid_cell(p, c)) return;
  const long long n = c.n;
  const int t = type[n] & 3;
  R *M = (R *)p.M, *phi = (R *)p.phi;
  p.flags[n] = (uint8_t)t;
  M[n] = 0;
  phi[n] = t == T_LIQ ? (R)1 : (t == T_IFC ? (R)alpha[n] : (R)0);
  if (t == T_LIQ || t == T_IFC) {
    const R uu[3] = {(R)u[3 * n], (R)u[3 * n + 1], (R)u[3 * n + 2]};
    write_equilibrium<D, S>(p, c, n, par, (R)rho[n], uu, (R)conc[n]);
    if (t == T_IFC) M[n] = (R)alpha[n] * (R)rho[n];
  }
}

// liquid next to gas becomes interface with alpha = 1 (two passes)
template <int D>
__global__ void k_separate_mark(Params p) {
  Cell c;
  if (!grid_cell(p, c)) return;
  const long long n = c.n;
  const uint8_t fl = p.flags[n];
  if (ftype(fl) != T_LIQ) return;
#pragma unroll
  for (int i = 1; i < Lat<D>::Q; ++i)
    if (ftype(p.flags[nb<D>(p, c, i)]) == T_GAS) {
      p.flags[n] = (uint8_t)(fl | (MK_LI << 2));
      return;
    }
}

template <int D, class S>
__global__ void k_separate_apply(Params p, int par) {
  using R = typename ST<S>::R;
  Cell c;
  if (!grid_cell(p, c)) return;
  const long long n = c.n;
  const uint8_t fl = p.flags[n];
  if (fmark(fl) != MK_LI) return;
  p.flags[n] = (uint8_t)(T_IFC | (fl & NEARWALL));
  ((R *)p.phi)[n] = 1;
  ((R *)p.M)[n] = sum_out_f<D, S>(p, c, n, par, nullptr);
}

template <int D>
__global__ void k_nearwall(Params p) {
  Cell c;
  if (!grid_cell(p, c)) return;
  const long long n = c.n;
  // bit i of the wall mask: the source x - e_i of direction i is a wall
  unsigned wm = 0;
#pragma unroll
  for (int i = 1; i < Lat<D>::Q; ++i) wm |= (ftype(p.flags[src<D>(p, c, i)]) == T_WALL ? 1u : 0u) << i;
  const uint8_t fl = p.flags[n];
  p.flags[n] = (uint8_t)(wm ? (fl | NEARWALL) : (fl & ~NEARWALL));
  p.wmask[n] = wm;
}

// Sec. 3.4: carve one nucleus (sphere or disk of radius R at (cx,cy,cz))
// into liquid cells of its bounding box [x0,x0+bx) x [y0,..) x [z0,..)
template <int D, class S>
__global__ void k_nucleate(Params p, int par, double cx, double cy, double cz, double R0, int x0, int y0,
                           int z0, int bx, int by, int bz) {
  using R = typename ST<S>::R;
  const long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (t >= (long long)bx * by * bz) return;
  const int X = x0 + (int)(t % bx);
  const int Y = y0 + (int)((t / bx) % by);
  const int Z = z0 + (int)(t / ((long long)bx * by));
  const long long n = at_far(p, X, Y, Z);
  if (ftype(p.flags[n]) != T_LIQ) return;
  const int total = D == 3 ? 64 : 16;
  int nout = 0;
  for (int k = 0; k < (D == 3 ? 4 : 1); ++k)
    for (int b = 0; b < 4; ++b)
      for (int a = 0; a < 4; ++a) {
        const double px = X + (a + 0.5) / 4.0 - 0.5 - cx;
        const double py = Y + (b + 0.5) / 4.0 - 0.5 - cy;
        const double pz = D == 3 ? Z + (k + 0.5) / 4.0 - 0.5 - cz : 0.0;
        nout += px * px + py * py + pz * pz >= R0 * R0;
      }
  if (nout == total) return;
  const Cell c = make_cell(p, n);
  const double rho = (double)sum_out_f<D, S>(p, c, n, par, nullptr);
  R *M = (R *)p.M, *phi = (R *)p.phi;
  const uint8_t keep = p.flags[n] & NEARWALL;
  if (nout == 0) {
    p.flags[n] = (uint8_t)(T_GAS | keep);
    phi[n] = 0;
    M[n] = 0;
    atomicAdd(p.led + 2, rho);
    atomicAdd(p.led + 5, (double)sum_out_g<D, S>(p, c, n, par));
  } else {
    const double al = (double)nout / total;
    p.flags[n] = (uint8_t)(T_IFC | keep);
    phi[n] = (R)al;
    M[n] = (R)(al * rho);
    atomicAdd(p.led + 2, rho - al * rho);
  }
}

// ---------------------------------------------------------------------------
// export and ledgers

template <int D, class S>
__global__ void k_fields(Params p, int par, int which, void *out, int dtype) {
  using R = typename ST<S>::R;
  Cell c;
  if (!grid_cell(p, c)) return;
  const long long n = c.n;
  const int t = ftype(p.flags[n]);
  const bool fluid = t == T_LIQ || t == T_IFC;
  double v[3] = {0.0, 0.0, 0.0};
  int width = 1;
  switch (which) {
    case FLD_RHO: if (fluid) v[0] = (double)sum_out_f<D, S>(p, c, n, par, nullptr); break;
    case FLD_U:
      width = 3;
      if (fluid) {
        R u[3];
        sum_out_f<D, S>(p, c, n, par, u);
        v[0] = u[0]; v[1] = u[1]; v[2] = u[2];
      }
      break;
    case FLD_ALPHA: v[0] = (double)((const R *)p.phi)[n]; break;
    case FLD_MASS:
      if (t == T_IFC) v[0] = (double)((const R *)p.M)[n];
      else if (t == T_LIQ) v[0] = (double)sum_out_f<D, S>(p, c, n, par, nullptr);
      break;
    case FLD_CONC: if (fluid) v[0] = (double)sum_out_g<D, S>(p, c, n, par); break;
    case FLD_KAPPA: if (t == T_IFC) v[0] = (double)((const R *)p.kappa)[n]; break;
    case FLD_PI: if (t == T_IFC) v[0] = (double)((const R *)p.Pi)[n]; break;
    case FLD_DSTAR: if (t == T_IFC) v[0] = (double)((const R *)p.dst)[n]; break;
    case FLD_NORMAL:
      width = 3;
      if (t == T_IFC) {
        const R *nr = (const R *)p.nrm;
        v[0] = nr[n]; v[1] = nr[p.N + n]; v[2] = nr[2 * p.N + n];
      }
      break;
    case FLD_FLAGS: ((int *)out)[n] = t; return;
    case FLD_LABEL: ((int *)out)[n] = (t == T_GAS || t == T_IFC) ? p.label_new[n] : -1; return;
  }
  for (int k = 0; k < width; ++k) {
    if (dtype == 1)
      ((double *)out)[width * n + k] = v[k];
    else
      ((float *)out)[width * n + k] = (float)v[k];
  }
}

// [0] liquid mass, [1] dissolved gas, [2] non-finite populations, plus cell
// counts of the four types
template <int D, class S>
__global__ void __launch_bounds__(128) k_ledger(Params p, int par, double *acc, unsigned long long *counts) {
  using R = typename ST<S>::R;
  __shared__ double sm[3][128];
  __shared__ unsigned long long sc[4];
  Cell c;
  const bool inr = grid_cell(p, c);
  const long long n = c.n;
  if (threadIdx.x < 4) sc[threadIdx.x] = 0;
  double mass = 0.0, gas = 0.0, bad = 0.0;
  __syncthreads();
  if (inr) {
    const int t = ftype(p.flags[n]);
    atomicAdd(&sc[t], 1ull);
    if (t == T_LIQ || t == T_IFC) {
      const S *f = (const S *)p.f;
      double rho = 0.0;
      for (int i = 0; i < Lat<D>::Q; ++i) {
        const double v = (double)ld(f, slot_out<D>(p, c, n, i, par), fshift<S, D>(p, i));
        rho += v;
        if (!isfinite(v)) bad += 1.0;
      }
      mass = t == T_LIQ ? rho : (double)((const R *)p.M)[n];
      gas = (double)sum_out_g<D, S>(p, c, n, par);
    }
  }
  sm[0][threadIdx.x] = mass;
  sm[1][threadIdx.x] = gas;
  sm[2][threadIdx.x] = bad;
  __syncthreads();
  for (int s = blockDim.x >> 1; s > 0; s >>= 1) {
    if (threadIdx.x < s)
      for (int k = 0; k < 3; ++k) sm[k][threadIdx.x] += sm[k][threadIdx.x + s];
    __syncthreads();
  }
  if (threadIdx.x == 0)
    for (int k = 0; k < 3; ++k) atomicAdd(acc + k, sm[k][0]);
  if (threadIdx.x < 4 && sc[threadIdx.x]) atomicAdd(counts + threadIdx.x, sc[threadIdx.x]);
}

}  // namespace lbf

// lbf_label.cuh -- per-step bubble labelling and bubble table update
// (Sec. 3.5: every iteration tags the gas cells of each bubble with a unique
// id and carries volume and gas content; merges and splits share the gas in
// proportion to volume; Sec. 2.2 Eq. idealgas gives the pressure).
//
// Gas cells connected over lattice links (D2Q9: 8 neighbours, D3Q19: 18)
// form a bubble.  A lock-free union-find links every root under the smaller
// index, so the root of a component is its smallest linear cell index; the
// bubbles are numbered in the order of those roots.  Interface cells join the
// bubble of their gas neighbour with the smallest number.  Old and new
// bubbles that share gas or interface cells form groups; within a group the
// old gas content is split over the new bubbles in proportion to volume.
#pragma once
#include "lbf_common.cuh"

namespace lbf {

constexpr unsigned long long HASH_EMPTY = ~0ull;
constexpr int UF_ITERS = 1 << 22;

// find with path halving: a node's parent is replaced by its grandparent
// on the way up.  Parents only move towards smaller indices, so the writes
// keep every node's parent an ancestor; a concurrent link that such a write
// overwrites is retried by the union that made it (its atomicMin returns a
// value other than the expected root).
__device__ __forceinline__ int uf_find(int *par, int a) {
  for (int it = 0; it < UF_ITERS; ++it) {
    const int b = __ldcg(par + a);
    if (b == a) return a;
    const int c = __ldcg(par + b);
    if (c == b) return b;
    __stcg(par + a, c);
    a = c;
  }
  return a;
}

// the same on arrays that may live in shared or global memory
__device__ __forceinline__ int uf_find_any(const int *par, int a) {
  for (int it = 0; it < UF_ITERS; ++it) {
    const int b = *(const volatile int *)(par + a);
    if (b == a) return a;
    a = b;
  }
  return a;
}
__device__ __forceinline__ bool uf_union_any(int *par, int a, int b) {
  for (int it = 0; it < UF_ITERS; ++it) {
    a = uf_find_any(par, a);
    b = uf_find_any(par, b);
    if (a == b) return true;
    if (a > b) {
      const int t = a;
      a = b;
      b = t;
    }
    const int old = atomicMin(par + b, a);
    if (old == b) return true;
    b = old;
  }
  return false;
}

// returns false when the iteration cap was reached (kept out of line: it is
// called from unrolled direction loops)
static __device__ __noinline__ bool uf_union(int *par, int a, int b) {
  for (int it = 0; it < UF_ITERS; ++it) {
    a = uf_find(par, a);
    b = uf_find(par, b);
    if (a == b) return true;
    if (a > b) {
      const int t = a;
      a = b;
      b = t;
    }
    const int old = atomicMin(par + b, a);
    if (old == b) return true;
    b = old;
  }
  return false;
}

static __global__ void k_label_prep(Params p) {
  const int cap = p.cap;
  for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < cap; k += gridDim.x * blockDim.x) {
    p.tnew.V[k] = 0.0;
    p.tnew.atm[k] = 0;
    p.tnew.ng[k] = 0;
  }
  if (blockIdx.x == 0 && threadIdx.x == 0) *p.nroots = 0;
}

// union-find tiles: the local pass joins gas cells of one tile in shared
// memory, the merge pass joins tiles across their faces in global memory
constexpr int TILE_THREADS = 1024;  // one thread per cell of a tile, one x-row per warp

// parents only ever point to smaller indices, so a chain has at most TN
// links; the caps below are never reached by a consistent forest
__device__ __forceinline__ int sm_find(volatile int *lp, int a) {
  for (int it = 0; it < 4096; ++it) {
    const int b = lp[a];
    if (b == a) break;
    a = b;
  }
  return a;
}

static __device__ __noinline__ bool sm_union(int *lp, int a, int b) {
  for (int it = 0; it < 65536; ++it) {
    a = sm_find(lp, a);
    b = sm_find(lp, b);
    if (a == b) return true;
    if (a > b) {
      const int t = a;
      a = b;
      b = t;
    }
    const int old = atomicMin(lp + b, a);
    if (old == b) return true;
    b = old;
  }
  return false;
}

template <int D> struct TileGrid {
  int ntx, nty, ntz;
  __device__ __forceinline__ TileGrid(const Params &p)
      : ntx((p.nx + Tile<D>::TX - 1) / Tile<D>::TX),
        nty((p.ny + Tile<D>::TY - 1) / Tile<D>::TY),
        ntz((p.nz + Tile<D>::TZ - 1) / Tile<D>::TZ) {}
  __device__ __forceinline__ int id(int tx, int ty, int tz) const {
    tx = (tx + ntx) % ntx;
    ty = (ty + nty) % nty;
    tz = (tz + ntz) % ntz;
    return tx + ntx * (ty + nty * tz);
  }
};

// the row-to-row links of the tile-local pass: one of each opposite pair of
// the lattice vectors that leave the x-row (x-links join runs directly);
// (dx, dy, dz)
template <int D> struct RowLinks;
template <> struct RowLinks<3> {
  static constexpr int n = 8;
  __device__ static constexpr int dx(int k) { return k == 2 ? -1 : k == 3 ? 1 : k == 4 ? -1 : k == 5 ? 1 : 0; }
  __device__ static constexpr int dy(int k) { return k == 0 ? -1 : k == 2 || k == 3 ? -1 : k == 6 ? -1 : k == 7 ? 1 : 0; }
  __device__ static constexpr int dz(int k) { return k == 1 || k == 4 || k == 5 || k == 6 || k == 7 ? -1 : 0; }
};
template <> struct RowLinks<2> {
  static constexpr int n = 3;
  __device__ static constexpr int dx(int k) { return k == 1 ? -1 : k == 2 ? 1 : 0; }
  __device__ static constexpr int dy(int) { return -1; }
  __device__ static constexpr int dz(int) { return 0; }
};

// One block per tile: status, local union-find in shared memory, parents
// and local component sizes.  A tile is 32 rows of 32 cells along x; a
// warp's ballot gives each row's gas mask, every gas cell starts out
// pointing at the first cell of its x-run, and two rows are joined once per
// overlapping segment of their runs (at the segment's first cell), so the
// number of unions grows with the number of runs rather than of cells.
// Roots are the smallest local index of each component, which orders cells
// like their global index.
template <int D>
__global__ void __launch_bounds__(TILE_THREADS) k_uf_local(Params p) {
  constexpr int TX = Tile<D>::TX, TY = Tile<D>::TY, TZ = Tile<D>::TZ, TN = TX * TY * TZ, NR = TY * TZ;
  static_assert(TX == 32 && NR == 32, "a tile is 32 rows of 32 cells");
  if (label_fast(p)) return;
  const int mode = label_mode(p);
  if (mode == LABEL_SKIP) return;
  __shared__ int lp[TN];
  __shared__ int lsz[TN];
  __shared__ unsigned rowm[NR];
  __shared__ int sg, sc, nroot, rfirst;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const long long nx = p.nx, nxy = (long long)p.nx * p.ny;
  const TileGrid<D> tgd(p);
  const int ntiles = tgd.ntx * tgd.nty * tgd.ntz;
  // blocks walk the tiles (one block per tile when the grid has as many)
  for (int tile = block_id(); tile < ntiles; tile += block_count()) {
    // a step that only added gas cells redoes the tiles it touched only
    if (mode == LABEL_ADDED && !p.tdirty[tile]) continue;
    const int bx = tile % tgd.ntx, by = (tile / tgd.ntx) % tgd.nty, bz = tile / (tgd.ntx * tgd.nty);
    const int x0 = bx * TX, y0 = by * TY, z0 = bz * TZ;
    __syncthreads();  // the shared arrays of the last tile are no longer read
    if (threadIdx.x == 0) {
      sg = 0;
      sc = 0;
      nroot = 0;
      rfirst = TN;
    }
    __syncthreads();
    // row masks, runs
    for (int r = warp; r < NR; r += TILE_THREADS / 32) {
      const int x = x0 + lane, y = y0 + r % TY, z = z0 + r / TY;
      const bool inside = x < p.nx && y < p.ny && z < p.nz;
      const bool gas = inside && post_type(p.flags[x + nx * y + nxy * z]) == T_GAS;
      const unsigned m = __ballot_sync(0xffffffffu, gas), in = __ballot_sync(0xffffffffu, inside);
      if (lane == 0) {
        rowm[r] = m;
        if (m) atomicAdd(&sg, __popc(m));
        atomicAdd(&sc, __popc(in));
      }
      const unsigned starts = m & ~(m << 1);
      lp[r * TX + lane] = gas ? r * TX + (31 - __clz(starts & (0xffffffffu >> (31 - lane)))) : -1;
      lsz[r * TX + lane] = 0;
    }
    __syncthreads();
    const long long root0 = x0 + nx * y0 + nxy * z0;
    if (sg == 0) {
      if (threadIdx.x == 0) p.tstat[tile] = 0;
      continue;
    }
    if (sg == sc) {  // every cell is gas: one component rooted at the first cell
      if (threadIdx.x == 0) {
        p.tstat[tile] = 1;
        p.troot[tile] = (int)root0;
      }
      for (int t = threadIdx.x; t < TN; t += TILE_THREADS) {
        const int x = x0 + t % TX, y = y0 + (t / TX) % TY, z = z0 + t / (TX * TY);
        if (x < p.nx && y < p.ny && z < p.nz) {
          const long long n = x + nx * y + nxy * z;
          p.parent[n] = (int)root0;
          p.lsize[n] = t == 0 ? sg : 0;
        }
      }
      continue;
    }
    // rows joined at the first cell of each overlapping segment
    bool ok = true;
    for (int r = warp; r < NR; r += TILE_THREADS / 32) {
      const unsigned a = rowm[r];
      if (!a) continue;
      const int ly = r % TY, lz = r / TY;
#pragma unroll
      for (int k = 0; k < RowLinks<D>::n; ++k) {
        const int dx = RowLinks<D>::dx(k), ry = ly + RowLinks<D>::dy(k), rz = lz + RowLinks<D>::dz(k);
        if (ry < 0 || ry >= TY || rz < 0 || rz >= TZ) continue;  // across the tile face: the merge pass
        const int rr = ry + TY * rz;
        const unsigned b = rowm[rr];
        const unsigned bs = dx > 0 ? (b >> 1) : (dx < 0 ? (b << 1) : b);  // bit x: gas at x + dx in row rr
        const unsigned ov = a & bs;
        const unsigned seg = ov & ~(ov << 1);
        if ((seg >> lane) & 1u) ok &= sm_union(lp, r * TX + lane, rr * TX + lane + dx);
      }
    }
    if (!ok) atomicOr(p.err, ERR_NOTCONV);
    __syncthreads();
    // flatten, count roots, sizes per run
    for (int r = warp; r < NR; r += TILE_THREADS / 32) {
      const unsigned m = rowm[r];
      const int t = r * TX + lane;
      int root = -1;
      if ((m >> lane) & 1u) root = sm_find(lp, t);
      __syncwarp();
      if (root >= 0) lp[t] = root;
      const unsigned starts = m & ~(m << 1);
      if ((starts >> lane) & 1u) {
        const int len = __ffs(~(m >> lane)) - 1;
        atomicAdd(&lsz[root], len > 0 ? len : 32 - lane);
      }
      if (root == t) {
        atomicAdd(&nroot, 1);
        atomicMin(&rfirst, t);
      }
    }
    __syncthreads();
    if (threadIdx.x == 0) {
      p.tstat[tile] = nroot == 1 ? 1 : 2;
      const int r = rfirst;
      p.troot[tile] = (int)(x0 + r % TX + nx * (y0 + (r / TX) % TY) + nxy * (z0 + r / (TX * TY)));
    }
    for (int t = threadIdx.x; t < TN; t += TILE_THREADS) {
      const int x = x0 + t % TX, y = y0 + (t / TX) % TY, z = z0 + t / (TX * TY);
      if (lp[t] < 0 || x >= p.nx || y >= p.ny || z >= p.nz) continue;
      const int r = lp[t];
      const int rx = x0 + r % TX, ry = y0 + (r / TX) % TY, rz = z0 + r / (TX * TY);
      const long long n = x + nx * y + nxy * z;
      p.parent[n] = (int)(rx + nx * ry + nxy * rz);
      p.lsize[n] = r == t ? lsz[t] : 0;
    }
  }
}

// one block per tile: join gas components across tile faces (and the
// periodic boundary).  Two all-gas tiles are joined by one union of their
// roots; otherwise every crossing link of a gas cell is joined.
template <int D>
__global__ void __launch_bounds__(TILE_THREADS) k_uf_merge(Params p) {
  constexpr int TX = Tile<D>::TX, TY = Tile<D>::TY, TZ = Tile<D>::TZ, TN = TX * TY * TZ;
  if (label_fast(p)) return;
  const int mode = label_mode(p);
  if (mode == LABEL_SKIP) return;
  const TileGrid<D> tgd(p);
  const long long nx = p.nx, nxy = (long long)p.nx * p.ny;
  const int ntiles = tgd.ntx * tgd.nty * tgd.ntz;
  // statuses of the 3^d neighbouring tiles (periodic); after a step that
  // only added gas cells, only links near a touched tile can be new
  __shared__ int nst[27];
  __shared__ int near_dirty;
  // one gas link suffices between two single-component tiles: the first
  // thread that meets one claims the neighbour offset
  __shared__ int claimed[27];
  // per neighbouring tile, the last pair of representatives joined: links
  // between the same two local components need one union only
  __shared__ unsigned long long lastpair[27];
  for (int tile = block_id(); tile < ntiles; tile += block_count()) {
    const int own = p.tstat[tile];
    if (own == 0) continue;
    const int bx = tile % tgd.ntx, by = (tile / tgd.ntx) % tgd.nty, bz = tile / (tgd.ntx * tgd.nty);
    const int x0 = bx * TX, y0 = by * TY, z0 = bz * TZ;
    __syncthreads();  // the shared arrays of the last tile are no longer read
    if (threadIdx.x == 0) near_dirty = 0;
    __syncthreads();
    if (threadIdx.x < 27) {
      const int ox = threadIdx.x % 3 - 1, oy = (threadIdx.x / 3) % 3 - 1, oz = threadIdx.x / 9 - 1;
      const bool in = !(D == 2 && oz != 0);
      const int nt = tgd.id(bx + ox, by + oy, bz + oz);
      nst[threadIdx.x] = in ? p.tstat[nt] : 0;
      if (mode == LABEL_ADDED && in && p.tdirty[nt]) near_dirty = 1;
      claimed[threadIdx.x] = 0;
      lastpair[threadIdx.x] = ~0ull;
    }
    __syncthreads();
    if (mode == LABEL_ADDED && !near_dirty) continue;
    bool ok = true;
    for (int t = threadIdx.x; t < TN; t += TILE_THREADS) {
      const int lx = t % TX, ly = (t / TX) % TY, lz = t / (TX * TY);
      const int x = x0 + lx, y = y0 + ly, z = z0 + lz;
      if (x >= p.nx || y >= p.ny || z >= p.nz) continue;
      const bool onface = lx == 0 || lx == TX - 1 || x == p.nx - 1 || ly == 0 || ly == TY - 1 || y == p.ny - 1 ||
                          (D == 3 && (lz == 0 || lz == TZ - 1 || z == p.nz - 1));
      if (!onface) continue;
      const long long n = x + nx * y + nxy * z;
      if (post_type(p.flags[n]) != T_GAS) continue;
#pragma unroll
      for (int i = 1; i < Lat<D>::Q; i += 2) {
        const int dx = Lat<D>::cx(i), dy = Lat<D>::cy(i), dz = Lat<D>::cz(i);
        const int ax = x + dx, ay = y + dy, az = z + dz;
        const bool wraps = ax < 0 || ax >= p.nx || ay < 0 || ay >= p.ny || az < 0 || az >= p.nz;
        // tile offset of the link's far end
        const int ox = (lx + dx < 0) ? -1 : ((lx + dx >= TX || ax >= p.nx) ? 1 : 0);
        const int oy = (ly + dy < 0) ? -1 : ((ly + dy >= TY || ay >= p.ny) ? 1 : 0);
        const int oz = (lz + dz < 0) ? -1 : ((lz + dz >= TZ || az >= p.nz) ? 1 : 0);
        if (!wraps && ox == 0 && oy == 0 && oz == 0) continue;  // joined by the local pass
        const int oi = (ox + 1) + 3 * (oy + 1) + 9 * (oz + 1);
        const int ns = nst[oi];
        if (ns == 0) continue;
        if (own == 1 && ns == 1 && claimed[oi]) continue;
        const long long m = at_far(p, ax, ay, az);
        if (post_type(p.flags[m]) != T_GAS) continue;
        if (own == 1 && ns == 1 && atomicExch(&claimed[oi], 1)) continue;
        // representatives: the parents the local pass left (any ancestor
        // stands for the same component)
        const int ra = __ldcg(p.parent + n), rb = __ldcg(p.parent + m);
        const unsigned long long key = ((unsigned long long)(unsigned)ra << 32) | (unsigned)rb;
        if (lastpair[oi] == key) continue;
        lastpair[oi] = key;
        ok &= uf_union(p.parent, ra, rb);
      }
    }
    if (!ok) atomicOr(p.err, ERR_NOTCONV);
  }
}

// one block per tile: every gas cell points at its component's root; roots
// are registered
template <int D>
__global__ void __launch_bounds__(TILE_THREADS) k_uf_compress(Params p) {
  constexpr int TX = Tile<D>::TX, TY = Tile<D>::TY, TZ = Tile<D>::TZ, TN = TX * TY * TZ;
  if (label_fast(p) || gas_unchanged(p)) return;
  const TileGrid<D> tgd(p);
  const int ntiles = tgd.ntx * tgd.nty * tgd.ntz;
  const long long nx = p.nx, nxy = (long long)p.nx * p.ny;
  __shared__ int sroot;
  for (int tile = block_id(); tile < ntiles; tile += block_count()) {
    // the merge pass has read the touched-tile marks: clear them for the next step
    if (threadIdx.x == 0 && p.tdirty) p.tdirty[tile] = 0;
    const int own = p.tstat[tile];
    if (own == 0) continue;
    const int bx = tile % tgd.ntx, by = (tile / tgd.ntx) % tgd.nty, bz = tile / (tgd.ntx * tgd.nty);
    const int x0 = bx * TX, y0 = by * TY, z0 = bz * TZ;
    if (own == 1) {
      const int r0 = p.troot[tile];
      __syncthreads();  // sroot of the last tile is no longer read
      if (threadIdx.x == 0) {
        sroot = uf_find(p.parent, r0);
        if (sroot == r0) {
          const int k = atomicAdd(p.nroots, 1);
          if (k < p.cap) {
            p.roots[k] = r0;
          } else {
            atomicOr(p.err, ERR_CAPACITY);
            if (p.rlabel) p.rlabel[r0] = -1;
          }
        }
      }
      __syncthreads();
      const int r = sroot;
      for (int t = threadIdx.x; t < TN; t += TILE_THREADS) {
        const int x = x0 + t % TX, y = y0 + (t / TX) % TY, z = z0 + t / (TX * TY);
        if (x < p.nx && y < p.ny && z < p.nz) {
          const long long n = x + nx * y + nxy * z;
          if (post_type(p.flags[n]) == T_GAS) p.parent[n] = r;
        }
      }
      continue;
    }
    for (int t = threadIdx.x; t < TN; t += TILE_THREADS) {
      const int x = x0 + t % TX, y = y0 + (t / TX) % TY, z = z0 + t / (TX * TY);
      if (x >= p.nx || y >= p.ny || z >= p.nz) continue;
      const long long n = x + nx * y + nxy * z;
      if (post_type(p.flags[n]) != T_GAS) continue;
      const int r = uf_find(p.parent, (int)n);
      p.parent[n] = r;
      if (r == (int)n) {
        const int k = atomicAdd(p.nroots, 1);
        if (k < p.cap) {
          p.roots[k] = r;
        } else {
          atomicOr(p.err, ERR_CAPACITY);
          if (p.rlabel) p.rlabel[r] = -1;
        }
      }
    }
  }
}

// one block: sort the roots (bitonic, in shared memory) and publish the count
static __global__ void k_sort_roots(Params p) {
  extern __shared__ int sr[];
  if (label_fast(p)) return;
  if (gas_unchanged(p)) {  // the sorted roots of the last labelling stand
    if (threadIdx.x == 0) *p.tnew.count = *p.told.count;
    return;
  }
  const int total = *p.nroots;
  const int cnt = total < p.cap ? total : p.cap;
  int P = 1;
  while (P < cnt) P <<= 1;
  for (int k = threadIdx.x; k < P; k += blockDim.x) sr[k] = k < cnt ? p.roots[k] : 0x7fffffff;
  __syncthreads();
  for (int size = 2; size <= P; size <<= 1)
    for (int stride = size >> 1; stride > 0; stride >>= 1) {
      for (int k = threadIdx.x; k < P; k += blockDim.x) {
        const int j = k ^ stride;
        if (j > k) {
          const bool up = (k & size) == 0;
          const int a = sr[k], b = sr[j];
          if ((a > b) == up) {
            sr[k] = b;
            sr[j] = a;
          }
        }
      }
      __syncthreads();
    }
  for (int k = threadIdx.x; k < cnt; k += blockDim.x) {
    p.roots[k] = sr[k];
    if (p.rlabel) p.rlabel[sr[k]] = k;
  }
  if (threadIdx.x == 0) {
    *p.tnew.count = cnt;
    // every thread read the labelling mode before the sort's barriers: the
    // forest is current again
    if (p.forest_stale) *p.forest_stale = 0;
  }
}

__device__ __forceinline__ int root_index(const int *roots, int cnt, int r) {
  int lo = 0, hi = cnt;
  while (lo < hi) {
    const int mid = (lo + hi) >> 1;
    if (roots[mid] < r)
      lo = mid + 1;
    else
      hi = mid;
  }
  return (lo < cnt && roots[lo] == r) ? lo : -1;
}

__device__ __forceinline__ void hash_insert(const Params &p, unsigned long long key) {
  unsigned long long h = key * 0x9E3779B97F4A7C15ull;
  unsigned idx = (unsigned)(h >> 32) & (unsigned)(p.hash_size - 1);
  for (int probe = 0; probe < p.hash_size; ++probe) {
    const unsigned long long cur = __ldcg(p.hash + idx);
    if (cur == key) return;
    if (cur == HASH_EMPTY) {
      const unsigned long long prev = atomicCAS(p.hash + idx, HASH_EMPTY, key);
      if (prev == HASH_EMPTY) {
        p.hlist[atomicAdd(p.hcount, 1)] = (int)idx;
        return;
      }
      if (prev == key) return;
    }
    idx = (idx + 1) & (unsigned)(p.hash_size - 1);
  }
  atomicOr(p.err, ERR_HASH);
}

// new labels, volumes, atmosphere flags and old->new overlap pairs
template <int D, class R>
__global__ void __launch_bounds__(256) k_relabel(Params p) {
  __shared__ double wbuf[256];
  if (label_fast(p)) return;
  // row blocks of blockDim.x cells along x, walked by a grid of any size
  const int nbx = (p.nx + (int)blockDim.x - 1) / (int)blockDim.x;
  const int nrb = nbx * p.ny * p.nz;
  for (int rb = block_id(); rb < nrb; rb += block_count()) {
  const int yz = rb / nbx, xb = (rb - yz * nbx) * (int)blockDim.x + (int)threadIdx.x;
  Cell c = cell_at(p, xb < p.nx ? xb : p.nx - 1, yz % p.ny, yz / p.ny);
  const bool inr = xb < p.nx;
  const long long n = c.n;
  const uint8_t fl = inr ? p.flags[n] : (uint8_t)T_WALL;
  const int t = post_type(fl);
  int knew = -1, ngas = 0;
  double v = 0.0;
  if (t == T_GAS) {
    knew = p.rlabel[p.parent[n]];
    ngas = p.lsize[n];  // non-zero only at tile-local roots
    if (p.atmosphere && knew >= 0 && (D == 2 ? c.y : c.z) == p.top_layer && !p.tnew.atm[knew]) p.tnew.atm[knew] = 1;
  } else if (t == T_IFC) {
#pragma unroll
    for (int i = 1; i < Lat<D>::Q; ++i) {
      const long long m = nb<D>(p, c, i);
      if (post_type(p.flags[m]) == T_GAS) {
        const int k = p.rlabel[p.parent[m]];
        if (k >= 0 && (knew < 0 || k < knew)) knew = k;
      }
    }
    if (knew >= 0) v = 1.0 - (double)((const R *)p.phi)[n];
  }
  if (inr) p.label_new[n] = knew;
  // gas cells are counted (the bubble update adds them to the volume),
  // interface cells add their gas share 1 - alpha
  const bool gcontrib = knew >= 0 && ngas != 0;
  if (__any_sync(0xffffffffu, gcontrib)) agg_count(p.tnew.ng, gcontrib ? knew : -1, ngas);
  const bool contrib = knew >= 0 && v != 0.0;
  if (__any_sync(0xffffffffu, contrib)) agg_add(p.tnew.V, contrib ? knew : -1, v, wbuf + (threadIdx.x & ~31));
  // old -> new overlap pairs (cells without a new label have none: no
  // old label read, and warps without any pair skip the match)
  const int kold = (inr && knew >= 0) ? p.label_old[n] : -1;
  const bool pair = kold >= 0 && knew >= 0;
  if (!__any_sync(0xffffffffu, pair)) continue;
  const unsigned long long key = pair ? (((unsigned long long)kold << 32) | (unsigned)knew) : HASH_EMPTY;
  const unsigned peers = __match_any_sync(0xffffffffu, key);
  if (pair && (threadIdx.x & 31) == __ffs(peers) - 1) hash_insert(p, key);
  }
}

// one block of 1024 threads: carry gas content from the old to the new table.
// Group bookkeeping lives in shared memory when there are at most
// K10_SMEM old + new bubbles, in the global scratch arrays otherwise.
constexpr int K10_SMEM = 512;
static __global__ void __launch_bounds__(1024) k_bubble_update(Params p) {
  if (label_fast(p)) return;
  __shared__ int sfresh[1024];
  __shared__ int sbase;
  __shared__ int s_par[K10_SMEM], s_nold[K10_SMEM], s_nnew[K10_SMEM], s_atm[K10_SMEM], s_minid[K10_SMEM],
      s_heir[K10_SMEM];
  __shared__ double s_mold[K10_SMEM], s_vnew[K10_SMEM];
  __shared__ unsigned long long s_vmax[K10_SMEM];
  const int nold = *p.told.count, nnew = *p.tnew.count;
  const int T = nold + nnew;
  const bool sm = T <= K10_SMEM;
  int *gpar = sm ? s_par : p.gpar, *gnold = sm ? s_nold : p.gnold, *gnnew = sm ? s_nnew : p.gnnew;
  int *gatm = sm ? s_atm : p.gatm, *gminid = sm ? s_minid : p.gminid, *gheir = sm ? s_heir : p.gheir;
  double *gmold = sm ? s_mold : p.gmold, *gvnew = sm ? s_vnew : p.gvnew;
  unsigned long long *gvmax = sm ? s_vmax : p.gvmax;
  const int tid = threadIdx.x, nt = blockDim.x;
  const int nh = *p.hcount;
  for (int k = tid; k < T; k += nt) {
    gpar[k] = k;
    gnold[k] = 0;
    gnnew[k] = 0;
    gatm[k] = 0;
    gminid[k] = 0x7fffffff;
    gmold[k] = 0.0;
    gvnew[k] = 0.0;
    gvmax[k] = 0ull;
  }
  for (int j = tid; j < nold; j += nt) p.told.m[j] += p.told.dm[j];
  for (int k = tid; k < nnew; k += nt) p.tnew.V[k] += (double)p.tnew.ng[k];
  __syncthreads();
  bool ok = true;
  for (int h = tid; h < nh; h += nt) {
    const unsigned long long key = p.hash[p.hlist[h]];
    const int j = (int)(key >> 32), k = (int)(key & 0xffffffffu);
    if (j < nold && k < nnew) ok &= uf_union_any(gpar, j, nold + k);
  }
  if (!ok) atomicOr(p.err, ERR_NOTCONV);
  __threadfence_block();
  __syncthreads();
  // group of every node (read-only finds into a separate array)
  for (int k = tid; k < T; k += nt) gheir[k] = uf_find_any(gpar, k);
  __syncthreads();
  for (int k = tid; k < T; k += nt) gpar[k] = gheir[k];
  __syncthreads();
  for (int k = tid; k < T; k += nt) gheir[k] = 0x7fffffff;
  __syncthreads();
  const int *grp = gpar;
  for (int j = tid; j < nold; j += nt) {
    const int g = grp[j];
    atomicAdd(gmold + g, p.told.m[j]);
    atomicAdd(gnold + g, 1);
    atomicMin(gminid + g, p.told.id[j]);
  }
  for (int k = tid; k < nnew; k += nt) {
    const int g = grp[nold + k];
    atomicAdd(gvnew + g, p.tnew.V[k]);
    atomicAdd(gnnew + g, 1);
    if (p.tnew.atm[k]) gatm[g] = 1;
    atomicMax(gvmax + g, (unsigned long long)__double_as_longlong(p.tnew.V[k]));
  }
  __syncthreads();
  for (int k = tid; k < nnew; k += nt) {
    const int g = grp[nold + k];
    if ((unsigned long long)__double_as_longlong(p.tnew.V[k]) == gvmax[g]) atomicMin(gheir + g, k);
  }
  __syncthreads();
  for (int j = tid; j < nold; j += nt) {
    const int g = grp[j];
    if (gnnew[g] == 0 || gatm[g]) atomicAdd(p.led + 5, p.told.m[j]);
  }
  // new rows; fresh ids are numbered in bubble order
  const int chunk = (nnew + nt - 1) / nt;
  const int k0 = tid * chunk, k1 = min(nnew, k0 + chunk);
  int myfresh = 0;
  for (int k = k0; k < k1; ++k) {
    const int g = grp[nold + k];
    const double V = p.tnew.V[k];
    double m, pr;
    if (gatm[g]) {
      pr = p.p0;
      m = p.p0 * V / p.RT;
      atomicAdd(p.led + 5, -m);
    } else if (gnold[g] == 0) {
      const double Req = p.dim == 3 ? cbrt(3.0 * V / (4.0 * 3.14159265358979323846)) : sqrt(V / 3.14159265358979323846);
      pr = p.p0 + (p.dim - 1) * p.sigma / Req;
      m = pr * V / p.RT;
      atomicAdd(p.led + 5, -m);
    } else {
      m = gmold[g] * V / gvnew[g];
      pr = m * p.RT / V;
    }
    p.tnew.m[k] = m;
    p.tnew.p[k] = pr;
    p.tnew.dm[k] = 0.0;
    p.tnew.root[k] = p.roots[k];
    myfresh += !(gnold[g] > 0 && gheir[g] == k);
  }
  // inclusive scan of myfresh over the block: within each warp by shuffles,
  // then over the warp totals by the first warp
  const int lane = tid & 31, wid = tid >> 5;
  int incl = myfresh;
#pragma unroll
  for (int off = 1; off < 32; off <<= 1) {
    const int v = __shfl_up_sync(0xffffffffu, incl, off);
    if (lane >= off) incl += v;
  }
  if (lane == 31) sfresh[wid] = incl;
  if (tid == 0) sbase = *p.next_id;
  __syncthreads();
  if (wid == 0) {
    int w = lane < (nt >> 5) ? sfresh[lane] : 0;
#pragma unroll
    for (int off = 1; off < 32; off <<= 1) {
      const int v = __shfl_up_sync(0xffffffffu, w, off);
      if (lane >= off) w += v;
    }
    sfresh[32 + lane] = w;  // inclusive totals of warps 0..lane
  }
  __syncthreads();
  const int before = (wid > 0 ? sfresh[32 + wid - 1] : 0) + incl - myfresh;
  int fid = sbase + before;
  for (int k = k0; k < k1; ++k) {
    const int g = grp[nold + k];
    if (gnold[g] > 0 && gheir[g] == k)
      p.tnew.id[k] = gminid[g];
    else
      p.tnew.id[k] = fid++;
  }
  __syncthreads();
  if (tid == nt - 1) *p.next_id = sbase + sfresh[32 + (nt >> 5) - 1];
  for (int h = tid; h < nh; h += nt) p.hash[p.hlist[h]] = HASH_EMPTY;
  if (tid == 0) {
    *p.hcount = 0;
    *p.nroots = 0;
    if (p.gas_dirty) *p.gas_dirty = 0;
  }
  // the old table is the next step's new table: clear its accumulators
  for (int k = tid; k < p.cap; k += nt) {
    p.told.V[k] = 0.0;
    p.told.atm[k] = 0;
    p.told.ng[k] = 0;
  }
}

// ---------------------------------------------------------------------------
// Labelling of a step whose conversion kept every bubble's cells, number and
// root: added gas cells touch no gas cell of another bubble and lie above
// their bubble's root (checked by the marking), removed gas cells leave
// their bubble connected (k_label_check); otherwise lab_slow is set.  Every
// bubble keeps its cells, its number and its root, so the labels of the last
// step stand except at the filled cells (-1), the added gas cells (the label
// they had as interface cells, which is their bubble's) and the interface
// cells after the conversion (smallest label of their gas neighbours).  The
// result equals the full labelling's.  The step graph picks this branch or
// the full one on the device: k_label_choose sets lab_fast, and the kernels
// of the branch not taken return at once.
static __global__ void k_label_choose(Params p) {
  const int d = *p.gas_dirty;  // -1: the state was set from outside
  const bool fast = d >= 0 && *p.lab_slow == 0;
  *p.lab_fast = fast;
  *p.lab_full = !fast;
  *p.lab_slow = 0;
}

// At the start of a step, before its marking: bring label_new (the labels
// of the step before last) up to the last labels wherever they differ.
// After a patched step they differ only at that step's interface cells
// before and after its conversion (every cell it patched), which are the
// two interface lists at hand; otherwise (lab_full) everything is copied,
// as int4 words and a tail.  The patch of this step then writes only its
// own cells; a full labelling overwrites every label.
static __global__ void k_label_sync(Params p) {
  const long long tid = blockIdx.x * (long long)blockDim.x + threadIdx.x, nt = (long long)gridDim.x * blockDim.x;
  // the roots of the next table start from the last ones (a patched step
  // lowers a bubble's root to the gas cells it adds below it)
  const int nbub = *p.told.count;
  for (long long k = tid; k < nbub; k += nt) p.tnew.root[k] = p.told.root[k];
  if (*p.lab_full) {
    const long long n4 = p.N >> 2;
    const int4 *src = reinterpret_cast<const int4 *>(p.label_old);
    int4 *dst = reinterpret_cast<int4 *>(p.label_new);
    for (long long k = tid; k < n4; k += nt) dst[k] = __ldcs(src + k);
    for (long long k = (n4 << 2) + tid; k < p.N; k += nt) p.label_new[k] = p.label_old[k];
    return;
  }
  const int np = *p.inext_count, nc = *p.icount;  // the last step's interface list, this step's
  for (long long k = tid; k < np + nc; k += nt) {
    const int n = k < np ? p.inext[k] : p.ilist[k - np];
    p.label_new[n] = p.label_old[n];
  }
}

// label_new holds the last labels when this runs (k_label_sync).  One thread per marked
// cell, then per interface cell after the conversion; gas counts grow by the
// added cells; volumes collect the interface shares 1 - alpha.
template <int D, class R>
__global__ void __launch_bounds__(128) k_label_fast(Params p) {
  __shared__ double wbuf[128];
  if (!label_fast(p)) return;
  const int nbub = *p.told.count, nm = *p.mcount, ni = *p.inext_count, nn = *p.ncount;
  const int tid = blockIdx.x * blockDim.x + threadIdx.x, nthreads = gridDim.x * blockDim.x;
  if (tid == 0) {
    *p.tnew.count = nbub;
    // the forest lacks the added gas cells (bit 0: redo the touched tiles)
    // or still holds removed ones (bit 1: rebuild it)
    const int d = *p.gas_dirty;
    if (d & 1) atomicOr(p.forest_stale, 1);
    if (d & 2) atomicOr(p.forest_stale, 2);
  }
  for (int k = tid; k < nbub; k += nthreads) {
    atomicAdd(p.tnew.ng + k, p.told.ng[k]);
    if (p.told.atm[k]) p.tnew.atm[k] = 1;
  }
  const int total = nm + ni + nn;
  for (int base = 0; base < total; base += nthreads) {
    const int k = base + tid;
    int kg = -1, kv = -1, dg = 1;
    double v = 0.0;
    if (k >= nm + ni) {
      // a new interface cell that was gas (it carries its bubble's label)
      // leaves its bubble's gas count
      if (k < total) {
        kg = p.label_old[p.nlist[k - nm - ni]];
        dg = -1;
      }
    } else if (k < nm) {
      const int n = p.mlist[k];
      const int t = post_type(p.flags[n]);
      if (t == T_LIQ) {
        p.label_new[n] = -1;
      } else if (t == T_GAS) {
        kg = p.label_old[n];
        if (kg >= 0) atomicMin(p.tnew.root + kg, n);
        if (p.atmosphere && kg >= 0) {
          const Cell c = make_cell(p, n);
          if ((D == 2 ? c.y : c.z) == p.top_layer) p.tnew.atm[kg] = 1;
        }
      }
    } else if (k < total) {
      const int n = p.inext[k - nm];
      const Cell c = make_cell(p, n);
      int knew = -1;
      // the neighbours' flags and labels in one round of loads
      uint8_t fn[Lat<D>::Q];
      int ln[Lat<D>::Q];
#pragma unroll
      for (int i = 1; i < Lat<D>::Q; ++i) {
        const int m = nb<D>(p, c, i);
        fn[i] = p.flags[m];
        ln[i] = p.label_old[m];
      }
#pragma unroll
      for (int i = 1; i < Lat<D>::Q; ++i) {
        if (post_type(fn[i]) == T_GAS) {
          const int l = ln[i];
          if (l >= 0 && (knew < 0 || l < knew)) knew = l;
        }
      }
      p.label_new[n] = knew;
      if (knew >= 0) {
        v = 1.0 - (double)((const R *)p.phi)[n];
        if (v != 0.0) kv = knew;
      }
    }
    if (__any_sync(0xffffffffu, kg >= 0)) agg_count(p.tnew.ng, kg, dg);
    if (__any_sync(0xffffffffu, kv >= 0)) agg_add(p.tnew.V, kv, v, wbuf + (threadIdx.x & ~31));
  }
}

// the bubble update of such a step: every group is one old and one new
// bubble with the same number, so each bubble keeps its id and gas (plus the
// flux of this step); the arithmetic is the general update's for such a
// group.  One thread per bubble.
static __global__ void k_bubble_update_fast(Params p) {
  if (!label_fast(p)) return;
  const int nbub = *p.tnew.count;
  const int tid = blockIdx.x * blockDim.x + threadIdx.x, nt = gridDim.x * blockDim.x;
  for (int k = tid; k < nbub; k += nt) {
    const double mold = p.told.m[k] + p.told.dm[k];
    p.told.m[k] = mold;
    const double V = p.tnew.V[k] + (double)p.tnew.ng[k];
    p.tnew.V[k] = V;
    double m, pr;
    if (p.tnew.atm[k]) {
      atomicAdd(p.led + 5, mold);
      pr = p.p0;
      m = p.p0 * V / p.RT;
      atomicAdd(p.led + 5, -m);
    } else {
      m = mold * V / V;
      pr = m * p.RT / V;
    }
    p.tnew.m[k] = m;
    p.tnew.p[k] = pr;
    p.tnew.dm[k] = 0.0;
    p.tnew.id[k] = p.told.id[k];
  }
  if (tid == 0) {
    *p.hcount = 0;
    *p.nroots = 0;
    if (p.gas_dirty) *p.gas_dirty = 0;
  }
  // the old table is the next step's new table: clear its accumulators
  for (int k = tid; k < p.cap; k += nt) {
    p.told.V[k] = 0.0;
    p.told.atm[k] = 0;
    p.told.ng[k] = 0;
  }
}

}  // namespace lbf

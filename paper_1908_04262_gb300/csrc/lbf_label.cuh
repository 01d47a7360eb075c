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

__device__ __forceinline__ int uf_find(const int *par, int a) {
  for (int it = 0; it < UF_ITERS; ++it) {
    const int b = __ldcg(par + a);
    if (b == a) return a;
    a = b;
  }
  return a;
}

// returns false when the iteration cap was reached
__device__ __forceinline__ bool uf_union(int *par, int a, int b) {
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
  }
  if (blockIdx.x == 0 && threadIdx.x == 0) *p.nroots = 0;
}

// union-find tiles: the local pass joins gas cells of one tile in shared
// memory, the merge pass joins tiles across their faces in global memory
template <int D> struct Tile;
template <> struct Tile<3> { static constexpr int TX = 32, TY = 8, TZ = 4; };
template <> struct Tile<2> { static constexpr int TX = 32, TY = 32, TZ = 1; };
constexpr int TILE_THREADS = 256;

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

__device__ __forceinline__ bool sm_union(int *lp, int a, int b) {
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

template <int D>
__global__ void __launch_bounds__(TILE_THREADS) k_uf_local(Params p) {
  constexpr int TX = Tile<D>::TX, TY = Tile<D>::TY, TZ = Tile<D>::TZ, TN = TX * TY * TZ;
  __shared__ int lp[TN];
  const int x0 = blockIdx.x * TX, y0 = blockIdx.y * TY, z0 = blockIdx.z * TZ;
  const long long nx = p.nx, nxy = (long long)p.nx * p.ny;
  for (int t = threadIdx.x; t < TN; t += TILE_THREADS) {
    const int x = x0 + t % TX, y = y0 + (t / TX) % TY, z = z0 + t / (TX * TY);
    bool gas = false;
    if (x < p.nx && y < p.ny && z < p.nz) gas = ftype(p.flags_out[x + nx * y + nxy * z]) == T_GAS;
    lp[t] = gas ? t : -1;
  }
  __syncthreads();
  bool ok = true;
  for (int t = threadIdx.x; t < TN; t += TILE_THREADS) {
    if (lp[t] < 0) continue;
    const int lx = t % TX, ly = (t / TX) % TY, lz = t / (TX * TY);
#pragma unroll
    for (int i = 1; i < Lat<D>::Q; i += 2) {  // one vector of each opposite pair
      const int ax = lx + Lat<D>::cx(i), ay = ly + Lat<D>::cy(i), az = lz + Lat<D>::cz(i);
      if (ax < 0 || ax >= TX || ay < 0 || ay >= TY || az < 0 || az >= TZ) continue;
      const int u = ax + TX * (ay + TY * az);
      if (lp[u] >= 0) ok &= sm_union(lp, t, u);
    }
  }
  if (!ok) atomicOr(p.err, ERR_NOTCONV);
  __syncthreads();
  for (int t = threadIdx.x; t < TN; t += TILE_THREADS) {
    if (lp[t] < 0) continue;
    const int r = sm_find(lp, t);
    const int x = x0 + t % TX, y = y0 + (t / TX) % TY, z = z0 + t / (TX * TY);
    const int rx = x0 + r % TX, ry = y0 + (r / TX) % TY, rz = z0 + r / (TX * TY);
    p.parent[x + nx * y + nxy * z] = (int)(rx + nx * ry + nxy * rz);
  }
}

// gas cells join their gas neighbours in other tiles (or across the
// periodic boundary)
template <int D>
__global__ void k_uf_merge(Params p) {
  Cell c;
  if (!grid_cell(p, c)) return;
  const long long n = c.n;
  if (ftype(p.flags_out[n]) != T_GAS) return;
  constexpr int TX = Tile<D>::TX, TY = Tile<D>::TY, TZ = Tile<D>::TZ;
  const int lx = c.x % TX, ly = c.y % TY, lz = c.z % TZ;
  bool ok = true;
#pragma unroll
  for (int i = 1; i < Lat<D>::Q; i += 2) {
    const int dx = Lat<D>::cx(i), dy = Lat<D>::cy(i), dz = Lat<D>::cz(i);
    const int ax = c.x + dx, ay = c.y + dy, az = c.z + dz;
    const bool wraps = ax < 0 || ax >= p.nx || ay < 0 || ay >= p.ny || az < 0 || az >= p.nz;
    const bool crosses = wraps || lx + dx < 0 || lx + dx >= TX || ly + dy < 0 || ly + dy >= TY ||
                         lz + dz < 0 || lz + dz >= TZ;
    if (!crosses) continue;
    const long long m = nb<D>(p, c, i);
    if (ftype(p.flags_out[m]) == T_GAS) ok &= uf_union(p.parent, (int)n, (int)m);
  }
  if (!ok) atomicOr(p.err, ERR_NOTCONV);
}

static __global__ void k_uf_compress(Params p) {
  Cell c;
  if (!grid_cell(p, c)) return;
  const long long n = c.n;
  if (ftype(p.flags_out[n]) != T_GAS) return;
  const int r = uf_find(p.parent, (int)n);
  p.parent[n] = r;
  if (r == (int)n) {
    const int k = atomicAdd(p.nroots, 1);
    if (k < p.cap)
      p.roots[k] = r;
    else
      atomicOr(p.err, ERR_CAPACITY);
  }
}

// one block: sort the roots (bitonic, in shared memory) and publish the count
static __global__ void k_sort_roots(Params p) {
  extern __shared__ int sr[];
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
  for (int k = threadIdx.x; k < cnt; k += blockDim.x) p.roots[k] = sr[k];
  if (threadIdx.x == 0) *p.tnew.count = cnt;
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
      if (prev == HASH_EMPTY || prev == key) return;
    }
    idx = (idx + 1) & (unsigned)(p.hash_size - 1);
  }
  atomicOr(p.err, ERR_HASH);
}

// new labels, volumes, atmosphere flags and old->new overlap pairs
template <int D, class R>
__global__ void __launch_bounds__(256) k_relabel(Params p) {
  __shared__ double wbuf[256];
  Cell c;
  const bool inr = grid_cell(p, c);
  const long long n = c.n;
  const int t = inr ? ftype(p.flags_out[n]) : T_WALL;
  const int cnt = *p.tnew.count;
  int knew = -1;
  double v = 0.0;
  if (t == T_GAS) {
    knew = root_index(p.roots, cnt, p.parent[n]);
    v = 1.0;
    if (p.atmosphere && knew >= 0) {
          if ((D == 2 ? c.y : c.z) == p.top_layer) p.tnew.atm[knew] = 1;
    }
  } else if (t == T_IFC) {
  #pragma unroll
    for (int i = 1; i < Lat<D>::Q; ++i) {
      const long long m = nb<D>(p, c, i);
      if (ftype(p.flags_out[m]) == T_GAS) {
        const int k = root_index(p.roots, cnt, p.parent[m]);
        if (k >= 0 && (knew < 0 || k < knew)) knew = k;
      }
    }
    if (knew >= 0) v = 1.0 - (double)((const R *)p.phi)[n];
  }
  if (inr) p.label_new[n] = knew;
  if (__any_sync(0xffffffffu, knew >= 0)) agg_add(p.tnew.V, knew, v, wbuf + (threadIdx.x & ~31));
  const int kold = inr ? p.label_old[n] : -1;
  const bool pair = kold >= 0 && knew >= 0;
  const unsigned long long key = pair ? (((unsigned long long)kold << 32) | (unsigned)knew) : HASH_EMPTY;
  const unsigned peers = __match_any_sync(0xffffffffu, key);
  if (pair && (threadIdx.x & 31) == __ffs(peers) - 1) hash_insert(p, key);
}

// one block of 1024 threads: carry gas content from the old to the new table
static __global__ void __launch_bounds__(1024) k_bubble_update(Params p) {
  __shared__ int sfresh[1024];
  __shared__ int sbase;
  const int nold = *p.told.count, nnew = *p.tnew.count;
  const int T = nold + nnew;
  const int tid = threadIdx.x, nt = blockDim.x;
  for (int k = tid; k < T; k += nt) {
    p.gpar[k] = k;
    p.gnold[k] = 0;
    p.gnnew[k] = 0;
    p.gatm[k] = 0;
    p.gminid[k] = 0x7fffffff;
    p.gheir[k] = 0x7fffffff;
    p.gmold[k] = 0.0;
    p.gvnew[k] = 0.0;
    p.gvmax[k] = 0ull;
  }
  for (int j = tid; j < nold; j += nt) p.told.m[j] += p.told.dm[j];
  __syncthreads();
  bool ok = true;
  for (int h = tid; h < p.hash_size; h += nt) {
    const unsigned long long key = p.hash[h];
    if (key == HASH_EMPTY) continue;
    const int j = (int)(key >> 32), k = (int)(key & 0xffffffffu);
    if (j < nold && k < nnew) ok &= uf_union(p.gpar, j, nold + k);
  }
  if (!ok) atomicOr(p.err, ERR_NOTCONV);
  __threadfence_block();
  __syncthreads();
  // group of every node (read-only finds into a separate array)
  for (int k = tid; k < T; k += nt) p.gheir[k] = uf_find(p.gpar, k);
  __syncthreads();
  for (int k = tid; k < T; k += nt) p.gpar[k] = p.gheir[k];
  __syncthreads();
  for (int k = tid; k < T; k += nt) p.gheir[k] = 0x7fffffff;
  __syncthreads();
  const int *grp = p.gpar;
  for (int j = tid; j < nold; j += nt) {
    const int g = grp[j];
    atomicAdd(p.gmold + g, p.told.m[j]);
    atomicAdd(p.gnold + g, 1);
    atomicMin(p.gminid + g, p.told.id[j]);
  }
  for (int k = tid; k < nnew; k += nt) {
    const int g = grp[nold + k];
    atomicAdd(p.gvnew + g, p.tnew.V[k]);
    atomicAdd(p.gnnew + g, 1);
    if (p.tnew.atm[k]) p.gatm[g] = 1;
    atomicMax(p.gvmax + g, (unsigned long long)__double_as_longlong(p.tnew.V[k]));
  }
  __syncthreads();
  for (int k = tid; k < nnew; k += nt) {
    const int g = grp[nold + k];
    if ((unsigned long long)__double_as_longlong(p.tnew.V[k]) == p.gvmax[g]) atomicMin(p.gheir + g, k);
  }
  __syncthreads();
  for (int j = tid; j < nold; j += nt) {
    const int g = grp[j];
    if (p.gnnew[g] == 0 || p.gatm[g]) atomicAdd(p.led + 5, p.told.m[j]);
  }
  // new rows; fresh ids are numbered in bubble order
  const int chunk = (nnew + nt - 1) / nt;
  const int k0 = tid * chunk, k1 = min(nnew, k0 + chunk);
  int myfresh = 0;
  for (int k = k0; k < k1; ++k) {
    const int g = grp[nold + k];
    const double V = p.tnew.V[k];
    double m, pr;
    if (p.gatm[g]) {
      pr = p.p0;
      m = p.p0 * V / p.RT;
      atomicAdd(p.led + 5, -m);
    } else if (p.gnold[g] == 0) {
      const double Req = p.dim == 3 ? cbrt(3.0 * V / (4.0 * 3.14159265358979323846)) : sqrt(V / 3.14159265358979323846);
      pr = p.p0 + (p.dim - 1) * p.sigma / Req;
      m = pr * V / p.RT;
      atomicAdd(p.led + 5, -m);
    } else {
      m = p.gmold[g] * V / p.gvnew[g];
      pr = m * p.RT / V;
    }
    p.tnew.m[k] = m;
    p.tnew.p[k] = pr;
    p.tnew.dm[k] = 0.0;
    p.tnew.root[k] = p.roots[k];
    myfresh += !(p.gnold[g] > 0 && p.gheir[g] == k);
  }
  sfresh[tid] = myfresh;
  __syncthreads();
  for (int off = 1; off < nt; off <<= 1) {  // inclusive scan
    const int v = tid >= off ? sfresh[tid - off] : 0;
    __syncthreads();
    sfresh[tid] += v;
    __syncthreads();
  }
  if (tid == 0) sbase = *p.next_id;
  __syncthreads();
  int fid = sbase + sfresh[tid] - myfresh;
  for (int k = k0; k < k1; ++k) {
    const int g = grp[nold + k];
    if (p.gnold[g] > 0 && p.gheir[g] == k)
      p.tnew.id[k] = p.gminid[g];
    else
      p.tnew.id[k] = fid++;
  }
  __syncthreads();
  if (tid == nt - 1) *p.next_id = sbase + sfresh[nt - 1];
  for (int h = tid; h < p.hash_size; h += nt) p.hash[h] = HASH_EMPTY;
}

}  // namespace lbf

// lbf_noalloc.cu -- bubble labelling of a caller-supplied cell-type field
// that allocates nothing: its union-find scratch is one file-scope device
// array, sized for at most kMaxCells cells.
//
// Who needs it: code that may not call cudaMalloc at all -- for example a
// host framework whose caching allocator has already reserved the device's
// memory, or a real-time loop in which an allocation (and the implicit
// synchronisation it can cause) is not acceptable.  Such callers pass their
// own input and output buffers and get the same labels as lbf_fields(LABEL)
// after lbf_set_cells.
#include <cuda_runtime.h>

#include <cstring>
#include <mutex>

#include "../../include/lbf.h"
#include "lbf_label.cuh"
#include "lbf_ops_api.h"

using namespace lbf;

namespace {

constexpr long long kMaxCells = 1 << 20;  // 1,048,576 cells
constexpr int kMaxTiles = 1 << 16;
constexpr int kMaxBubbles = 4096;

struct Scratch {
  int parent[kMaxCells];
  int lsize[kMaxCells];
  int troot[kMaxTiles];
  int roots[kMaxBubbles];
  int nroots, count, err;
  uint8_t tstat[kMaxTiles];
};

// every GPU that loads the library holds this array until the process exits
static __device__ __align__(256) Scratch g_scratch;

std::mutex g_mu;
Scratch *g_addr[256] = {nullptr};

int fail(int code, const char *msg) {
  lbf::set_last_error(msg);
  return code;
}

// final labels: gas cells get the rank of their root among the sorted roots,
// interface cells the smallest label of their gas neighbours, others -1
template <int D>
__global__ void k_cc_label(Params p, int32_t *label, int32_t *count) {
  Cell c;
  const bool inr = grid_cell(p, c);
  const int cnt = *p.tnew.count;
  if (inr) {
    const long long n = c.n;
    const int t = ftype(p.flags[n]);
    int k = -1;
    if (t == T_GAS) {
      k = root_index(p.roots, cnt, p.parent[n]);
    } else if (t == T_IFC) {
#pragma unroll
      for (int i = 1; i < Lat<D>::Q; ++i) {
        const long long m = nb<D>(p, c, i);
        if (ftype(p.flags[m]) == T_GAS) {
          const int r = root_index(p.roots, cnt, p.parent[m]);
          if (r >= 0 && (k < 0 || r < k)) k = r;
        }
      }
    }
    label[n] = k;
  }
  if (blockIdx.x == 0 && blockIdx.y == 0 && blockIdx.z == 0 && threadIdx.x == 0) *count = *p.err ? -1 : cnt;
}

__global__ void k_cc_reset(Scratch *s) {
  s->nroots = 0;
  s->err = 0;
  s->count = 0;
}

template <int D>
int run(Scratch *s, const uint8_t *type, int nx, int ny, int nz, int32_t *label, int32_t *count, cudaStream_t st) {
  Params p;
  memset(&p, 0, sizeof p);
  p.nx = nx;
  p.ny = ny;
  p.nz = nz;
  p.dim = D;
  p.N = (long long)nx * ny * nz;
  p.flags = const_cast<uint8_t *>(type);
  p.parent = s->parent;
  p.lsize = s->lsize;
  p.tstat = s->tstat;
  p.troot = s->troot;
  p.roots = s->roots;
  p.nroots = &s->nroots;
  p.cap = kMaxBubbles;
  p.err = &s->err;
  p.tnew.count = &s->count;
  const dim3 tg((unsigned)((nx + Tile<D>::TX - 1) / Tile<D>::TX), (unsigned)((ny + Tile<D>::TY - 1) / Tile<D>::TY),
                (unsigned)((nz + Tile<D>::TZ - 1) / Tile<D>::TZ));
  const int b = nx >= 96 ? 128 : (nx > 32 ? 64 : 32);
  const dim3 rg((unsigned)((nx + b - 1) / b), (unsigned)ny, (unsigned)nz);
  k_cc_reset<<<1, 1, 0, st>>>(s);
  k_uf_local<D><<<tg, TILE_THREADS, 0, st>>>(p);
  k_uf_merge<D><<<tg, TILE_THREADS, 0, st>>>(p);
  k_uf_compress<D><<<tg, TILE_THREADS, 0, st>>>(p);
  k_sort_roots<<<1, 1024, kMaxBubbles * sizeof(int), st>>>(p);
  k_cc_label<D><<<rg, b, 0, st>>>(p, label, count);
  const cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return fail(LBF_ECUDA, cudaGetErrorString(e));
  return 0;
}

}  // namespace

extern "C" int lbf_label_gas_noalloc(const uint8_t *type, int nx, int ny, int nz, int32_t *label, int32_t *count,
                                     void *stream) {
  if (!type || !label || !count) return fail(LBF_EINVAL, "NULL buffer");
  if (nx < 3 || ny < 3 || (nz != 1 && nz < 3)) return fail(LBF_EINVAL, "each extent must be >= 3 (nz == 1 for 2D)");
  if (ny > 65535 || nz > 65535) return fail(LBF_EINVAL, "ny and nz must be <= 65535");
  const long long N = (long long)nx * ny * nz;
  if (N > kMaxCells) return fail(LBF_EINVAL, "more cells than the static scratch holds (1,048,576)");
  const int D = nz == 1 ? 2 : 3;
  const long long tiles = D == 3 ? (long long)((nx + 31) / 32) * ((ny + 7) / 8) * ((nz + 3) / 4)
                                 : (long long)((nx + 31) / 32) * ((ny + 31) / 32);
  if (tiles > kMaxTiles) return fail(LBF_EINVAL, "more union-find tiles than the static scratch holds (65,536)");
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 256) return fail(LBF_ECUDA, "cudaGetDevice failed");
  cudaStream_t st = (cudaStream_t)stream;
  // the symbol's device address, looked up with the device current (in host
  // code g_scratch is only a host-side stand-in).  It is looked up again on
  // every call made outside stream capture, so that a device reset or another
  // context on the device never leaves a stale address behind; under capture
  // the address of the last uncaptured call on this device is used.
  cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
  if (cudaStreamIsCapturing(st, &cs) != cudaSuccess) return fail(LBF_ECUDA, "cudaStreamIsCapturing failed");
  Scratch *s = nullptr;
  {
    std::lock_guard<std::mutex> lock(g_mu);
    if (cs == cudaStreamCaptureStatusNone || !g_addr[dev]) {
      if (cs != cudaStreamCaptureStatusNone)
        return fail(LBF_EINVAL, "the first call on a device must come before any stream capture");
      void *a = nullptr;
      const cudaError_t e = cudaGetSymbolAddress(&a, g_scratch);
      if (e != cudaSuccess) return fail(LBF_ECUDA, cudaGetErrorString(e));
      g_addr[dev] = (Scratch *)a;
    }
    s = g_addr[dev];
  }
  return D == 2 ? run<2>(s, type, nx, ny, nz, label, count, st) : run<3>(s, type, nx, ny, nz, label, count, st);
}

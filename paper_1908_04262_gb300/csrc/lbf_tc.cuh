// lbf_tc.cuh -- the learned-curvature network's products on the
// fifth-generation tensor cores (tcgen05): operand tiles in shared memory
// (K-major, no swizzle), the FP32 accumulators in tensor memory, one
// elected thread issuing the BF16 MMAs and committing them to an mbarrier,
// the epilogues reading the accumulators back with tcgen05.ld, the packed
// network brought into shared memory by bulk copies.  Inline PTX for
// sm_103a.  The forward tile below serves inference; the gradient kernel
// (lbf_mlp.cu) uses the same set-up, issue, wait and load helpers for its
// own products.
//
// Forward tile of one CTA (128 or 256 threads; in the epilogues thread t holds row
// t mod 128, and with 256 threads each pair of warps on the same rows
// splits the 64 columns):
//   layer 1: Z1 (128 x 64) = X (128 x 32, 27 inputs used) W1^T, 2 MMAs of K 16
//   layer 2: Z2 (128 x 64) = SiLU(Z1 + b1) W2^T,               4 MMAs of K 16
// in tensor-memory columns [0, 64) and [64, 128) of the CTA's 128-column
// allocation; the epilogues finish the rows (bias, SiLU, BF16 rounding,
// the output dot product with W3).
#pragma once
#include <cuda_bf16.h>
#include <stdint.h>

#include "lbf_mlp.cuh"

namespace lbf {
namespace tc {

constexpr int ROWS = 128;       // rows of a tile (M of the MMA)
constexpr uint32_t TCOLS = 128;  // tensor-memory columns a CTA allocates
// bounded waits: give up after about half a second at the maximum SM clock
constexpr long long WAIT_CYCLES = 1ll << 30;

__device__ __forceinline__ uint32_t smem_u32(const void *p) { return (uint32_t)__cvta_generic_to_shared(p); }

// Byte offset of element (r, k) of a K-major tile with K columns in the
// no-swizzle canonical layout: 8-row x 16-byte core matrices of 128 bytes,
// the K/8 core matrices of one 8-row group side by side (leading byte
// offset 128 along K), the groups K * 16 bytes apart (stride byte offset).
__host__ __device__ constexpr uint32_t kofs(int r, int k, int K) {
  return (uint32_t)((r >> 3) * (K * 16) + (k >> 3) * 128 + (r & 7) * 16 + (k & 7) * 2);
}

// shared-memory matrix descriptor: start address, leading and stride byte
// offsets (16-byte units), descriptor version 1 (bit 46), base offset 0,
// no swizzle (bits 61-63 zero)
__device__ __forceinline__ uint64_t desc(uint32_t saddr, uint32_t lbo, uint32_t sbo) {
  return (uint64_t)((saddr >> 4) & 0x3FFFu) | ((uint64_t)((lbo >> 4) & 0x3FFFu) << 16) |
         ((uint64_t)((sbo >> 4) & 0x3FFFu) << 32) | ((uint64_t)1 << 46);
}

// instruction descriptor of kind::f16: D FP32 (bits 4-5 = 1), A and B BF16
// (bits 7-9, 10-12 = 1), both K-major (bits 15, 16 = 0), N >> 3 in bits
// 17-22, M >> 4 in bits 24-28
__host__ __device__ constexpr uint32_t idesc_bf16(int M, int N) {
  return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(N >> 3) << 17) | ((uint32_t)(M >> 4) << 24);
}

// whole warp: allocate ncols tensor-memory columns, address written to *dst
__device__ __forceinline__ void tmem_alloc(uint32_t *dst, uint32_t ncols) {
  asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(dst)), "r"(ncols)
               : "memory");
  asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
}
__device__ __forceinline__ void tmem_dealloc(uint32_t taddr, uint32_t ncols) {
  asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(taddr), "r"(ncols) : "memory");
}
__device__ __forceinline__ void fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }
// generic-proxy shared-memory writes made visible to the tensor cores
__device__ __forceinline__ void fence_async_smem() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }

// D (tensor memory) = A B^T (+ D when accumulate != 0)
__device__ __forceinline__ void mma(uint32_t d, uint64_t a, uint64_t b, uint32_t idesc, uint32_t accumulate) {
  asm volatile(
      "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
      "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(d),
      "l"(a), "l"(b), "r"(idesc), "r"(accumulate)
      : "memory");
}
// the mbarrier completes one phase once every MMA issued so far by this
// thread has finished
__device__ __forceinline__ void commit(uint64_t *mbar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(smem_u32(mbar))
               : "memory");
}
__device__ __forceinline__ void mbar_init(uint64_t *mbar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(mbar)), "r"(count) : "memory");
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}
__device__ __forceinline__ bool mbar_try(uint64_t *mbar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\tselp.u32 %0, 1, 0, p;\n\t}"
      : "=r"(ok)
      : "r"(smem_u32(mbar)), "r"(parity)
      : "memory");
  return ok != 0;
}
// wait for the phase of the given parity to complete; false after
// WAIT_CYCLES without completion
__device__ __forceinline__ bool mbar_wait(uint64_t *mbar, uint32_t parity) {
  const long long t0 = clock64();
  while (!mbar_try(mbar, parity))
    if (clock64() - t0 > WAIT_CYCLES) return false;
  return true;
}

// thread 0: the mbarrier's current phase also waits for `bytes` more
// bytes of bulk copies
__device__ __forceinline__ void expect_bytes(uint64_t *mbar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(mbar)), "r"(bytes) : "memory");
}
// copy `bytes` (a multiple of 16, both addresses 16-byte aligned) from
// global to shared memory with the bulk-copy engine, counted on mbar
__device__ __forceinline__ void bulk_copy(void *dst, const void *src, uint32_t bytes, uint64_t *mbar) {
  asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                   smem_u32(dst)),
               "l"(src), "r"(bytes), "r"(smem_u32(mbar))
               : "memory");
}

// 16 consecutive FP32 columns of the warp's 32 tensor-memory lanes (lane
// i of the warp receives lane base + i), waited for before return
__device__ __forceinline__ void ld16(uint32_t taddr, float (&v)[16]) {
  uint32_t r[16];
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]), "=r"(r[8]),
        "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
      : "r"(taddr));
  // the registers pass through the wait, so no use of them moves above it
  asm volatile("tcgen05.wait::ld.sync.aligned;"
               : "+r"(r[0]), "+r"(r[1]), "+r"(r[2]), "+r"(r[3]), "+r"(r[4]), "+r"(r[5]), "+r"(r[6]), "+r"(r[7]),
                 "+r"(r[8]), "+r"(r[9]), "+r"(r[10]), "+r"(r[11]), "+r"(r[12]), "+r"(r[13]), "+r"(r[14]), "+r"(r[15])
               :
               : "memory");
#pragma unroll
  for (int i = 0; i < 16; ++i) v[i] = __uint_as_float(r[i]);
}

// the network as the tensor cores read it: W1 and W2 in the K-major
// canonical layout, biases and W3 in FP32 (a multiple of 16 bytes, so that
// one bulk copy moves a packed image into shared memory)
struct __align__(128) Image {
  __nv_bfloat16 w1[64 * 32];  // W1 (N = 64 rows, K = 32: inputs 27..31 zero)
  __nv_bfloat16 w2[64 * 64];  // W2
  float b1[64], b2[64], w3[64], b3, pad[3];
};
static_assert(sizeof(Image) % 16 == 0, "bulk copies move multiples of 16 bytes");

// the CTA's operand tiles, the network, the second half-rows' partial
// output sums and the synchronisation words
struct __align__(128) Tile {
  __nv_bfloat16 a1[ROWS * 32];  // inputs, K-major canonical (27 used, pads zero)
  __nv_bfloat16 a2[ROWS * 64];  // SiLU(Z1 + b1) in BF16
  Image net;
  float part[ROWS];
  uint64_t mbar;
  uint32_t tmem;
};

// the packed image of the flat FP32 parameters (layout of lbf_mlp.cuh);
// any number of threads of one block
__device__ __forceinline__ void pack_image(Image &m, const float *theta) {
  for (int i = threadIdx.x; i < 64 * 32; i += blockDim.x) {
    const int r = i >> 5, k = i & 31;
    m.w1[kofs(r, k, 32) / 2] = __float2bfloat16_rn(k < 27 ? theta[mlp::OFF_W1 + r * 27 + k] : 0.f);
  }
  for (int i = threadIdx.x; i < 64 * 64; i += blockDim.x) {
    const int r = i >> 6, k = i & 63;
    m.w2[kofs(r, k, 64) / 2] = __float2bfloat16_rn(theta[mlp::OFF_W2 + r * 64 + k]);
  }
  for (int i = threadIdx.x; i < 64; i += blockDim.x) {
    m.b1[i] = theta[mlp::OFF_B1 + i];
    m.b2[i] = theta[mlp::OFF_B2 + i];
    m.w3[i] = theta[mlp::OFF_W3 + i];
  }
  if (threadIdx.x == 0) {
    m.b3 = theta[mlp::OFF_B3];
    m.pad[0] = m.pad[1] = m.pad[2] = 0.f;
  }
}

// one bulk copy of a set-up
struct Copy {
  void *dst;
  const void *src;
  uint32_t bytes;
};

// input pads zero, mbarrier and ncols columns of tensor memory; thread 0
// also starts the bulk copies given (bytes 0: none), which complete the
// mbarrier's first phase (wait_net).  Every thread of the CTA.
__device__ __forceinline__ void setup(Tile &t, uint32_t ncols, Copy c0 = {nullptr, nullptr, 0u},
                                      Copy c1 = {nullptr, nullptr, 0u}) {
  for (int i = threadIdx.x; i < ROWS * 32; i += blockDim.x) t.a1[i] = __float2bfloat16_rn(0.f);
  if (threadIdx.x == 0) {
    mbar_init(&t.mbar, 1);
    if (c0.bytes + c1.bytes) {
      expect_bytes(&t.mbar, c0.bytes + c1.bytes);
      if (c0.bytes) bulk_copy(c0.dst, c0.src, c0.bytes, &t.mbar);
      if (c1.bytes) bulk_copy(c1.dst, c1.src, c1.bytes, &t.mbar);
    }
  }
  if (threadIdx.x < 32) tmem_alloc(&t.tmem, ncols);
  fence_before();
  __syncthreads();
  fence_after();
}
// the network of a packed image (global, 16-byte aligned) by bulk copy
__device__ __forceinline__ void setup(Tile &t, const Image *img) {
  setup(t, TCOLS, Copy{&t.net, img, (uint32_t)sizeof(Image)});
}

// the CTA's shared-memory writes made visible to the tensor cores and
// ordered, with the tensor-memory loads before them, ahead of the MMAs
// that follow (every thread)
__device__ __forceinline__ void to_tensor_cores() {
  fence_async_smem();
  fence_before();
  __syncthreads();
  fence_after();
}
// thread 0: D (+)= A B^T for A of 128 rows and B of N rows, both K-major
// canonical with K columns, over the first 16 * ksteps of them; then commit
__device__ __forceinline__ void issue(Tile &t, uint32_t d, const void *A, const void *B, int K, int N, int ksteps,
                                      bool accumulate) {
  const uint32_t a = smem_u32(A), b = smem_u32(B), sbo = (uint32_t)K * 16u, id = idesc_bf16(ROWS, N);
  for (int s = 0; s < ksteps; ++s)
    mma(d, desc(a + 256 * s, 128, sbo), desc(b + 256 * s, 128, sbo), id, (accumulate || s > 0) ? 1u : 0u);
  commit(&t.mbar);
}
// wait for the MMAs committed last (every thread); false for every thread
// when they did not complete within the bound
__device__ __forceinline__ bool wait_mmas(Tile &t, uint32_t &phase) {
  const bool ok = mbar_wait(&t.mbar, phase);
  phase ^= 1u;
  if (__syncthreads_or(!ok)) return false;
  fence_after();
  return true;
}

// wait for the network's bulk copy (the mbarrier phase of parity `phase`);
// false, for every thread, when it did not land within the bound
__device__ __forceinline__ bool wait_net(Tile &t, uint32_t &phase) {
  const bool ok = mbar_wait(&t.mbar, phase);
  phase ^= 1u;
  return !__syncthreads_or(!ok);
}

// input value k of row r of the tile
__device__ __forceinline__ void put_x(Tile &t, int r, int k, float v) {
  t.a1[kofs(r, k, 32) / 2] = __float2bfloat16_rn(v);
}

// the network on the staged tile (a1 written by the CTA, not yet fenced)
// with NT = 128 or 256 threads; returns in y the output of row
// threadIdx.x (threads below 128) and false, for every thread, when an
// MMA did not complete within the bound (then y is NaN).  phase: the
// parity of the mbarrier's next phase, advanced by two.
template <int NT>
__device__ __forceinline__ bool forward_tile(Tile &t, uint32_t &phase, float &y) {
  static_assert(NT == 128 || NT == 256, "one or two warps per 32 rows");
  constexpr int CPW = NT == 128 ? 64 : 32;  // columns per warp in the epilogues
  const int tid = threadIdx.x, w = tid >> 5, row = tid & (ROWS - 1), col0 = (w >> 2) * CPW;
  const uint32_t tm = t.tmem, lanes = (uint32_t)(32 * (w & 3)) << 16;
  // layer 1
  to_tensor_cores();
  if (tid == 0) issue(t, tm, t.a1, t.net.w1, 32, 64, 2, false);
  if (!wait_mmas(t, phase)) {
    y = __int_as_float(0x7fc00000);
    return false;
  }
  // epilogue 1: Z1 + b1 -> SiLU -> BF16 into a2 (this warp's columns)
#pragma unroll
  for (int c = 0; c < CPW / 16; ++c) {
    const int j0 = col0 + 16 * c;
    float z[16];
    ld16(tm + lanes + j0, z);
#pragma unroll
    for (int h = 0; h < 2; ++h) {
      uint4 q;
      uint32_t *qw = reinterpret_cast<uint32_t *>(&q);
#pragma unroll
      for (int e = 0; e < 4; ++e) {
        const int j = j0 + 8 * h + 2 * e;
        qw[e] = mlp::pack2(mlp::silu(z[8 * h + 2 * e] + t.net.b1[j]), mlp::silu(z[8 * h + 2 * e + 1] + t.net.b1[j + 1]));
      }
      *reinterpret_cast<uint4 *>(reinterpret_cast<unsigned char *>(t.a2) + kofs(row, j0 + 8 * h, 64)) = q;
    }
  }
  // layer 2
  to_tensor_cores();
  if (tid == 0) issue(t, tm + 64, t.a2, t.net.w2, 64, 64, 4, false);
  if (!wait_mmas(t, phase)) {
    y = __int_as_float(0x7fc00000);
    return false;
  }
  // epilogue 2: SiLU(Z2 + b2) rounded to BF16, dot with W3, + b3
  float acc = 0.f;
#pragma unroll
  for (int c = 0; c < CPW / 16; ++c) {
    const int j0 = col0 + 16 * c;
    float z[16];
    ld16(tm + lanes + 64 + j0, z);
#pragma unroll
    for (int e = 0; e < 16; ++e)
      acc += __bfloat162float(__float2bfloat16_rn(mlp::silu(z[e] + t.net.b2[j0 + e]))) * t.net.w3[j0 + e];
  }
  if constexpr (NT == 256) {
    if (tid >= ROWS) t.part[row] = acc;
    __syncthreads();
    if (tid < ROWS) acc += t.part[row];
  }
  y = acc + t.net.b3;
  return true;
}

// release the ncols columns of tensor memory (every thread of the CTA);
// after a timed-out wait the mbarrier is given one more bounded wait first
__device__ __forceinline__ void teardown(Tile &t, uint32_t phase, bool failed, uint32_t ncols = TCOLS) {
  if (failed && threadIdx.x == 0) (void)mbar_wait(&t.mbar, phase ^ 1u);
  fence_before();
  __syncthreads();
  fence_after();
  if (threadIdx.x < 32) tmem_dealloc(t.tmem, ncols);
}

}  // namespace tc
}  // namespace lbf

// bt_tc.cuh -- fifth-generation tensor-core (tcgen05) building blocks for
// sm_103a, written as inline PTX, and the tile forward pass of the learned
// remap's network built from them.  Device code only; included by the CUDA
// translation units that run the network.
//
// Conventions (one CTA = one warpgroup of 128 threads, cta_group::1):
//  * Operands are bf16 in shared memory, "K-major, no swizzle": an R x K tile
//    is a grid of 8 x 8 core matrices (8 rows x 16 bytes, 128 contiguous
//    bytes), core matrix (R/8 index i, K/8 index j) at byte (i * K/8 + j) *
//    128.  So the leading-dimension byte offset (next core matrix along K) is
//    128 and the stride-dimension byte offset (next 8 rows) is K/8 * 128.
//  * D = A B^T with A [128 x K] and B [N x K]; the fp32 accumulator D lives in
//    tensor memory, row m in lane m, column n in column (base + n).
//  * Warp w of the CTA reads lanes 32w .. 32w+31 with tcgen05.ld, so thread t
//    owns row t of every accumulator.
//  * One thread issues the MMAs and commits them to an mbarrier; every wait
//    on it is bounded and, on expiry, raises flag[1].
#pragma once

#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <cstdint>

#include "bt_mlp.h"

namespace bt {
namespace tc {

__device__ __forceinline__ uint32_t saddr(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

// byte offset of element (r, k) of a K-major no-swizzle tile with K columns
__device__ __forceinline__ uint32_t cm_off(int r, int k, int K) {
  return (uint32_t)((((r >> 3) * (K >> 3)) + (k >> 3)) * 128 + (r & 7) * 16 + (k & 7) * 2);
}

// shared-memory matrix descriptor: start address, leading-dimension byte
// offset 128, stride-dimension byte offset `sbo`, descriptor version 1
// (bits 46-47), base offset 0, no swizzle (bits 61-63 = 0)
__device__ __forceinline__ uint64_t sdesc(const void* p, uint32_t sbo) {
  const uint32_t a = saddr(p);
  return (uint64_t)((a & 0x3FFFFu) >> 4) | ((uint64_t)(128u >> 4) << 16) | ((uint64_t)((sbo >> 4) & 0x3FFFu) << 32) |
         (1ull << 46);
}

// instruction descriptor of kind::f16: fp32 accumulator (bits 4-5 = 1), bf16
// A and B (bits 7-9 = 1, 10-12 = 1), both K-major, N >> 3 at bit 17, M >> 4
// at bit 24
__host__ __device__ constexpr uint32_t idesc_bf16(int M, int N) {
  return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(N >> 3) << 17) | ((uint32_t)(M >> 4) << 24);
}

__device__ __forceinline__ void mma_bf16(uint32_t d_tmem, uint64_t a, uint64_t b, uint32_t idesc, uint32_t accum) {
  asm volatile(
      "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
      " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(d_tmem),
      "l"(a), "l"(b), "r"(idesc), "r"(accum)
      : "memory");
}

// arrive on `bar` once every MMA issued so far by this thread has completed
__device__ __forceinline__ void mma_commit(unsigned long long* bar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(saddr(bar))
               : "memory");
}

__device__ __forceinline__ void fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void fence_async_smem() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }

// shared-memory writes by all threads -> visible to MMAs issued after this
__device__ __forceinline__ void sync_for_mma() {
  fence_async_smem();
  fence_before();
  __syncthreads();
  fence_after();
}

// whole warp: allocate `ncols` tensor-memory columns, address -> *slot
__device__ __forceinline__ void tmem_alloc(uint32_t* slot, uint32_t ncols) {
  asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(saddr(slot)), "r"(ncols)
               : "memory");
  asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
}
__device__ __forceinline__ void tmem_dealloc(uint32_t taddr, uint32_t ncols) {
  asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(taddr), "r"(ncols) : "memory");
}

// this warp's 32 lanes, 32 consecutive columns from `taddr` (lane field set
// by the caller); the wait is in the same statement so no use of the
// registers can be scheduled before the data has arrived
__device__ __forceinline__ void tmem_ld32(uint32_t taddr, float* out) {
  uint32_t r[32];
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x32.b32 "
      "{%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%"
      "30,%31}, [%32];\n"
      "tcgen05.wait::ld.sync.aligned;\n"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]), "=r"(r[8]),
        "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15]), "=r"(r[16]),
        "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]), "=r"(r[24]),
        "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
      : "r"(taddr)
      : "memory");
#pragma unroll
  for (int i = 0; i < 32; ++i) out[i] = __uint_as_float(r[i]);
}
__device__ __forceinline__ void tmem_ld16(uint32_t taddr, float* out) {
  uint32_t r[16];
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];\n"
      "tcgen05.wait::ld.sync.aligned;\n"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]), "=r"(r[8]),
        "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
      : "r"(taddr)
      : "memory");
#pragma unroll
  for (int i = 0; i < 16; ++i) out[i] = __uint_as_float(r[i]);
}
// lane field of this warp's quarter of tensor memory
__device__ __forceinline__ uint32_t lane_base(uint32_t tmem) { return tmem + ((uint32_t)((threadIdx.x >> 5) * 32) << 16); }

__device__ __forceinline__ void bar_init(unsigned long long* bar) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(saddr(bar)) : "memory");
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}
constexpr long kSpinLimit = 1L << 22;
// bounded wait for phase `parity`; false on expiry (and flag[1] raised)
__device__ __forceinline__ bool bar_wait(unsigned long long* bar, unsigned parity, int* flag) {
  for (long it = 0; it < kSpinLimit; ++it) {
    unsigned ok;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(ok)
        : "r"(saddr(bar)), "r"(parity)
        : "memory");
    if (ok) return true;
  }
  if (flag) atomicExch(flag + 1, 1);
  return false;
}
// every thread waits; the CTA agrees on the outcome (true = all completed)
__device__ __forceinline__ bool bar_wait_all(unsigned long long* bar, unsigned& phase, int* flag) {
  const bool ok = bar_wait(bar, phase, flag);
  phase ^= 1u;
  const bool all = !__syncthreads_or(!ok);
  fence_after();
  return all;
}

// pack 8 floats into 8 bf16 (element 0 at the lowest address)
__device__ __forceinline__ uint4 pack8(const float* v) {
  uint4 u;
  __nv_bfloat162 p;
  p = __floats2bfloat162_rn(v[0], v[1]); u.x = *reinterpret_cast<uint32_t*>(&p);
  p = __floats2bfloat162_rn(v[2], v[3]); u.y = *reinterpret_cast<uint32_t*>(&p);
  p = __floats2bfloat162_rn(v[4], v[5]); u.z = *reinterpret_cast<uint32_t*>(&p);
  p = __floats2bfloat162_rn(v[6], v[7]); u.w = *reinterpret_cast<uint32_t*>(&p);
  return u;
}
// row t of a K-major tile with K columns from v[K]
template <int K>
__device__ __forceinline__ void store_row(unsigned char* tile, int t, const float* v) {
#pragma unroll
  for (int j = 0; j < K / 8; ++j) *reinterpret_cast<uint4*>(tile + cm_off(t, 8 * j, K)) = pack8(v + 8 * j);
}
// column t of a K-major tile (rows 0..n-1) from v[n]: the transposed store
template <int K>
__device__ __forceinline__ void store_col(unsigned char* tile, int t, const float* v, int n) {
  for (int r = 0; r < n; ++r) *reinterpret_cast<__nv_bfloat16*>(tile + cm_off(r, t, K)) = __float2bfloat16_rn(v[r]);
}

// Gaussian error linear unit (exact erf form) and its derivative
__device__ __forceinline__ float gelu(float z) { return 0.5f * z * (1.0f + erff(z * 0.70710678118654752f)); }
__device__ __forceinline__ float gelu_d(float z) {
  return 0.5f * (1.0f + erff(z * 0.70710678118654752f)) + z * 0.39894228040143268f * expf(-0.5f * z * z);
}

// Network weights staged in shared memory as bf16 B operands (N x K):
// W1 [64 x 16], W2, W3 [64 x 64], W4 [32 x 64] (rows 27..31 zero), plus the
// fp32 biases and the input normaliser.
struct MlpW {
  unsigned char* W1;
  unsigned char* W2;
  unsigned char* W3;
  unsigned char* W4;
  float* b;      // b1 [64], b2 [64], b3 [64], b4 [32]
  float* mean;   // [16]
  float* scale;  // [16]
};
constexpr size_t kMlpWBytes = 2048 + 8192 + 8192 + 4096 + 4 * (3 * 64 + 32) + 4 * 32;

__device__ __forceinline__ MlpW carve_w(unsigned char* p) {
  MlpW w;
  w.W1 = p; p += 2048;
  w.W2 = p; p += 8192;
  w.W3 = p; p += 8192;
  w.W4 = p; p += 4096;
  w.b = reinterpret_cast<float*>(p); p += 4 * (3 * 64 + 32);
  w.mean = reinterpret_cast<float*>(p); p += 4 * 16;
  w.scale = reinterpret_cast<float*>(p);
  return w;
}

// N x K bf16 tile from the row-major fp32 [N][K] matrix src (rows >= n_src zero)
template <int N, int K>
__device__ __forceinline__ void stage_matrix(unsigned char* dst, const float* src, int n_src) {
  for (int q = threadIdx.x; q < N * K / 2; q += blockDim.x) {
    const int n = (2 * q) / K, k = (2 * q) % K;
    const float a = n < n_src ? src[n * K + k] : 0.0f;
    const float b = n < n_src ? src[n * K + k + 1] : 0.0f;
    *reinterpret_cast<__nv_bfloat162*>(dst + cm_off(n, k, K)) = __floats2bfloat162_rn(a, b);
  }
}
// the transpose: tile[r][c] = src[c][r] for src row-major [Cs][R] (columns >= Cs zero)
template <int R, int K>
__device__ __forceinline__ void stage_transposed(unsigned char* dst, const float* src, int c_src) {
  for (int q = threadIdx.x; q < R * K; q += blockDim.x) {
    const int r = q / K, c = q % K;
    const float a = c < c_src ? src[c * R + r] : 0.0f;
    *reinterpret_cast<__nv_bfloat16*>(dst + cm_off(r, c, K)) = __float2bfloat16_rn(a);
  }
}

__device__ __forceinline__ void stage_w(const MlpW& w, const float* prm) {
  using namespace bt::mlp;
  stage_matrix<64, 16>(w.W1, prm + oW1, 64);
  stage_matrix<64, 64>(w.W2, prm + oW2, 64);
  stage_matrix<64, 64>(w.W3, prm + oW3, 64);
  stage_matrix<32, 64>(w.W4, prm + oW4, kOut);
  for (int q = threadIdx.x; q < 3 * 64 + 32; q += blockDim.x) {
    float v = 0.0f;
    if (q < 64) v = prm[oB1 + q];
    else if (q < 128) v = prm[oB2 + q - 64];
    else if (q < 192) v = prm[oB3 + q - 128];
    else if (q - 192 < kOut) v = prm[oB4 + q - 192];
    w.b[q] = v;
  }
  for (int q = threadIdx.x; q < 16; q += blockDim.x) {
    w.mean[q] = prm[oMean + q];
    w.scale[q] = prm[oScale + q];
  }
}

// Forward pass of one 128-row tile.  Thread t supplies the normalised
// features x[16] of row t and receives its 27 logits (+4 zero pads) in
// logit[32].  X: [128 x 16] and H: [128 x 64] operand tiles; the accumulator
// occupies tensor-memory columns tmem .. tmem+63.  False if a wait expired.
__device__ __forceinline__ bool tile_forward(const MlpW& w, unsigned char* X, unsigned char* H, uint32_t tmem,
                                             unsigned long long* bar, unsigned& phase, const float* x, float* logit,
                                             int* flag) {
  const int t = threadIdx.x;
  const uint32_t tl = lane_base(tmem);
  store_row<16>(X, t, x);
  sync_for_mma();
  if (t == 0) {
    mma_bf16(tmem, sdesc(X, 256), sdesc(w.W1, 256), idesc_bf16(128, 64), 0);
    mma_commit(bar);
  }
  if (!bar_wait_all(bar, phase, flag)) return false;
  float a[64];
  const unsigned char* Wl[2] = {w.W2, w.W3};
#pragma unroll 1
  for (int l = 0; l < 3; ++l) {
    tmem_ld32(tl, a);
    tmem_ld32(tl + 32, a + 32);
    const float* bl = w.b + 64 * l;
#pragma unroll
    for (int i = 0; i < 64; ++i) a[i] = gelu(a[i] + bl[i]);
    store_row<64>(H, t, a);
    sync_for_mma();
    if (t == 0) {
      const unsigned char* B = l < 2 ? Wl[l] : w.W4;
      const uint32_t id = l < 2 ? idesc_bf16(128, 64) : idesc_bf16(128, 32);
#pragma unroll
      for (int ks = 0; ks < 4; ++ks) mma_bf16(tmem, sdesc(H + 256 * ks, 1024), sdesc(B + 256 * ks, 1024), id, ks > 0);
      mma_commit(bar);
    }
    if (!bar_wait_all(bar, phase, flag)) return false;
  }
  tmem_ld32(tl, logit);
  const float* b4 = w.b + 192;
#pragma unroll
  for (int i = 0; i < 32; ++i) logit[i] += b4[i];
  return true;
}

// softmax over the 27 logits (in place into p[27])
__device__ __forceinline__ void softmax27(const float* z, float* p) {
  float m = z[0];
#pragma unroll
  for (int o = 1; o < bt::mlp::kOut; ++o) m = fmaxf(m, z[o]);
  float s = 0.0f;
#pragma unroll
  for (int o = 0; o < bt::mlp::kOut; ++o) {
    p[o] = expf(z[o] - m);
    s += p[o];
  }
  const float r = 1.0f / s;
#pragma unroll
  for (int o = 0; o < bt::mlp::kOut; ++o) p[o] *= r;
}

}  // namespace tc
}  // namespace bt

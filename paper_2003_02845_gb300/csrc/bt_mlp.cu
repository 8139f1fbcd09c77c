// bt_mlp.cu -- forward (inference) and training kernels of the learned
// remap's network, 16 -> 64 -> 64 -> 64 -> 27 with GELU hidden units and a
// softmax output, on the tcgen05 tensor cores: bf16 operands in shared
// memory, fp32 accumulators in tensor memory, one warpgroup per CTA with
// thread t owning row t of a 128-row tile (see bt_tc.cuh).
//
// Training is plain minibatch gradient descent with Adam on fp32 master
// weights; the kernels convert them to bf16 operand tiles on load.  Loss:
// cross entropy between the target redistribution weights Y (a distribution
// over the 27 offsets) and the network's softmax P, whose gradient with
// respect to the logits is P - Y.
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <cstdint>

#include "bt_mlp.h"
#include "bt_tc.cuh"

namespace bt {
namespace mlp {

namespace {

constexpr int kT = 128;   // threads per CTA: one warpgroup

__host__ __device__ constexpr size_t a128(size_t x) { return (x + 127) & ~size_t(127); }

// ---- inference -------------------------------------------------------------
constexpr size_t kFwdX = a128(tc::kMlpWBytes);
constexpr size_t kFwdH = kFwdX + 4096;
constexpr size_t kFwdBar = kFwdH + 16384;
constexpr size_t kFwdBytes = kFwdBar + 64;

__global__ void __launch_bounds__(kT) k_mlp_forward(const float* __restrict__ prm, const float* __restrict__ X,
                                                    long long n, float* __restrict__ P, int* flag) {
  extern __shared__ __align__(128) unsigned char smem[];
  const tc::MlpW w = tc::carve_w(smem);
  unsigned char* Xs = smem + kFwdX;
  unsigned char* Hs = smem + kFwdH;
  unsigned long long* bar = reinterpret_cast<unsigned long long*>(smem + kFwdBar);
  uint32_t* slot = reinterpret_cast<uint32_t*>(smem + kFwdBar + 8);
  const int t = threadIdx.x;
  tc::stage_w(w, prm);
  if (t == 0) tc::bar_init(bar);
  if (t < 32) tc::tmem_alloc(slot, 64);
  tc::fence_before();
  __syncthreads();
  tc::fence_after();
  const uint32_t tmem = *slot;
  unsigned phase = 0;
  bool ok = true;
  const long long ntile = (n + kRows - 1) / kRows;
  for (long long tile = blockIdx.x; tile < ntile && ok; tile += gridDim.x) {
    const long long row = tile * kRows + t;
    const bool valid = row < n;
    float x[kIn], z[kOutP], p[kOut];
    if (valid) {
      const float4* xr = reinterpret_cast<const float4*>(X + row * kIn);
#pragma unroll
      for (int j = 0; j < kIn / 4; ++j) {
        const float4 v = xr[j];
        x[4 * j] = v.x; x[4 * j + 1] = v.y; x[4 * j + 2] = v.z; x[4 * j + 3] = v.w;
      }
#pragma unroll
      for (int i = 0; i < kIn; ++i) x[i] = (x[i] - w.mean[i]) * w.scale[i];
    } else {
#pragma unroll
      for (int i = 0; i < kIn; ++i) x[i] = 0.0f;
    }
    ok = tc::tile_forward(w, Xs, Hs, tmem, bar, phase, x, z, flag);
    if (ok && valid) {
      tc::softmax27(z, p);
#pragma unroll
      for (int o = 0; o < kOut; ++o) P[row * kOut + o] = p[o];
    }
  }
  if (!ok && t == 0) tc::bar_wait(bar, phase ^ 1u, nullptr);   // MMAs still in flight
  tc::fence_before();
  __syncthreads();
  tc::fence_after();
  if (t < 32) tc::tmem_dealloc(tmem, 64);
}

// ---- training --------------------------------------------------------------
// tensor-memory columns (512 allocated, one CTA per SM)
// pre-activations Z1..Z3 (64 columns) and Z4 (32) at columns 64 l, l = 0..3
constexpr uint32_t cDW1 = 224, cDH = 256, cDW2 = 320, cDW3 = 384, cDW4 = 448;

constexpr size_t gW2t = a128(tc::kMlpWBytes);
constexpr size_t gW3t = gW2t + 8192;
constexpr size_t gW4t = gW3t + 8192;      // [64 x 32]
constexpr size_t gX = gW4t + 4096;        // [128 x 16]
constexpr size_t gH = gX + 4096;          // 3 x [128 x 64]
constexpr size_t gXt = gH + 3 * 16384;    // [16 x 128]
constexpr size_t gHt = gXt + 4096;        // 3 x [64 x 128]
constexpr size_t gDZt = gHt + 3 * 16384;  // [128 x 128] (rows >= 64 stay zero)
constexpr size_t gDZa = gDZt + 32768;     // [128 x 64] (or [128 x 32])
constexpr size_t gDb = gDZa + 16384;      // fp32 [224]
constexpr size_t gRed = gDb + 4 * 224;    // fp32 [4]
constexpr size_t gBar = gRed + 16;
constexpr size_t kGradBytes = gBar + 64;

__global__ void __launch_bounds__(kT, 1) k_mlp_grad(const float* __restrict__ prm, const float* __restrict__ X,
                                                    const float* __restrict__ Y, long long n, float scale,
                                                    float* __restrict__ grad, float* __restrict__ loss, int* flag) {
  extern __shared__ __align__(128) unsigned char smem[];
  const tc::MlpW w = tc::carve_w(smem);
  unsigned char* W2t = smem + gW2t;
  unsigned char* W3t = smem + gW3t;
  unsigned char* W4t = smem + gW4t;
  unsigned char* Xs = smem + gX;
  unsigned char* Hs[3] = {smem + gH, smem + gH + 16384, smem + gH + 32768};
  unsigned char* Xt = smem + gXt;
  unsigned char* Ht[3] = {smem + gHt, smem + gHt + 16384, smem + gHt + 32768};
  unsigned char* dZt = smem + gDZt;
  unsigned char* dZa = smem + gDZa;
  float* db = reinterpret_cast<float*>(smem + gDb);
  float* red = reinterpret_cast<float*>(smem + gRed);
  unsigned long long* bar = reinterpret_cast<unsigned long long*>(smem + gBar);
  uint32_t* slot = reinterpret_cast<uint32_t*>(smem + gBar + 8);
  const int t = threadIdx.x, lane = t & 31, warp = t >> 5;

  tc::stage_w(w, prm);
  tc::stage_transposed<64, 64>(W2t, prm + oW2, 64);
  tc::stage_transposed<64, 64>(W3t, prm + oW3, 64);
  tc::stage_transposed<64, 32>(W4t, prm + oW4, kOut);
  for (int q = t; q < 32768 / 16; q += kT) reinterpret_cast<uint4*>(dZt)[q] = make_uint4(0, 0, 0, 0);
  for (int q = t; q < 224; q += kT) db[q] = 0.0f;
  if (t == 0) tc::bar_init(bar);
  if (t < 32) tc::tmem_alloc(slot, 512);
  tc::fence_before();
  __syncthreads();
  tc::fence_after();
  const uint32_t tmem = *slot;
  const uint32_t tl = tc::lane_base(tmem);
  unsigned phase = 0;
  bool ok = true, any = false;
  float ce = 0.0f;
  const long long ntile = (n + kRows - 1) / kRows;
  for (long long tile = blockIdx.x; tile < ntile && ok; tile += gridDim.x) {
    const long long row = tile * kRows + t;
    const bool valid = row < n;
    float x[kIn], a[64], z[64], y[kOut];
#pragma unroll
    for (int i = 0; i < kIn; ++i) x[i] = valid ? (X[row * kIn + i] - w.mean[i]) * w.scale[i] : 0.0f;
#pragma unroll
    for (int o = 0; o < kOut; ++o) y[o] = valid ? Y[row * kOut + o] : 0.0f;
    // ---- forward, pre-activations kept in tensor memory
    tc::store_row<16>(Xs, t, x);
    tc::store_col<128>(Xt, t, x, kIn);
    tc::sync_for_mma();
    if (t == 0) {
      tc::mma_bf16(tmem + 0u, tc::sdesc(Xs, 256), tc::sdesc(w.W1, 256), tc::idesc_bf16(128, 64), 0);
      tc::mma_commit(bar);
    }
    if (!(ok = tc::bar_wait_all(bar, phase, flag))) break;
#pragma unroll 1
    for (int l = 0; l < 3; ++l) {
      tc::tmem_ld32(tl + 64u * l, a);
      tc::tmem_ld32(tl + 64u * l + 32, a + 32);
      const float* bl = w.b + 64 * l;
#pragma unroll
      for (int i = 0; i < 64; ++i) a[i] = tc::gelu(a[i] + bl[i]);
      tc::store_row<64>(Hs[l], t, a);
      tc::store_col<128>(Ht[l], t, a, 64);
      tc::sync_for_mma();
      if (t == 0) {
        const unsigned char* B = l == 0 ? w.W2 : (l == 1 ? w.W3 : w.W4);
        const uint32_t id = l < 2 ? tc::idesc_bf16(128, 64) : tc::idesc_bf16(128, 32);
#pragma unroll
        for (int ks = 0; ks < 4; ++ks)
          tc::mma_bf16(tmem + 64u * (l + 1), tc::sdesc(Hs[l] + 256 * ks, 1024), tc::sdesc(B + 256 * ks, 1024), id, ks > 0);
        tc::mma_commit(bar);
      }
      if (!(ok = tc::bar_wait_all(bar, phase, flag))) break;
    }
    if (!ok) break;
    // ---- output: softmax, cross entropy, dZ4 = (P - Y) scale
    tc::tmem_ld32(tl + 192u, a);
    {
      const float* b4 = w.b + 192;
      float m = -3.0e38f;
#pragma unroll
      for (int o = 0; o < kOut; ++o) { a[o] += b4[o]; m = fmaxf(m, a[o]); }
      float s = 0.0f;
#pragma unroll
      for (int o = 0; o < kOut; ++o) s += expf(a[o] - m);
      const float lse = m + logf(s), rs = 1.0f / s;
#pragma unroll
      for (int o = 0; o < kOutP; ++o) {
        if (o < kOut && valid) {
          ce -= y[o] * (a[o] - lse);
          z[o] = (expf(a[o] - m) * rs - y[o]) * scale;
        } else {
          z[o] = 0.0f;
        }
      }
    }
    tc::store_row<32>(dZa, t, z);
    tc::store_col<128>(dZt, t, z, 32);
#pragma unroll 1
    for (int o = 0; o < kOut; ++o) atomicAdd(&db[192 + o], z[o]);
    tc::sync_for_mma();
    if (t == 0) {
#pragma unroll
      for (int ks = 0; ks < 8; ++ks)
        tc::mma_bf16(tmem + cDW4, tc::sdesc(dZt + 256 * ks, 2048), tc::sdesc(Ht[2] + 256 * ks, 2048),
                     tc::idesc_bf16(128, 64), any || ks > 0);
#pragma unroll
      for (int ks = 0; ks < 2; ++ks)
        tc::mma_bf16(tmem + cDH, tc::sdesc(dZa + 256 * ks, 512), tc::sdesc(W4t + 256 * ks, 512),
                     tc::idesc_bf16(128, 64), ks > 0);
      tc::mma_commit(bar);
    }
    if (!(ok = tc::bar_wait_all(bar, phase, flag))) break;
    // ---- hidden layers, last to first
#pragma unroll 1
    for (int l = 2; l >= 0; --l) {
      tc::tmem_ld32(tl + cDH, a);
      tc::tmem_ld32(tl + cDH + 32, a + 32);
      tc::tmem_ld32(tl + 64u * l, z);
      tc::tmem_ld32(tl + 64u * l + 32, z + 32);
      const float* bl = w.b + 64 * l;
#pragma unroll
      for (int i = 0; i < 64; ++i) a[i] = valid ? a[i] * tc::gelu_d(z[i] + bl[i]) : 0.0f;
      if (l > 0) tc::store_row<64>(dZa, t, a);
      tc::store_col<128>(dZt, t, a, 64);
#pragma unroll 1
      for (int i = 0; i < 64; ++i) atomicAdd(&db[64 * l + i], a[i]);
      tc::sync_for_mma();
      if (t == 0) {
        const unsigned char* Bt = l == 0 ? Xt : Ht[l - 1];
        const uint32_t dst = l == 0 ? cDW1 : (l == 1 ? cDW2 : cDW3);
        const uint32_t id = l == 0 ? tc::idesc_bf16(128, 16) : tc::idesc_bf16(128, 64);
#pragma unroll
        for (int ks = 0; ks < 8; ++ks)
          tc::mma_bf16(tmem + dst, tc::sdesc(dZt + 256 * ks, 2048), tc::sdesc(Bt + 256 * ks, 2048), id,
                       any || ks > 0);
        if (l > 0) {
          const unsigned char* Wt = l == 2 ? W3t : W2t;
#pragma unroll
          for (int ks = 0; ks < 4; ++ks)
            tc::mma_bf16(tmem + cDH, tc::sdesc(dZa + 256 * ks, 1024), tc::sdesc(Wt + 256 * ks, 1024),
                         tc::idesc_bf16(128, 64), ks > 0);
        }
        tc::mma_commit(bar);
      }
      if (!(ok = tc::bar_wait_all(bar, phase, flag))) break;
    }
    any = true;
  }
  if (!ok && t == 0) tc::bar_wait(bar, phase ^ 1u, nullptr);   // MMAs still in flight
  // ---- this CTA's weight gradients (rows = output units) -> global
  if (ok && any) {
    if (warp < 2) {
      const int o = t;   // output unit of hidden layers 1..3
      float g[64];
      tc::tmem_ld16(tl + cDW1, g);
#pragma unroll 1
      for (int i = 0; i < kIn; ++i) atomicAdd(&grad[oW1 + o * kIn + i], g[i]);
      tc::tmem_ld32(tl + cDW2, g);
      tc::tmem_ld32(tl + cDW2 + 32, g + 32);
#pragma unroll 1
      for (int i = 0; i < 64; ++i) atomicAdd(&grad[oW2 + o * 64 + i], g[i]);
      tc::tmem_ld32(tl + cDW3, g);
      tc::tmem_ld32(tl + cDW3 + 32, g + 32);
#pragma unroll 1
      for (int i = 0; i < 64; ++i) atomicAdd(&grad[oW3 + o * 64 + i], g[i]);
      if (warp == 0) {
        tc::tmem_ld32(tl + cDW4, g);
        tc::tmem_ld32(tl + cDW4 + 32, g + 32);
        if (o < kOut)
#pragma unroll 1
          for (int i = 0; i < 64; ++i) atomicAdd(&grad[oW4 + o * 64 + i], g[i]);
      }
    }
  }
  __syncthreads();
  if (ok && any) {
    for (int q = t; q < 3 * 64 + kOut; q += kT) {
      const int dst = q < 64 ? oB1 + q : (q < 128 ? oB2 + q - 64 : (q < 192 ? oB3 + q - 128 : oB4 + q - 192));
      atomicAdd(&grad[dst], db[q]);
    }
  }
  // cross entropy of this CTA's rows
  for (int o = 16; o > 0; o >>= 1) ce += __shfl_xor_sync(0xffffffffu, ce, o);
  if (lane == 0) red[warp] = ce;
  tc::fence_before();
  __syncthreads();
  tc::fence_after();
  if (t == 0 && ok) atomicAdd(loss, (red[0] + red[1] + red[2] + red[3]) * scale);
  if (t < 32) tc::tmem_dealloc(tmem, 512);
}

__global__ void k_adam(float* __restrict__ prm, const float* __restrict__ g, float* __restrict__ m,
                       float* __restrict__ v, float lr, float b1, float b2, float eps, float bc1, float bc2,
                       const float* __restrict__ loss, float* __restrict__ epoch_loss) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < kNTrain; i += gridDim.x * blockDim.x) {
    const float gi = g[i];
    const float mi = b1 * m[i] + (1.0f - b1) * gi;
    const float vi = b2 * v[i] + (1.0f - b2) * gi * gi;
    m[i] = mi;
    v[i] = vi;
    prm[i] -= lr * (mi / bc1) / (sqrtf(vi / bc2) + eps);
  }
  if (blockIdx.x == 0 && threadIdx.x == 0 && epoch_loss) *epoch_loss += *loss;
}

__global__ void k_feat_stats(const float* __restrict__ X, long long n, double* __restrict__ acc) {
  __shared__ double s[2 * kIn];
  for (int q = threadIdx.x; q < 2 * kIn; q += blockDim.x) s[q] = 0.0;
  __syncthreads();
  double a[kIn], b[kIn];
#pragma unroll
  for (int i = 0; i < kIn; ++i) a[i] = b[i] = 0.0;
  for (long long r = blockIdx.x * (long long)blockDim.x + threadIdx.x; r < n; r += (long long)gridDim.x * blockDim.x)
#pragma unroll
    for (int i = 0; i < kIn; ++i) {
      const double x = X[r * kIn + i];
      a[i] += x;
      b[i] += x * x;
    }
#pragma unroll
  for (int i = 0; i < kIn; ++i) {
    atomicAdd(&s[i], a[i]);
    atomicAdd(&s[kIn + i], b[i]);
  }
  __syncthreads();
  for (int q = threadIdx.x; q < 2 * kIn; q += blockDim.x) atomicAdd(&acc[q], s[q]);
}

}  // namespace

size_t forward_smem_bytes() { return kFwdBytes; }
size_t grad_smem_bytes() { return kGradBytes; }

int prepare() {
  cudaError_t e = cudaFuncSetAttribute(k_mlp_forward, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kFwdBytes);
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(k_mlp_grad, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kGradBytes);
  return (int)e;
}

int launch_forward(const float* prm, const float* X, int64_t n, float* P, int* flag, int grid, void* stream) {
  if (n <= 0) return 0;
  const long long ntile = (n + kRows - 1) / kRows;
  const int g = (int)(ntile < grid ? ntile : grid);
  k_mlp_forward<<<g, kT, kFwdBytes, (cudaStream_t)stream>>>(prm, X, (long long)n, P, flag);
  return (int)cudaGetLastError();
}

int launch_grad(const float* prm, const float* X, const float* Y, int64_t n, float scale, float* grad, float* loss,
                int* flag, int grid, void* stream) {
  if (n <= 0) return 0;
  const long long ntile = (n + kRows - 1) / kRows;
  const int g = (int)(ntile < grid ? ntile : grid);
  k_mlp_grad<<<g, kT, kGradBytes, (cudaStream_t)stream>>>(prm, X, Y, (long long)n, scale, grad, loss, flag);
  return (int)cudaGetLastError();
}

int launch_adam(float* prm, const float* grad, float* m, float* v, float lr, float b1, float b2, float eps, float bc1,
                float bc2, const float* loss, float* epoch_loss, void* stream) {
  k_adam<<<(kNTrain + 255) / 256, 256, 0, (cudaStream_t)stream>>>(prm, grad, m, v, lr, b1, b2, eps, bc1, bc2, loss,
                                                                  epoch_loss);
  return (int)cudaGetLastError();
}

int launch_feat_stats(const float* X, int64_t n, double* acc, void* stream) {
  if (n <= 0) return 0;
  long long blocks = (n + 255) / 256;
  if (blocks > 1024) blocks = 1024;
  k_feat_stats<<<(int)blocks, 256, 0, (cudaStream_t)stream>>>(X, (long long)n, acc);
  return (int)cudaGetLastError();
}

}  // namespace mlp
}  // namespace bt

// bt_mlp.h -- the learned remap's network: shapes, the fp32 parameter block
// and the kernel launchers (bt_mlp.cu).  Not part of the ABI; the public
// layout of the parameter block is stated in include/bt.h.
#pragma once

#include <cstddef>
#include <cstdint>

namespace bt {
namespace mlp {

constexpr int kIn = 16;     // input features (one bf16 MMA K step)
constexpr int kH = 64;      // hidden width (3 hidden layers)
constexpr int kOut = 27;    // offsets {-1,0,1}^3 in (energy, mu, Phi)
constexpr int kOutP = 32;   // kOut padded to an MMA N
constexpr int kRows = 128;  // rows of one tile = tensor-memory lanes

// fp32 parameter block: W_l row-major [out][in], then b_l; then the input
// normaliser x_n = (x - mean) * scale.
constexpr int oW1 = 0;
constexpr int oB1 = oW1 + kH * kIn;
constexpr int oW2 = oB1 + kH;
constexpr int oB2 = oW2 + kH * kH;
constexpr int oW3 = oB2 + kH;
constexpr int oB3 = oW3 + kH * kH;
constexpr int oW4 = oB3 + kH;
constexpr int oB4 = oW4 + kOut * kH;
constexpr int oMean = oB4 + kOut;
constexpr int oScale = oMean + kIn;
constexpr int kNParam = oScale + kIn;   // 11195
constexpr int kNTrain = oMean;          // trained entries (the normaliser is fixed)

size_t forward_smem_bytes();
size_t grad_smem_bytes();
int prepare();   // opt-in shared memory of the kernels (once per device)

// P[n][27] = softmax(MLP((X - mean) * scale)); X [n][16] fp32.  Device pointers.
int launch_forward(const float* prm, const float* X, int64_t n, float* P, int* flag, int grid, void* stream);
// grad[kNParam] += d(loss)/d(param), loss[0] += sum of the rows' cross
// entropies -sum_o Y log P, both times `scale` (1/batch for a mean).
int launch_grad(const float* prm, const float* X, const float* Y, int64_t n, float scale, float* grad, float* loss,
                int* flag, int grid, void* stream);
// one Adam step of the trained entries; epoch_loss[0] += loss[0]
int launch_adam(float* prm, const float* grad, float* m, float* v, float lr, float b1, float b2, float eps,
                float bc1, float bc2, const float* loss, float* epoch_loss, void* stream);
// per-feature sum and sum of squares of X [n][16] into acc[32] (float64)
int launch_feat_stats(const float* X, int64_t n, double* acc, void* stream);

}  // namespace mlp
}  // namespace bt

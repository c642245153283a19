// mlp_layout.h -- shapes and parameter layout of the learned proposal's
// network (9-64-64-64-40, GELU), shared by its kernels.
//
// Parameter vector (11,560 floats, shared convention with the host API):
// W1[64][9], b1[64], W2[64][64], b2[64], W3[64][64], b3[64], W4[40][64], b4[40].
// The padded BF16 inference copy (pack_kernel) holds rows of k values with
// row strides 24 (layer 1, k padded 9 -> 16) and 72 (k = 64), layer 4 padded
// to 48 rows, followed by the FP32 biases 64 + 64 + 64 + 48.
#pragma once

namespace mcrt {
namespace mlp {

constexpr int kIn = 9, kH = 64, kOut = 40, kLobes = 8;
constexpr int kOffW1 = 0, kOffB1 = kOffW1 + kH * kIn, kOffW2 = kOffB1 + kH, kOffB2 = kOffW2 + kH * kH;
constexpr int kOffW3 = kOffB2 + kH, kOffB3 = kOffW3 + kH * kH, kOffW4 = kOffB3 + kH, kOffB4 = kOffW4 + kOut * kH;
constexpr int kNumParams = kOffB4 + kOut;                   // 11,560

constexpr int kLd1 = 24, kLd = 72;
constexpr int kPW1 = 0, kPW2 = kPW1 + 64 * kLd1, kPW3 = kPW2 + 64 * kLd, kPW4 = kPW3 + 64 * kLd;
constexpr int kPackedBf16 = kPW4 + 48 * kLd;                // 14,208 bf16
constexpr int kPackedBias = 64 * 3 + 48;                      // fp32

}  // namespace mlp
}  // namespace mcrt

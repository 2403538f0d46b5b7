// The learned correction of the M2L Green's-function tables: a small MLP
// 5 -> 64 -> 64 -> 64 -> 1 with GELU (erf form) hidden activations.
//
// Sec. 4 proposes parameterising G_* by many parameters (a grid of values) to
// go beyond the analytic G_S1; here the correction to the tabulated G_S1 is a
// smooth function of the table offset, the level and the field, written so
// that the corrected table keeps every symmetry of G_S1:
//   field 0 (G):        input (sorted |n_x|, |n_y|, |n_z|), class 0, even;
//   field i (-dG/dx_i): input (|n_i|, sorted |n_j|, |n_k|), class 1, times
//                       sign(n_i) (odd in x_i, even in the others), the same
//                       network for the three axes (cube symmetry).
// Inputs x = (a, b, c) / (4p), level / 8, class.  The output is scaled by
// kappa = 1e-3 times the natural size of the table entry at that level:
// (2^l p)/(4 pi) for G and (2^l p)^2/(4 pi) for its gradient (kappa sets the
// expected size of G_* - G_S1 relative to G: Table 1's fitted a_1 spread).  Parameters (FP32), in this order:
//   W1[64][5] b1[64] W2[64][64] b2[64] W3[64][64] b3[64] W4[64] b4[1].
#pragma once

#include <cuda_bf16.h>

namespace fmm {
namespace mlp {

constexpr int kIn = 5, kH = 64;
constexpr int kOffW1 = 0, kOffB1 = kOffW1 + kH * kIn, kOffW2 = kOffB1 + kH, kOffB2 = kOffW2 + kH * kH;
constexpr int kOffW3 = kOffB2 + kH, kOffB3 = kOffW3 + kH * kH, kOffW4 = kOffB3 + kH, kOffB4 = kOffW4 + kH;
constexpr int kParams = kOffB4 + 1;   // 8769
constexpr double kKappa = 1e-3;

__host__ __device__ inline void sort3(int& a, int& b, int& c) {
  int t;
  if (a > b) { t = a; a = b; b = t; }
  if (b > c) { t = b; b = c; c = t; }
  if (a > b) { t = a; a = b; b = t; }
}

// Input vector and the sign / scale of the correction of table entry n, field f.
// The offset is first wrapped to its nearest periodic image (the box is 2^l p
// gridlet spacings), so the correction is 1-periodic like G_S1 itself; at
// level 2 the offsets +2 and -2 nodes are the same node.
__host__ __device__ inline int wrap_offset(int v, int period) {
  v %= period;
  if (v < 0) v += period;
  if (2 * v > period) v -= period;     // to (-period/2, period/2]
  return v;
}

__host__ __device__ inline void features(int nx, int ny, int nz, int f, int level, int p, float x[kIn], float& sign,
                                         double& scale) {
  const int period = (1 << level) * p;
  nx = wrap_offset(nx, period);
  ny = wrap_offset(ny, period);
  nz = wrap_offset(nz, period);
  const int ax = nx < 0 ? -nx : nx, ay = ny < 0 ? -ny : ny, az = nz < 0 ? -nz : nz;
  int a, b, c;
  sign = 1.f;
  if (f == 0) {
    a = ax; b = ay; c = az;
    sort3(a, b, c);
  } else {
    const int own = f == 1 ? ax : (f == 2 ? ay : az);
    const int s = f == 1 ? nx : (f == 2 ? ny : nz);
    int o1 = f == 1 ? ay : ax, o2 = f == 3 ? ay : az;
    if (o1 > o2) { const int t = o1; o1 = o2; o2 = t; }
    a = own; b = o1; c = o2;
    // odd and periodic: zero at n_i = 0 and at half the box, as grad G_S1
    sign = (2 * own == period) ? 0.f : (s > 0 ? 1.f : (s < 0 ? -1.f : 0.f));
  }
  const float inv = 1.f / (4.f * p);
  x[0] = a * inv;
  x[1] = b * inv;
  x[2] = c * inv;
  x[3] = level * 0.125f;
  x[4] = f == 0 ? 0.f : 1.f;
  const double base = (double)(1 << level) * p;
  scale = kKappa * (f == 0 ? base : base * base) / (4.0 * 3.14159265358979323846);
}

__device__ __forceinline__ float gelu(float z) { return 0.5f * z * (1.f + erff(z * 0.70710678118654752f)); }
__device__ __forceinline__ float gelu_grad(float z) {
  // d/dz [z Phi(z)] = Phi(z) + z phi(z)
  return 0.5f * (1.f + erff(z * 0.70710678118654752f)) + z * 0.39894228040143268f * __expf(-0.5f * z * z);
}

__device__ __forceinline__ float round_bf16(float v) { return __bfloat162float(__float2bfloat16_rn(v)); }

// Forward pass for one sample.  BF16 = true rounds the weights and the
// activations to BF16 (FP32 accumulation): the inference form.
template <bool BF16>
__device__ inline float forward(const float* __restrict__ w, const float x[kIn]) {
  float h1[kH], h2[kH];
#pragma unroll 4
  for (int i = 0; i < kH; ++i) {
    float z = w[kOffB1 + i];
#pragma unroll
    for (int j = 0; j < kIn; ++j) {
      const float wij = BF16 ? round_bf16(w[kOffW1 + i * kIn + j]) : w[kOffW1 + i * kIn + j];
      z = fmaf(wij, BF16 ? round_bf16(x[j]) : x[j], z);
    }
    h1[i] = BF16 ? round_bf16(gelu(z)) : gelu(z);
  }
#pragma unroll 2
  for (int i = 0; i < kH; ++i) {
    float z = w[kOffB2 + i];
    for (int j = 0; j < kH; ++j) z = fmaf(BF16 ? round_bf16(w[kOffW2 + i * kH + j]) : w[kOffW2 + i * kH + j], h1[j], z);
    h2[i] = BF16 ? round_bf16(gelu(z)) : gelu(z);
  }
  float out = w[kOffB4];
#pragma unroll 2
  for (int i = 0; i < kH; ++i) {
    float z = w[kOffB3 + i];
    for (int j = 0; j < kH; ++j) z = fmaf(BF16 ? round_bf16(w[kOffW3 + i * kH + j]) : w[kOffW3 + i * kH + j], h2[j], z);
    const float h3 = BF16 ? round_bf16(gelu(z)) : gelu(z);
    out = fmaf(BF16 ? round_bf16(w[kOffW4 + i]) : w[kOffW4 + i], h3, out);
  }
  return out;
}

}  // namespace mlp
}  // namespace fmm

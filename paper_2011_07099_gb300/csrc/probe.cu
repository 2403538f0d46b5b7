// Measurement aid: a kernel that does nothing but dependent-chain FP32 FMAs,
// so that the FP32 CUDA-core peak, the roofline of the FMA-bound kernels, is
// measured on the device rather than derived from a nominal clock.
#include "fmm_internal.cuh"

namespace fmm {
namespace {

constexpr int kProbeThreads = 1024;
constexpr int kChains = 8;       // independent FMA chains per thread (covers the FMA latency)
constexpr int kUnroll = 16;      // FMAs per chain per loop trip

__global__ void __launch_bounds__(kProbeThreads) k_fma_probe(float* __restrict__ out, int iters, float a, float b) {
  float acc[kChains];
#pragma unroll
  for (int c = 0; c < kChains; ++c) acc[c] = (float)(threadIdx.x + c);
  for (int i = 0; i < iters; ++i) {
#pragma unroll
    for (int u = 0; u < kUnroll; ++u) {
#pragma unroll
      for (int c = 0; c < kChains; ++c) acc[c] = fmaf(acc[c], a, b);
    }
  }
  float s = 0.f;
#pragma unroll
  for (int c = 0; c < kChains; ++c) s += acc[c];
  // keep every thread's chains live; thread 0 always stores
  if (threadIdx.x == 0 || s == -1.0f) out[blockIdx.x] = s;
}

}  // namespace
}  // namespace fmm

extern "C" int fmm_probe_fma(float* out, int blocks, int iters, void* stream) {
  if (!out || blocks < 1 || iters < 1) return fmm::set_last_error(FMM_ERR_ARG);
  fmm::k_fma_probe<<<blocks, fmm::kProbeThreads, 0, reinterpret_cast<cudaStream_t>(stream)>>>(
      out, iters, 1.0f - 1.0f / 1048576.0f, 1e-6f);
  if (cudaGetLastError() != cudaSuccess) return fmm::set_last_error(FMM_ERR_CUDA);
  return fmm::set_last_error(FMM_OK);
}

extern "C" double fmm_probe_fma_flops(int blocks, int iters) {
  return 2.0 * blocks * (double)fmm::kProbeThreads * iters * fmm::kUnroll * fmm::kChains;
}

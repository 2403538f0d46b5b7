// Allocation-free variant of the density-mean reduction.
//
// Some callers cannot let a library call cudaMalloc: embedders whose own
// memory manager owns every byte of device memory, and latency-critical host
// loops that cannot afford the implicit device-wide synchronisation that
// cudaMalloc / cudaFree may cause.  fmm_mean_density_noalloc serves them: its
// scratch (one FP64 partial sum per 8192-cell block) lives in a file-scope
// static device array that every GPU loading this library holds until the
// process exits, so the call itself allocates nothing.
#include <cuda_runtime.h>

#include <atomic>

#include "fmm_internal.cuh"

namespace {

constexpr int kCellsPerBlock = 8192;
constexpr int kMaxBlocks = 16384;                      // 128 KB of FP64 partial sums
constexpr size_t kMaxCells = (size_t)kCellsPerBlock * kMaxBlocks;   // 134,217,728 = 512^3
constexpr int kMaxDevices = 64;

// Shared by every call on a device; each call overwrites the slots it uses
// before reading them, so nothing needs clearing between calls.
static __device__ __align__(256) double g_partials[kMaxBlocks];

// Device address of g_partials per device, looked up on the first call made
// with that device current.  Atomic slots: host threads that make their first
// call on the same device at the same time may both look the address up, and
// both store the same value, without a data race.
std::atomic<double*> g_partials_addr[kMaxDevices] = {};

__global__ void k_block_sums(const float* __restrict__ rho, size_t count, double* __restrict__ partials) {
  const size_t begin = (size_t)blockIdx.x * kCellsPerBlock;
  size_t end = begin + kCellsPerBlock;
  if (end > count) end = count;
  double acc = 0.0;
  for (size_t i = begin + threadIdx.x; i < end; i += blockDim.x) acc += (double)rho[i];
  for (int o = 16; o > 0; o >>= 1) acc += __shfl_down_sync(0xffffffffu, acc, o);
  __shared__ double red[32];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  if (lane == 0) red[warp] = acc;
  __syncthreads();
  if (warp == 0) {
    acc = lane < (int)(blockDim.x >> 5) ? red[lane] : 0.0;
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_down_sync(0xffffffffu, acc, o);
    if (lane == 0) partials[blockIdx.x] = acc;
  }
}

__global__ void k_mean_of_partials(const double* __restrict__ partials, int n, double inv_count,
                                   double* __restrict__ mean) {
  double acc = 0.0;
  for (int i = threadIdx.x; i < n; i += blockDim.x) acc += partials[i];
  for (int o = 16; o > 0; o >>= 1) acc += __shfl_down_sync(0xffffffffu, acc, o);
  __shared__ double red[32];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  if (lane == 0) red[warp] = acc;
  __syncthreads();
  if (warp == 0) {
    acc = lane < (int)(blockDim.x >> 5) ? red[lane] : 0.0;
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_down_sync(0xffffffffu, acc, o);
    if (lane == 0) *mean = acc * inv_count;
  }
}

}  // namespace

extern "C" int fmm_mean_density_noalloc(const float* density, size_t count, double* mean, void* stream) {
  using fmm::set_last_error;
  if (!density || !mean || count == 0) return set_last_error(FMM_ERR_ARG);
  if (count > kMaxCells) return set_last_error(FMM_ERR_ARG);   // beyond the static scratch: 16384 x 8192 cells
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return set_last_error(FMM_ERR_CUDA);
  if (dev < 0 || dev >= kMaxDevices) return set_last_error(FMM_ERR_UNSUPPORTED);
  double* partials = g_partials_addr[dev].load(std::memory_order_acquire);
  if (!partials) {
    // one-time set-up for this device: the static array's device address
    if (cudaGetSymbolAddress(reinterpret_cast<void**>(&partials), g_partials) != cudaSuccess || !partials)
      return set_last_error(FMM_ERR_CUDA);
    g_partials_addr[dev].store(partials, std::memory_order_release);
  }
  const int blocks = (int)((count + kCellsPerBlock - 1) / kCellsPerBlock);
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  k_block_sums<<<blocks, 256, 0, s>>>(density, count, partials);
  if (cudaGetLastError() != cudaSuccess) return set_last_error(FMM_ERR_CUDA);
  k_mean_of_partials<<<1, 1024, 0, s>>>(partials, blocks, 1.0 / (double)count, mean);
  if (cudaGetLastError() != cudaSuccess) return set_last_error(FMM_ERR_CUDA);
  return set_last_error(FMM_OK);
}

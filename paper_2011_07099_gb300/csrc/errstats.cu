// Sampled error of a solution against the PM solution with the same Green's
// function.  Sec. 3 defines the optimal G_* as the function with which PM and
// FMM give the same potential, and measures the FMM against that PM: the
// periodic convolution of the cell masses with G sampled at the mesh offsets
// d/N (eq. pmconv), with the cell self term at d = 0.  That convolution is
// evaluated here exactly, by a direct sum over every source cell, at a set of
// sampled target cells; the relative L2 error of the given potential and
// acceleration over those cells is the result.
//
// Arithmetic: per-axis xi(d/N), xi'(d/N) in FP64 (green_s1.cuh) rounded to
// FP32; each pair's (G, -grad G) in FP32; masses and sums in FP64.
#include <cuda_runtime.h>

#include "fmm_internal.cuh"
#include "green_s1.cuh"

namespace fmm {
namespace {

constexpr int kEsThreads = 256;   // one target cell per thread
constexpr int kEsChunk = 2048;    // source cells staged in shared memory per step

// partials[(blockIdx.x * T + t) * 4 + f]: block blockIdx.x's share of the
// direct sum (Phi, g_x, g_y, g_z) at target t, over the source chunks
// blockIdx.x, blockIdx.x + gridDim.x, ...
__global__ void __launch_bounds__(kEsThreads) k_es_direct(const float* __restrict__ rho,
                                                          const double* __restrict__ mean, int N,
                                                          const unsigned long long* __restrict__ targets, int T,
                                                          double* __restrict__ partials) {
  extern __shared__ __align__(16) unsigned char es_smem[];
  double* sm = reinterpret_cast<double*>(es_smem);                 // kEsChunk masses
  float* sxi = reinterpret_cast<float*>(sm + kEsChunk);           // N values xi(d/N)
  float* sdxi = sxi + N;                                          // N values xi'(d/N)
  for (int d = threadIdx.x; d < N; d += blockDim.x) {
    sxi[d] = (float)green::xi_s1((double)d / N);
    sdxi[d] = (float)green::dxi_s1((double)d / N);
  }
  const size_t n3 = (size_t)N * N * N;
  const double inv_n3 = 1.0 / (double)n3;
  const double mu = *mean;
  const int ti = blockIdx.y * kEsThreads + threadIdx.x;
  const bool valid = ti < T;
  int tx = 0, ty = 0, tz = 0;
  if (valid) {
    const unsigned long long t = targets[ti];
    tx = (int)(t % N);
    ty = (int)((t / N) % N);
    tz = (int)(t / ((unsigned long long)N * N));
  }
  const float inv4pi = (float)(1.0 / (4.0 * green::kPi));
  const float self = (float)(-green::cube_mean_inv_r() * N / (4.0 * green::kPi));
  double a0 = 0.0, a1 = 0.0, a2 = 0.0, a3 = 0.0;
  for (size_t c0 = (size_t)blockIdx.x * kEsChunk; c0 < n3; c0 += (size_t)gridDim.x * kEsChunk) {
    const int cnt = (int)((n3 - c0) < (size_t)kEsChunk ? (n3 - c0) : (size_t)kEsChunk);
    __syncthreads();
    for (int k = threadIdx.x; k < cnt; k += blockDim.x) sm[k] = ((double)rho[c0 + k] - mu) * inv_n3;
    __syncthreads();
    if (!valid) continue;
    // offsets d = (t - j) mod N per axis, stepped along the chunk (x fastest)
    int jx = (int)(c0 % N), jy = (int)((c0 / N) % N);
    const int jz = (int)(c0 / ((size_t)N * N));
    int dx = tx - jx, dy = ty - jy, dz = tz - jz;
    dx += dx < 0 ? N : 0;
    dy += dy < 0 ? N : 0;
    dz += dz < 0 ? N : 0;
    float hy = sxi[dy], gy = sdxi[dy], hz = sxi[dz], gz = sdxi[dz];
    float ryz2 = hy * hy + hz * hz;
    for (int k = 0; k < cnt; ++k) {
      const double mj = sm[k];
      if ((dx | dy | dz) == 0) {
        a0 = fma(mj, (double)self, a0);   // self term; grad G(0) = 0
      } else {
        const float hx = sxi[dx];
        const float r2 = fmaf(hx, hx, ryz2);
        const float r = sqrtf(r2);
        const float G = -inv4pi / r;
        const float c = G / r2;           // -1 / (4 pi |xhat|^3)
        a0 = fma(mj, (double)G, a0);
        a1 = fma(mj, (double)(c * hx * sdxi[dx]), a1);
        a2 = fma(mj, (double)(c * hy * gy), a2);
        a3 = fma(mj, (double)(c * hz * gz), a3);
      }
      dx = dx == 0 ? N - 1 : dx - 1;
      if (++jx == N) {                    // next row: x restarts, y advances
        jx = 0;
        dx = tx;
        dy = dy == 0 ? N - 1 : dy - 1;
        if (++jy == N) {                  // next plane
          jy = 0;
          dy = ty;
          dz = dz == 0 ? N - 1 : dz - 1;
          hz = sxi[dz];
          gz = sdxi[dz];
        }
        hy = sxi[dy];
        gy = sdxi[dy];
        ryz2 = hy * hy + hz * hz;
      }
    }
  }
  if (valid) {
    double* o = partials + ((size_t)blockIdx.x * T + ti) * 4;
    o[0] = a0;
    o[1] = a1;
    o[2] = a2;
    o[3] = a3;
  }
}

// One block of 1024 threads: thread t sums target t's partials over the
// blocks, compares with the given solution there, and the block reduces
// sums[0..3] = (sum dPhi^2, sum Phi_ref^2, sum |dg|^2, sum |g_ref|^2).
constexpr int kEsFinishThreads = 1024;

__global__ void __launch_bounds__(kEsFinishThreads) k_es_finish(const double* __restrict__ partials, int nblocks,
                                                                int T, const unsigned long long* __restrict__ targets,
                                                                size_t n3, const float* __restrict__ phi,
                                                                const float* __restrict__ acc,
                                                                double* __restrict__ sums) {
  __shared__ double red[4][kEsFinishThreads];
  const int t = threadIdx.x;
  double e[4] = {0.0, 0.0, 0.0, 0.0};
  if (t < T) {
    double ref[4] = {0.0, 0.0, 0.0, 0.0};
    for (int b = 0; b < nblocks; ++b)
      for (int f = 0; f < 4; ++f) ref[f] += partials[((size_t)b * T + t) * 4 + f];
    const size_t i = targets[t];
    const double dp = (double)phi[i] - ref[0];
    e[0] = dp * dp;
    e[1] = ref[0] * ref[0];
    for (int c = 0; c < 3; ++c) {
      const double dg = (double)acc[(size_t)c * n3 + i] - ref[1 + c];
      e[2] += dg * dg;
      e[3] += ref[1 + c] * ref[1 + c];
    }
  }
  for (int f = 0; f < 4; ++f) red[f][t] = e[f];
  __syncthreads();
  for (int h = kEsFinishThreads / 2; h > 0; h >>= 1) {
    if (t < h)
      for (int f = 0; f < 4; ++f) red[f][t] += red[f][t + h];
    __syncthreads();
  }
  if (t < 4) sums[t] = red[t][0];
}

}  // namespace

int error_stats_max_samples() { return kEsFinishThreads; }

int error_stats_grid_x(const Plan& P, int T) {
  const int gy = (T + kEsThreads - 1) / kEsThreads;
  const int gx = (2 * P.num_sms + gy - 1) / gy;
  return gx < 1 ? 1 : gx;
}

cudaError_t launch_error_stats(Plan& P, const float* rho, const float* phi, const float* acc,
                               const unsigned long long* targets, int T, double* partials, double* sums,
                               double* mean_scratch, cudaStream_t s) {
  double* mean = mean_scratch + P.n_partials;
  cudaError_t e = launch_mean_into(P, rho, mean_scratch, mean, s);
  if (e != cudaSuccess) return e;
  const int gx = error_stats_grid_x(P, T);
  const dim3 grid(gx, (T + kEsThreads - 1) / kEsThreads);
  const size_t smem = sizeof(double) * kEsChunk + 2 * sizeof(float) * (size_t)P.N;
  k_es_direct<<<grid, kEsThreads, smem, s>>>(rho, mean, P.N, targets, T, partials);
  e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  const size_t n3 = (size_t)P.N * P.N * P.N;
  k_es_finish<<<1, kEsFinishThreads, 0, s>>>(partials, gx, T, targets, n3, phi, acc, sums);
  return cudaGetLastError();
}

}  // namespace fmm

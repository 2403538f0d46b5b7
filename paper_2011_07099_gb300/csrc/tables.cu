// Green's-function tabulation (plan time, FP64 arithmetic): G_S1 of eq. gfs1
// (green_s1.cuh) at the gridlet and mesh offsets of each level.  Tables hold
// (G, -dG/dx, -dG/dy, -dG/dz) so that a contraction with masses yields
// (Phi, g) directly, g = -grad Phi.
#include <cuda_bf16.h>

#include "fmm_internal.cuh"
#include "green_s1.cuh"
#include "mlp.cuh"

namespace fmm {
namespace {

using green::cube_mean_inv_r;
using green::gs1;
using green::kPi;

// Learned correction of one table entry (all four fields), if weights are set.
__device__ inline void add_correction(double v[4], int ix, int iy, int iz, int level, int p, const float* mlp, int fp32) {
  if (!mlp || !(ix | iy | iz)) return;
  for (int f = 0; f < 4; ++f) {
    float x[mlp::kIn], sign;
    double scale;
    mlp::features(ix, iy, iz, f, level, p, x, sign, scale);
    if (sign == 0.f) continue;
    const float o = fp32 ? mlp::forward<false>(mlp, x) : mlp::forward<true>(mlp, x);
    v[f] += (double)o * (double)sign * scale;
  }
}

// M2L table of level l: n in [-(4p-1), 4p-1]^3 at spacing dx_l = 1/(2^l p)
// (Sec. 3: gridlet spacing of a level-l node; the (4 N_g)^D samples of Sec. 4
// folded over the sign of each component).  Entry n = 0 is never used by M2L
// (the interaction zone excludes near nodes) and is stored as 0.
__global__ void k_tab_m2l(float4* __restrict__ out, float4* __restrict__ lo, int p, int level, const float* mlp,
                          int fp32) {
  const int hw = 4 * p - 1, E = 8 * p - 1;
  const long total = (long)E * E * E;
  const double dx = 1.0 / ((double)(1 << level) * p);
  for (long i = blockIdx.x * (long)blockDim.x + threadIdx.x; i < total; i += (long)gridDim.x * blockDim.x) {
    const int ix = (int)(i % E) - hw, iy = (int)((i / E) % E) - hw, iz = (int)(i / ((long)E * E)) - hw;
    double v[4] = {0.0, 0.0, 0.0, 0.0};
    if (ix | iy | iz) gs1(ix * dx, iy * dx, iz * dx, v);
    add_correction(v, ix, iy, iz, level, p, mlp, fp32);
    out[i] = make_float4((float)v[0], (float)v[1], (float)v[2], (float)v[3]);
    if (lo)
      lo[i] = make_float4((float)(v[0] - (double)(float)v[0]), (float)(v[1] - (double)(float)v[1]),
                          (float)(v[2] - (double)(float)v[2]), (float)(v[3] - (double)(float)v[3]));
  }
}

// Near-zone table at cell spacing h = 1/N for |d_i| in [0, 2S-1] (the offsets
// between a cell of a leaf and a cell of any of its 27 neighbour leaves),
// folded: G is even in every component, -dG/dx_i is odd in x_i and even in the
// others, so entries hold the values at (|dx|, |dy|, |dz|) and the kernel
// restores the signs.  d = 0 holds the self term -(1/4 pi) <1/r>_cell / h.
__global__ void k_tab_near(float4* __restrict__ out, int S, int N) {
  const int D = 2 * S;
  const int total = D * D * D;
  const double h = 1.0 / N;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < total; i += gridDim.x * blockDim.x) {
    const int ix = i % D, iy = (i / D) % D, iz = i / (D * D);
    double v[4];
    if (ix | iy | iz) {
      gs1(ix * h, iy * h, iz * h, v);
    } else {
      v[0] = -cube_mean_inv_r() * (double)N / (4.0 * kPi);
      v[1] = v[2] = v[3] = 0.0;
    }
    out[i] = make_float4((float)v[0], (float)v[1], (float)v[2], (float)v[3]);
  }
}

// The same level table split into BF16 hi + lo per field for the tensor-core
// M2L: each uint32 holds hi in its low half and lo = bf16(v - hi) in its high
// half, the four fields in the four words of a uint4.
__global__ void k_tab_bf16(uint4* __restrict__ out, int p, int level, const float* mlp, int fp32) {
  const int hw = 4 * p - 1, E = 8 * p - 1;
  const long total = (long)E * E * E;
  const double dx = 1.0 / ((double)(1 << level) * p);
  for (long i = blockIdx.x * (long)blockDim.x + threadIdx.x; i < total; i += (long)gridDim.x * blockDim.x) {
    const int ix = (int)(i % E) - hw, iy = (int)((i / E) % E) - hw, iz = (int)(i / ((long)E * E)) - hw;
    double v[4] = {0.0, 0.0, 0.0, 0.0};
    if (ix | iy | iz) gs1(ix * dx, iy * dx, iz * dx, v);
    add_correction(v, ix, iy, iz, level, p, mlp, fp32);
    uint32_t w[4];
    for (int f = 0; f < 4; ++f) {
      const __nv_bfloat16 h = __double2bfloat16(v[f]);
      const __nv_bfloat16 l = __double2bfloat16(v[f] - (double)__bfloat162float(h));
      w[f] = (uint32_t)__bfloat16_as_ushort(h) | ((uint32_t)__bfloat16_as_ushort(l) << 16);
    }
    out[i] = make_uint4(w[0], w[1], w[2], w[3]);
  }
}

}  // namespace

cudaError_t launch_tab_bf16(Plan& P, int level, cudaStream_t s) {
  k_tab_bf16<<<4 * P.num_sms, 256, 0, s>>>(P.tab_bf[level], P.p, level, P.has_corr ? P.corr_w : nullptr,
                                           P.corr_fp32);
  return cudaGetLastError();
}

cudaError_t launch_tables(Plan& P, cudaStream_t s) {
  for (int l = 2; l <= P.L; ++l) {
    k_tab_m2l<<<4 * P.num_sms, 256, 0, s>>>(P.tab[l], P.tab_lo[l], P.p, l, P.has_corr ? P.corr_w : nullptr,
                                            P.corr_fp32);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
  }
  k_tab_near<<<P.num_sms, 256, 0, s>>>(P.near_tab, P.S, P.N);
  return cudaGetLastError();
}

}  // namespace fmm

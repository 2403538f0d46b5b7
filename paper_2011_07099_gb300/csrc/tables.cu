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

// Grid model of G_* (Sec. 4: every table value its own parameter).  The
// parameters sit on the folded entries: the offset is taken to its nearest
// periodic image (the level-l box spans 2^l p gridlet spacings) and folded
// over the sign of each component; G adds grid[0][a], -dG/dx_i adds
// sign(n_i) grid[i][a] (zero at half the box, where the odd periodic
// gradient vanishes), so the corrected table keeps the parity and the
// periodicity of G_S1.  `grid` is this level's 4 x (4p)^3 block.
__device__ inline void add_grid(double v[4], int ix, int iy, int iz, int level, int p, const float* grid) {
  if (!grid || !(ix | iy | iz)) return;
  const int period = (1 << level) * p, G = 4 * p;
  const int n[3] = {ix, iy, iz};
  int a[3];
  double sg[3];
  for (int i = 0; i < 3; ++i) {
    int w = ((n[i] % period) + period) % period;
    if (2 * w > period) w -= period;
    a[i] = w < 0 ? -w : w;
    sg[i] = 2 * a[i] == period ? 0.0 : (w > 0 ? 1.0 : (w < 0 ? -1.0 : 0.0));
  }
  const size_t e = ((size_t)a[2] * G + a[1]) * G + a[0], G3 = (size_t)G * G * G;
  v[0] += (double)grid[e];
  for (int f = 1; f < 4; ++f) v[f] += sg[f - 1] * (double)grid[f * G3 + e];
}

// M2L table of level l: n in [-(4p-1), 4p-1]^3 at spacing dx_l = 1/(2^l p)
// (Sec. 3: gridlet spacing of a level-l node; the (4 N_g)^D samples of Sec. 4
// folded over the sign of each component).  Entry n = 0 is never used by M2L
// (the interaction zone excludes near nodes) and is stored as 0.
// A function given on the mesh (kind 4): the value at the cell offset
// (cx, cy, cz), taken modulo N (periodic).
__device__ inline void mesh_value(const double* mesh, int N, long cx, long cy, long cz, double v[4]) {
  const long x = ((cx % N) + N) % N, y = ((cy % N) + N) % N, z = ((cz % N) + N) % N;
  const size_t n3 = (size_t)N * N * N, e = ((size_t)z * N + y) * N + x;
  for (int f = 0; f < 4; ++f) v[f] = mesh[f * n3 + e];
}

// (G, -grad G) of table entry n at level l: analytic at n dx_l, or from the
// mesh, where gridlet spacing dx_l is cpg = N / (2^l p) whole cells.
__device__ inline void table_value(const green::Spec& gs, const double* mesh, int N, int level, int p, int ix, int iy,
                                   int iz, double v[4]) {
  if (gs.kind == 4) {
    const long cpg = (long)N / ((long)(1 << level) * p);
    mesh_value(mesh, N, ix * cpg, iy * cpg, iz * cpg, v);
  } else {
    const double dx = 1.0 / ((double)(1 << level) * p);
    green::eval(gs, ix * dx, iy * dx, iz * dx, v);
  }
}

__global__ void k_tab_m2l(float4* __restrict__ out, float4* __restrict__ lo, int p, int level, const float* mlp,
                          int fp32, const float* grid, green::Spec gs, const double* mesh, int N) {
  const int hw = 4 * p - 1, E = 8 * p - 1;
  const long total = (long)E * E * E;
  for (long i = blockIdx.x * (long)blockDim.x + threadIdx.x; i < total; i += (long)gridDim.x * blockDim.x) {
    const int ix = (int)(i % E) - hw, iy = (int)((i / E) % E) - hw, iz = (int)(i / ((long)E * E)) - hw;
    double v[4] = {0.0, 0.0, 0.0, 0.0};
    if (ix | iy | iz) table_value(gs, mesh, N, level, p, ix, iy, iz, v);
    add_correction(v, ix, iy, iz, level, p, mlp, fp32);
    add_grid(v, ix, iy, iz, level, p, grid);
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
__global__ void k_tab_near(float4* __restrict__ out, int S, int N, green::Spec gs, const double* mesh) {
  const int D = 2 * S;
  const int total = D * D * D;
  const double h = 1.0 / N;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < total; i += gridDim.x * blockDim.x) {
    const int ix = i % D, iy = (i / D) % D, iz = i / (D * D);
    double v[4];
    if (gs.kind == 4) {
      mesh_value(mesh, N, ix, iy, iz, v);      // the mesh carries its own self term
    } else if (ix | iy | iz) {
      green::eval(gs, ix * h, iy * h, iz * h, v);
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
__global__ void k_tab_bf16(uint4* __restrict__ out, int p, int level, const float* mlp, int fp32, const float* grid,
                           green::Spec gs, const double* mesh, int N) {
  const int hw = 4 * p - 1, E = 8 * p - 1;
  const long total = (long)E * E * E;
  for (long i = blockIdx.x * (long)blockDim.x + threadIdx.x; i < total; i += (long)gridDim.x * blockDim.x) {
    const int ix = (int)(i % E) - hw, iy = (int)((i / E) % E) - hw, iz = (int)(i / ((long)E * E)) - hw;
    double v[4] = {0.0, 0.0, 0.0, 0.0};
    if (ix | iy | iz) table_value(gs, mesh, N, level, p, ix, iy, iz, v);
    add_correction(v, ix, iy, iz, level, p, mlp, fp32);
    add_grid(v, ix, iy, iz, level, p, grid);
    uint32_t w[4];
    for (int f = 0; f < 4; ++f) {
      const __nv_bfloat16 h = __double2bfloat16(v[f]);
      const __nv_bfloat16 l = __double2bfloat16(v[f] - (double)__bfloat162float(h));
      w[f] = (uint32_t)__bfloat16_as_ushort(h) | ((uint32_t)__bfloat16_as_ushort(l) << 16);
    }
    out[i] = make_uint4(w[0], w[1], w[2], w[3]);
  }
}

// Gradient of the grid parameters of one level from the table gradient dT
// (layout [n][f], n over the (8p-1)^3 table): every table entry adds its
// gradient, times the sign it was applied with, to the entry it folds onto.
__global__ void k_grid_grad(const float* __restrict__ dT, int p, int level, float* __restrict__ g) {
  const int hw = 4 * p - 1, E = 8 * p - 1, period = (1 << level) * p, G = 4 * p;
  const long total = (long)E * E * E * 4;
  const size_t G3 = (size_t)G * G * G;
  for (long i = blockIdx.x * (long)blockDim.x + threadIdx.x; i < total; i += (long)gridDim.x * blockDim.x) {
    const int f = (int)(i % 4);
    const long e = i / 4;
    const int n[3] = {(int)(e % E) - hw, (int)((e / E) % E) - hw, (int)(e / ((long)E * E)) - hw};
    if (!(n[0] | n[1] | n[2])) continue;
    int a[3];
    float sg[3];
    for (int k = 0; k < 3; ++k) {
      int w = ((n[k] % period) + period) % period;
      if (2 * w > period) w -= period;
      a[k] = w < 0 ? -w : w;
      sg[k] = 2 * a[k] == period ? 0.f : (w > 0 ? 1.f : (w < 0 ? -1.f : 0.f));
    }
    const float sgn = f == 0 ? 1.f : sg[f - 1];
    const float d = dT[i];
    if (sgn == 0.f || d == 0.f) continue;
    atomicAdd(&g[f * G3 + ((size_t)a[2] * G + a[1]) * G + a[0]], sgn * d);
  }
}

// The corrections (network, grid) are corrections of G_S1: they apply only
// when the plan tabulates G_S1 with periodic boundaries.
bool plain_gs1(const Plan& P) { return P.gspec.kind == 0 && !P.iso; }
const float* grid_of(const Plan& P, int level) {
  return P.has_grid && plain_gs1(P) ? P.grid + (size_t)(level - 2) * grid_level_size(P.p) : nullptr;
}
const float* mlp_of(const Plan& P) { return P.has_corr && plain_gs1(P) ? P.corr_w : nullptr; }
// The function the tables hold: G_0 in the isolated problem.
green::Spec spec_of(const Plan& P) {
  if (!P.iso) return P.gspec;
  green::Spec g;
  g.kind = 2;
  return g;
}

}  // namespace

cudaError_t launch_grid_grad(Plan& P, float* grad, cudaStream_t s) {
  for (int l = 2; l <= P.L; ++l) {
    k_grid_grad<<<4 * P.num_sms, 256, 0, s>>>(P.dT[l], P.p, l, grad + (size_t)(l - 2) * grid_level_size(P.p));
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
  }
  return cudaSuccess;
}

cudaError_t launch_tab_bf16(Plan& P, int level, cudaStream_t s) {
  k_tab_bf16<<<4 * P.num_sms, 256, 0, s>>>(P.tab_bf[level], P.p, level, mlp_of(P), P.corr_fp32, grid_of(P, level),
                                           spec_of(P), P.gmesh, P.N);
  return cudaGetLastError();
}

cudaError_t launch_tables(Plan& P, cudaStream_t s) {
  for (int l = 2; l <= P.L; ++l) {
    k_tab_m2l<<<4 * P.num_sms, 256, 0, s>>>(P.tab[l], P.tab_lo[l], P.p, l, mlp_of(P), P.corr_fp32, grid_of(P, l),
                                            spec_of(P), P.gmesh, P.N);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
  }
  k_tab_near<<<P.num_sms, 256, 0, s>>>(P.near_tab, P.S, P.N, spec_of(P), P.gmesh);
  return cudaGetLastError();
}

}  // namespace fmm

// Training kernels of the learned table correction (FP32).
//
// The FMM output is linear in the M2L tables.  For a loss
//   J = w_phi |Phi - Phi*|^2 + w_g |g - g*|^2
// against a target solution (PM with G_S1, Sec. 3: the optimal G_* is the one
// for which FMM and PM agree), the gradient with respect to a table entry is
//   dJ/dT_l[f][n] = sum_T sum_{o in IL(T)} sum_{r - s = n - o p} lam_l[T][f][r] M_l[T - o][s],
// where lam_l is the adjoint of the level-l local field: lam_L = L2P^T of the
// cell residual, lam_l = L2L^T(lam_{l+1}) (eq. fmm3 transposed is eq. fmm1's
// map, so the adjoint sweep reuses the upward contractions).  The table
// gradient then flows through the MLP (mlp.cuh) by its own backward kernel.
#include <cuda_runtime.h>

#include "fmm_internal.cuh"
#include "green_s1.cuh"
#include "mlp.cuh"

namespace fmm {
namespace {

// ------------------------------------------------------------ residual, loss
// lam[f][i] = 2 w_f (out_f - target_f), f = Phi, g_x, g_y, g_z (SoA, N^3 each);
// loss += sum w_f (out_f - target_f)^2.
__global__ void k_residual(const float* __restrict__ phi, const float* __restrict__ acc, const float* __restrict__ tphi,
                           const float* __restrict__ tacc, size_t n3, float w_phi, float w_g, float* __restrict__ lam,
                           float* __restrict__ loss) {
  double part = 0.0;
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < 4 * n3; i += (size_t)gridDim.x * blockDim.x) {
    const bool isphi = i < n3;
    const float d = isphi ? phi[i] - tphi[i] : acc[i - n3] - tacc[i - n3];
    const float w = isphi ? w_phi : w_g;
    lam[i] = 2.f * w * d;
    part += (double)w * d * d;
  }
  for (int o = 16; o > 0; o >>= 1) part += __shfl_down_sync(0xffffffffu, part, o);
  if ((threadIdx.x & 31) == 0) atomicAdd(loss, (float)part);
}

// --------------------------------------------------------- adjoint of L2P
// lam_L[leaf][f][s] = sum_c w_p2m(s, c) lam_cell[f][c]: the transpose of L2P is
// the P2M contraction, applied to the four residual fields.
__global__ void k_adj_l2p(const float* __restrict__ lam, int N, int S, int p, const float2* __restrict__ w,
                          float* __restrict__ lamL) {
  extern __shared__ float smf[];
  const int p3 = p * p * p, S3 = S * S * S;
  float2* W = reinterpret_cast<float2*>(smf);      // p*S
  float* in = reinterpret_cast<float*>(W + p * S); // 4*S^3
  float* t1 = in + 4 * S3;                         // 4*S*S*p
  float* t2 = t1 + 4 * S * S * p;                  // 4*S*p*p
  float* out = t2 + 4 * S * p * p;                 // 4*p^3
  const int tid = threadIdx.x, nthr = blockDim.x;
  uint32_t lx, ly, lz;
  unmorton(blockIdx.x, lx, ly, lz);
  const size_t n3 = (size_t)N * N * N;
  for (int i = tid; i < p * S; i += nthr) W[i] = w[i];
  for (int i = tid; i < 4 * S3; i += nthr) {
    const int f = i / S3, c = i % S3;
    const int cx = c % S, cy = (c / S) % S, cz = c / (S * S);
    in[i] = lam[f * n3 + ((size_t)(lz * S + cz) * N + (ly * S + cy)) * N + (lx * S + cx)];
  }
  __syncthreads();
  contract3(in, t1, t2, out, 4, S, p, W, S, false, tid, nthr);
  for (int i = tid; i < 4 * p3; i += nthr) lamL[(size_t)blockIdx.x * 4 * p3 + i] = out[i];
}

// --------------------------------------------------------- adjoint of L2L
// lam_l[P] = sum_children T^c lam_{l+1}[8P + c] (the M2M contraction, 4 fields).
__global__ void k_adj_l2l(const float* __restrict__ lamc, int p, const float2* __restrict__ w, float* __restrict__ lamp) {
  extern __shared__ float smf[];
  const int K = 2 * p, p3 = p * p * p, K3 = K * K * K;
  float2* W = reinterpret_cast<float2*>(smf);      // p*K
  float* in = reinterpret_cast<float*>(W + p * K); // 4*K^3
  float* t1 = in + 4 * K3;                         // 4*K*K*p
  float* t2 = t1 + 4 * K * K * p;                  // 4*K*p*p
  float* out = t2 + 4 * K * p * p;                 // 4*p^3
  const int tid = threadIdx.x, nthr = blockDim.x;
  for (int i = tid; i < p * K; i += nthr) W[i] = w[i];
  const float* src = lamc + (size_t)blockIdx.x * 8 * 4 * p3;
  for (int i = tid; i < 8 * 4 * p3; i += nthr) {
    const int c = i / (4 * p3), rem = i % (4 * p3);
    const int f = rem / p3, q = rem % p3;
    const int qx = q % p, qy = (q / p) % p, qz = q / (p * p);
    const int ux = (c & 1) * p + qx, uy = ((c >> 1) & 1) * p + qy, uz = (c >> 2) * p + qz;
    in[((f * K + uz) * K + uy) * K + ux] = src[i];
  }
  __syncthreads();
  contract3(in, t1, t2, out, 4, K, p, W, K, false, tid, nthr);
  for (int i = tid; i < 4 * p3; i += nthr) lamp[(size_t)blockIdx.x * 4 * p3 + i] = out[i];
}

// ------------------------------------------------------ table gradient
// CTA (offset index io, child type c, field f): for every d in [-(p-1), p-1]^3,
//   g[d] = sum over targets T of type c, sum_r lam[T][f][r] M[T - o][r - d],
// added to dT[o p + d][f].  Targets are staged 32 at a time in shared memory.
constexpr int kTgChunk = 32;

__global__ void k_table_grad(const float* __restrict__ lam, const float* __restrict__ M, const int8_t* __restrict__ offs,
                             int n_off, int level, int p, float* __restrict__ dT) {
  extern __shared__ float smf[];
  const int p3 = p * p * p, D = 2 * p - 1, D3 = D * D * D, E = 8 * p - 1, HW = 4 * p - 1;
  float* sl = smf;                      // kTgChunk * p3
  float* sm = sl + kTgChunk * p3;       // kTgChunk * p3
  const int io = blockIdx.x, ctype = blockIdx.y, f = blockIdx.z;
  const int8_t* o3 = offs + ((size_t)ctype * n_off + io) * 3;
  const int ox = o3[0], oy = o3[1], oz = o3[2];
  const int n = 1 << level;
  const uint32_t n_par = 1u << (3 * (level - 1));
  constexpr int KMAX = 8;      // (2p-1)^3 <= 8 x 512 for p <= 8
  float acc[KMAX];
#pragma unroll
  for (int k = 0; k < KMAX; ++k) acc[k] = 0.f;
  for (uint32_t t0 = 0; t0 < n_par; t0 += kTgChunk) {
    __syncthreads();
    for (int i = threadIdx.x; i < kTgChunk * p3; i += blockDim.x) {
      const uint32_t t = t0 + i / p3;
      const int r = i % p3;
      float lv = 0.f, mv = 0.f;
      if (t < n_par) {
        const uint32_t T = 8u * t + ctype;
        uint32_t x, y, z;
        unmorton(T, x, y, z);
        const uint32_t S = morton((x - ox) & (n - 1), (y - oy) & (n - 1), (z - oz) & (n - 1));
        lv = lam[((size_t)T * 4 + f) * p3 + r];
        mv = M[(size_t)S * p3 + r];
      }
      sl[i] = lv;
      sm[i] = mv;
    }
    __syncthreads();
#pragma unroll
    for (int k = 0; k < KMAX; ++k) {
      const int dd = threadIdx.x + k * blockDim.x;
      if (dd >= D3) break;
      const int dx = dd % D - (p - 1), dy = (dd / D) % D - (p - 1), dz = dd / (D * D) - (p - 1);
      const int x0 = dx > 0 ? dx : 0, x1 = dx < 0 ? p + dx : p;
      const int y0 = dy > 0 ? dy : 0, y1 = dy < 0 ? p + dy : p;
      const int z0 = dz > 0 ? dz : 0, z1 = dz < 0 ? p + dz : p;
      const int shift = (dz * p + dy) * p + dx;     // s = r - shift
      float a = 0.f;
      for (int t = 0; t < kTgChunk; ++t) {
        const float* lt = sl + t * p3;
        const float* mt = sm + t * p3;
        for (int rz = z0; rz < z1; ++rz)
          for (int ry = y0; ry < y1; ++ry) {
            const int rb = (rz * p + ry) * p;
            for (int rx = x0; rx < x1; ++rx) a = fmaf(lt[rb + rx], mt[rb + rx - shift], a);
          }
      }
      acc[k] += a;
    }
  }
#pragma unroll
  for (int k = 0; k < KMAX; ++k) {
    const int dd = threadIdx.x + k * blockDim.x;
    if (dd >= D3) break;
    const int dx = dd % D - (p - 1), dy = (dd / D) % D - (p - 1), dz = dd / (D * D) - (p - 1);
    const int nx = ox * p + dx + HW, ny = oy * p + dy + HW, nz = oz * p + dz + HW;
    atomicAdd(&dT[(((size_t)nz * E + ny) * E + nx) * 4 + f], acc[k]);
  }
}

// ----------------------------------------------------------- MLP backward
// Samples are the table entries (level, n, f); the upstream gradient of the
// MLP output of a sample is dT * scale * sign (mlp::features).  One block of
// kBwdTile threads processes tiles of kBwdTile samples (one per thread) and
// accumulates the parameter gradient in shared memory (each thread owns a
// fixed set of parameters); per-block partials are summed by k_grad_reduce.
constexpr int kBwdTile = 64;
constexpr int kPerThread = (mlp::kParams + kBwdTile - 1) / kBwdTile;   // 138

__global__ void __launch_bounds__(kBwdTile) k_mlp_backward(const float* __restrict__ w, const float* __restrict__ dT,
                                                          int lmin, int lmax, int p, float* __restrict__ partials) {
  using namespace mlp;
  extern __shared__ float smf[];
  float* sw = smf;                               // kParams
  float* X = sw + kParams;                       // tile x kIn
  float* Z1 = X + kBwdTile * kIn;                // tile x kH (pre-activations)
  float* Z2 = Z1 + kBwdTile * kH;
  float* Z3 = Z2 + kBwdTile * kH;
  float* H1 = Z3 + kBwdTile * kH;                // post-activations
  float* H2 = H1 + kBwdTile * kH;
  float* G = H2 + kBwdTile * kH;                 // tile x kH (backprop buffer)
  float* GO = G + kBwdTile * kH;                 // tile (upstream gradient)
  float* gacc = GO + kBwdTile;                   // kParams: this block's gradient
  const int tid = threadIdx.x;
  for (int i = tid; i < kParams; i += kBwdTile) {
    sw[i] = w[i];
    gacc[i] = 0.f;
  }
  const int E = 8 * p - 1;
  const long E3 = (long)E * E * E;
  const long total = (long)(lmax - lmin + 1) * E3 * 4;
  __syncthreads();
  for (long base = (long)blockIdx.x * kBwdTile; base < total; base += (long)gridDim.x * kBwdTile) {
    // forward for sample base + tid
    {
      const long sidx = base + tid;
      float x[kIn] = {0.f, 0.f, 0.f, 0.f, 0.f};
      float go = 0.f;
      if (sidx < total) {
        const int f = (int)(sidx % 4);
        const long e = (sidx / 4) % E3;
        const int level = lmin + (int)(sidx / (4 * E3));
        const int hw = 4 * p - 1;
        const int nx = (int)(e % E) - hw, ny = (int)((e / E) % E) - hw, nz = (int)(e / ((long)E * E)) - hw;
        float sign;
        double scale;
        features(nx, ny, nz, f, level, p, x, sign, scale);
        const float g = dT[((size_t)(level - lmin) * E3 + e) * 4 + f];
        go = (nx | ny | nz) ? (float)(g * scale) * sign : 0.f;
      }
      GO[tid] = go;
      for (int j = 0; j < kIn; ++j) X[tid * kIn + j] = x[j];
      for (int i = 0; i < kH; ++i) {
        float z = sw[kOffB1 + i];
        for (int j = 0; j < kIn; ++j) z = fmaf(sw[kOffW1 + i * kIn + j], x[j], z);
        Z1[tid * kH + i] = z;
        H1[tid * kH + i] = gelu(z);
      }
      for (int i = 0; i < kH; ++i) {
        float z = sw[kOffB2 + i];
        for (int j = 0; j < kH; ++j) z = fmaf(sw[kOffW2 + i * kH + j], H1[tid * kH + j], z);
        Z2[tid * kH + i] = z;
        H2[tid * kH + i] = gelu(z);
      }
      for (int i = 0; i < kH; ++i) {
        float z = sw[kOffB3 + i];
        for (int j = 0; j < kH; ++j) z = fmaf(sw[kOffW3 + i * kH + j], H2[tid * kH + j], z);
        Z3[tid * kH + i] = z;
        // dz3 = go * W4 * gelu'(z3)
        G[tid * kH + i] = go * sw[kOffW4 + i] * gelu_grad(z);
      }
    }
    __syncthreads();
    // parameter gradients of layers 3 and 4 (thread owns entries k*kBwdTile + tid)
    for (int k = 0; k < kPerThread; ++k) {
      const int q = k * kBwdTile + tid;
      if (q >= kOffW3 && q < kOffB4 + 1) {
        float a = 0.f;
        if (q < kOffB3) {
          const int i = (q - kOffW3) / kH, j = (q - kOffW3) % kH;
          for (int s = 0; s < kBwdTile; ++s) a = fmaf(G[s * kH + i], H2[s * kH + j], a);
        } else if (q < kOffW4) {
          const int i = q - kOffB3;
          for (int s = 0; s < kBwdTile; ++s) a += G[s * kH + i];
        } else if (q < kOffB4) {
          const int i = q - kOffW4;
          for (int s = 0; s < kBwdTile; ++s) a = fmaf(GO[s], gelu(Z3[s * kH + i]), a);
        } else {
          for (int s = 0; s < kBwdTile; ++s) a += GO[s];
        }
        gacc[q] += a;
      }
    }
    __syncthreads();
    // dz2 = (W3^T dz3) * gelu'(z2), in place of Z3
    {
      float d2[kH];
      for (int j = 0; j < kH; ++j) d2[j] = 0.f;
      for (int i = 0; i < kH; ++i) {
        const float g3 = G[tid * kH + i];
        for (int j = 0; j < kH; ++j) d2[j] = fmaf(sw[kOffW3 + i * kH + j], g3, d2[j]);
      }
      for (int j = 0; j < kH; ++j) Z3[tid * kH + j] = d2[j] * gelu_grad(Z2[tid * kH + j]);
    }
    __syncthreads();
    for (int k = 0; k < kPerThread; ++k) {
      const int q = k * kBwdTile + tid;
      if (q >= kOffW2 && q < kOffW3) {
        float a = 0.f;
        if (q < kOffB2) {
          const int i = (q - kOffW2) / kH, j = (q - kOffW2) % kH;
          for (int s = 0; s < kBwdTile; ++s) a = fmaf(Z3[s * kH + i], H1[s * kH + j], a);
        } else {
          const int i = q - kOffB2;
          for (int s = 0; s < kBwdTile; ++s) a += Z3[s * kH + i];
        }
        gacc[q] += a;
      }
    }
    __syncthreads();
    // dz1 = (W2^T dz2) * gelu'(z1), into G
    {
      float d1[kH];
      for (int j = 0; j < kH; ++j) d1[j] = 0.f;
      for (int i = 0; i < kH; ++i) {
        const float g2 = Z3[tid * kH + i];
        for (int j = 0; j < kH; ++j) d1[j] = fmaf(sw[kOffW2 + i * kH + j], g2, d1[j]);
      }
      for (int j = 0; j < kH; ++j) G[tid * kH + j] = d1[j] * gelu_grad(Z1[tid * kH + j]);
    }
    __syncthreads();
    for (int k = 0; k < kPerThread; ++k) {
      const int q = k * kBwdTile + tid;
      if (q < kOffW2) {
        float a = 0.f;
        if (q < kOffB1) {
          const int i = q / kIn, j = q % kIn;
          for (int s = 0; s < kBwdTile; ++s) a = fmaf(G[s * kH + i], X[s * kIn + j], a);
        } else {
          const int i = q - kOffB1;
          for (int s = 0; s < kBwdTile; ++s) a += G[s * kH + i];
        }
        gacc[q] += a;
      }
    }
    __syncthreads();
  }
  __syncthreads();
  for (int q = tid; q < kParams; q += kBwdTile) partials[(size_t)blockIdx.x * kParams + q] = gacc[q];
}

__global__ void k_grad_reduce(const float* __restrict__ partials, int nblocks, float* __restrict__ grad) {
  for (int q = blockIdx.x * blockDim.x + threadIdx.x; q < mlp::kParams; q += gridDim.x * blockDim.x) {
    double a = 0.0;
    for (int b = 0; b < nblocks; ++b) a += partials[(size_t)b * mlp::kParams + q];
    grad[q] += (float)a;
  }
}

// ------------------------------------------------------------------ Adam
__global__ void k_adam(float* __restrict__ w, const float* __restrict__ g, float* __restrict__ m, float* __restrict__ v,
                       size_t n, float lr, float b1, float b2, float eps, float c1, float c2) {
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) {
    const float gi = g[i];
    const float mi = b1 * m[i] + (1.f - b1) * gi;
    const float vi = b2 * v[i] + (1.f - b2) * gi * gi;
    m[i] = mi;
    v[i] = vi;
    w[i] -= lr * (mi / c1) / (sqrtf(vi / c2) + eps);
  }
}

// ------------------------------------------------- mesh Green's function
// G_S1 and -grad G_S1 at the periodic mesh offsets d/N, d in [0, N)^3, with
// the cell self term at d = 0 (for the PM target, Sec. 3 eq. pmconv).
__global__ void k_mesh_green(int N, float* __restrict__ out) {
  const size_t n3 = (size_t)N * N * N;
  const double inv4pi = 1.0 / (4.0 * green::kPi);
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n3; i += (size_t)gridDim.x * blockDim.x) {
    const int ix = (int)(i % N), iy = (int)((i / N) % N), iz = (int)(i / ((size_t)N * N));
    double v[4] = {0.0, 0.0, 0.0, 0.0};
    if (ix | iy | iz)
      green::gs1((double)ix / N, (double)iy / N, (double)iz / N, v);
    else
      v[0] = -green::cube_mean_inv_r() * N * inv4pi;
    for (int f = 0; f < 4; ++f) out[f * n3 + i] = (float)v[f];
  }
}

// The plan's Green's function on a mesh, for the PM references of Sec. 3:
// periodic (M = N): offsets d/N, d in [0, N)^3, the function the plan
// tabulates; isolated (M = 2N, the zero-padded Hockney mesh): G_0 at signed
// offsets k/N, k in [-N, N) in FFT order.  Self term at d = 0.
__global__ void k_mesh_green_plan(int N, int M, green::Spec gs, double* __restrict__ out) {
  const size_t m3 = (size_t)M * M * M;
  const double inv4pi = 1.0 / (4.0 * green::kPi);
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < m3; i += (size_t)gridDim.x * blockDim.x) {
    int k[3] = {(int)(i % M), (int)((i / M) % M), (int)(i / ((size_t)M * M))};
    if (M != N)
      for (int c = 0; c < 3; ++c)
        if (k[c] >= N) k[c] -= M;
    double v[4] = {0.0, 0.0, 0.0, 0.0};
    if (k[0] | k[1] | k[2])
      green::eval(gs, (double)k[0] / N, (double)k[1] / N, (double)k[2] / N, v);
    else
      v[0] = -green::cube_mean_inv_r() * N * inv4pi;
    for (int f = 0; f < 4; ++f) out[f * m3 + i] = v[f];
  }
}

}  // namespace

cudaError_t launch_mesh_green_plan(const Plan& P, double* out, cudaStream_t s) {
  if (!P.iso && P.gspec.kind == 4)   // the function is the mesh itself
    return cudaMemcpyAsync(out, P.gmesh, sizeof(double) * 4 * (size_t)P.N * P.N * P.N, cudaMemcpyDeviceToDevice, s);
  green::Spec g = P.gspec;
  if (P.iso) {
    g = green::Spec();
    g.kind = 2;
  }
  k_mesh_green_plan<<<4 * P.num_sms, 256, 0, s>>>(P.N, P.iso ? 2 * P.N : P.N, g, out);
  return cudaGetLastError();
}

// --------------------------------------------------------------- launchers
cudaError_t launch_residual(const float* phi, const float* acc, const float* tphi, const float* tacc, size_t n3,
                            float w_phi, float w_g, float* lam, float* loss, int sms, cudaStream_t s) {
  k_residual<<<4 * sms, 256, 0, s>>>(phi, acc, tphi, tacc, n3, w_phi, w_g, lam, loss);
  return cudaGetLastError();
}

cudaError_t launch_adjoint_and_table_grad(Plan& P, const float* lam_cells, cudaStream_t s) {
  const int p = P.p, S = P.S, p3 = p * p * p, K = 2 * p;
  // leaf adjoint
  {
    const size_t smem = sizeof(float2) * p * S + sizeof(float) * (4 * S * S * S + 4 * S * S * p + 4 * S * p * p + 4 * p3);
    k_adj_l2p<<<1u << (3 * P.L), 128, smem, s>>>(lam_cells, P.N, S, p, P.w_p2m, P.lam[P.L]);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
  }
  for (int l = P.L - 1; l >= 2; --l) {
    const size_t smem = sizeof(float2) * p * K + sizeof(float) * (4 * K * K * K + 4 * K * K * p + 4 * K * p * p + 4 * p3);
    k_adj_l2l<<<1u << (3 * l), 256, smem, s>>>(P.lam[l + 1], p, P.w_m2m, P.lam[l]);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
  }
  const size_t E = 8 * p - 1;
  for (int l = 2; l <= P.L; ++l) {
    cudaError_t e = cudaMemsetAsync(P.dT[l], 0, sizeof(float) * E * E * E * 4, s);
    if (e != cudaSuccess) return e;
    const size_t smem = sizeof(float) * 2 * kTgChunk * p3;
    dim3 grid(P.n_off[l], 8, 4);
    k_table_grad<<<grid, 512, smem, s>>>(P.lam[l], P.M[l], P.offsets[l], P.n_off[l], l, p, P.dT[l]);
    e = cudaGetLastError();
    if (e != cudaSuccess) return e;
  }
  return cudaSuccess;
}

size_t mlp_backward_smem() {
  return sizeof(float) * (2 * mlp::kParams + kBwdTile * mlp::kIn + 6 * kBwdTile * mlp::kH + kBwdTile);
}

int mlp_backward_blocks(const Plan& P) { return 2 * P.num_sms; }

cudaError_t setup_learn() {
  cudaError_t e = cudaFuncSetAttribute(k_mlp_backward, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)mlp_backward_smem());
  if (e != cudaSuccess) return e;
  e = cudaFuncSetAttribute(k_table_grad, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
  if (e != cudaSuccess) return e;
  e = cudaFuncSetAttribute(k_adj_l2l, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
  if (e != cudaSuccess) return e;
  return cudaFuncSetAttribute(k_adj_l2p, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
}

cudaError_t launch_mlp_backward(Plan& P, const float* w, float* grad, cudaStream_t s) {
  // dT of levels 2..L are contiguous per level in P.dT_all
  const int nb = mlp_backward_blocks(P);
  k_mlp_backward<<<nb, kBwdTile, mlp_backward_smem(), s>>>(w, P.dT_all, 2, P.L, P.p, P.grad_partials);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  k_grad_reduce<<<(mlp::kParams + 255) / 256, 256, 0, s>>>(P.grad_partials, nb, grad);
  return cudaGetLastError();
}

cudaError_t launch_adam(float* w, const float* g, float* m, float* v, size_t n, int step, float lr, float b1, float b2,
                        float eps, cudaStream_t s) {
  const float c1 = 1.f - powf(b1, (float)step), c2 = 1.f - powf(b2, (float)step);
  k_adam<<<64, 256, 0, s>>>(w, g, m, v, n, lr, b1, b2, eps, c1, c2);
  return cudaGetLastError();
}

cudaError_t launch_mesh_green(int N, float* out, int sms, cudaStream_t s) {
  k_mesh_green<<<4 * sms, 256, 0, s>>>(N, out);
  return cudaGetLastError();
}

}  // namespace fmm

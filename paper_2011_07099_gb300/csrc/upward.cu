// Upward pass: mean removal, P2M at the leaves and M2M up to level 2
// (double-float arithmetic, see fmm_internal.cuh).
//
// Gridlet masses (Sec. 2): a node's order^3 effective masses on its
// cell-centred mini-mesh must reproduce every Cartesian multipole Q_n,
// n_i < order, of the mass they stand for.  The unique solution of that
// Vandermonde system is separable: M_s = sum_c l_s(x_c) m_c with l_s the 1-D
// Lagrange basis on the gridlet points, one factor per axis.  M2M (eq. fmm1)
// is the same map with the children's gridlet points as sources: the 8 child
// gridlets form a uniform (2 order)^3 cell-centred mesh over the parent.
#include "fmm_internal.cuh"

namespace fmm {
namespace {

// a0: block partial sums of the density in FP64.
__global__ void k_partial_sum(const float4* __restrict__ rho4, size_t n4, double* __restrict__ partials) {
  double acc = 0.0;
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n4; i += (size_t)gridDim.x * blockDim.x) {
    const float4 v = __ldg(rho4 + i);
    acc += ((double)v.x + (double)v.y) + ((double)v.z + (double)v.w);
  }
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

__global__ void k_final_mean(const double* __restrict__ partials, int n, double inv_cells, double* __restrict__ mean) {
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
    if (lane == 0) *mean = acc * inv_cells;
  }
}

// a3: one CTA per leaf (Morton key = blockIdx.x).  Cell masses
// m = (rho - mean) / N^3 are formed exactly as double-float pairs from the
// FP32 density and the mean split into hi + lo, and contracted in
// double-float with (hi, lo) Lagrange weights; the gridlet masses are rounded
// once to FP32 (and kept as FP64 at high order).  FP32 arithmetic here fails
// the point-source test: every node of the uniform background rounds the
// same way, so the errors add up coherently across the mesh.
__global__ void k_p2m(const float* __restrict__ rho, const double* __restrict__ mean, int N, int S, int p,
                      const float2* __restrict__ w, float* __restrict__ Mout, double* __restrict__ Mout64) {
  extern __shared__ float2 smdf[];
  float2* W = smdf;                      // p*S
  float2* in = W + p * S;                // S^3
  float2* t1 = in + S * S * S;           // S*S*p
  float2* t2 = t1 + S * S * p;           // S*p*p
  float2* out = t2 + S * p * p;          // p^3
  const int tid = threadIdx.x, nthr = blockDim.x;
  uint32_t lx, ly, lz;
  unmorton(blockIdx.x, lx, ly, lz);
  const double mu = *mean;
  const float mu_hi = (float)mu, mu_lo = (float)(mu - (double)mu_hi);
  const double ivd = 1.0 / ((double)N * N * N);
  const float iv = (float)ivd, iv_lo = (float)(ivd - (double)iv);
  for (int i = tid; i < p * S; i += nthr) W[i] = w[i];
  for (int i = tid; i < S * S * S; i += nthr) {
    const int cx = i % S, cy = (i / S) % S, cz = i / (S * S);
    const size_t g = ((size_t)(lz * S + cz) * N + (ly * S + cy)) * N + (lx * S + cx);
    const float2 d = df_two_sum(__ldg(rho + g), -mu_hi);      // rho - mu_hi exactly
    const float dlo = __fsub_rn(d.y, mu_lo);
    const float ph = __fmul_rn(d.x, iv);                        // (d.x + dlo) (iv + iv_lo)
    const float pe = fmaf(d.x, iv, -ph);
    const float lo = fmaf(d.x, iv_lo, fmaf(dlo, iv, pe));
    const float sum = __fadd_rn(ph, lo);
    in[i] = make_float2(sum, __fsub_rn(lo, __fsub_rn(sum, ph)));
  }
  __syncthreads();
  contract3_df(in, t1, t2, out, S, p, W, S, false, tid, nthr);
  const int p3 = p * p * p;
  for (int i = tid; i < p3; i += nthr) {
    Mout[(size_t)blockIdx.x * p3 + i] = out[i].x;
    if (Mout64) Mout64[(size_t)blockIdx.x * p3 + i] = df_to_double(out[i]);
  }
}

// a4: one CTA per parent; the 8 children (keys 8P + c) are gathered into a
// (2p)^3 mesh and contracted with the [p][2p] (hi, lo) Lagrange matrix on each
// axis in double-float.  At high order the FP64 copies are read (Mc64, when
// the children keep one) and written (Mp64).
__global__ void k_m2m(const float* __restrict__ Mc, const double* __restrict__ Mc64, int p,
                      const float2* __restrict__ w, float* __restrict__ Mp, double* __restrict__ Mp64) {
  extern __shared__ float2 smdf[];
  const int K = 2 * p, p3 = p * p * p;
  float2* W = smdf;              // p*K
  float2* in = W + p * K;        // K^3
  float2* t1 = in + K * K * K;   // K*K*p
  float2* t2 = t1 + K * K * p;   // K*p*p
  float2* out = t2 + K * p * p;  // p^3
  const int tid = threadIdx.x, nthr = blockDim.x;
  for (int i = tid; i < p * K; i += nthr) W[i] = w[i];
  const size_t base = (size_t)blockIdx.x * 8 * p3;
  for (int i = tid; i < 8 * p3; i += nthr) {
    const int c = i / p3, q = i % p3;
    const int qx = q % p, qy = (q / p) % p, qz = q / (p * p);
    const int ux = (c & 1) * p + qx, uy = ((c >> 1) & 1) * p + qy, uz = (c >> 2) * p + qz;
    in[(uz * K + uy) * K + ux] = Mc64 ? df_from_double(Mc64[base + i]) : make_float2(__ldg(Mc + base + i), 0.f);
  }
  __syncthreads();
  contract3_df(in, t1, t2, out, K, p, W, K, false, tid, nthr);
  for (int i = tid; i < p3; i += nthr) {
    Mp[(size_t)blockIdx.x * p3 + i] = out[i].x;
    if (Mp64) Mp64[(size_t)blockIdx.x * p3 + i] = df_to_double(out[i]);
  }
}

}  // namespace

cudaError_t setup_upward(const Plan& P) {
  cudaError_t e = cudaFuncSetAttribute(k_p2m, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
  if (e != cudaSuccess) return e;
  return cudaFuncSetAttribute(k_m2m, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
}

cudaError_t launch_mean_into(const Plan& P, const float* rho, double* partials, double* mean, cudaStream_t s) {
  const size_t n4 = (size_t)P.N * P.N * P.N / 4;
  k_partial_sum<<<P.n_partials, 256, 0, s>>>(reinterpret_cast<const float4*>(rho), n4, partials);
  k_final_mean<<<1, 1024, 0, s>>>(partials, P.n_partials, 1.0 / ((double)P.N * P.N * P.N), mean);
  return cudaGetLastError();
}

cudaError_t launch_mean(Plan& P, const float* rho, cudaStream_t s) {
  return launch_mean_into(P, rho, P.d_partials, P.d_mean, s);
}

cudaError_t launch_p2m(Plan& P, const float* rho, cudaStream_t s) {
  const int S = P.S, p = P.p;
  const size_t smem = sizeof(float2) * (p * S + S * S * S + S * S * p + S * p * p + p * p * p);
  const unsigned leaves = 1u << (3 * P.L);
  k_p2m<<<leaves, 128, smem, s>>>(rho, P.d_mean, P.N, S, p, P.w_p2m, P.M[P.L], P.M64[P.L]);
  return cudaGetLastError();
}

cudaError_t launch_m2m(Plan& P, int level, cudaStream_t s) {
  const int p = P.p, K = 2 * p;
  const size_t smem = sizeof(float2) * (p * K + K * K * K + K * K * p + K * p * p + p * p * p);
  const unsigned parents = 1u << (3 * level);
  k_m2m<<<parents, 128, smem, s>>>(P.M[level + 1], P.M64[level + 1], p, P.w_m2m, P.M[level], P.M64[level]);
  return cudaGetLastError();
}

}  // namespace fmm

// Downward pass: L2L (eq. fmm3).
//
// The local field of a child is the parent's local field projected with the
// transpose of the child's M2M matrix: Phi_child[q] = sum_r T_{r q} Phi_parent[r]
// (Sec. 3 eq. fmm3).  With T the separable Lagrange matrix, that is the parent
// field interpolated at the child's gridlet points.  The 8 children's points
// form one uniform (2p)^3 mesh over the parent, so one CTA expands all four
// fields of a parent onto that mesh and adds them to the children's fields
// (which already hold their own M2L result).
#include "fmm_internal.cuh"

namespace fmm {
namespace {

__global__ void k_l2l(const float* __restrict__ Fp, int p, const float2* __restrict__ w, float* __restrict__ Fc) {
  extern __shared__ float2 sm2[];
  const int K = 2 * p, p3 = p * p * p;
  float2* W = sm2;                       // p*K  ([p][2p], used transposed)
  float* in = reinterpret_cast<float*>(W + p * K);   // 4*p^3
  float* t1 = in + 4 * p3;               // 4*p*p*K
  float* t2 = t1 + 4 * p * p * K;        // 4*p*K*K
  float* out = t2 + 4 * p * K * K;       // 4*K^3
  const int tid = threadIdx.x, nthr = blockDim.x;
  for (int i = tid; i < p * K; i += nthr) W[i] = w[i];
  const float* src = Fp + (size_t)blockIdx.x * 4 * p3;
  for (int i = tid; i < 4 * p3; i += nthr) in[i] = src[i];
  __syncthreads();
  contract3(in, t1, t2, out, 4, p, K, W, K, true, tid, nthr);
  float* dst = Fc + (size_t)blockIdx.x * 8 * 4 * p3;
  for (int i = tid; i < 8 * 4 * p3; i += nthr) {
    const int c = i / (4 * p3), rem = i % (4 * p3);
    const int f = rem / p3, q = rem % p3;
    const int qx = q % p, qy = (q / p) % p, qz = q / (p * p);
    const int ux = (c & 1) * p + qx, uy = ((c >> 1) & 1) * p + qy, uz = (c >> 2) * p + qz;
    dst[i] += out[((f * K + uz) * K + uy) * K + ux];
  }
}

// Variant for parents at the wide levels (the coarse levels 2 and 3; at
// order >= 7 every level above the leaves): FP64 local fields, interpolated
// in double-float (fmm_internal.cuh), one field
// at a time (shared memory).  The child field is F64 (a coarse child, whose
// FP32 copy is refreshed too) or the FP32 field of the first fine level, to
// which the FP64 contribution is added before a single rounding.
__global__ void k_l2l64(const double* __restrict__ Fp, int p, const float2* __restrict__ w,
                        double* __restrict__ Fc64, float* __restrict__ Fc) {
  extern __shared__ float2 smdf[];
  const int K = 2 * p, p3 = p * p * p;
  float2* W = smdf;                  // p*K  ([p][2p], used transposed)
  float2* in = W + p * K;            // p^3
  float2* t1 = in + p3;              // p*p*K
  float2* t2 = t1 + p * p * K;       // p*K*K
  float2* out = t2 + p * K * K;      // K^3
  const int tid = threadIdx.x, nthr = blockDim.x;
  for (int i = tid; i < p * K; i += nthr) W[i] = w[i];
  for (int f = 0; f < 4; ++f) {
    const double* src = Fp + ((size_t)blockIdx.x * 4 + f) * p3;
    for (int i = tid; i < p3; i += nthr) in[i] = df_from_double(src[i]);
    __syncthreads();
    contract3_df(in, t1, t2, out, p, K, W, K, true, tid, nthr);
    for (int i = tid; i < 8 * p3; i += nthr) {
      const int c = i / p3, q = i % p3;
      const int qx = q % p, qy = (q / p) % p, qz = q / (p * p);
      const int ux = (c & 1) * p + qx, uy = ((c >> 1) & 1) * p + qy, uz = (c >> 2) * p + qz;
      const size_t d = (((size_t)blockIdx.x * 8 + c) * 4 + f) * p3 + q;
      const double v = df_to_double(out[(uz * K + uy) * K + ux]);
      if (Fc64) {
        const double t = Fc64[d] + v;
        Fc64[d] = t;
        Fc[d] = (float)t;
      } else {
        Fc[d] = (float)((double)Fc[d] + v);
      }
    }
    __syncthreads();   // `in` and `out` are reused by the next field
  }
}

}  // namespace

cudaError_t setup_downward(const Plan& P) {
  cudaError_t e = cudaFuncSetAttribute(k_l2l64, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
  if (e != cudaSuccess) return e;
  return cudaFuncSetAttribute(k_l2l, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
}

cudaError_t launch_l2l(Plan& P, int level, cudaStream_t s) {
  const int p = P.p, K = 2 * p, p3 = p * p * p;
  const size_t smem = sizeof(float2) * p * K + sizeof(float) * (4 * p3 + 4 * p * p * K + 4 * p * K * K + 4 * K * K * K);
  const unsigned parents = 1u << (3 * level);
  if (wide_level(P, level)) {
    const size_t smem64 = sizeof(float2) * (p * K + p3 + p * p * K + p * K * K + K * K * K);
    k_l2l64<<<parents, 256, smem64, s>>>(P.F64[level], p, P.w_m2m, wide_level(P, level + 1) ? P.F64[level + 1] : nullptr,
                                         P.F[level + 1]);
    return cudaGetLastError();
  }
  k_l2l<<<parents, 256, smem, s>>>(P.F[level], p, P.w_m2m, P.F[level + 1]);
  return cudaGetLastError();
}

}  // namespace fmm

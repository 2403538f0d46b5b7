// M2L by FFT over each parent's children (the HPM form of the interaction
// zone, Sec. 2), an ablation against the dense contraction of the other
// M2L kernels.
//
// The interaction zones of the 8 children of a parent P lie in the 6 x 6 x 6
// block of P's neighbours' children (Sec. 2, Fig. fmm).  Their gridlet masses
// form a (6p)^3 uniform grid; the potential at the children's gridlet points
// is a discrete convolution of that grid with the level table (eq. fmm2:
// every term is G at a gridlet offset).  Target and source points differ by
// at most 4p - 1 gridlet spacings per axis, so a circular convolution of
// size M = 8p reproduces the linear one exactly where it is read (the
// (6 N_g)^D grid of the text would wrap offsets around).  Per parent: the
// zero-padded M^3 grid is transformed once (cuFFT, R2C, batched over
// parents), multiplied by the table's spectrum per field, transformed back
// (C2R), and the block sum at the children's points has the 27 near nodes'
// terms, computed directly over the same table, subtracted.  FP32 throughout.
#include <cufft.h>

#include <vector>

#include "fmm_internal.cuh"

namespace fmm {
namespace {

// The level table as an M^3 circular kernel per field: index a <-> offset
// a (a < 4p) or a - M (a >= M - 4p + 1); the unused offset -4p holds 0.
__global__ void k_fft_kernel(const float4* __restrict__ tab, int p, int M, float* __restrict__ out) {
  const int hw = 4 * p - 1, E = 8 * p - 1;
  const size_t m3 = (size_t)M * M * M;
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < m3; i += (size_t)gridDim.x * blockDim.x) {
    int d[3] = {(int)(i % M), (int)((i / M) % M), (int)(i / ((size_t)M * M))};
    bool ok = true;
    for (int c = 0; c < 3; ++c) {
      if (d[c] >= M - hw) d[c] -= M;
      if (d[c] > hw || d[c] < -hw) ok = false;
    }
    float4 v = make_float4(0.f, 0.f, 0.f, 0.f);
    if (ok) v = tab[((size_t)(d[2] + hw) * E + (d[1] + hw)) * E + (d[0] + hw)];
    out[i] = v.x;
    out[m3 + i] = v.y;
    out[2 * m3 + i] = v.z;
    out[3 * m3 + i] = v.w;
  }
}

// Per parent (blockIdx.x): the 6 x 6 x 6 children block's gridlet masses on
// the M^3 grid (block node i at gridlet rows [i p, (i + 1) p)), zero beyond.
__global__ void k_fft_gather(const float* __restrict__ Mlev, int level, int p, int M, float* __restrict__ X) {
  const uint32_t par = blockIdx.x;
  uint32_t px, py, pz;
  unmorton(par, px, py, pz);
  const int n = 1 << level, p3 = p * p * p, w = 6 * p;
  const size_t m3 = (size_t)M * M * M;
  float* dst = X + (size_t)par * m3;
  for (size_t i = threadIdx.x; i < m3; i += blockDim.x) {
    const int x = (int)(i % M), y = (int)((i / M) % M), z = (int)(i / ((size_t)M * M));
    float v = 0.f;
    if (x < w && y < w && z < w) {
      const uint32_t sx = (uint32_t)(2 * (int)px - 2 + x / p) & (n - 1);
      const uint32_t sy = (uint32_t)(2 * (int)py - 2 + y / p) & (n - 1);
      const uint32_t sz = (uint32_t)(2 * (int)pz - 2 + z / p) & (n - 1);
      v = Mlev[(size_t)morton(sx, sy, sz) * p3 + ((z % p) * p + (y % p)) * p + (x % p)];
    }
    dst[i] = v;
  }
}

// Y = X^ K_f^ for one field (complex, per parent).
__global__ void k_fft_mul(const cufftComplex* __restrict__ Xh, const cufftComplex* __restrict__ Kh, size_t per,
                          size_t total, cufftComplex* __restrict__ Yh) {
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < total; i += (size_t)gridDim.x * blockDim.x) {
    const cufftComplex a = Xh[i], b = Kh[i % per];
    Yh[i] = make_cuFloatComplex(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
  }
}

// F[child][f][r] = (block sum at the child's point r) / M^3 - F (the near
// nodes' terms, written there beforehand).
__global__ void k_fft_extract(const float* __restrict__ Y, int f, int p, int M, float* __restrict__ F) {
  const uint32_t par = blockIdx.x;
  const int p3 = p * p * p;
  const size_t m3 = (size_t)M * M * M;
  const float scale = 1.f / (float)m3;
  const float* src = Y + (size_t)par * m3;
  for (int i = threadIdx.x; i < 8 * p3; i += blockDim.x) {
    const int c = i / p3, r = i % p3;
    const int rx = r % p, ry = (r / p) % p, rz = r / (p * p);
    const int x = (2 + (c & 1)) * p + rx, y = (2 + ((c >> 1) & 1)) * p + ry, z = (2 + (c >> 2)) * p + rz;
    float* dst = F + ((size_t)(8u * par + c) * 4 + f) * p3 + r;
    *dst = src[((size_t)z * M + y) * M + x] * scale - *dst;
  }
}

}  // namespace

struct FftLevel {
  cufftHandle r2c = 0, c2r = 0;
  float* X = nullptr;            // parents x M^3 (real grid; reused for the back transforms)
  cufftComplex* Xh = nullptr;    // parents x M^2 (M/2 + 1)
  cufftComplex* Yh = nullptr;
  cufftComplex* Kh = nullptr;    // 4 fields x M^2 (M/2 + 1)
};

struct FftState {
  FftLevel lev[kMaxLevel + 1];
  int8_t* near27 = nullptr;      // 8 child types x 27 offsets x 3
};

void free_fft(Plan& P) {
  FftState* S = static_cast<FftState*>(P.fft);
  if (!S) return;
  for (auto& l : S->lev) {
    if (l.r2c) cufftDestroy(l.r2c);
    if (l.c2r) cufftDestroy(l.c2r);
    cudaFree(l.X);
    cudaFree(l.Xh);
    cudaFree(l.Yh);
    cudaFree(l.Kh);
  }
  cudaFree(S->near27);
  delete S;
  P.fft = nullptr;
}

bool fft_level(const Plan& P, int l) { return P.m2l_fft && !P.iso && !wide_level(P, l) && l >= 3; }

int prepare_fft(Plan& P) {
  if (P.fft) return FMM_OK;
  FftState* S = new FftState();
  P.fft = S;
  const int p = P.p, M = 8 * p, hc = M / 2 + 1;
  const size_t m3 = (size_t)M * M * M, mc = (size_t)M * M * hc;
  std::vector<int8_t> near;
  for (int c = 0; c < 8; ++c)
    for (int z = -1; z <= 1; ++z)
      for (int y = -1; y <= 1; ++y)
        for (int x = -1; x <= 1; ++x) {
          near.push_back((int8_t)x);
          near.push_back((int8_t)y);
          near.push_back((int8_t)z);
        }
  if (cudaMalloc(&S->near27, near.size()) != cudaSuccess ||
      cudaMemcpy(S->near27, near.data(), near.size(), cudaMemcpyHostToDevice) != cudaSuccess)
    return FMM_ERR_ALLOC;
  int dims[3] = {M, M, M};
  for (int l = 2; l <= P.L; ++l) {
    if (!fft_level(P, l)) continue;
    FftLevel& F = S->lev[l];
    const int np = 1 << (3 * (l - 1));
    if (cudaMalloc(&F.X, sizeof(float) * m3 * np) != cudaSuccess ||
        cudaMalloc(&F.Xh, sizeof(cufftComplex) * mc * np) != cudaSuccess ||
        cudaMalloc(&F.Yh, sizeof(cufftComplex) * mc * np) != cudaSuccess ||
        cudaMalloc(&F.Kh, sizeof(cufftComplex) * mc * 4) != cudaSuccess)
      return FMM_ERR_ALLOC;
    if (cufftPlanMany(&F.r2c, 3, dims, nullptr, 1, (int)m3, nullptr, 1, (int)mc, CUFFT_R2C, np) != CUFFT_SUCCESS ||
        cufftPlanMany(&F.c2r, 3, dims, nullptr, 1, (int)mc, nullptr, 1, (int)m3, CUFFT_C2R, np) != CUFFT_SUCCESS)
      return FMM_ERR_CUDA;
    // the table's spectrum, one field at a time (the parents' grid buffer
    // holds the 4 kernels: np >= 4 at the levels that use this path)
    k_fft_kernel<<<4 * P.num_sms, 256>>>(P.tab[l], p, M, F.X);
    cufftHandle k4 = 0;
    if (cudaGetLastError() != cudaSuccess ||
        cufftPlanMany(&k4, 3, dims, nullptr, 1, (int)m3, nullptr, 1, (int)mc, CUFFT_R2C, 4) != CUFFT_SUCCESS)
      return FMM_ERR_CUDA;
    const bool ok = cufftExecR2C(k4, F.X, F.Kh) == CUFFT_SUCCESS;
    cufftDestroy(k4);
    if (!ok || cudaDeviceSynchronize() != cudaSuccess) return FMM_ERR_CUDA;
  }
  return FMM_OK;
}

cudaError_t launch_m2l_fft(Plan& P, int level, cudaStream_t s) {
  FftState* S = static_cast<FftState*>(P.fft);
  FftLevel& F = S->lev[level];
  const int p = P.p, M = 8 * p, hc = M / 2 + 1;
  const size_t mc = (size_t)M * M * hc;
  const int np = 1 << (3 * (level - 1));
  // the near nodes' terms first (the extract kernel subtracts them)
  cudaError_t e = launch_m2l_fp32_list(P, level, S->near27, 27, s);
  if (e != cudaSuccess) return e;
  k_fft_gather<<<np, 256, 0, s>>>(P.M[level], level, p, M, F.X);
  if ((e = cudaGetLastError()) != cudaSuccess) return e;
  if (cufftSetStream(F.r2c, s) != CUFFT_SUCCESS || cufftSetStream(F.c2r, s) != CUFFT_SUCCESS ||
      cufftExecR2C(F.r2c, F.X, F.Xh) != CUFFT_SUCCESS)
    return cudaErrorUnknown;
  for (int f = 0; f < 4; ++f) {
    k_fft_mul<<<8 * P.num_sms, 256, 0, s>>>(F.Xh, F.Kh + (size_t)f * mc, mc, mc * np, F.Yh);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    if (cufftExecC2R(F.c2r, F.Yh, F.X) != CUFFT_SUCCESS) return cudaErrorUnknown;
    k_fft_extract<<<np, 256, 0, s>>>(F.X, f, p, M, P.F[level]);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
  }
  return cudaSuccess;
}

}  // namespace fmm

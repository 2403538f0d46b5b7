// M2L on CUDA cores in FP32 (the plain form).
//
// Eq. fmm2 (Sec. 3): for a target node T at level l and every source node S
// of its interaction zone (the children of the parent's neighbours that are
// not T's neighbours, with periodic wrap, Sec. 2),
//   Phi_T[r] += sum_s G(d + dx_l (r - s)) M_S[s],   d = (T - S) H_l,
// and the three acceleration fields with -grad G.  Since H_l = p dx_l every
// argument is dx_l (o p + r - s) with o = T - S in node units, so each
// offset's translation matrix is a window of the level table.
//
// Work split: a CTA owns NT targets of one child type (the 8 types have
// different interaction lists, Sec. 2 Fig. fmm); thread r owns one target
// gridlet point and keeps NT x 4 accumulators.  Per offset the CTA stages the
// (2p-1)^3 table window and the NT source gridlets in shared memory, so every
// table value read feeds 4 x NT FMAs and every mass read (a broadcast) feeds 4.
//
// Rounding: the far-field sum cancels heavily (mean-free masses, G < 0), so a
// plain running FP32 sum over all 189 p^3 terms loses several digits.  Within
// one offset the terms of every field mostly share a sign (G < 0 and grad G
// points one way across a distant node, while a node's gridlet masses mostly
// share the sign of its net mass), so a running sum grows ~p^3 times larger
// than a term.  The terms are therefore summed as a tree: p-term rows, rows
// into planes, and each plane is added to the total with Kahan compensation.
// At the top two levels the potential also takes the low half of the split
// table, G = G_hi + G_lo: rounding G to FP32 errs coherently across targets
// and is the largest remaining error of the long-range potential.  At high
// order (p >= 7) the rounding of the gradient tables matters as well (1.5e-5
// on g at p = 8), so all four fields take their low halves there (EXT = 2).
#include "fmm_internal.cuh"

namespace fmm {
namespace {

template <int P>
struct M2LShape {
  static constexpr int P3 = P * P * P;
  static constexpr int THREADS = ((P3 + 31) / 32) * 32 < 64 ? 64 : ((P3 + 31) / 32) * 32;
  static constexpr int NT = P3 > 256 ? 4 : 8;            // targets per CTA (register budget)
};

// EXT: 0 = FP32 table; 1 = the potential also takes G_lo; 2 = all four fields
// take their low halves.
template <int P, int EXT>
__global__ void __launch_bounds__(M2LShape<P>::THREADS)
k_m2l_fp32(const float* __restrict__ M, float* __restrict__ F, const float4* __restrict__ tab,
           const float4* __restrict__ tab_lo, const int8_t* __restrict__ offs, int n_off, int level) {
  constexpr int P3 = P * P * P;
  constexpr int NT = M2LShape<P>::NT;
  constexpr int D = 2 * P - 1;          // table window per dimension
  constexpr int D3 = D * D * D;
  constexpr int HW = 4 * P - 1, E = 8 * P - 1;
  extern __shared__ float4 sm4[];
  float4* win = sm4;                                     // D3 float4
  float4* msrc = win + D3;                               // P3 x (NT/4) float4: [s][k]
  float* win_lo = reinterpret_cast<float*>(msrc + P3 * (NT / 4));   // D3 floats (EXT == 1)
  float4* win_lo4 = msrc + P3 * (NT / 4);                            // D3 float4 (EXT == 2)
  const int tid = threadIdx.x, nthr = blockDim.x;
  const int ctype = blockIdx.y;
  const int n = 1 << level;
  const uint32_t n_par = 1u << (3 * (level - 1));
  const uint32_t par0 = blockIdx.x * NT;
  const int8_t* my_offs = offs + (size_t)ctype * n_off * 3;

  __shared__ int tx[NT], ty[NT], tz[NT];
  if (tid < NT) {
    uint32_t x = 0, y = 0, z = 0;
    if (par0 + tid < n_par) unmorton(8u * (par0 + tid) + ctype, x, y, z);
    tx[tid] = x; ty[tid] = y; tz[tid] = z;
  }

  float acc[4][NT], comp[4][NT];
#pragma unroll
  for (int f = 0; f < 4; ++f)
#pragma unroll
    for (int k = 0; k < NT; ++k) acc[f][k] = comp[f][k] = 0.f;

  const int r = tid;
  const int rx = r % P, ry = (r / P) % P, rz = r / (P * P);
  const int rbase = ((rz + P - 1) * D + (ry + P - 1)) * D + (rx + P - 1);

  for (int io = 0; io < n_off; ++io) {
    const int ox = my_offs[3 * io + 0], oy = my_offs[3 * io + 1], oz = my_offs[3 * io + 2];
    __syncthreads();   // previous offset's compute is done with the buffers (and tx.. are set)
    for (int i = tid; i < D3; i += nthr) {
      const int dx = i % D - (P - 1), dy = (i / D) % D - (P - 1), dz = i / (D * D) - (P - 1);
      const int nx = ox * P + dx + HW, ny = oy * P + dy + HW, nz = oz * P + dz + HW;
      win[i] = __ldg(tab + ((size_t)nz * E + ny) * E + nx);
      if (EXT == 1) win_lo[i] = __ldg(&tab_lo[((size_t)nz * E + ny) * E + nx].x);
      if (EXT == 2) win_lo4[i] = __ldg(tab_lo + ((size_t)nz * E + ny) * E + nx);
    }
    float* ms = reinterpret_cast<float*>(msrc);
    for (int i = tid; i < NT * P3; i += nthr) {
      const int k = i / P3, s = i % P3;
      float v = 0.f;
      if (par0 + k < n_par) {
        const uint32_t sx = (uint32_t)(tx[k] - ox) & (n - 1), sy = (uint32_t)(ty[k] - oy) & (n - 1),
                       sz = (uint32_t)(tz[k] - oz) & (n - 1);
        v = __ldg(M + (size_t)morton(sx, sy, sz) * P3 + s);
      }
      ms[s * NT + k] = v;
    }
    __syncthreads();
    if (r < P3) {
      constexpr int NLO = EXT == 2 ? 4 : 1;
      float plo[NLO][NT];
#pragma unroll
      for (int f = 0; f < NLO; ++f)
#pragma unroll
        for (int k = 0; k < NT; ++k) plo[f][k] = 0.f;
#pragma unroll 1
      for (int sz = 0; sz < P; ++sz) {
        float plane[4][NT];
#pragma unroll
        for (int f = 0; f < 4; ++f)
#pragma unroll
          for (int k = 0; k < NT; ++k) plane[f][k] = 0.f;
#pragma unroll 1
        for (int sy = 0; sy < P; ++sy) {
          float row[4][NT];
#pragma unroll
          for (int f = 0; f < 4; ++f)
#pragma unroll
            for (int k = 0; k < NT; ++k) row[f][k] = 0.f;
#pragma unroll
          for (int sx = 0; sx < P; ++sx) {
            const int s = (sz * P + sy) * P + sx;
            const int w = rbase - ((sz * D + sy) * D + sx);
            const float4 t = win[w];
            const float4 tl = EXT == 2 ? win_lo4[w] : make_float4(EXT == 1 ? win_lo[w] : 0.f, 0.f, 0.f, 0.f);
            const float4* mv = msrc + s * (NT / 4);
#pragma unroll
            for (int q = 0; q < NT / 4; ++q) {
              const float4 m = mv[q];
              const float mm[4] = {m.x, m.y, m.z, m.w};
#pragma unroll
              for (int j = 0; j < 4; ++j) {
                row[0][4 * q + j] = fmaf(t.x, mm[j], row[0][4 * q + j]);
                row[1][4 * q + j] = fmaf(t.y, mm[j], row[1][4 * q + j]);
                row[2][4 * q + j] = fmaf(t.z, mm[j], row[2][4 * q + j]);
                row[3][4 * q + j] = fmaf(t.w, mm[j], row[3][4 * q + j]);
                if (EXT >= 1) plo[0][4 * q + j] = fmaf(tl.x, mm[j], plo[0][4 * q + j]);
                if (EXT == 2) {
                  plo[NLO - 3][4 * q + j] = fmaf(tl.y, mm[j], plo[NLO - 3][4 * q + j]);
                  plo[NLO - 2][4 * q + j] = fmaf(tl.z, mm[j], plo[NLO - 2][4 * q + j]);
                  plo[NLO - 1][4 * q + j] = fmaf(tl.w, mm[j], plo[NLO - 1][4 * q + j]);
                }
              }
            }
          }
#pragma unroll
          for (int f = 0; f < 4; ++f)
#pragma unroll
            for (int k = 0; k < NT; ++k) plane[f][k] += row[f][k];
        }
        // Kahan-compensated add of the plane partial into the total
#pragma unroll
        for (int f = 0; f < 4; ++f)
#pragma unroll
          for (int k = 0; k < NT; ++k) {
            const float y = plane[f][k] - comp[f][k];
            const float t = acc[f][k] + y;
            comp[f][k] = (t - acc[f][k]) - y;
            acc[f][k] = t;
          }
      }
      if (EXT) {
#pragma unroll
        for (int f = 0; f < NLO; ++f)
#pragma unroll
          for (int k = 0; k < NT; ++k) comp[f][k] -= plo[f][k];
      }
    }
  }
  if (r < P3) {
#pragma unroll
    for (int k = 0; k < NT; ++k) {
      if (par0 + k >= n_par) break;
      float* dst = F + (size_t)(8u * (par0 + k) + ctype) * 4 * P3;
#pragma unroll
      for (int f = 0; f < 4; ++f) dst[f * P3 + r] = acc[f][k];
    }
  }
}

template <int P>
cudaError_t launch_p(Plan& Pl, int level, cudaStream_t s) {
  constexpr int P3 = P * P * P;
  constexpr int D = 2 * P - 1;
  constexpr int NT = M2LShape<P>::NT;
  constexpr int EXT_TOP = P >= 7 ? 2 : 1;
  const int threads = M2LShape<P>::THREADS;
  const bool ext = level <= kExtTopLevel;
  const size_t lo_bytes = ext ? (EXT_TOP == 2 ? sizeof(float4) : sizeof(float)) * D * D * D : 0;
  const size_t smem = sizeof(float4) * (D * D * D + P3 * (NT / 4)) + lo_bytes;
  const uint32_t n_par = 1u << (3 * (level - 1));
  dim3 grid((n_par + NT - 1) / NT, 8);
  if (ext)
    k_m2l_fp32<P, EXT_TOP><<<grid, threads, smem, s>>>(Pl.M[level], Pl.F[level], Pl.tab[level], Pl.tab_lo[level],
                                                       Pl.offsets[level], Pl.n_off[level], level);
  else
    k_m2l_fp32<P, 0><<<grid, threads, smem, s>>>(Pl.M[level], Pl.F[level], Pl.tab[level], nullptr,
                                                 Pl.offsets[level], Pl.n_off[level], level);
  return cudaGetLastError();
}

template <int P>
cudaError_t setup_p() {
  constexpr int EXT_TOP = P >= 7 ? 2 : 1;
  cudaError_t e = cudaFuncSetAttribute(k_m2l_fp32<P, EXT_TOP>, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
  if (e != cudaSuccess) return e;
  return cudaFuncSetAttribute(k_m2l_fp32<P, 0>, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
}

}  // namespace

cudaError_t setup_m2l_fp32(const Plan& P) {
  switch (P.p) {
    case 1: return setup_p<1>();
    case 2: return setup_p<2>();
    case 3: return setup_p<3>();
    case 4: return setup_p<4>();
    case 5: return setup_p<5>();
    case 6: return setup_p<6>();
    case 7: return setup_p<7>();
    case 8: return setup_p<8>();
    default: return cudaErrorInvalidValue;
  }
}

cudaError_t launch_m2l_fp32(Plan& P, int level, cudaStream_t s) {
  switch (P.p) {
    case 1: return launch_p<1>(P, level, s);
    case 2: return launch_p<2>(P, level, s);
    case 3: return launch_p<3>(P, level, s);
    case 4: return launch_p<4>(P, level, s);
    case 5: return launch_p<5>(P, level, s);
    case 6: return launch_p<6>(P, level, s);
    case 7: return launch_p<7>(P, level, s);
    case 8: return launch_p<8>(P, level, s);
    default: return cudaErrorInvalidValue;
  }
}

}  // namespace fmm

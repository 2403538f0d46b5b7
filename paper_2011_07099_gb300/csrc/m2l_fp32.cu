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
// different interaction lists, Sec. 2 Fig. fmm) and one contiguous range of
// the interaction offsets; thread r owns one target gridlet point and keeps
// NT x 4 accumulators.  The coarse levels have few targets (64 at level 2,
// 512 at level 3), so there the offsets are split over enough CTAs to fill
// the GPU, each range writes its own partial field, and a second kernel adds
// the partials in range order.  Per offset the CTA stages the
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

// NT targets per CTA (register budget: NT x 4 fields x (sum, compensation,
// plane, row) accumulators per thread).  The level-3 split-table kernel
// (EXT 1) takes 4, so that two CTAs share an SM: with 8 its 169 registers
// left one 7-warp CTA per SM, waiting on the table-window loads.
template <int P, int EXT = 0>
struct M2LShape {
  static constexpr int P3 = P * P * P;
  static constexpr int THREADS = ((P3 + 31) / 32) * 32 < 64 ? 64 : ((P3 + 31) / 32) * 32;
  static constexpr int NT = (P3 > 256 || EXT == 1) ? 4 : 8;
  static constexpr int PER_SM = EXT == 1 ? 2 : 1;        // CTAs per SM the launch bounds ask for
};

// EXT: 0 = FP32 table; 1 = the potential also takes G_lo; 2 = all four fields
// take their low halves; 3 = as 2, and the gridlet masses are read from their
// FP64 copy as hi + lo (the wide levels of high orders, whose masses are
// large alternating sums).
template <int P, int EXT>
__global__ void __launch_bounds__(M2LShape<P, EXT>::THREADS, M2LShape<P, EXT>::PER_SM)
k_m2l_fp32(const float* __restrict__ M, float* __restrict__ F, const float4* __restrict__ tab,
           const float4* __restrict__ tab_lo, const int8_t* __restrict__ offs, int n_off, int level,
           int per_split, size_t split_stride, int pairs, const double* __restrict__ M64, int iso) {
  constexpr int P3 = P * P * P;
  constexpr int NT = M2LShape<P, EXT>::NT;
  constexpr int D = 2 * P - 1;          // table window per dimension
  constexpr int D3 = D * D * D;
  constexpr int HW = 4 * P - 1, E = 8 * P - 1;
  extern __shared__ float4 sm4[];
  float4* win = sm4;                                     // D3 float4
  float4* msrc = win + D3;                               // P3 x (NT/4) float4: [s][k]
  float* win_lo = reinterpret_cast<float*>(msrc + P3 * (NT / 4));   // D3 floats (EXT == 1)
  float4* win_lo4 = msrc + P3 * (NT / 4);                            // D3 float4 (EXT >= 2)
  float4* msrc_lo = win_lo4 + D3;                                    // P3 x (NT/4) float4 (EXT == 3)
  const int tid = threadIdx.x, nthr = blockDim.x;
  const int ctype = blockIdx.y;
  const int n = 1 << level;
  const uint32_t n_par = 1u << (3 * (level - 1));
  const uint32_t par0 = blockIdx.x * NT;
  const int8_t* my_offs = offs + (size_t)ctype * n_off * 3;
  const int io0 = blockIdx.z * per_split;
  const int io1 = io0 + per_split < n_off ? io0 + per_split : n_off;
  // with `pairs`, each range writes (sum, -compensation): [range][hi | lo][field]
  const bool split = pairs != 0;
  F += 2 * (size_t)blockIdx.z * split_stride;

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

  __syncthreads();     // tx.. are set (also when the range is empty)
  for (int io = io0; io < io1; ++io) {
    const int ox = my_offs[3 * io + 0], oy = my_offs[3 * io + 1], oz = my_offs[3 * io + 2];
    __syncthreads();   // previous offset's compute is done with the buffers
    for (int i = tid; i < D3; i += nthr) {
      const int dx = i % D - (P - 1), dy = (i / D) % D - (P - 1), dz = i / (D * D) - (P - 1);
      const int nx = ox * P + dx + HW, ny = oy * P + dy + HW, nz = oz * P + dz + HW;
      win[i] = __ldg(tab + ((size_t)nz * E + ny) * E + nx);
      if (EXT == 1) win_lo[i] = __ldg(&tab_lo[((size_t)nz * E + ny) * E + nx].x);
      if (EXT >= 2) win_lo4[i] = __ldg(tab_lo + ((size_t)nz * E + ny) * E + nx);
    }
    float* ms = reinterpret_cast<float*>(msrc);
    float* ms_lo = reinterpret_cast<float*>(msrc_lo);
    for (int i = tid; i < NT * P3; i += nthr) {
      const int k = i / P3, s = i % P3;
      float v = 0.f, vlo = 0.f;
      // the source node T - o, wrapped (periodic) or, in the isolated
      // problem, skipped when it lies outside the box
      const int ux = tx[k] - ox, uy = ty[k] - oy, uz = tz[k] - oz;
      const bool inbox = (unsigned)ux < (unsigned)n && (unsigned)uy < (unsigned)n && (unsigned)uz < (unsigned)n;
      if (par0 + k < n_par && (inbox || !iso)) {
        const uint32_t sx = (uint32_t)ux & (n - 1), sy = (uint32_t)uy & (n - 1), sz = (uint32_t)uz & (n - 1);
        const size_t g = (size_t)morton(sx, sy, sz) * P3 + s;
        if (EXT == 3) {
          const double d = __ldg(M64 + g);
          v = (float)d;
          vlo = (float)(d - (double)v);
        } else {
          v = __ldg(M + g);
        }
      }
      ms[s * NT + k] = v;
      if (EXT == 3) ms_lo[s * NT + k] = vlo;
    }
    __syncthreads();
    if (r < P3) {
      constexpr int NLO = EXT >= 2 ? 4 : 1;
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
            const float4 tl = EXT >= 2 ? win_lo4[w] : make_float4(EXT == 1 ? win_lo[w] : 0.f, 0.f, 0.f, 0.f);
            const float4* mv = msrc + s * (NT / 4);
            const float4* mvl = msrc_lo + s * (NT / 4);
#pragma unroll
            for (int q = 0; q < NT / 4; ++q) {
              const float4 m = mv[q];
              const float mm[4] = {m.x, m.y, m.z, m.w};
              const float4 ml = EXT == 3 ? mvl[q] : make_float4(0.f, 0.f, 0.f, 0.f);
              const float mml[4] = {ml.x, ml.y, ml.z, ml.w};
#pragma unroll
              for (int j = 0; j < 4; ++j) {
                row[0][4 * q + j] = fmaf(t.x, mm[j], row[0][4 * q + j]);
                row[1][4 * q + j] = fmaf(t.y, mm[j], row[1][4 * q + j]);
                row[2][4 * q + j] = fmaf(t.z, mm[j], row[2][4 * q + j]);
                row[3][4 * q + j] = fmaf(t.w, mm[j], row[3][4 * q + j]);
                if (EXT >= 1) plo[0][4 * q + j] = fmaf(tl.x, mm[j], plo[0][4 * q + j]);
                if (EXT >= 2) {
                  plo[NLO - 3][4 * q + j] = fmaf(tl.y, mm[j], plo[NLO - 3][4 * q + j]);
                  plo[NLO - 2][4 * q + j] = fmaf(tl.z, mm[j], plo[NLO - 2][4 * q + j]);
                  plo[NLO - 1][4 * q + j] = fmaf(tl.w, mm[j], plo[NLO - 1][4 * q + j]);
                }
                if (EXT == 3) {
                  plo[0][4 * q + j] = fmaf(t.x, mml[j], plo[0][4 * q + j]);
                  plo[NLO - 3][4 * q + j] = fmaf(t.y, mml[j], plo[NLO - 3][4 * q + j]);
                  plo[NLO - 2][4 * q + j] = fmaf(t.z, mml[j], plo[NLO - 2][4 * q + j]);
                  plo[NLO - 1][4 * q + j] = fmaf(t.w, mml[j], plo[NLO - 1][4 * q + j]);
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
      for (int f = 0; f < 4; ++f) {
        if (split) {
          dst[f * P3 + r] = acc[f][k];
          dst[split_stride + f * P3 + r] = -comp[f][k];
        } else {
          dst[f * P3 + r] = acc[f][k] - comp[f][k];
        }
      }
    }
  }
}

// Level 2 (the first far-field level, 37 periodic interaction nodes, Sec. 2)
// carries the long-range potential: its terms are ~100 times larger than the
// potential they sum to, so FP32 products alone cost ~1e-6.  At order 8 on
// point-like clumps the cancellation reaches ~1000-fold at every level, so
// there every level above the leaves uses this kernel.  This kernel sums
// eq. fmm2 there in double-float arithmetic: every product with the split
// table value G_hi + G_lo is accumulated as an unevaluated sum (s, c) with
// error-free transformations (TwoProd by FMA, TwoSum; Ogita, Rump and Oishi,
// "Accurate sum and dot product", 2005), about 48 significant bits in FP32
// instructions; the FP64 pipe of this part would be ~6x slower.
// At high order (512 threads) one CTA per SM is the shared-memory limit
// anyway; saying so lets each thread keep its 2 x 4 x NT sums in registers.
template <int P>
__global__ void __launch_bounds__(M2LShape<P>::THREADS, P >= kWideOrder ? 1 : 2)
k_m2l_df(const float* __restrict__ M, float* __restrict__ F, const float4* __restrict__ tab,
         const float4* __restrict__ tab_lo, const int8_t* __restrict__ offs, int n_off, int level, int per_split,
         size_t split_stride, int pairs, const double* __restrict__ M64, int iso) {
  constexpr int P3 = P * P * P;
  constexpr int NT = M2LShape<P>::NT;
  constexpr int D = 2 * P - 1;
  constexpr int D3 = D * D * D;
  constexpr int HW = 4 * P - 1, E = 8 * P - 1;
  extern __shared__ float4 sm4[];
  float4* win = sm4;                       // D3
  float4* wlo = win + D3;                  // D3
  float4* msrc = wlo + D3;                 // P3 x (NT/4): [s][k]
  float4* mlo4 = msrc + P3 * (NT / 4);     // low halves of FP64 masses (M64 given)
  const int tid = threadIdx.x, nthr = blockDim.x;
  const int ctype = blockIdx.y;
  const int n = 1 << level;
  const uint32_t n_par = 1u << (3 * (level - 1));
  const uint32_t par0 = blockIdx.x * NT;
  const int8_t* my_offs = offs + (size_t)ctype * n_off * 3;
  const int io0 = blockIdx.z * per_split;
  const int io1 = io0 + per_split < n_off ? io0 + per_split : n_off;
  const bool split = pairs != 0;
  F += 2 * (size_t)blockIdx.z * split_stride;

  __shared__ int tx[NT], ty[NT], tz[NT];
  if (tid < NT) {
    uint32_t x = 0, y = 0, z = 0;
    if (par0 + tid < n_par) unmorton(8u * (par0 + tid) + ctype, x, y, z);
    tx[tid] = x; ty[tid] = y; tz[tid] = z;
  }
  float hs[4][NT], lc[4][NT];
#pragma unroll
  for (int f = 0; f < 4; ++f)
#pragma unroll
    for (int k = 0; k < NT; ++k) hs[f][k] = lc[f][k] = 0.f;
  const int r = tid;
  const int rx = r % P, ry = (r / P) % P, rz = r / (P * P);
  const int rbase = ((rz + P - 1) * D + (ry + P - 1)) * D + (rx + P - 1);

  __syncthreads();
  for (int io = io0; io < io1; ++io) {
    const int ox = my_offs[3 * io + 0], oy = my_offs[3 * io + 1], oz = my_offs[3 * io + 2];
    __syncthreads();
    for (int i = tid; i < D3; i += nthr) {
      const int dx = i % D - (P - 1), dy = (i / D) % D - (P - 1), dz = i / (D * D) - (P - 1);
      const size_t g = ((size_t)(oz * P + dz + HW) * E + (oy * P + dy + HW)) * E + (ox * P + dx + HW);
      win[i] = __ldg(tab + g);
      wlo[i] = __ldg(tab_lo + g);
    }
    float* ms = reinterpret_cast<float*>(msrc);
    float* msl = reinterpret_cast<float*>(mlo4);
    for (int i = tid; i < NT * P3; i += nthr) {
      const int k = i / P3, s = i % P3;
      float v = 0.f, vlo = 0.f;
      // the source node T - o, wrapped (periodic) or, in the isolated
      // problem, skipped when it lies outside the box
      const int ux = tx[k] - ox, uy = ty[k] - oy, uz = tz[k] - oz;
      const bool inbox = (unsigned)ux < (unsigned)n && (unsigned)uy < (unsigned)n && (unsigned)uz < (unsigned)n;
      if (par0 + k < n_par && (inbox || !iso)) {
        const uint32_t sx = (uint32_t)ux & (n - 1), sy = (uint32_t)uy & (n - 1), sz = (uint32_t)uz & (n - 1);
        const size_t g = (size_t)morton(sx, sy, sz) * P3 + s;
        if (M64) {
          const double d = __ldg(M64 + g);
          v = (float)d;
          vlo = (float)(d - (double)v);
        } else {
          v = __ldg(M + g);
        }
      }
      ms[s * NT + k] = v;
      if (M64) msl[s * NT + k] = vlo;
    }
    __syncthreads();
    if (r < P3) {
#pragma unroll 1
      for (int sz = 0; sz < P; ++sz)
#pragma unroll 1
        for (int sy = 0; sy < P; ++sy)
#pragma unroll
          for (int sx = 0; sx < P; ++sx) {
            const int s = (sz * P + sy) * P + sx;
            const int w = rbase - ((sz * D + sy) * D + sx);
            const float4 th = win[w], tl = wlo[w];
            const float gh[4] = {th.x, th.y, th.z, th.w}, gl[4] = {tl.x, tl.y, tl.z, tl.w};
            const float4* mv = msrc + s * (NT / 4);
#pragma unroll
            for (int q = 0; q < NT / 4; ++q) {
              const float4 m4 = mv[q];
              const float mm[4] = {m4.x, m4.y, m4.z, m4.w};
              const float4 l4 = M64 ? mlo4[s * (NT / 4) + q] : make_float4(0.f, 0.f, 0.f, 0.f);
              const float ml[4] = {l4.x, l4.y, l4.z, l4.w};
#pragma unroll
              for (int j = 0; j < 4; ++j) {
                const int k = 4 * q + j;
#pragma unroll
                for (int f = 0; f < 4; ++f) {
                  // _rn intrinsics: the compiler must not contract these into FMAs
                  const float pr = __fmul_rn(gh[f], mm[j]);
                  const float pe = fmaf(gh[f], mm[j], -pr);          // exact product error
                  const float t = __fadd_rn(hs[f][k], pr);            // TwoSum(hs, pr)
                  const float z = __fsub_rn(t, hs[f][k]);
                  const float se = __fadd_rn(__fsub_rn(hs[f][k], __fsub_rn(t, z)), __fsub_rn(pr, z));
                  hs[f][k] = t;
                  lc[f][k] = fmaf(gh[f], ml[j], fmaf(gl[f], mm[j], __fadd_rn(lc[f][k], __fadd_rn(pe, se))));
                }
              }
            }
          }
    }
  }
  if (r < P3) {
#pragma unroll
    for (int k = 0; k < NT; ++k) {
      if (par0 + k >= n_par) break;
      float* dst = F + (size_t)(8u * (par0 + k) + ctype) * 4 * P3;
#pragma unroll
      for (int f = 0; f < 4; ++f) {
        if (split) {
          dst[f * P3 + r] = hs[f][k];
          dst[split_stride + f * P3 + r] = lc[f][k];
        } else {
          dst[f * P3 + r] = hs[f][k] + lc[f][k];
        }
      }
    }
  }
}

// Coarse levels: F64[i] = sum over the offset ranges z = 0, 1, ... of the
// range sums part[z][0][i] plus their low parts part[z][1][i], in FP64 (the
// ranges' partial sums cancel heavily); F[i] gets the FP32 rounding.
__global__ void k_sum_ranges(const float* __restrict__ part, int nsplit, size_t n, double* __restrict__ F64,
                             float* __restrict__ F) {
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) {
    double v = 0.0;
    for (int z = 0; z < nsplit; ++z) v += (double)part[2 * z * n + i] + (double)part[(2 * z + 1) * n + i];
    F64[i] = v;
    F[i] = (float)v;
  }
}

template <int P>
cudaError_t launch_p(Plan& Pl, int level, cudaStream_t s) {
  constexpr int P3 = P * P * P;
  constexpr int D = 2 * P - 1;
  constexpr int EXT_TOP = P >= 7 ? 2 : 1;
  const int threads = M2LShape<P>::THREADS;
  const bool ext = level <= kExtTopLevel;          // split table
  const bool wide = wide_level(Pl, level);         // (sum, low part) outputs reduced in FP64
  const double* m64 = wide ? Pl.M64[level] : nullptr;   // FP64 masses: wide levels of the high orders
  const bool df = level == 2 || m64 || Pl.S >= kWideLeaf;
  // targets per CTA of the kernel that runs (m2l_fp32_pick)
  const int NT = (!df && ext) ? M2LShape<P, EXT_TOP>::NT : M2LShape<P>::NT;
  const size_t lo_bytes = ext ? (EXT_TOP == 2 ? sizeof(float4) : sizeof(float)) * D * D * D : 0;
  const size_t smem = sizeof(float4) * (D * D * D + P3 * (NT / 4)) + lo_bytes;
  const uint32_t n_par = 1u << (3 * (level - 1));
  const int nsplit = m2l_fp32_splits(Pl, level);
  const int n_off = Pl.n_off[level];
  const int per = (n_off + nsplit - 1) / nsplit;
  const size_t field = ((size_t)1 << (3 * level)) * 4 * P3;
  // wide levels write (sum, low part) pairs per offset range, reduced in FP64
  float* out = wide ? Pl.m2l_part : Pl.F[level];
  dim3 grid((n_par + NT - 1) / NT, 8, nsplit);
  // double-float sums: level 2, every wide level of the high orders, and
  // every level with 16-cell leaves (whose L2P amplifies the rounding of the
  // sums that varies from one gridlet point to the next)
  if (df)
    k_m2l_df<P><<<grid, threads, sizeof(float4) * (2 * D * D * D + 2 * P3 * (NT / 4)), s>>>(
        Pl.M[level], out, Pl.tab[level], Pl.tab_lo[level], Pl.offsets[level], n_off, level, per, field, 1, m64,
        Pl.iso);
  else if (m64)
    k_m2l_fp32<P, 3><<<grid, threads, sizeof(float4) * (2 * D * D * D + 2 * P3 * (NT / 4)), s>>>(
        Pl.M[level], out, Pl.tab[level], Pl.tab_lo[level], Pl.offsets[level], n_off, level, per, field, 1, m64,
        Pl.iso);
  else if (ext)
    k_m2l_fp32<P, EXT_TOP><<<grid, threads, smem, s>>>(Pl.M[level], out, Pl.tab[level], Pl.tab_lo[level],
                                                       Pl.offsets[level], n_off, level, per, field, 1, nullptr,
                                                       Pl.iso);
  else
    k_m2l_fp32<P, 0><<<grid, threads, smem, s>>>(Pl.M[level], out, Pl.tab[level], nullptr, Pl.offsets[level],
                                                 n_off, level, per, field, wide ? 1 : 0, nullptr, Pl.iso);
  if (wide) k_sum_ranges<<<4 * Pl.num_sms, 256, 0, s>>>(Pl.m2l_part, nsplit, field, Pl.F64[level], Pl.F[level]);
  return cudaGetLastError();
}

// FP32 M2L over a caller's offset list (same list for the 8 child types),
// written straight into F[level]: the near-node part that the FFT form of
// the interaction zone subtracts (m2l_fft.cu).
template <int P>
cudaError_t launch_list_p(Plan& Pl, int level, const int8_t* offs, int n_off, cudaStream_t s) {
  constexpr int P3 = P * P * P, D = 2 * P - 1, NT = M2LShape<P>::NT;
  const size_t smem = sizeof(float4) * (D * D * D + P3 * (NT / 4));
  const uint32_t n_par = 1u << (3 * (level - 1));
  dim3 grid((n_par + NT - 1) / NT, 8, 1);
  k_m2l_fp32<P, 0><<<grid, M2LShape<P>::THREADS, smem, s>>>(Pl.M[level], Pl.F[level], Pl.tab[level], nullptr, offs,
                                                            n_off, level, n_off, 0, 0, nullptr, Pl.iso);
  return cudaGetLastError();
}

template <int P>
cudaError_t setup_p() {
  constexpr int EXT_TOP = P >= 7 ? 2 : 1;
  cudaError_t e = cudaFuncSetAttribute(k_m2l_df<P>, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
  if (e != cudaSuccess) return e;
  e = cudaFuncSetAttribute(k_m2l_fp32<P, 3>, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
  if (e != cudaSuccess) return e;
  e = cudaFuncSetAttribute(k_m2l_fp32<P, EXT_TOP>, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
  if (e != cudaSuccess) return e;
  return cudaFuncSetAttribute(k_m2l_fp32<P, 0>, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
}

}  // namespace

int m2l_fp32_splits(const Plan& P, int level) {
  if (level > kExtTopLevel) return 1;     // fine levels have targets enough
  // the level-3 split-table kernel of orders < 7: 4 targets per CTA, two
  // CTAs per SM (M2LShape); the others 8 (4 above 256 gridlet points), one
  const bool df = level == 2 || (P.p >= kWideOrder && wide_level(P, level)) || P.S >= kWideLeaf;
  const bool ext1 = !df && P.p < kWideOrder;
  const int nt = (P.p * P.p * P.p > 256 || ext1) ? 4 : 8;
  const long ctas = (long)(((1u << (3 * (level - 1))) + nt - 1) / nt) * 8;
  const long sms = (P.num_sms > 0 ? P.num_sms : 1) * (ext1 ? 2 : 1);
  // at least ~4 waves of one CTA per SM, and the range count whose last wave
  // is fullest (these CTAs hold one SM each: registers)
  long lo = (4 * sms + ctas - 1) / ctas, hi = 3 * lo;
  if (hi > P.n_off[level]) hi = P.n_off[level];
  if (lo > hi) lo = hi;
  long best = lo < 1 ? 1 : lo;
  double best_eff = -1.0;
  for (long ns = best; ns <= hi; ++ns) {
    const long waves = (ctas * ns + sms - 1) / sms;
    const double eff = (double)(ctas * ns) / (double)(waves * sms);
    if (eff > best_eff + 1e-9) {
      best_eff = eff;
      best = ns;
    }
  }
  return (int)best;
}

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

cudaError_t launch_m2l_fp32_list(Plan& P, int level, const int8_t* offs, int n_off, cudaStream_t s) {
  switch (P.p) {
    case 1: return launch_list_p<1>(P, level, offs, n_off, s);
    case 2: return launch_list_p<2>(P, level, offs, n_off, s);
    case 3: return launch_list_p<3>(P, level, offs, n_off, s);
    case 4: return launch_list_p<4>(P, level, offs, n_off, s);
    case 5: return launch_list_p<5>(P, level, offs, n_off, s);
    case 6: return launch_list_p<6>(P, level, offs, n_off, s);
    case 7: return launch_list_p<7>(P, level, offs, n_off, s);
    case 8: return launch_list_p<8>(P, level, offs, n_off, s);
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

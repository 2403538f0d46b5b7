// Leaf stage: L2P plus the near-zone direct sum (P2P), fused, writing the
// final potential and acceleration of every cell.
//
// Far field (eq. fmm3 at the leaves): the leaf's local field interpolated at
// its cell centres by the transpose of the P2M matrix.
// Near field (Sec. 2, part 3 of the potential; Sec. 3: it must use the same G
// as the PM solution): for the 27 periodic neighbour leaves of the target leaf,
//   Phi_i += sum_j G_S1(x_i - x_j) m_j,   g_i += sum_j (-grad G_S1)(x_i - x_j) m_j.
//
// Work split: one CTA per target leaf.  The (3S)^3 source window (masses
// m = (rho - mean)/N^3 with periodic wrap) and the near table folded over the
// sign of each offset component are staged in shared memory.  Thread
// (cz, cy, zg) owns one target row of S cells x 4 fields and sums the source
// planes zg, zg + NZG, ...; the groups are reduced through shared memory.
// Within a source row the x offsets between the S targets and 3S sources are
// compile-time constants, so each table value is a register and each FMA's
// sign is resolved at compile time.
#include "fmm_internal.cuh"

namespace fmm {
namespace {

template <int S>
struct P2PShape {
  static constexpr int W = 3 * S;                 // window width
  static constexpr int TD = 2 * S;                // folded table extent
  static constexpr int TS = 2 * S + 1;            // padded x stride (bank spread)
  static constexpr int ROWS = S * S;
  static constexpr int NZG = (256 / ROWS) < W ? ((256 / ROWS) > 0 ? 256 / ROWS : 1) : W;
  static constexpr int THREADS = ROWS * NZG;
};

template <int S>
__global__ void __launch_bounds__(P2PShape<S>::THREADS)
k_p2p(const float* __restrict__ rho, const double* __restrict__ mean, int N, int p,
      const float4* __restrict__ near_tab, const float* __restrict__ Fleaf, const float2* __restrict__ wp2m,
      float* __restrict__ phi, float* __restrict__ acc_out, int region_floats) {
  using Sh = P2PShape<S>;
  constexpr int W = Sh::W, TD = Sh::TD, TS = Sh::TS, ROWS = Sh::ROWS, NZG = Sh::NZG;
  extern __shared__ float4 sm4[];
  float4* tab = sm4;                                        // TD*TD*TS
  float* far = reinterpret_cast<float*>(tab + TD * TD * TS);  // 4*S^3
  float* region = far + 4 * S * S * S;                      // window / L2P scratch / reduction
  const int tid = threadIdx.x, nthr = blockDim.x;
  uint32_t lx, ly, lz;
  unmorton(blockIdx.x, lx, ly, lz);
  const int p3 = p * p * p;

  // folded near table
  for (int i = tid; i < TD * TD * TD; i += nthr) {
    const int dx = i % TD, dy = (i / TD) % TD, dz = i / (TD * TD);
    tab[(dz * TD + dy) * TS + dx] = __ldg(near_tab + i);
  }
  // L2P: far[f][cz][cy][cx] = sum_s l_s(cz) l_s(cy) l_s(cx) F[f][s]
  {
    float2* W8 = reinterpret_cast<float2*>(region);   // p*S weights (region is 16-byte aligned)
    float* in = reinterpret_cast<float*>(W8 + p * S); // 4*p^3
    float* t1 = in + 4 * p3;              // 4*p*p*S
    float* t2 = t1 + 4 * p * p * S;       // 4*p*S*S
    for (int i = tid; i < p * S; i += nthr) W8[i] = wp2m[i];
    const float* src = Fleaf + (size_t)blockIdx.x * 4 * p3;
    for (int i = tid; i < 4 * p3; i += nthr) in[i] = src[i];
    __syncthreads();
    contract3(in, t1, t2, far, 4, p, S, W8, S, true, tid, nthr);
  }
  // source window with periodic wrap
  float* win = region;
  {
    const double mu = *mean;
    const double inv_vol = 1.0 / ((double)N * N * N);
    const int x0 = (int)lx * S - S, y0 = (int)ly * S - S, z0 = (int)lz * S - S;
    for (int i = tid; i < W * W * W; i += nthr) {
      const int wx = i % W, wy = (i / W) % W, wz = i / (W * W);
      const int gx = (x0 + wx + N) % N, gy = (y0 + wy + N) % N, gz = (z0 + wz + N) % N;
      win[i] = (float)(((double)__ldg(rho + ((size_t)gz * N + gy) * N + gx) - mu) * inv_vol);
    }
  }
  __syncthreads();

  const int row = tid % ROWS, zg = tid / ROWS;
  const int cz = row / S, cy = row % S;
  float a[4][S];
#pragma unroll
  for (int f = 0; f < 4; ++f)
#pragma unroll
    for (int x = 0; x < S; ++x) a[f][x] = 0.f;

  // Rounding: each source row's 3S terms go into a fresh row partial, rows into
  // a plane partial, planes into the total, so no running FP32 sum is longer
  // than 3S terms (a single running sum over the 27 S^3 sources loses about
  // log10(sqrt(27 S^3)) more digits).
  if (zg < NZG) {
    for (int zp = zg; zp < W; zp += NZG) {
      const int dz = cz + S - zp;                         // target z - source z (cells)
      const int adz = dz < 0 ? -dz : dz;
      const float sz = dz > 0 ? 1.f : (dz < 0 ? -1.f : 0.f);
      float pl[4][S];
#pragma unroll
      for (int f = 0; f < 4; ++f)
#pragma unroll
        for (int x = 0; x < S; ++x) pl[f][x] = 0.f;
#pragma unroll 1
      for (int yp = 0; yp < W; ++yp) {
        const int dy = cy + S - yp;
        const int ady = dy < 0 ? -dy : dy;
        const float sy = dy > 0 ? 1.f : (dy < 0 ? -1.f : 0.f);
        const float4* trow = tab + (adz * TD + ady) * TS;
        float4 t[TD];
#pragma unroll
        for (int j = 0; j < TD; ++j) t[j] = trow[j];
        const float* mrow = win + (zp * W + yp) * W;
        float rw[4][S];
#pragma unroll
        for (int f = 0; f < 4; ++f)
#pragma unroll
          for (int x = 0; x < S; ++x) rw[f][x] = 0.f;
#pragma unroll
        for (int xp = 0; xp < W; ++xp) {
          const float m = mrow[xp];
          const float my = sy * m, mz = sz * m;
#pragma unroll
          for (int x = 0; x < S; ++x) {
            const int dx = x + S - xp;                    // compile-time after unrolling
            const int adx = dx < 0 ? -dx : dx;
            const float4 v = t[adx];
            rw[0][x] = fmaf(v.x, m, rw[0][x]);
            rw[1][x] = dx >= 0 ? fmaf(v.y, m, rw[1][x]) : fmaf(-v.y, m, rw[1][x]);
            rw[2][x] = fmaf(v.z, my, rw[2][x]);
            rw[3][x] = fmaf(v.w, mz, rw[3][x]);
          }
        }
#pragma unroll
        for (int f = 0; f < 4; ++f)
#pragma unroll
          for (int x = 0; x < S; ++x) pl[f][x] += rw[f][x];
      }
#pragma unroll
      for (int f = 0; f < 4; ++f)
#pragma unroll
        for (int x = 0; x < S; ++x) a[f][x] += pl[f][x];
    }
  }
  __syncthreads();   // window no longer needed: reuse the region for the reduction
  float* red = region;   // [NZG][4][S][ROWS]
  if (zg < NZG && zg > 0) {
#pragma unroll
    for (int f = 0; f < 4; ++f)
#pragma unroll
      for (int x = 0; x < S; ++x) red[((zg * 4 + f) * S + x) * ROWS + row] = a[f][x];
  }
  __syncthreads();
  if (zg == 0) {
    for (int g = 1; g < NZG; ++g)
#pragma unroll
      for (int f = 0; f < 4; ++f)
#pragma unroll
        for (int x = 0; x < S; ++x) a[f][x] += red[((g * 4 + f) * S + x) * ROWS + row];
    const size_t N3 = (size_t)N * N * N;
    const size_t base = ((size_t)(lz * S + cz) * N + (ly * S + cy)) * N + lx * S;
#pragma unroll
    for (int x = 0; x < S; ++x) {
      const int c = (cz * S + cy) * S + x;
      phi[base + x] = a[0][x] + far[0 * S * S * S + c];
      acc_out[base + x] = a[1][x] + far[1 * S * S * S + c];
      acc_out[N3 + base + x] = a[2][x] + far[2 * S * S * S + c];
      acc_out[2 * N3 + base + x] = a[3][x] + far[3 * S * S * S + c];
    }
  }
  (void)region_floats;
}

template <int S>
cudaError_t launch_s(Plan& P, const float* rho, float* phi, float* acc, cudaStream_t s) {
  using Sh = P2PShape<S>;
  const int p = P.p, p3 = p * p * p;
  const int win = Sh::W * Sh::W * Sh::W;
  const int l2p = 2 * p * S + 4 * p3 + 4 * p * p * S + 4 * p * S * S;
  const int red = Sh::NZG * 4 * S * Sh::ROWS;
  int region = win;
  if (l2p > region) region = l2p;
  if (red > region) region = red;
  const size_t smem = sizeof(float4) * Sh::TD * Sh::TD * Sh::TS + sizeof(float) * (4 * S * S * S + region);
  const unsigned leaves = 1u << (3 * P.L);
  k_p2p<S><<<leaves, Sh::THREADS, smem, s>>>(rho, P.d_mean, P.N, p, P.near_tab, P.F[P.L], P.w_p2m, phi, acc,
                                             region);
  return cudaGetLastError();
}

template <int S>
cudaError_t setup_s() {
  return cudaFuncSetAttribute(k_p2p<S>, cudaFuncAttributeMaxDynamicSharedMemorySize, 220 * 1024);
}

}  // namespace

cudaError_t setup_p2p(const Plan& P) {
  switch (P.S) {
    case 1: return setup_s<1>();
    case 2: return setup_s<2>();
    case 3: return setup_s<3>();
    case 4: return setup_s<4>();
    case 6: return setup_s<6>();
    case 8: return setup_s<8>();
    default: return cudaErrorInvalidValue;
  }
}

cudaError_t launch_p2p(Plan& P, const float* rho, float* phi, float* acc, cudaStream_t s) {
  switch (P.S) {
    case 1: return launch_s<1>(P, rho, phi, acc, s);
    case 2: return launch_s<2>(P, rho, phi, acc, s);
    case 3: return launch_s<3>(P, rho, phi, acc, s);
    case 4: return launch_s<4>(P, rho, phi, acc, s);
    case 6: return launch_s<6>(P, rho, phi, acc, s);
    case 8: return launch_s<8>(P, rho, phi, acc, s);
    default: return cudaErrorInvalidValue;
  }
}

}  // namespace fmm

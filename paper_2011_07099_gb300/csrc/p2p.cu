// Leaf stage: L2P plus the near-zone direct sum (P2P), fused, writing the
// final potential and acceleration of every cell.
//
// Far field (eq. fmm3 at the leaves): the leaf's local field interpolated at
// its cell centres by the transpose of the P2M matrix.
// Near field (Sec. 2, part 3 of the potential; Sec. 3: it must use the same G
// as the PM solution): for the 27 periodic neighbour leaves of the target leaf,
//   Phi_i += sum_j G_S1(x_i - x_j) m_j,   g_i += sum_j (-grad G_S1)(x_i - x_j) m_j.
//
// Work split: a persistent CTA (one per SM, or as many as fit) walks the
// leaves blockIdx.x, blockIdx.x + gridDim.x, ...  The near table, folded over
// the sign of each offset component, is staged in shared memory once per CTA.
// Per leaf, the (3S)^3 density window (periodic wrap) and the leaf's local
// field are fetched with cp.async one leaf ahead, into the other half of a
// double buffer, so the copies of leaf i+1 run under the arithmetic of leaf
// i.  Masses m = (rho - mean)/N^3 are formed in FP32 from the mean split into
// hi + lo (one rounding more than an FP64 subtraction, well inside FP32
// parity; the FP64 pipe would otherwise hold every warp for ~8 % of the
// kernel).  Thread (cz, cy, zg) owns one target row of S cells x 4 fields and
// sums the source planes zg, zg + NZG, ...; the groups are reduced through
// shared memory.  Within a source row the x offsets between the S targets
// and 3S sources are compile-time constants, so each table value is a
// register and each FMA's sign is resolved at compile time.
#include "fmm_internal.cuh"
#include "tc_ptx.cuh"

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
  static constexpr int RED = NZG * 4 * S * ROWS;  // reduction floats
  static constexpr int WIN = W * W * W;
  // one window buffer, also the reduction scratch of its leaf (16-byte multiple)
  static constexpr int WBUF = ((WIN > RED ? WIN : RED) + 3) / 4 * 4;
};

// Shared-memory carve-up (floats after the float4 table), for order p.
template <int S>
struct P2PSmem {
  int far, w8, t1, t2, in0, in1, win0, win1, total;   // offsets in floats from the table end
  __host__ __device__ P2PSmem(int p) {
    using Sh = P2PShape<S>;
    const int p3 = p * p * p;
    far = 0;
    w8 = far + 4 * S * S * S;                       // p*S float2 (16-byte aligned: 4 S^3 floats)
    w8 = (w8 + 3) / 4 * 4;
    t1 = w8 + 2 * p * S;
    t2 = t1 + 4 * p * p * S;
    in0 = (t2 + 4 * p * S * S + 3) / 4 * 4;
    in1 = in0 + 4 * p3;                             // 4 p^3 floats: a 16-byte multiple
    win0 = in1 + 4 * p3;
    win1 = win0 + Sh::WBUF;
    total = win1 + Sh::WBUF;
  }
};

template <int S>
__global__ void __launch_bounds__(P2PShape<S>::THREADS, 1)
k_p2p(const float* __restrict__ rho, const double* __restrict__ mean, int N, int L, int p,
      const float4* __restrict__ near_tab, const float* __restrict__ Fleaf, const float2* __restrict__ wp2m,
      float* __restrict__ phi, float* __restrict__ acc_out, int vec) {
  using Sh = P2PShape<S>;
  constexpr int W = Sh::W, TD = Sh::TD, TS = Sh::TS, ROWS = Sh::ROWS, NZG = Sh::NZG;
  extern __shared__ float4 sm4[];
  float4* tab = sm4;                                             // TD*TD*TS
  float* base = reinterpret_cast<float*>(tab + TD * TD * TS);
  const P2PSmem<S> lay(p);
  float* far = base + lay.far;
  float2* W8 = reinterpret_cast<float2*>(base + lay.w8);
  float* t1 = base + lay.t1;
  float* t2 = base + lay.t2;
  const int tid = threadIdx.x, nthr = blockDim.x;
  const int p3 = p * p * p;
  const unsigned nleaves = 1u << (3 * L);
  const size_t N3 = (size_t)N * N * N;

  for (int i = tid; i < TD * TD * TD; i += nthr) {
    const int dx = i % TD, dy = (i / TD) % TD, dz = i / (TD * TD);
    tab[(dz * TD + dy) * TS + dx] = __ldg(near_tab + i);
  }
  for (int i = tid; i < p * S; i += nthr) W8[i] = wp2m[i];
  const double mu = *mean;
  const float mu_hi = (float)mu, mu_lo = (float)(mu - (double)mu_hi);
  const float inv_vol = (float)(1.0 / ((double)N * N * N));

  // cp.async of one leaf's density window and local field into buffer b
  auto fetch = [&](unsigned leaf, int b) {
    uint32_t lx, ly, lz;
    unmorton(leaf, lx, ly, lz);
    const int x0 = (int)lx * S - S, y0 = (int)ly * S - S, z0 = (int)lz * S - S;
    float* win = base + (b ? lay.win1 : lay.win0);
    float* in = base + (b ? lay.in1 : lay.in0);
    if (S % 4 == 0 && vec) {         // 16-byte aligned density: 4 cells per copy
      constexpr int C = S % 4 == 0 ? W / 4 : 1;
      for (int i = tid; i < W * W * C; i += nthr) {
        const int c = i % C, wy = (i / C) % W, wz = i / (C * W);
        const int gx = (x0 + 4 * c + N) % N, gy = (y0 + wy + N) % N, gz = (z0 + wz + N) % N;
        tc::cp_async16(tc::smem_u32(win + (wz * W + wy) * W + 4 * c), rho + ((size_t)gz * N + gy) * N + gx, 16u);
      }
    } else {
      for (int i = tid; i < W * W * W; i += nthr) {
        const int wx = i % W, wy = (i / W) % W, wz = i / (W * W);
        const int gx = (x0 + wx + N) % N, gy = (y0 + wy + N) % N, gz = (z0 + wz + N) % N;
        tc::cp_async4(tc::smem_u32(win + i), rho + ((size_t)gz * N + gy) * N + gx);
      }
    }
    const float* src = Fleaf + (size_t)leaf * 4 * p3;
    for (int i = tid; i < p3; i += nthr) tc::cp_async16(tc::smem_u32(in + 4 * i), src + 4 * i, 16u);
    tc::cp_async_commit();
  };

  unsigned leaf = blockIdx.x;
  if (leaf < nleaves) fetch(leaf, 0);
  for (int b = 0; leaf < nleaves; leaf += gridDim.x, b ^= 1) {
    float* win = base + (b ? lay.win1 : lay.win0);
    float* in = base + (b ? lay.in1 : lay.in0);
    tc::cp_async_wait<0>();
    __syncthreads();     // the leaf's data landed; the previous leaf's epilogue is done
    for (int i = tid; i < W * W * W; i += nthr) win[i] = ((win[i] - mu_hi) - mu_lo) * inv_vol;
    // L2P: far[f][cz][cy][cx] = sum_s l_s(cz) l_s(cy) l_s(cx) F[f][s]  (ends with a barrier,
    // which also publishes the masses)
    contract3(in, t1, t2, far, 4, p, S, W8, S, true, tid, nthr);
    if (leaf + gridDim.x < nleaves) fetch(leaf + gridDim.x, b ^ 1);
    uint32_t lx, ly, lz;
    unmorton(leaf, lx, ly, lz);

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
#pragma unroll
            for (int x = 0; x < S; ++x) {
              const int dx = x + S - xp;                    // compile-time after unrolling
              const int adx = dx < 0 ? -dx : dx;
              const float4 v = t[adx];
              rw[0][x] = fmaf(v.x, m, rw[0][x]);
              rw[1][x] = dx >= 0 ? fmaf(v.y, m, rw[1][x]) : fmaf(-v.y, m, rw[1][x]);
              rw[2][x] = fmaf(v.z, m, rw[2][x]);            // sign of dy applied per row
              rw[3][x] = fmaf(v.w, m, rw[3][x]);            // sign of dz applied per plane
            }
          }
#pragma unroll
          for (int x = 0; x < S; ++x) {
            pl[0][x] += rw[0][x];
            pl[1][x] += rw[1][x];
            pl[2][x] = fmaf(sy, rw[2][x], pl[2][x]);       // sy in {-1, 0, 1}: exact
            pl[3][x] += rw[3][x];
          }
        }
#pragma unroll
        for (int x = 0; x < S; ++x) {
          a[0][x] += pl[0][x];
          a[1][x] += pl[1][x];
          a[2][x] += pl[2][x];
          a[3][x] = fmaf(sz, pl[3][x], a[3][x]);
        }
      }
    }
    __syncthreads();   // window no longer read: it becomes the reduction scratch
    float* red = win;   // [NZG][4][S][ROWS]
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
      const size_t o = ((size_t)(lz * S + cz) * N + (ly * S + cy)) * N + lx * S;
#pragma unroll
      for (int x = 0; x < S; ++x) {
        const int c = (cz * S + cy) * S + x;
        phi[o + x] = a[0][x] + far[0 * S * S * S + c];
        acc_out[o + x] = a[1][x] + far[1 * S * S * S + c];
        acc_out[N3 + o + x] = a[2][x] + far[2 * S * S * S + c];
        acc_out[2 * N3 + o + x] = a[3][x] + far[3 * S * S * S + c];
      }
    }
  }
}

template <int S>
size_t smem_s(int p) {
  using Sh = P2PShape<S>;
  return sizeof(float4) * Sh::TD * Sh::TD * Sh::TS + sizeof(float) * (size_t)P2PSmem<S>(p).total;
}

template <int S>
cudaError_t launch_s(Plan& P, const float* rho, float* phi, float* acc, cudaStream_t s) {
  using Sh = P2PShape<S>;
  const size_t smem = smem_s<S>(P.p);
  const unsigned leaves = 1u << (3 * P.L);
  int per_sm = 1;
  cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_p2p<S>, Sh::THREADS, smem);
  if (e != cudaSuccess) return e;
  if (per_sm < 1) return cudaErrorInvalidConfiguration;
  const unsigned slots = (unsigned)(per_sm * P.num_sms);
  const unsigned grid = leaves < slots ? leaves : slots;
  const int vec = (S % 4 == 0) && ((reinterpret_cast<uintptr_t>(rho) & 15u) == 0);
  k_p2p<S><<<grid, Sh::THREADS, smem, s>>>(rho, P.d_mean, P.N, P.L, P.p, P.near_tab, P.F[P.L], P.w_p2m, phi, acc, vec);
  return cudaGetLastError();
}

template <int S>
cudaError_t setup_s() {
  return cudaFuncSetAttribute(k_p2p<S>, cudaFuncAttributeMaxDynamicSharedMemorySize, 225 * 1024);
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

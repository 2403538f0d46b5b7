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
      float* __restrict__ phi, float* __restrict__ acc_out, int vec, int iso) {
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
        const int ux = x0 + 4 * c, uy = y0 + wy, uz = z0 + wz;
        const int gx = (ux + N) % N, gy = (uy + N) % N, gz = (uz + N) % N;
        // isolated problem: cells outside the box hold no mass (zero fill)
        const bool out = iso && (gx != ux || gy != uy || gz != uz);
        tc::cp_async16(tc::smem_u32(win + (wz * W + wy) * W + 4 * c), rho + ((size_t)gz * N + gy) * N + gx,
                       out ? 0u : 16u);
      }
    } else {
      for (int i = tid; i < W * W * W; i += nthr) {
        const int wx = i % W, wy = (i / W) % W, wz = i / (W * W);
        const int ux = x0 + wx, uy = y0 + wy, uz = z0 + wz;
        const int gx = (ux + N) % N, gy = (uy + N) % N, gz = (uz + N) % N;
        const bool out = iso && (gx != ux || gy != uy || gz != uz);
        tc::cp_async4_zfill(tc::smem_u32(win + i), rho + ((size_t)gz * N + gy) * N + gx, out ? 0u : 4u);
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
          // 16-byte aligned rows (S % 4 == 0: W and the buffers are multiples
          // of 4 floats): the masses come in as float4, four at a time
          float mq[4];
#pragma unroll
          for (int xp = 0; xp < W; ++xp) {
            if (S % 4 == 0 && xp % 4 == 0) {
              const float4 q4 = *reinterpret_cast<const float4*>(mrow + xp);
              mq[0] = q4.x;
              mq[1] = q4.y;
              mq[2] = q4.z;
              mq[3] = q4.w;
            }
            const float m = S % 4 == 0 ? mq[xp % 4] : mrow[xp];
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

// Leaf size 16, the sub-grid of the paper's accuracy experiment (Sec. 3:
// 16^3 cells per node, significantly more than the gridlet).  The 48^3 window
// and the 32^3 folded table do not fit in shared memory, so the window is
// streamed one source plane at a time (cp.async double buffer) and the table
// is read through the L1 cache.  Two CTAs per leaf (target planes 0-7 and
// 8-15) of 256 threads: thread (cz, cy, h) owns the 8 cells x in [8h, 8h + 8)
// of target row (cz, cy), 4 fields.  A source row's 48 cells are taken 8 at a
// time: for chunk c the offsets dx = 8 (2 + h - c) + (x - xs) span 15
// consecutive values, whose table entries are loaded into registers once per
// chunk; the sign of dx is the same for the whole chunk except in the
// target's own chunk (base 0), where it is resolved at compile time.  The
// summation keeps the row -> plane -> total partial sums of the kernel above.
// L2P runs in double-float from the leaf's FP64 local field (every level is
// wide with 16-cell leaves, fmm_internal.cuh): the cells at the edges of a
// 16-cell leaf lie well outside the order-p gridlet's hull (absolute weight
// sums up to 835 at p = 6 against 46 for 8-cell leaves), which amplifies any
// FP32 rounding of the field or of the partial sums at the leaf's edges.
constexpr int kS16 = 16, kW16 = 48, kT16 = 256;

struct P2P16Smem {
  int far, w8, t1, t2, o2, in2, pl0, pl1, total;   // offsets in floats
  __host__ __device__ P2P16Smem(int p) {
    far = 0;                                      // 4 S^3 floats
    w8 = 4 * kS16 * kS16 * kS16;                  // p S float2
    t1 = w8 + 2 * p * kS16;                       // p p S float2
    t2 = t1 + 2 * p * p * kS16;                   // p S S float2
    o2 = t2 + 2 * p * kS16 * kS16;                // S^3 float2
    in2 = o2 + 2 * kS16 * kS16 * kS16;            // p^3 float2
    pl0 = (in2 + 2 * p * p * p + 3) / 4 * 4;
    pl1 = pl0 + kW16 * kW16;
    total = pl1 + kW16 * kW16;
  }
};

template <int SGN>   // +1: every dx > 0, -1: every dx < 0, 0: dx = x - xs
__device__ __forceinline__ void p2p16_chunk(float rw[4][8], const float4 t[15], const float m[8]) {
#pragma unroll
  for (int xs = 0; xs < 8; ++xs) {
#pragma unroll
    for (int x = 0; x < 8; ++x) {
      const float4 v = t[x - xs + 7];
      rw[0][x] = fmaf(v.x, m[xs], rw[0][x]);
      const bool neg = SGN < 0 || (SGN == 0 && x < xs);
      rw[1][x] = neg ? fmaf(-v.y, m[xs], rw[1][x]) : fmaf(v.y, m[xs], rw[1][x]);
      rw[2][x] = fmaf(v.z, m[xs], rw[2][x]);
      rw[3][x] = fmaf(v.w, m[xs], rw[3][x]);
    }
  }
}

__global__ void __launch_bounds__(kT16, 1)
k_p2p16(const float* __restrict__ rho, const double* __restrict__ mean, int N, int L, int p,
        const float4* __restrict__ near_tab, const double* __restrict__ Fleaf, const float2* __restrict__ wp2m,
        float* __restrict__ phi, float* __restrict__ acc_out, int vec, int iso) {
  extern __shared__ float4 sm4[];
  float* base = reinterpret_cast<float*>(sm4);
  const P2P16Smem lay(p);
  float* far = base + lay.far;
  float2* W8 = reinterpret_cast<float2*>(base + lay.w8);
  const int tid = threadIdx.x, nthr = blockDim.x;
  const int p3 = p * p * p;
  const unsigned leaf = blockIdx.x >> 1;
  const int zh = blockIdx.x & 1;
  const size_t N3 = (size_t)N * N * N;
  uint32_t lx, ly, lz;
  unmorton(leaf, lx, ly, lz);
  const int x0 = (int)lx * kS16 - kS16, y0 = (int)ly * kS16 - kS16, z0 = (int)lz * kS16 - kS16;
  const double mu = *mean;
  const float mu_hi = (float)mu, mu_lo = (float)(mu - (double)mu_hi);
  const float inv_vol = (float)(1.0 / ((double)N * N * N));

  // cp.async of source plane zp of the window (periodic wrap; zero fill
  // outside the box in the isolated problem) into plane buffer b
  auto fetch = [&](int zp, int b) {
    float* pln = base + (b ? lay.pl1 : lay.pl0);
    const int uz = z0 + zp, gz = (uz + N) % N;
    const bool outz = iso && gz != uz;
    if (vec) {
      for (int i = tid; i < kW16 * (kW16 / 4); i += nthr) {
        const int c = i % (kW16 / 4), wy = i / (kW16 / 4);
        const int ux = x0 + 4 * c, uy = y0 + wy;
        const int gx = (ux + N) % N, gy = (uy + N) % N;
        const bool out = outz || (iso && (gx != ux || gy != uy));
        tc::cp_async16(tc::smem_u32(pln + wy * kW16 + 4 * c), rho + ((size_t)gz * N + gy) * N + gx, out ? 0u : 16u);
      }
    } else {
      for (int i = tid; i < kW16 * kW16; i += nthr) {
        const int wx = i % kW16, wy = i / kW16;
        const int ux = x0 + wx, uy = y0 + wy;
        const int gx = (ux + N) % N, gy = (uy + N) % N;
        const bool out = outz || (iso && (gx != ux || gy != uy));
        tc::cp_async4_zfill(tc::smem_u32(pln + i), rho + ((size_t)gz * N + gy) * N + gx, out ? 0u : 4u);
      }
    }
    tc::cp_async_commit();
  };

  fetch(0, 0);
  for (int i = tid; i < p * kS16; i += nthr) W8[i] = wp2m[i];
  // L2P of the whole leaf, one field at a time, in double-float
  {
    float2* in2 = reinterpret_cast<float2*>(base + lay.in2);
    float2* o2 = reinterpret_cast<float2*>(base + lay.o2);
    constexpr int S3 = kS16 * kS16 * kS16;
    for (int f = 0; f < 4; ++f) {
      for (int i = tid; i < p3; i += nthr) in2[i] = df_from_double(Fleaf[((size_t)leaf * 4 + f) * p3 + i]);
      __syncthreads();
      contract3_df(in2, reinterpret_cast<float2*>(base + lay.t1), reinterpret_cast<float2*>(base + lay.t2), o2, p,
                   kS16, W8, kS16, true, tid, nthr);      // ends with a barrier
      for (int i = tid; i < S3; i += nthr) far[f * S3 + i] = o2[i].x + o2[i].y;
    }
    __syncthreads();
  }

  const int row = tid & 127, h = tid >> 7;
  const int cz = zh * 8 + (row >> 4), cy = row & 15;
  float a[4][8];
#pragma unroll
  for (int f = 0; f < 4; ++f)
#pragma unroll
    for (int x = 0; x < 8; ++x) a[f][x] = 0.f;

  for (int zp = 0; zp < kW16; ++zp) {
    float* pln = base + ((zp & 1) ? lay.pl1 : lay.pl0);
    tc::cp_async_wait<0>();
    __syncthreads();   // plane zp landed; plane zp - 1 is no longer read
    for (int i = tid; i < kW16 * kW16; i += nthr) pln[i] = ((pln[i] - mu_hi) - mu_lo) * inv_vol;
    __syncthreads();
    if (zp + 1 < kW16) fetch(zp + 1, (zp + 1) & 1);
    const int dz = cz + kS16 - zp;
    const int adz = dz < 0 ? -dz : dz;
    const float sz = dz > 0 ? 1.f : (dz < 0 ? -1.f : 0.f);
    float pl[4][8];
#pragma unroll
    for (int f = 0; f < 4; ++f)
#pragma unroll
      for (int x = 0; x < 8; ++x) pl[f][x] = 0.f;
#pragma unroll 1
    for (int yp = 0; yp < kW16; ++yp) {
      const int dy = cy + kS16 - yp;
      const int ady = dy < 0 ? -dy : dy;
      const float sy = dy > 0 ? 1.f : (dy < 0 ? -1.f : 0.f);
      const float4* trow = near_tab + ((size_t)adz * 2 * kS16 + ady) * 2 * kS16;
      const float* mrow = pln + yp * kW16;
      float rw[4][8];
#pragma unroll
      for (int f = 0; f < 4; ++f)
#pragma unroll
        for (int x = 0; x < 8; ++x) rw[f][x] = 0.f;
#pragma unroll 1
      for (int c = 0; c < kW16 / 8; ++c) {
        const int b8 = 8 * (2 + h - c);       // dx = b8 + x - xs
        float4 t[15];
#pragma unroll
        for (int j = 0; j < 15; ++j) {
          const int d = b8 + j - 7;
          t[j] = __ldg(trow + (d < 0 ? -d : d));
        }
        const float4 m0 = *reinterpret_cast<const float4*>(mrow + 8 * c);
        const float4 m1 = *reinterpret_cast<const float4*>(mrow + 8 * c + 4);
        const float m[8] = {m0.x, m0.y, m0.z, m0.w, m1.x, m1.y, m1.z, m1.w};
        if (b8 > 0)
          p2p16_chunk<1>(rw, t, m);
        else if (b8 < 0)
          p2p16_chunk<-1>(rw, t, m);
        else
          p2p16_chunk<0>(rw, t, m);
      }
#pragma unroll
      for (int x = 0; x < 8; ++x) {
        pl[0][x] += rw[0][x];
        pl[1][x] += rw[1][x];
        pl[2][x] = fmaf(sy, rw[2][x], pl[2][x]);
        pl[3][x] += rw[3][x];
      }
    }
#pragma unroll
    for (int x = 0; x < 8; ++x) {
      a[0][x] += pl[0][x];
      a[1][x] += pl[1][x];
      a[2][x] += pl[2][x];
      a[3][x] = fmaf(sz, pl[3][x], a[3][x]);
    }
  }
  const size_t o = ((size_t)(lz * kS16 + cz) * N + (ly * kS16 + cy)) * N + lx * kS16 + 8 * h;
#pragma unroll
  for (int x = 0; x < 8; ++x) {
    const int c = (cz * kS16 + cy) * kS16 + 8 * h + x;
    const int S3 = kS16 * kS16 * kS16;
    phi[o + x] = a[0][x] + far[c];
    acc_out[o + x] = a[1][x] + far[S3 + c];
    acc_out[N3 + o + x] = a[2][x] + far[2 * S3 + c];
    acc_out[2 * N3 + o + x] = a[3][x] + far[3 * S3 + c];
  }
}

cudaError_t launch_s16(Plan& P, const float* rho, float* phi, float* acc, cudaStream_t s) {
  const size_t smem = sizeof(float) * (size_t)P2P16Smem(P.p).total;
  const unsigned leaves = 1u << (3 * P.L);
  const int vec = (reinterpret_cast<uintptr_t>(rho) & 15u) == 0;
  k_p2p16<<<2 * leaves, kT16, smem, s>>>(rho, P.d_mean, P.N, P.L, P.p, P.near_tab, P.F64[P.L], P.w_p2m, phi, acc, vec,
                                        P.iso);
  return cudaGetLastError();
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
  k_p2p<S><<<grid, Sh::THREADS, smem, s>>>(rho, P.d_mean, P.N, P.L, P.p, P.near_tab, P.F[P.L], P.w_p2m, phi, acc, vec,
                                           P.iso);
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
    case 8: {
      const cudaError_t e = setup_s<8>();
      return e != cudaSuccess ? e : setup_near_fft(P);
    }
    case 16: return cudaFuncSetAttribute(k_p2p16, cudaFuncAttributeMaxDynamicSharedMemorySize, 225 * 1024);
    default: return cudaErrorInvalidValue;
  }
}

cudaError_t launch_p2p(Plan& P, const float* rho, float* phi, float* acc, cudaStream_t s, bool near_fwd_done) {
  if (P.near_fft) return launch_near_fft(P, rho, phi, acc, s, near_fwd_done);
  switch (P.S) {
    case 1: return launch_s<1>(P, rho, phi, acc, s);
    case 2: return launch_s<2>(P, rho, phi, acc, s);
    case 3: return launch_s<3>(P, rho, phi, acc, s);
    case 4: return launch_s<4>(P, rho, phi, acc, s);
    case 6: return launch_s<6>(P, rho, phi, acc, s);
    case 8: return launch_s<8>(P, rho, phi, acc, s);
    case 16: return launch_s16(P, rho, phi, acc, s);
    default: return cudaErrorInvalidValue;
  }
}

}  // namespace fmm

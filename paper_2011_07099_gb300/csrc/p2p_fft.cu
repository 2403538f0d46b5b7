// Leaf stage by fast Fourier transforms: the near zone (P2P) as a sum of
// zero-padded convolutions, added to the leaf's L2P far field.
//
// Sec. 3 computes the near zone of a regular grid with an FFT under
// non-periodic boundary conditions, obtained by doubling the grid.  Here that
// is done per pair of leaves.  For a target leaf T of S = 8 cells per side and
// one of its 27 neighbour leaves T + o (o in {-1, 0, 1}^3), the near-zone
// field at cell r of T is the linear convolution
//   Phi_T(r) += sum_{r'} K(r - r' - S o) m_{T+o}(r'),   r, r' in [0, S)^3,
// whose lags r - r' lie in [-(S-1), S-1]^3.  Padded to M = 2S points per axis
// that linear convolution is a circular one with no lag wrapped onto another,
// so on the M^3 spectrum
//   Phi^_T(k) = sum_o K^_o(k) m^_{T+o}(k),
// K^_o the transform of u -> K(u - S o) placed at u mod M (u in [-(S-1), S-1]^3,
// the lag S never occurs and holds 0).  K = (G, -dG/dx, -dG/dy, -dG/dz) at the
// cell offsets: the plan's near table (the same FP32 values the direct sum
// uses), so the result is the direct sum's up to rounding.
//
// Kernels (all spectra are real-input half spectra, kx in [0, M/2]):
//   k_nz_kernel  plan time: the 27 x 4 kernel spectra, in FP64, rounded once
//   k_nz_fwd     per leaf: the spectrum of its zero-padded masses (direct
//                line DFTs of the 8 nonzero inputs per axis)
//   k_nz_mac     per (tile of 4^3 target leaves, 8 chunks of 32 frequencies):
//                the 27-term sums for 4 fields, written per target leaf
//   k_nz_l2p     per leaf: the L2P far field, written to the outputs
//   k_nz_inv     persistent over the target leaves: 4 inverse transforms
//                (radix-2 in registers, only the S^3 cells kept) added to the
//                far field in the outputs.
// Twiddles come from sincospi in FP64.
#include "fmm_internal.cuh"
#include "tc_ptx.cuh"

namespace fmm {
namespace {

constexpr int kNS = 8;                       // leaf cells per side
constexpr int kNM = 2 * kNS;                 // padded transform size
constexpr int kNX = kNM / 2 + 1;             // half-spectrum extent along x
constexpr int kNK = kNM * kNM * kNX;         // frequencies per spectrum (2304)
constexpr int kNC = 32;                      // frequencies per chunk
constexpr int kNCH = kNK / kNC;              // chunks (72)
constexpr int kNO = 27;                      // neighbour offsets
constexpr int kNT = 4;                       // target leaves per tile side
constexpr int kNH = kNT + 2;                 // source leaves per halo side
constexpr int kThr = 256;
static_assert(kNK % kNC == 0, "chunking");

// linear frequency index: k = (kz * M + ky) * (M/2 + 1) + kx

__device__ __forceinline__ void cfma(float2& acc, float2 a, float2 b) {
  acc.x = fmaf(a.x, b.x, acc.x);
  acc.x = fmaf(-a.y, b.y, acc.x);
  acc.y = fmaf(a.x, b.y, acc.y);
  acc.y = fmaf(a.y, b.x, acc.y);
}

// e^{-2 pi i j / M}, j = 0 .. M-1, into shared memory (FP64 -> FP32)
__device__ __forceinline__ void twiddles(float2* w, int tid) {
  if (tid < kNM) {
    double s, c;
    sincospi((double)tid / (kNM / 2), &s, &c);
    w[tid] = make_float2((float)c, (float)-s);
  }
}

// The kernel's value for field f at lag d (cells), from the folded near table
// (|d_i| in [0, 2S-1]); the gradient fields take the sign of their own
// component as the direct sum does, and vanish where that component is 0
// (the table holds exact zeros there for G_S1 and G_0), so that every field
// is exactly even (Phi) or odd (g) under d -> -d.
__device__ __forceinline__ double near_value(const float4* __restrict__ tab, int f, int dx, int dy, int dz) {
  constexpr int TD = 2 * kNS;
  const int ax = dx < 0 ? -dx : dx, ay = dy < 0 ? -dy : dy, az = dz < 0 ? -dz : dz;
  const float4 t = __ldg(tab + (az * TD + ay) * TD + ax);
  switch (f) {
    case 0: return (double)t.x;
    case 1: return dx > 0 ? (double)t.y : (dx < 0 ? -(double)t.y : 0.0);
    case 2: return dy > 0 ? (double)t.z : (dy < 0 ? -(double)t.z : 0.0);
    default: return dz > 0 ? (double)t.w : (dz < 0 ? -(double)t.w : 0.0);
  }
}

// Kernel spectra: CTA (o, f) transforms u -> K_f(u - S o) on the M^3 grid in
// FP64 (three separable passes), writing K^[chunk][o][f][32] as FP32.
__global__ void __launch_bounds__(kThr) k_nz_kernel(const float4* __restrict__ near_tab, float2* __restrict__ Khat) {
  __shared__ double2 w64[kNM];
  extern __shared__ double2 sd[];
  double2* T1 = sd;                 // [vz][vy][kx]
  double2* T2 = sd + kNM * kNM * kNX;   // [vz][ky][kx]
  const int o = blockIdx.x / 4, f = blockIdx.x % 4, tid = threadIdx.x;
  const int ox = o % 3 - 1, oy = (o / 3) % 3 - 1, oz = o / 9 - 1;
  if (tid < kNM) {
    double s, c;
    sincospi((double)tid / (kNM / 2), &s, &c);
    w64[tid] = make_double2(c, -s);
  }
  __syncthreads();
  auto lag = [](int v) { return v < kNS ? v : v - kNM; };   // v = M/2 = S is never a lag
  for (int i = tid; i < kNM * kNM * kNX; i += blockDim.x) {
    const int kx = i % kNX, vy = (i / kNX) % kNM, vz = i / (kNX * kNM);
    double re = 0.0, im = 0.0;
    if (vy != kNS && vz != kNS) {
      for (int vx = 0; vx < kNM; ++vx) {
        if (vx == kNS) continue;
        const double a = near_value(near_tab, f, lag(vx) - kNS * ox, lag(vy) - kNS * oy, lag(vz) - kNS * oz);
        const double2 t = w64[(kx * vx) % kNM];
        re += a * t.x;
        im += a * t.y;
      }
    }
    T1[i] = make_double2(re, im);
  }
  __syncthreads();
  for (int i = tid; i < kNM * kNM * kNX; i += blockDim.x) {
    const int kx = i % kNX, ky = (i / kNX) % kNM, vz = i / (kNX * kNM);
    double re = 0.0, im = 0.0;
    for (int vy = 0; vy < kNM; ++vy) {
      const double2 a = T1[(vz * kNM + vy) * kNX + kx], t = w64[(ky * vy) % kNM];
      re += a.x * t.x - a.y * t.y;
      im += a.x * t.y + a.y * t.x;
    }
    T2[i] = make_double2(re, im);
  }
  __syncthreads();
  for (int k = tid; k < kNK; k += blockDim.x) {
    const int kx = k % kNX, ky = (k / kNX) % kNM, kz = k / (kNX * kNM);
    double re = 0.0, im = 0.0;
    for (int vz = 0; vz < kNM; ++vz) {
      const double2 a = T2[(vz * kNM + ky) * kNX + kx], t = w64[(kz * vz) % kNM];
      re += a.x * t.x - a.y * t.y;
      im += a.x * t.y + a.y * t.x;
    }
    Khat[(((size_t)(k / kNC) * kNO + o) * 4 + f) * kNC + k % kNC] = make_float2((float)re, (float)im);
  }
}

// Source spectra: CTA per leaf; masses m = (rho - mean) / N^3 (mean as hi + lo,
// as in the direct kernel) zero-padded to M^3.  Writes m^[chunk][leaf][32];
// the slot after the last leaf is the all-zero spectrum of an out-of-box
// neighbour (isolated problem), cleared at allocation.  Each pass gives a
// thread whole lines: the line's nonzero inputs in registers, the twiddles in
// registers at compile-time indices.
constexpr int kFwdThr = kNM * kNX;           // 144: one thread per (ky, kx) line of the last pass
__global__ void __launch_bounds__(kFwdThr) k_nz_fwd(const float* __restrict__ rho, const double* __restrict__ mean,
                                                   int N, int L, float2* __restrict__ Mhat) {
  __shared__ float2 w[kNM];
  __shared__ float m[kNS * kNS * kNS];
  __shared__ float2 A[kNS * kNS * kNX];    // [z][y][kx]
  __shared__ float2 B[kNS * kNM * kNX];    // [z][ky][kx]
  const int tid = threadIdx.x;
  const unsigned leaf = blockIdx.x, nl3 = 1u << (3 * L);
  twiddles(w, tid);
  uint32_t lx, ly, lz;
  unmorton(leaf, lx, ly, lz);
  const double mu = *mean;
  const float mu_hi = (float)mu, mu_lo = (float)(mu - (double)mu_hi);
  const float inv_vol = (float)(1.0 / ((double)N * N * N));
  for (int i = tid; i < kNS * kNS * kNS; i += blockDim.x) {
    const int x = i % kNS, y = (i / kNS) % kNS, z = i / (kNS * kNS);
    const float r = __ldg(rho + ((size_t)(lz * kNS + z) * N + (ly * kNS + y)) * N + lx * kNS + x);
    m[i] = ((r - mu_hi) - mu_lo) * inv_vol;
  }
  __syncthreads();
  float2 tw[kNM];
#pragma unroll
  for (int j = 0; j < kNM; ++j) tw[j] = w[j];
  if (tid < kNS * kNS) {                     // x: line (z, y), 8 real inputs -> kx in [0, M/2]
    float v[kNS];
#pragma unroll
    for (int x = 0; x < kNS; ++x) v[x] = m[tid * kNS + x];
#pragma unroll
    for (int kx = 0; kx < kNX; ++kx) {
      float2 a = make_float2(0.f, 0.f);
#pragma unroll
      for (int x = 0; x < kNS; ++x) {
        a.x = fmaf(v[x], tw[(kx * x) % kNM].x, a.x);
        a.y = fmaf(v[x], tw[(kx * x) % kNM].y, a.y);
      }
      A[tid * kNX + kx] = a;
    }
  }
  __syncthreads();
  if (tid < kNS * kNX) {                     // y: line (z, kx), 8 nonzero inputs -> 16
    const int kx = tid % kNX, z = tid / kNX;
    float2 v[kNS];
#pragma unroll
    for (int y = 0; y < kNS; ++y) v[y] = A[(z * kNS + y) * kNX + kx];
#pragma unroll
    for (int ky = 0; ky < kNM; ++ky) {
      float2 a = make_float2(0.f, 0.f);
#pragma unroll
      for (int y = 0; y < kNS; ++y) cfma(a, v[y], tw[(ky * y) % kNM]);
      B[(z * kNM + ky) * kNX + kx] = a;
    }
  }
  __syncthreads();
  {                                          // z: line (ky, kx), 8 nonzero inputs -> 16
    float2 v[kNS];
#pragma unroll
    for (int z = 0; z < kNS; ++z) v[z] = B[z * kNM * kNX + tid];
#pragma unroll
    for (int kz = 0; kz < kNM; ++kz) {
      float2 a = make_float2(0.f, 0.f);
#pragma unroll
      for (int z = 0; z < kNS; ++z) cfma(a, v[z], tw[(kz * z) % kNM]);
      const int k = kz * kNM * kNX + tid;
      Mhat[((size_t)(k / kNC) * (nl3 + 1) + leaf) * kNC + k % kNC] = a;
    }
  }
}

// Spectral sums: CTA (tile of 4^3 target leaves, 8 consecutive chunks of 32
// frequencies).  Thread (g, f): frequency f of the chunk for the 4 target
// leaves of row g (x = 0..3 at y = g % 4, z = g / 4), 4 fields each.  The
// next chunk's kernel and source spectra are copied (cp.async) while the
// current one is summed.  The kernels are real and Phi's is even, g's odd,
// under lag -> -lag, so K^_{-o} = s conj(K^_o) (s = +1 for Phi, -1 for g)
// and the 26 non-central offsets are taken in pairs (o, -o): with
// M+ = m^_{T+o}, M- = m^_{T-o}, K^_o = a + ib,
//   K^_o M+ + s conj(K^_o) M- = a (M+ + s M-) + i b (M+ - s M-).
// The pairs come in groups of the three x offsets: a group's 6 source spectra
// of the +o row and 6 of the -o row are read once for its 3 x 4 pair terms.
constexpr int kCPC = 8;                      // chunks per CTA
constexpr int kMacThr = 512;
constexpr int kNKO = kNO / 2 + 1;            // kernel spectra used per chunk: offsets 0..13
constexpr int kMacStage = kNKO * 4 * kNC + kNH * kNH * kNH * kNC;   // float2 per pipeline stage
static_assert(kNCH % kCPC == 0, "chunk groups");

// one pair term for the 4 fields of one target leaf
__device__ __forceinline__ void pair_term(float2 (&acc)[4], const float2 (&k)[4], float2 mp, float2 mm) {
  const float2 sum = make_float2(mp.x + mm.x, mp.y + mm.y), dif = make_float2(mp.x - mm.x, mp.y - mm.y);
  acc[0].x = fmaf(k[0].x, sum.x, acc[0].x);
  acc[0].x = fmaf(-k[0].y, dif.y, acc[0].x);
  acc[0].y = fmaf(k[0].x, sum.y, acc[0].y);
  acc[0].y = fmaf(k[0].y, dif.x, acc[0].y);
#pragma unroll
  for (int q = 1; q < 4; ++q) {
    acc[q].x = fmaf(k[q].x, dif.x, acc[q].x);
    acc[q].x = fmaf(-k[q].y, sum.y, acc[q].x);
    acc[q].y = fmaf(k[q].x, dif.y, acc[q].y);
    acc[q].y = fmaf(k[q].y, sum.x, acc[q].y);
  }
}

__global__ void __launch_bounds__(kMacThr, 1) k_nz_mac(const float2* __restrict__ Khat,
                                                      const float2* __restrict__ Mhat, float2* __restrict__ Phat,
                                                      int L, int iso) {
  extern __shared__ float4 sm4[];
  unsigned* hleaf = reinterpret_cast<unsigned*>(sm4);             // [216] source leaf of each halo slot
  float2* stage0 = reinterpret_cast<float2*>(sm4) + 128;           // 1 KB after the halo list
  const int tid = threadIdx.x;
  const int nl = 1 << L, nt = nl / kNT;
  const unsigned nl3 = 1u << (3 * L);
  const int t = blockIdx.x, c0 = blockIdx.y * kCPC;
  const int TX = t % nt, TY = (t / nt) % nt, TZ = t / (nt * nt);
  if (tid < kNH * kNH * kNH) {
    const int hx = tid % kNH, hy = (tid / kNH) % kNH, hz = tid / (kNH * kNH);
    int gx = TX * kNT + hx - 1, gy = TY * kNT + hy - 1, gz = TZ * kNT + hz - 1;
    if (iso && (gx < 0 || gy < 0 || gz < 0 || gx >= nl || gy >= nl || gz >= nl)) {
      hleaf[tid] = nl3;                                            // the all-zero spectrum
    } else {
      gx = (gx + nl) % nl;
      gy = (gy + nl) % nl;
      gz = (gz + nl) % nl;
      hleaf[tid] = morton((uint32_t)gx, (uint32_t)gy, (uint32_t)gz);
    }
  }
  __syncthreads();
  auto load = [&](int c, int st) {
    float2* sK = stage0 + st * kMacStage;
    float2* sM = sK + kNKO * 4 * kNC;
    const float2* src = Khat + (size_t)c * kNO * 4 * kNC;          // offsets 0..13 (the rest by symmetry)
    for (int i = tid; i < kNKO * 4 * kNC / 2; i += blockDim.x)
      tc::cp_async16(tc::smem_u32(sK + 2 * i), src + 2 * i, 16u);
    const float2* msrc = Mhat + (size_t)c * (nl3 + 1) * kNC;
    for (int i = tid; i < kNH * kNH * kNH * (kNC / 2); i += blockDim.x) {
      const int h = i / (kNC / 2), q = i % (kNC / 2);
      tc::cp_async16(tc::smem_u32(sM + h * kNC + 2 * q), msrc + (size_t)hleaf[h] * kNC + 2 * q, 16u);
    }
    tc::cp_async_commit();
  };
  const int f = tid % kNC, g = tid / kNC;
  const int ly = g % kNT, lz = g / kNT;
  // halo slot of (x, y, z) in [0, 6)^3, frequency f
  auto slot = [&](int x, int y, int z) { return ((z * kNH + y) * kNH + x) * kNC + f; };
  load(c0, 0);
  for (int it = 0; it < kCPC; ++it) {
    const int c = c0 + it;
    if (it + 1 < kCPC) {
      load(c + 1, (it + 1) & 1);
      tc::cp_async_wait<1>();
    } else {
      tc::cp_async_wait<0>();
    }
    __syncthreads();
    const float2* sK = stage0 + (it & 1) * kMacStage;
    const float2* sM = sK + kNKO * 4 * kNC;
    float2 acc[4][4];
    {                                                 // the central offset (index 13)
      float2 k[4];
#pragma unroll
      for (int q = 0; q < 4; ++q) k[q] = sK[(13 * 4 + q) * kNC + f];
#pragma unroll
      for (int j = 0; j < 4; ++j) {
        const float2 mv = sM[slot(j + 1, ly + 1, lz + 1)];
#pragma unroll
        for (int q = 0; q < 4; ++q) {
          acc[j][q] = make_float2(0.f, 0.f);
          cfma(acc[j][q], k[q], mv);
        }
      }
    }
    // groups of pairs sharing (oy, oz): offset index o = (ox+1) + 3 (oy+1) + 9 (oz+1)
#pragma unroll
    for (int grp = 0; grp < 5; ++grp) {
      // grp 0..2: oz = -1, oy = grp - 1, ox in {-1, 0, 1}; grp 3: oz = 0, oy = -1, ox in {-1, 0, 1};
      // grp 4: the single pair (-1, 0, 0)
      const int oz = grp < 3 ? -1 : 0, oy = grp < 3 ? grp - 1 : (grp == 3 ? -1 : 0);
      float2 mp[kNH], mm[kNH];
#pragma unroll
      for (int x = 0; x < kNH; ++x) {
        mp[x] = sM[slot(x, ly + oy + 1, lz + oz + 1)];
        mm[x] = sM[slot(x, ly - oy + 1, lz - oz + 1)];
      }
#pragma unroll
      for (int ox = -1; ox <= (grp == 4 ? -1 : 1); ++ox) {
        const int o = (ox + 1) + 3 * (oy + 1) + 9 * (oz + 1);
        float2 k[4];
#pragma unroll
        for (int q = 0; q < 4; ++q) k[q] = sK[(o * 4 + q) * kNC + f];
#pragma unroll
        for (int j = 0; j < 4; ++j) pair_term(acc[j], k, mp[j + ox + 1], mm[j - ox + 1]);
      }
    }
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      const size_t leaf = morton(TX * kNT + j, TY * kNT + ly, TZ * kNT + lz);
#pragma unroll
      for (int q = 0; q < 4; ++q) Phat[(leaf * 4 + q) * kNK + (size_t)c * kNC + f] = acc[j][q];
    }
    __syncthreads();                                  // this stage is refilled two chunks on
  }
}

// Complex helpers of the inverse transforms.
__device__ __forceinline__ float2 cadd(float2 a, float2 b) { return make_float2(a.x + b.x, a.y + b.y); }
__device__ __forceinline__ float2 csub(float2 a, float2 b) { return make_float2(a.x - b.x, a.y - b.y); }
__device__ __forceinline__ float2 cmul(float2 a, float2 b) {
  return make_float2(fmaf(a.x, b.x, -a.y * b.y), fmaf(a.x, b.y, a.y * b.x));
}
__device__ __forceinline__ float2 mul_i(float2 a) { return make_float2(-a.y, a.x); }

// 4-point inverse DFT, y_z = sum_m x_m e^{+2 pi i m z / 4}.
__device__ __forceinline__ void idft4(float2 x0, float2 x1, float2 x2, float2 x3, float2 (&y)[4]) {
  const float2 c0 = cadd(x0, x2), c1 = csub(x0, x2), d0 = cadd(x1, x3), d1 = mul_i(csub(x1, x3));
  y[0] = cadd(c0, d0);
  y[2] = csub(c0, d0);
  y[1] = cadd(c1, d1);
  y[3] = csub(c1, d1);
}
// 8-point inverse DFT of x[0], x[s], ..., x[7s] by one radix-2 split into two
// 4-point transforms; t1 = e^{+2 pi i / 8}, t3 = e^{+6 pi i / 8}.
template <int OFF, int STRIDE>
__device__ __forceinline__ void idft8(const float2 (&x)[16], float2 (&y)[8], float2 t1, float2 t3) {
  float2 a[4], b[4];
  idft4(x[OFF], x[OFF + 2 * STRIDE], x[OFF + 4 * STRIDE], x[OFF + 6 * STRIDE], a);
  idft4(x[OFF + STRIDE], x[OFF + 3 * STRIDE], x[OFF + 5 * STRIDE], x[OFF + 7 * STRIDE], b);
  const float2 b1 = cmul(b[1], t1), b2 = mul_i(b[2]), b3 = cmul(b[3], t3);
  y[0] = cadd(a[0], b[0]);
  y[4] = csub(a[0], b[0]);
  y[1] = cadd(a[1], b1);
  y[5] = csub(a[1], b1);
  y[2] = cadd(a[2], b2);
  y[6] = csub(a[2], b2);
  y[3] = cadd(a[3], b3);
  y[7] = csub(a[3], b3);
}
// Outputs 0..7 of the 16-point inverse DFT of v (decimation in time: the
// 8-point transforms E, O of the even and odd samples, X_z = E_z + t^z O_z);
// tw[j] = e^{+2 pi i j / 16}.
__device__ __forceinline__ void idft16_first_half(const float2 (&v)[16], float2 (&out)[8], const float2 (&tw)[kNM]) {
  float2 E[8], O[8];
  idft8<0, 2>(v, E, tw[2], tw[6]);
  idft8<1, 2>(v, O, tw[2], tw[6]);
  out[0] = cadd(E[0], O[0]);
  out[4] = cadd(E[4], mul_i(O[4]));
#pragma unroll
  for (int z = 1; z < 8; ++z)
    if (z != 4) out[z] = cadd(E[z], cmul(tw[z], O[z]));
}

// L2P of the 8-cell leaves: far[f][cz][cy][cx] = sum_s l_s(cz) l_s(cy)
// l_s(cx) F[f][s], as the separable contraction of the direct kernel (x, then
// y, then z; each output the FP32 sum over the gridlet points of the hi
// weights plus that of the lo weights, in the same order, so the far field is
// bitwise the direct kernel's), written to the outputs; the inverse
// transforms add the near field to it.  CTA per leaf; a thread takes whole
// lines (the P inputs in registers, all 8 outputs), the P x 8 weight pairs in
// registers.
constexpr int kL2pThr = 128;
template <int P>
__global__ void __launch_bounds__(kL2pThr) k_nz_l2p(int N, const float* __restrict__ Fleaf,
                                                   const float2* __restrict__ wp2m, float* __restrict__ phi,
                                                   float* __restrict__ acc_out) {
  __shared__ float F[4 * P * P * P];
  __shared__ float t1[4 * P * P * kNS];
  __shared__ float t2[4 * P * kNS * kNS];
  const int tid = threadIdx.x, nthr = blockDim.x;
  const unsigned leaf = blockIdx.x;
  const size_t N3 = (size_t)N * N * N;
  float2 wr[P][kNS];
#pragma unroll
  for (int k = 0; k < P; ++k)
#pragma unroll
    for (int c = 0; c < kNS; ++c) wr[k][c] = __ldg(wp2m + k * kNS + c);
  const float* src = Fleaf + (size_t)leaf * 4 * P * P * P;
  for (int i = tid; i < 4 * P * P * P; i += nthr) F[i] = __ldg(src + i);
  __syncthreads();
  auto line8 = [&](const float (&in)[P], float (&out)[kNS]) {
#pragma unroll
    for (int c = 0; c < kNS; ++c) {
      float acc = 0.f, lo = 0.f;
#pragma unroll
      for (int k = 0; k < P; ++k) {
        acc = fmaf(wr[k][c].x, in[k], acc);
        lo = fmaf(wr[k][c].y, in[k], lo);
      }
      out[c] = acc + lo;
    }
  };
  for (int l = tid; l < 4 * P * P; l += nthr) {              // x: line (f, sz, sy)
    float in[P], out[kNS];
#pragma unroll
    for (int k = 0; k < P; ++k) in[k] = F[l * P + k];
    line8(in, out);
#pragma unroll
    for (int c = 0; c < kNS; ++c) t1[l * kNS + c] = out[c];
  }
  __syncthreads();
  for (int l = tid; l < 4 * P * kNS; l += nthr) {            // y: line (f, sz, cx)
    const int cx = l % kNS, g = l / kNS;
    float in[P], out[kNS];
#pragma unroll
    for (int k = 0; k < P; ++k) in[k] = t1[(g * P + k) * kNS + cx];
    line8(in, out);
#pragma unroll
    for (int c = 0; c < kNS; ++c) t2[(g * kNS + c) * kNS + cx] = out[c];
  }
  __syncthreads();
  uint32_t lx, ly, lz;
  unmorton(leaf, lx, ly, lz);
  for (int l = tid; l < 4 * kNS * kNS; l += nthr) {          // z: line (f, cy, cx) -> the outputs
    const int cyx = l % (kNS * kNS), f = l / (kNS * kNS);
    float in[P], out[kNS];
#pragma unroll
    for (int k = 0; k < P; ++k) in[k] = t2[(f * P + k) * kNS * kNS + cyx];
    line8(in, out);
    float* dst = (f == 0 ? phi : acc_out + (size_t)(f - 1) * N3) +
                 ((size_t)(lz * kNS) * N + (ly * kNS + cyx / kNS)) * N + lx * kNS + cyx % kNS;
#pragma unroll
    for (int c = 0; c < kNS; ++c) dst[(size_t)c * N * N] = out[c];
  }
}

template <int P>
void launch_l2p_p(const Plan& Pl, float* phi, float* acc, cudaStream_t s) {
  k_nz_l2p<P><<<1u << (3 * Pl.L), kL2pThr, 0, s>>>(Pl.N, Pl.F[Pl.L], Pl.w_p2m, phi, acc);
}
void launch_l2p(const Plan& Pl, float* phi, float* acc, cudaStream_t s) {
  switch (Pl.p) {
    case 1: launch_l2p_p<1>(Pl, phi, acc, s); break;
    case 2: launch_l2p_p<2>(Pl, phi, acc, s); break;
    case 3: launch_l2p_p<3>(Pl, phi, acc, s); break;
    case 4: launch_l2p_p<4>(Pl, phi, acc, s); break;
    case 5: launch_l2p_p<5>(Pl, phi, acc, s); break;
    case 6: launch_l2p_p<6>(Pl, phi, acc, s); break;
    case 7: launch_l2p_p<7>(Pl, phi, acc, s); break;
    default: launch_l2p_p<8>(Pl, phi, acc, s); break;
  }
}

// Shared-memory carve-up of the inverse kernel (floats): two pipeline stages
// of (the 4 field spectra, the 4 x 64 rows of the leaf's outputs).
constexpr int kInvSpec = 4 * 2 * kNK;                 // floats of one stage's spectra
constexpr int kInvRows = 4 * kNS * kNS * kNS;         // floats of one stage's output rows
constexpr int kInvSmemFloats = 2 * (kInvSpec + kInvRows);
constexpr int kInvThr = 576;                 // one thread per z line of the 4 fields (288 y, 256 x lines)

// Inverse transforms of the target leaves' 4 field spectra (only the S^3
// cells of a leaf are formed), added to the far field k_nz_l2p left in the
// outputs.  Persistent: a CTA walks the leaves blockIdx.x, + gridDim.x, ...;
// the next leaf's spectra and output rows arrive by cp.async while the
// current one is transformed.  Each pass works in place: a thread holds a
// whole line in registers and writes its 8 kept outputs over the line's
// first 8 slots, so the z pass leaves [f][z < 8][ky][kx] and the y pass
// [f][z][y < 8][kx].
__global__ void __launch_bounds__(kInvThr, 1) k_nz_inv(const float2* __restrict__ Phat, int N, int L,
                                                      float* __restrict__ phi, float* __restrict__ acc_out) {
  __shared__ float2 w[kNM];
  extern __shared__ float4 sm4[];
  float* base = reinterpret_cast<float*>(sm4);
  const int tid = threadIdx.x, nthr = blockDim.x;
  const unsigned nl3 = 1u << (3 * L);
  const size_t N3 = (size_t)N * N * N;
  auto row_of = [&](unsigned leaf, int r) -> float* {   // output row r = (f, z, y) of a leaf
    uint32_t lx, ly, lz;
    unmorton(leaf, lx, ly, lz);
    const int y = r & 7, z = (r >> 3) & 7, f = r >> 6;
    const size_t o = ((size_t)(lz * kNS + z) * N + (ly * kNS + y)) * N + lx * kNS;
    return (f == 0 ? phi : acc_out + (size_t)(f - 1) * N3) + o;
  };
  auto fetch = [&](unsigned leaf, int b) {
    float2* spec = reinterpret_cast<float2*>(base + b * (kInvSpec + kInvRows));
    float* rows = base + b * (kInvSpec + kInvRows) + kInvSpec;
    const float2* src = Phat + (size_t)leaf * 4 * kNK;
    for (int i = tid; i < 4 * kNK / 2; i += nthr) tc::cp_async16(tc::smem_u32(spec + 2 * i), src + 2 * i, 16u);
    for (int i = tid; i < kInvRows / 4; i += nthr)
      tc::cp_async16(tc::smem_u32(rows + 4 * i), row_of(leaf, i >> 1) + 4 * (i & 1), 16u);
    tc::cp_async_commit();
  };
  twiddles(w, tid);
  unsigned leaf = blockIdx.x;
  if (leaf < nl3) fetch(leaf, 0);
  __syncthreads();
  float2 tw[kNM];                              // e^{+2 pi i j / M}
#pragma unroll
  for (int j = 0; j < kNM; ++j) tw[j] = make_float2(w[j].x, -w[j].y);
  const float scale = 1.f / (float)(kNM * kNM * kNM);
  constexpr int PL = kNM * kNX;                // one kz (or z) plane of a field: 144 values
  for (int b = 0; leaf < nl3; leaf += gridDim.x, b ^= 1) {
    if (leaf + gridDim.x < nl3) {
      fetch(leaf + gridDim.x, b ^ 1);
      tc::cp_async_wait<1>();
    } else {
      tc::cp_async_wait<0>();
    }
    __syncthreads();
    float2* spec = reinterpret_cast<float2*>(base + b * (kInvSpec + kInvRows));
    const float* rows = base + b * (kInvSpec + kInvRows) + kInvSpec;
    for (int u = tid; u < 4 * PL; u += nthr) {   // z: line (f, ky, kx), 16 -> the 8 kept planes
      float2* line = spec + (u / PL) * kNK + u % PL;
      float2 v[kNM], o[kNS];
#pragma unroll
      for (int kz = 0; kz < kNM; ++kz) v[kz] = line[kz * PL];
      idft16_first_half(v, o, tw);
#pragma unroll
      for (int z = 0; z < kNS; ++z) line[z * PL] = o[z];
    }
    __syncthreads();
    for (int u = tid; u < 4 * kNS * kNX; u += nthr) {   // y: line (f, z, kx), 16 -> the 8 kept rows
      const int kx = u % kNX, z = (u / kNX) % kNS, f = u / (kNX * kNS);
      float2* line = spec + f * kNK + z * PL + kx;
      float2 v[kNM], o[kNS];
#pragma unroll
      for (int ky = 0; ky < kNM; ++ky) v[ky] = line[ky * kNX];
      idft16_first_half(v, o, tw);
#pragma unroll
      for (int y = 0; y < kNS; ++y) line[y * kNX] = o[y];
    }
    __syncthreads();
    for (int u = tid; u < 4 * kNS * kNS; u += nthr) {   // x: line (f, z, y), half spectrum -> 8 real cells
      const int y = u % kNS, z = (u / kNS) % kNS, f = u / (kNS * kNS);
      const float2* line = spec + f * kNK + z * PL + y * kNX;
      float2 v[kNX];
#pragma unroll
      for (int kx = 0; kx < kNX; ++kx) v[kx] = line[kx];
      float* dst = row_of(leaf, u);
      const float* fr = rows + u * kNS;
#pragma unroll
      for (int x = 0; x < kNS; ++x) {
        float r = 0.f;                             // Re(v e^{+i theta}) = v.x cos - v.y sin
#pragma unroll
        for (int kx = 1; kx < kNX - 1; ++kx) {
          r = fmaf(v[kx].x, tw[(kx * x) % kNM].x, r);
          r = fmaf(-v[kx].y, tw[(kx * x) % kNM].y, r);
        }
        r = 2.f * r + v[0].x + ((x & 1) ? -v[kNX - 1].x : v[kNX - 1].x);
        dst[x] = r * scale + fr[x];
      }
    }
    __syncthreads();     // this stage is refilled two leaves on
  }
}

}  // namespace

bool near_fft_supported(const Plan& P) { return P.S == kNS && P.L >= 2; }

void near_fft_counts(const Plan& P, size_t& nK, size_t& nM, size_t& nP) {
  const size_t nl3 = (size_t)1 << (3 * P.L);
  nK = (size_t)kNCH * kNO * 4 * kNC;
  nM = (size_t)kNCH * (nl3 + 1) * kNC;
  nP = nl3 * 4 * kNK;
}

cudaError_t setup_near_fft(const Plan& P) {
  cudaError_t e = cudaFuncSetAttribute(k_nz_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)(2 * sizeof(double2) * kNM * kNM * kNX));
  if (e != cudaSuccess) return e;
  e = cudaFuncSetAttribute(k_nz_mac, cudaFuncAttributeMaxDynamicSharedMemorySize,
                           (int)(sizeof(float2) * (128 + 2 * kMacStage)));
  if (e != cudaSuccess) return e;
  return cudaFuncSetAttribute(k_nz_inv, cudaFuncAttributeMaxDynamicSharedMemorySize,
                              (int)(sizeof(float) * kInvSmemFloats));
}

cudaError_t launch_near_fft_kernels(Plan& P, cudaStream_t s) {
  k_nz_kernel<<<kNO * 4, kThr, 2 * sizeof(double2) * kNM * kNM * kNX, s>>>(P.near_tab, P.nz_K);
  return cudaGetLastError();
}

cudaError_t launch_near_fft_fwd(Plan& P, const float* rho, cudaStream_t s) {
  k_nz_fwd<<<1u << (3 * P.L), kFwdThr, 0, s>>>(rho, P.d_mean, P.N, P.L, P.nz_M);
  return cudaGetLastError();
}

cudaError_t launch_near_fft(Plan& P, const float* rho, float* phi, float* acc, cudaStream_t s, bool fwd_done) {
  const unsigned nl3 = 1u << (3 * P.L);
  const int nt = (1 << P.L) / kNT;
  if (!fwd_done) k_nz_fwd<<<nl3, kFwdThr, 0, s>>>(rho, P.d_mean, P.N, P.L, P.nz_M);
  k_nz_mac<<<dim3(nt * nt * nt, kNCH / kCPC), kMacThr, sizeof(float2) * (128 + 2 * kMacStage), s>>>(
      P.nz_K, P.nz_M, P.nz_P, P.L, P.iso);
  launch_l2p(P, phi, acc, s);
  const unsigned inv_grid = nl3 < (unsigned)P.num_sms ? nl3 : (unsigned)P.num_sms;
  k_nz_inv<<<inv_grid, kInvThr, sizeof(float) * kInvSmemFloats, s>>>(P.nz_P, P.N, P.L, phi, acc);
  return cudaGetLastError();
}

}  // namespace fmm

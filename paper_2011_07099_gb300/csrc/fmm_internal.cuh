// Internal declarations of libfmm (not part of the C-ABI).
#pragma once

#include <cuda_runtime.h>
#include <cstdint>
#include <cstddef>

#include "../../include/fmm.h"
#include "green_s1.cuh"

namespace fmm {

// Records `code` as the calling host thread's last error and returns it.
int set_last_error(int code);

constexpr int kMaxLevel = 8;
constexpr int kMaxOrder = 8;
constexpr int kFields = 4;          // Phi, g_x, g_y, g_z
constexpr int kMaxOffsets = 189;    // interaction-zone size below level 2 (Sec. 2)
// The top two far-field levels (2 and 3) carry the long-range potential, whose
// sum cancels most; their Phi contraction uses G = hi + lo split tables.
constexpr int kExtTopLevel = 3;
// Levels at or below kExtTopLevel always run the FP32 split-table kernel; the
// tensor-core precision modes apply from kTcMinLevel down to the leaves.
constexpr int kTcMinLevel = kExtTopLevel + 1;

// ---------------------------------------------------------------- Morton keys
// Node order at every level is Morton: bit 3b of the key is bit b of x, 3b+1
// of y, 3b+2 of z.  The 8 children of parent key P are 8P + c with
// c = cx | cy << 1 | cz << 2, so siblings are contiguous.
__host__ __device__ inline uint32_t spread3(uint32_t v) {
  v &= 0x3ffu;
  v = (v | (v << 16)) & 0x030000FFu;
  v = (v | (v << 8)) & 0x0300F00Fu;
  v = (v | (v << 4)) & 0x030C30C3u;
  v = (v | (v << 2)) & 0x09249249u;
  return v;
}
__host__ __device__ inline uint32_t compact3(uint32_t v) {
  v &= 0x09249249u;
  v = (v ^ (v >> 2)) & 0x030C30C3u;
  v = (v ^ (v >> 4)) & 0x0300F00Fu;
  v = (v ^ (v >> 8)) & 0xFF0000FFu;
  v = (v ^ (v >> 16)) & 0x000003FFu;
  return v;
}
__host__ __device__ inline uint32_t morton(uint32_t x, uint32_t y, uint32_t z) {
  return spread3(x) | (spread3(y) << 1) | (spread3(z) << 2);
}
__host__ __device__ inline void unmorton(uint32_t k, uint32_t& x, uint32_t& y, uint32_t& z) {
  x = compact3(k);
  y = compact3(k >> 1);
  z = compact3(k >> 2);
}

// At high order the downward interpolation amplifies the rounding of the
// local fields much more (absolute L2L weight sums ~1100 at p = 8 against ~160
// at p = 6), so from this order on every level above the leaves keeps FP64
// local fields, and the tensor cores take only the leaf level.
constexpr int kWideOrder = 7;

// ------------------------------------------------------------------- the plan
struct Plan {
  int N = 0, L = 0, p = 0, S = 0;
  int prec = FMM_PREC_FP32;
  // the tabulated Green's function (G_S1 by default) and the boundary: in the
  // isolated problem (iso = 1) every table holds G_0, no mean is removed and
  // interaction and near zones keep only in-box nodes
  green::Spec gspec;
  int iso = 0;
  double* gmesh = nullptr;          // kind 4: (G, -dG/dx, -dG/dy, -dG/dz) at the mesh offsets, 4 N^3
  int device = 0;
  int num_sms = 0;
  int solved = 0;

  // device buffers
  double* d_partials = nullptr;     // block partial sums for the mean
  double* d_mean = nullptr;         // mean density (1 value)
  int n_partials = 0;
  float* M[kMaxLevel + 1] = {};     // gridlet masses, 8^l x p^3, levels 2..L
  float* F[kMaxLevel + 1] = {};     // local fields, 8^l x 4 x p^3, levels 2..L
  float* m2l_part = nullptr;        // coarse FP32 M2L levels: ranges x (sum, low part) x 8^l x 4 p^3
  // Local fields of the wide levels in FP64: the L2L interpolation
  // to the children extrapolates to points outside the parent's gridlet
  // (weights up to ~160 in absolute sum at p = 6), so FP32 storage of the
  // coarse local fields would cost ~1e-6 of the potential.
  double* F64[kMaxLevel + 1] = {};
  // At order >= kWideOrder the gridlet masses of the wide levels are kept in
  // FP64 as well (M2M writes both copies; M2L reads them as hi + lo).
  double* M64[kMaxLevel + 1] = {};
  float4* tab[kMaxLevel + 1] = {};  // (G, -dG/dx, -dG/dy, -dG/dz) at n dx_l, n in [-(4p-1), 4p-1]^3
  float4* tab_lo[kMaxLevel + 1] = {};  // v - fl32(v) of the same entries, 4 fields (wide levels)
  float4* near_tab = nullptr;       // the same at cell spacing for |d_i| in [0, 2S-1], folded
  float2* w_p2m = nullptr;          // Lagrange weights [p][S] as (hi, lo): gridlet s at cell c
  float2* w_m2m = nullptr;          // Lagrange weights [p][2p] as (hi, lo): parent s at child point u
  int8_t* offsets[kMaxLevel + 1] = {};  // per level: [8 child types][n_off][3] (dx, dy, dz) = T - S
  // tensor-core M2L (levels >= kTcMinLevel, allocated on the first mixed-precision solve)
  uint4* tab_bf[kMaxLevel + 1] = {};       // per table entry, per field: bf16 hi | bf16 lo << 16
  void* Mbf_hi[kMaxLevel + 1] = {};        // gridlet masses split into BF16 parts (2; 3 at bf16x6 levels), per parity class with a halo
                                           // (layout in m2l_tc.cu, k_split_bf16), rows padded to KP
  void* tmapB[kMaxLevel + 1] = {};         // host CUtensorMap of each Mbf_hi level (the tensor loads of B)
  void* Apre[kMaxLevel + 1] = {};          // precomputed split translation tiles per offset slot
  int tc_group = 4;                        // offsets accumulated per TMEM partial before promotion
  int tc_tile[kMaxLevel + 1] = {};         // targets per tensor-core CTA per level: 0 (= 256) or 128
  int m2l_fft = 0;                         // FFT form of the interaction zone at the fine levels (ablation)
  void* fft = nullptr;                     // its cuFFT plans and buffers (m2l_fft.cu)
  int tc_min_level = kTcMinLevel;          // first level on the tensor cores in the mixed forms
  int tc_min_set = 0;                      // tc_min_level set by the caller (honoured at high order too)
  // near zone by FFT (p2p_fft.cu; 8-cell leaves): kernel spectra [72][27][4][32],
  // source spectra [72][leaves + 1][32] (last: all zero), target spectra [leaves][4][2304]
  int near_fft = 0;
  float2* nz_K = nullptr;
  float2* nz_M = nullptr;
  float2* nz_P = nullptr;
  // learned table correction (MLP weights) and its training buffers
  float* corr_w = nullptr;                 // mlp::kParams weights (device) or unset
  int has_corr = 0;
  int corr_fp32 = 0;                       // 0: BF16 inference (default), 1: FP32
  float* train_out = nullptr;              // 4 N^3: the solve's outputs during training
  float* lam_cells = nullptr;              // 4 N^3: cell residual adjoint
  float* lam[kMaxLevel + 1] = {};          // adjoint of the local fields, 8^l x 4 x p^3
  float* dT_all = nullptr;                 // table gradients, levels 2..L, (8p-1)^3 x 4 each
  float* dT[kMaxLevel + 1] = {};
  float* grad_partials = nullptr;          // per-block MLP gradient partials
  // grid model of G_* (Sec. 4): one free value per folded table entry and
  // field, per level: levels 2..L x 4 fields x (4p)^3, added to the tables
  float* grid = nullptr;
  int has_grid = 0;
  uint64_t wait_ns = 2000000000ull;        // limit of every bounded device-side wait
  int inject_stall = 0;                    // test hook: tensor-core MMA issuer stalls
  int tc_ready = 0;
  int* d_err = nullptr;                    // device error word (bounded waits that gave up)
  int n_off[kMaxLevel + 1] = {};

  // untimed solves of the tensor-core forms overlap independent stages on
  // two plan-owned streams (aux), joined by events (fev)
  cudaStream_t aux[2] = {};
  cudaEvent_t fev[4] = {};

  // per-stage timing: ev[2*k] / ev[2*k+1] bracket slot k
  int timing = 0;
  int timed = 0;
  cudaEvent_t ev[2 * FMM_TIME_SLOTS] = {};

  // host-buffer staging for fmm_solve_host
  float* stage_in = nullptr;
  float* stage_out = nullptr;
};

// ------------------------------------------------------- per-plan kernel setup
// Opt-in shared-memory limits (and other function attributes) are set once at
// plan creation, never inside a solve, so a solve is safe to capture.
cudaError_t setup_upward(const Plan& P);
// Levels whose local field is kept in FP64 (M2L output reduced in FP64, L2L
// from them in double-float): the two coarse levels, at high order every level
// above the leaves, and with 16-cell leaves every level: the L2P of a 16-cell
// leaf extrapolates far beyond the gridlet (absolute weight sums up to 835 at
// p = 6), which amplifies the FP32 rounding of the leaf field at the leaf's
// edge cells to ~1e-7 of the potential, so that leaf field stays FP64.
constexpr int kWideLeaf = 16;
inline bool wide_level(const Plan& P, int l) {
  return l <= kExtTopLevel || (P.p >= kWideOrder && l < P.L) || P.S >= kWideLeaf;
}
// First level of the tensor-core M2L in the mixed forms (above L: none; the
// tensor-core kernel writes FP32 fields, or the bf16x6 kernel FP64 ones, and
// 16-cell leaves use neither).  At high order the wide levels from
// kWideTcLevel down run the bf16x6 mode: measured on the 512^3 order-8
// clustered workload, level 5 in bf16x6 costs 2.6e-6 / 5.8e-6 (Phi / g)
// against the oracle, level 4 6.1e-5 (the coarser the level, the more its
// far-field sums cancel), so the coarser wide levels keep the double-float
// CUDA-core kernel.  A level set by the caller is taken as given.
constexpr int kWideTcLevel = 5;
inline int tc_first_level(const Plan& P) {
  if (P.S >= kWideLeaf) return P.L + 1;
  if (P.tc_min_set || P.p < kWideOrder) return P.tc_min_level;
  const int wide_first = P.L < kWideTcLevel ? P.L : kWideTcLevel;
  return P.tc_min_level > wide_first ? P.tc_min_level : wide_first;
}

cudaError_t setup_m2l_fp32(const Plan& P);
// Number of offset ranges the FP32 M2L of a level is split into (1 = none).
int m2l_fp32_splits(const Plan& P, int level);
cudaError_t setup_downward(const Plan& P);
cudaError_t setup_p2p(const Plan& P);

// ------------------------------------------------------------ kernel launchers
// Each returns cudaGetLastError() after the launch.
cudaError_t launch_tables(Plan& P, cudaStream_t s);
cudaError_t launch_mean(Plan& P, const float* rho, cudaStream_t s);
// The same reduction into caller scratch (P.n_partials partials, 1 mean).
cudaError_t launch_mean_into(const Plan& P, const float* rho, double* partials, double* mean, cudaStream_t s);
cudaError_t launch_p2m(Plan& P, const float* rho, cudaStream_t s);
cudaError_t launch_m2m(Plan& P, int level, cudaStream_t s);       // level+1 -> level
cudaError_t launch_m2l_fp32(Plan& P, int level, cudaStream_t s);  // writes F[level] (and F64[level] when coarse)
// FP32 M2L over one offset list for all child types, written into F[level].
cudaError_t launch_m2l_fp32_list(Plan& P, int level, const int8_t* offs, int n_off, cudaStream_t s);
// The FFT form of the interaction zone (m2l_fft.cu): levels that use it,
// set-up of plans/buffers/table spectra (FMM_* code), launch, release.
bool fft_level(const Plan& P, int level);
int prepare_fft(Plan& P);
cudaError_t launch_m2l_fft(Plan& P, int level, cudaStream_t s);
void free_fft(Plan& P);
cudaError_t launch_l2l(Plan& P, int level, cudaStream_t s);       // F[level] -> F[level+1] (adds)
// near_fwd_done: the FFT near zone's source spectra were already taken (launch_near_fft_fwd).
cudaError_t launch_p2p(Plan& P, const float* rho, float* phi, float* acc, cudaStream_t s,
                       bool near_fwd_done = false);
// The near zone by FFT (p2p_fft.cu): whether the plan's shape allows it, the
// float2 counts of its kernel, source and target spectra, function attributes, the plan-time kernel spectra (after every
// re-tabulation) and the leaf stage itself (launch_p2p dispatches to it).
bool near_fft_supported(const Plan& P);
void near_fft_counts(const Plan& P, size_t& nK, size_t& nM, size_t& nP);
cudaError_t setup_near_fft(const Plan& P);
cudaError_t launch_near_fft_kernels(Plan& P, cudaStream_t s);
cudaError_t launch_near_fft_fwd(Plan& P, const float* rho, cudaStream_t s);
cudaError_t launch_near_fft(Plan& P, const float* rho, float* phi, float* acc, cudaStream_t s, bool fwd_done);
cudaError_t setup_m2l_tc(const Plan& P);
cudaError_t setup_learn();
cudaError_t launch_residual(const float* phi, const float* acc, const float* tphi, const float* tacc, size_t n3,
                            float w_phi, float w_g, float* lam, float* loss, int sms, cudaStream_t s);
cudaError_t launch_adjoint_and_table_grad(Plan& P, const float* lam_cells, cudaStream_t s);
cudaError_t launch_mlp_backward(Plan& P, const float* w, float* grad, cudaStream_t s);
int mlp_backward_blocks(const Plan& P);
cudaError_t launch_adam(float* w, const float* g, float* m, float* v, size_t n, int step, float lr, float b1, float b2,
                        float eps, cudaStream_t s);
cudaError_t launch_mesh_green(int N, float* out, int sms, cudaStream_t s);
cudaError_t launch_mesh_green_plan(const Plan& P, double* out, cudaStream_t s);
// Sampled error against the direct periodic sum with G_S1 (errstats.cu):
// targets T <= error_stats_max_samples(), partials error_stats_grid_x(P, T)
// x T x 4 doubles, sums 4 doubles, mean_scratch P.n_partials + 1 doubles
// (the density mean of the statement is its own, the plan's mean stage is
// left as the last solve wrote it).
int error_stats_max_samples();
int error_stats_grid_x(const Plan& P, int T);
cudaError_t launch_error_stats(Plan& P, const float* rho, const float* phi, const float* acc,
                               const unsigned long long* targets, int T, double* partials, double* sums,
                               double* mean_scratch, cudaStream_t s);
cudaError_t launch_tab_bf16(Plan& P, int level, cudaStream_t s);
// Grid-model parameters per level: 4 fields x (4p)^3 folded entries.
inline size_t grid_level_size(int p) { return (size_t)4 * (4 * p) * (4 * p) * (4 * p); }
// dJ/d(grid) += the table gradients P.dT folded onto the grid's entries.
cudaError_t launch_grid_grad(Plan& P, float* grad, cudaStream_t s);
cudaError_t launch_split_bf16(Plan& P, int level, cudaStream_t s);
cudaError_t launch_m2l_tc(Plan& P, int level, int mode, cudaStream_t s);
int tc_padded_k(int p);
// Tensor-core levels with FP64 local fields (the wide levels of high orders)
// use the bf16x6 mode: operands split in three BF16 parts, partials added
// into a double-float total.
inline bool tc_wide(const Plan& P, int l) { return wide_level(P, l); }
inline int tc_splits(const Plan& P, int l) { return tc_wide(P, l) ? 3 : 2; }
// Targets per tensor-core CTA at level l: 128 in the wide mode, else the
// plan's tile (fmm_plan_set_tc_tile), 256 by default.
inline int tc_targets(const Plan& P, int l) { return tc_wide(P, l) || P.tc_tile[l] == 128 ? 128 : 256; }
size_t tc_apre_bytes(int p, int nsplit);
size_t tc_bsplit_bytes(int p, int level, int nsplit);
// Encodes P.tmapB[level] for P.Mbf_hi[level] (FMM_* code).
int make_tc_map(Plan& P, int level);
cudaError_t launch_build_a(Plan& P, int level, cudaStream_t s);

// Block-wide separable contraction over the middle axis of a [A][Kin][B]
// array: out[a][s][b] = sum_k W(s,k) in[a][k][b], W(s,k) = W[s*ldw+k] or, when
// wt is set, W[k*ldw+s].  Threads tid..nthr stride over the outputs.  Weights
// are (hi, lo) float pairs: the same weights apply to every node, so their
// FP32 rounding would err coherently across the whole mesh.
__device__ inline void contract_mid(const float* __restrict__ in, float* __restrict__ out, int A,
                                    int Kin, int Kout, int B, const float2* __restrict__ W, int ldw,
                                    bool wt, int tid, int nthr) {
  const int total = A * Kout * B;
  for (int i = tid; i < total; i += nthr) {
    const int b = i % B;
    const int s = (i / B) % Kout;
    const int a = i / (B * Kout);
    const float* src = in + (size_t)a * Kin * B + b;
    float acc = 0.f, lo = 0.f;
    for (int k = 0; k < Kin; ++k) {
      const float2 w = wt ? W[k * ldw + s] : W[s * ldw + k];
      const float x = src[k * B];
      acc = fmaf(w.x, x, acc);
      lo = fmaf(w.y, x, lo);
    }
    out[i] = acc + lo;
  }
}

// ---------------------------------------------------------- double-float
// Values as unevaluated sums hi + lo of two FP32 numbers (~48 significant
// bits) computed with error-free transformations (TwoProd by FMA, TwoSum;
// Ogita, Rump and Oishi, "Accurate sum and dot product", 2005).  The _rn
// intrinsics keep the compiler from contracting the transformations into
// FMAs.  On this part the FP64 pipe runs at 1/64 of the FP32 rate, so the
// upward pass and the coarse L2L run ~10x faster this way than in FP64.
__device__ __forceinline__ float2 df_two_sum(float a, float b) {
  const float s = __fadd_rn(a, b);
  const float z = __fsub_rn(s, a);
  return make_float2(s, __fadd_rn(__fsub_rn(a, __fsub_rn(s, z)), __fsub_rn(b, z)));
}
__device__ __forceinline__ float2 df_from_double(double d) {
  const float h = (float)d;
  return make_float2(h, (float)(d - (double)h));
}
__device__ __forceinline__ double df_to_double(float2 v) { return (double)v.x + (double)v.y; }

// contract_mid in double-float: inputs, weights and outputs are (hi, lo)
// pairs; each output is normalised (hi = the FP32 rounding of the sum).
__device__ inline void contract_mid_df(const float2* __restrict__ in, float2* __restrict__ out, int A, int Kin,
                                       int Kout, int B, const float2* __restrict__ W, int ldw, bool wt, int tid,
                                       int nthr) {
  const int total = A * Kout * B;
  for (int i = tid; i < total; i += nthr) {
    const int b = i % B;
    const int s = (i / B) % Kout;
    const int a = i / (B * Kout);
    const float2* src = in + (size_t)a * Kin * B + b;
    float hs = 0.f, lc = 0.f;
    for (int k = 0; k < Kin; ++k) {
      const float2 w = wt ? W[k * ldw + s] : W[s * ldw + k];
      const float2 x = src[k * B];
      const float pr = __fmul_rn(w.x, x.x);
      const float pe = fmaf(w.x, x.x, -pr);            // exact product error
      const float2 t = df_two_sum(hs, pr);
      hs = t.x;
      lc = fmaf(w.x, x.y, fmaf(w.y, x.x, __fadd_rn(lc, __fadd_rn(pe, t.y))));
    }
    const float sum = __fadd_rn(hs, lc);
    out[i] = make_float2(sum, __fsub_rn(lc, __fsub_rn(sum, hs)));
  }
}

// 3-D separable contraction [Kin]^3 -> [Kout]^3 of one field in double-float
// (scratch t1: Kin*Kin*Kout, t2: Kin*Kout*Kout pairs).  Ends with __syncthreads().
__device__ inline void contract3_df(const float2* in, float2* t1, float2* t2, float2* out, int Kin, int Kout,
                                    const float2* W, int ldw, bool wt, int tid, int nthr) {
  contract_mid_df(in, t1, Kin * Kin, Kin, Kout, 1, W, ldw, wt, tid, nthr);
  __syncthreads();
  contract_mid_df(t1, t2, Kin, Kin, Kout, Kout, W, ldw, wt, tid, nthr);
  __syncthreads();
  contract_mid_df(t2, out, 1, Kin, Kout, Kout * Kout, W, ldw, wt, tid, nthr);
  __syncthreads();
}

// 3-D separable contraction of `nf` fields [nf][Kin][Kin][Kin] -> [nf][Kout]^3,
// the same 1-D matrix on every axis.  t1, t2 are scratch of nf*Kin*Kin*Kout
// and nf*Kin*Kout*Kout floats.  Ends with __syncthreads().
__device__ inline void contract3(const float* in, float* t1, float* t2, float* out, int nf, int Kin,
                                 int Kout, const float2* W, int ldw, bool wt, int tid, int nthr) {
  contract_mid(in, t1, nf * Kin * Kin, Kin, Kout, 1, W, ldw, wt, tid, nthr);
  __syncthreads();
  contract_mid(t1, t2, nf * Kin, Kin, Kout, Kout, W, ldw, wt, tid, nthr);
  __syncthreads();
  contract_mid(t2, out, nf, Kin, Kout, Kout * Kout, W, ldw, wt, tid, nthr);
  __syncthreads();
}

}  // namespace fmm

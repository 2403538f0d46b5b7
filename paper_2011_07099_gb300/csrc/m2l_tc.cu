// M2L on the tcgen05 tensor cores (BF16 operands, FP32 accumulation in TMEM).
//
// Eq. fmm2 (Sec. 3) over a level is, for the targets T of one child type c
// (all of which share the interaction list IL(c), Sec. 2 Fig. fmm), the dense
// contraction
//     D[(f, r), T] = sum_{o in IL(c)} sum_s A_o[(f, r), s] * B_o[s, T],
//     A_o[(f, r), s] = Tab_f[o p + r - s]     (Toeplitz in r - s, from the table)
//     B_o[s, T]      = M_{T - o}[s]            (gridlet masses of the source node)
// with f over (G, -dG/dx, -dG/dy, -dG/dz).  Rows (f, r) run over 4 p^3, the
// reduction over 189 p^3.
//
// The translation operand A_o depends only on the offset (not on the target),
// so it is built once per plan, split into BF16 hi + lo, in the exact shared-
// memory tile layout (`k_build_a`), and each pipeline stage streams its two
// 8 KB tiles with one bulk asynchronous copy.
//
// CTA tile: 128 rows of (f, r) x 256 targets (one M = 128, N = 256 MMA per
// 16-deep k step, so every A byte staged feeds 256 targets).  Warp roles:
//   warp 0      issues the MMAs (one thread);
//   warps 1..4  per stage (32 reduction indices of one offset): one thread
//               arms the stage's A barrier with the A bytes and issues the
//               bulk copies; all gather B, the source nodes' split BF16
//               masses, with 16-byte cp.async whose completion arrives on the
//               stage barrier (hi and lo are interleaved every 8 values, so a
//               target's stage slice is one 128-byte line);
//   warps 5..8  drain TMEM: every G offsets accumulate into a fresh TMEM
//               partial, which the drain warps add into an FP32 total kept in
//               TMEM while the issuer waits.  A single TMEM accumulator over
//               all 189 p^3 terms drifts by ~1e-4 on the coherent, cancelling
//               far-field sums (the accumulation inside the MMA truncates);
//               per-group partials summed in FP32 with rounding to nearest
//               cost ~1e-7 (CPU emulation of the level's sums), far below the
//               bf16x3 operand error.
// Layout: canonical no-swizzle K-major core matrices (8 rows x 16 B).
// bf16x3 mode accumulates A_hi B_hi + A_hi B_lo + A_lo B_hi; bf16 mode A_hi B_hi.
// TMEM: 512 columns = partial (256) | total (256).
// Every wait is bounded; a timeout sets the plan's error word and later work
// is skipped without leaving any barrier sequence.  Before the CTA exits the
// issuer waits (bounded) for the completion of every MMA it issued and the
// copy thread for every A copy it issued, so nothing is still in flight into
// this CTA's TMEM or shared memory; then TMEM is freed and the kernel returns.
#include <cuda_bf16.h>

#include "fmm_internal.cuh"
#include "tc_ptx.cuh"

namespace fmm {
namespace {

constexpr int kKC = 32;          // reduction indices per pipeline stage
constexpr int kNT = 256;         // targets per CTA (MMA N)
constexpr int kProd = 128;       // producer threads (warps 1..4)
constexpr int kDrain = 128;      // drain threads (warps 5..8)
constexpr int kThreads = 32 + kProd + kDrain;
constexpr uint32_t kTmemCols = 512;
constexpr int kTileBytes = 128 * kKC * 2;     // one 128 x 32 BF16 tile of A
constexpr int kTileB = kNT * kKC * 2;         // one 256 x 32 BF16 tile of B

template <int P, int MODE>
struct TcShape {
  static constexpr int P3 = P * P * P;
  static constexpr int KP = ((P3 + kKC - 1) / kKC) * kKC;   // padded reduction length per offset
  static constexpr int NCH = KP / kKC;                       // stages per offset
  static constexpr int MT = (4 * P3 + 127) / 128;            // row tiles
  static constexpr int NSPLIT = MODE == 3 ? 2 : 1;
  static constexpr int STAGE_BYTES = NSPLIT * (kTileBytes + kTileB);
  static constexpr int EXTRA = 2 * kNT * 4 + 64;
  static constexpr int LIMIT = 225 * 1024;                  // dynamic shared memory budget
  static constexpr int FIT = (LIMIT - EXTRA) / STAGE_BYTES;
  static constexpr int ST = FIT > 6 ? 6 : FIT;              // pipeline depth
  static_assert(FIT >= 3, "pipeline needs at least 3 stages");
  static constexpr int SMEM = ST * STAGE_BYTES + EXTRA;
};

// Offsets o with |o_i| <= 3 are indexed ((oz+3) 7 + (oy+3)) 7 + (ox+3).
__host__ __device__ constexpr int off_index(int ox, int oy, int oz) { return ((oz + 3) * 7 + (oy + 3)) * 7 + (ox + 3); }
constexpr int kOffSlots = 343;

__device__ __forceinline__ void producer_bar() { asm volatile("bar.sync 1, %0;" ::"n"(kProd) : "memory"); }

template <int P, int MODE>
__global__ void __launch_bounds__(kThreads, 1)
k_m2l_tc(const __nv_bfloat16* __restrict__ Msp, const uint8_t* __restrict__ Apre,
         const int8_t* __restrict__ offs, int n_off, int level, int group,
         float* __restrict__ F, int* __restrict__ err, uint64_t kWaitNs, int stall, int iso) {
  using Sh = TcShape<P, MODE>;
  constexpr int P3 = Sh::P3, KP = Sh::KP, NCH = Sh::NCH, MT = Sh::MT, ST = Sh::ST, NSPLIT = Sh::NSPLIT;
  constexpr int STAGE_BYTES = Sh::STAGE_BYTES;
  static_assert(Sh::SMEM <= Sh::LIMIT, "shared-memory budget");
  constexpr uint32_t IDESC = tc::idesc_bf16_f32(128, kNT);
  constexpr uint32_t LBO_A = (128 / 8) * 128;      // next core matrix along K in an A tile
  constexpr uint32_t LBO_B = (kNT / 8) * 128;      // next core matrix along K in a B tile
  constexpr uint32_t A_TX = NSPLIT * kTileBytes;

  extern __shared__ __align__(1024) uint8_t smem[];
  uint8_t* stages = smem;                                                // ST x [A tiles | B tiles]
  int* srckey = reinterpret_cast<int*>(smem + ST * STAGE_BYTES);         // 2 x kNT
  // full: the producers' cp.async gathers of B landed; afull: the bulk copy of
  // A landed (its own barrier, so that a CTA that gives up can still wait for
  // exactly the copies it issued); empty: the MMAs reading the stage are done;
  // pfull / pfree: a group's partial is complete / has been added to the total.
  __shared__ uint64_t full[ST], afull[ST], empty[ST], pfull, pfree, mdone;
  __shared__ uint32_t tmem_holder;
  __shared__ int s_err;

  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int nt = blockIdx.x, mt = blockIdx.y, ctype = blockIdx.z;
  const int n = 1 << level;
  const uint32_t n_par = 1u << (3 * (level - 1));
  const uint32_t par0 = (uint32_t)nt * kNT;
  const int8_t* my_offs = offs + (size_t)ctype * n_off * 3;
  const int n_grp = (n_off + group - 1) / group;

  if (tid == 0) {
    s_err = 0;
    for (int i = 0; i < ST; ++i) {
      tc::mbar_init(&full[i], kProd);          // one cp.async-completion arrival per producer thread
      tc::mbar_init(&afull[i], 1);             // the A expect_tx arrival (+ its bytes)
      tc::mbar_init(&empty[i], 1);             // one MMA completion
    }
    tc::mbar_init(&pfull, 1);
    tc::mbar_init(&pfree, kDrain);
    tc::mbar_init(&mdone, 1);
    tc::mbar_fence_init();
  }
  if (warp == 0) tc::tmem_alloc(&tmem_holder, kTmemCols);
  tc::fence_before_sync();
  __syncthreads();
  tc::fence_after_sync();
  const uint32_t tmem = tmem_holder;
  const uint32_t t_tot = tmem + kNT;
  const uint32_t smem_base = tc::smem_u32(stages);

  if (warp == 0) {
    // ------------------------------------------------------------ MMA issuer
    // (`stall` is a test hook: the issuer does nothing, so every dependent
    // bounded wait of this CTA expires and the error path runs)
    if (lane == 0) {
      bool ok = true;
      for (int io = 0; io < n_off && ok && !stall; ++io) {
        const int g = io / group;
        const bool first = (io % group) == 0;
        // the partial is reused: the drain must have added group g - 1
        if (first && g >= 1 && !tc::mbar_wait_bounded(&pfree, (uint32_t)(g - 1) & 1u, kWaitNs)) {
          ok = false;
          break;
        }
        tc::fence_after_sync();
        for (int ch = 0; ch < NCH; ++ch) {
          const int it = io * NCH + ch, st = it % ST;
          const uint32_t ph = (uint32_t)(it / ST) & 1u;
          if (!tc::mbar_wait_bounded(&afull[st], ph, kWaitNs) || !tc::mbar_wait_bounded(&full[st], ph, kWaitNs)) {
            ok = false;
            break;
          }
          tc::fence_proxy_async_smem();     // cp.async (generic proxy) data -> tensor core
          tc::fence_after_sync();
          const uint32_t sA = smem_base + st * STAGE_BYTES;
          const uint32_t sB = sA + NSPLIT * kTileBytes;
#pragma unroll
          for (int j = 0; j < kKC / 16; ++j) {
            const uint64_t ah = tc::smem_desc(sA + j * 2 * LBO_A, LBO_A, 128);
            const uint64_t bh = tc::smem_desc(sB + j * 2 * LBO_B, LBO_B, 128);
            tc::mma_bf16(tmem, ah, bh, IDESC, (!first || ch > 0 || j > 0) ? 1u : 0u);
            if (MODE == 3) {
              const uint64_t al = tc::smem_desc(sA + kTileBytes + j * 2 * LBO_A, LBO_A, 128);
              const uint64_t bl = tc::smem_desc(sB + kTileB + j * 2 * LBO_B, LBO_B, 128);
              tc::mma_bf16(tmem, ah, bl, IDESC, 1u);
              tc::mma_bf16(tmem, al, bh, IDESC, 1u);
            }
          }
          tc::mma_commit(&empty[st]);
        }
        if (ok && ((io % group) == group - 1 || io == n_off - 1)) tc::mma_commit(&pfull);
      }
      // every MMA this thread issued has finished before TMEM is released,
      // also when a wait gave up part-way
      tc::mma_commit(&mdone);
      if (!tc::mbar_wait_bounded(&mdone, 0u, kWaitNs)) ok = false;
      if (!ok || stall) atomicExch(&s_err, 1);
    }
    __syncwarp();
  } else if (warp <= 4) {
    // ------------------------------------------------------------- producers
    const int pt = tid - 32;   // 0..127
    bool ok = true;            // sticky; after a timeout only the barrier sequence is kept
    int armed = 0;             // (pt == 0) stages whose A copy was issued: iterations [0, armed)
    const int piece = pt & 7, c8 = piece >> 1, split = piece & 1;
    for (int io = 0; io < n_off; ++io) {
      const int b = io & 1;
      const int ox = my_offs[3 * io + 0], oy = my_offs[3 * io + 1], oz = my_offs[3 * io + 2];
      // source keys of this offset (buffer b was last read two offsets ago)
      producer_bar();
#pragma unroll
      for (int h = 0; h < kNT / kProd; ++h) {
        const int t = pt + h * kProd;
        int key = 1 << (3 * level);   // no source: the all-zero node after the 8^l nodes
        if (par0 + t < n_par) {
          uint32_t x, y, z;
          unmorton(8u * (par0 + t) + ctype, x, y, z);
          // the source node, wrapped; in the isolated problem a source
          // outside the box contributes nothing (zero-filled like padding)
          const int ux = (int)x - ox, uy = (int)y - oy, uz = (int)z - oz;
          const bool inbox = (unsigned)ux < (unsigned)n && (unsigned)uy < (unsigned)n && (unsigned)uz < (unsigned)n;
          if (inbox || !iso) key = (int)morton((uint32_t)ux & (n - 1), (uint32_t)uy & (n - 1), (uint32_t)uz & (n - 1));
        }
        srckey[b * kNT + t] = key;
      }
      producer_bar();
      const int* sk = srckey + b * kNT;
      const uint8_t* atile = Apre + ((size_t)(off_index(ox, oy, oz) * MT + mt) * NCH) * 2 * kTileBytes;
      for (int ch = 0; ch < NCH; ++ch) {
        const int it = io * NCH + ch, st = it % ST;
        if (ok && !tc::mbar_wait_bounded(&empty[st], ((uint32_t)(it / ST) & 1u) ^ 1u, kWaitNs)) ok = false;
        if (!ok) continue;
        const uint32_t sA = smem_base + st * STAGE_BYTES;
        const uint32_t sB = sA + NSPLIT * kTileBytes;
        if (pt == 0) {
          tc::mbar_arrive_expect_tx(&afull[st], A_TX);
          tc::bulk_g2s(sA, atile + (size_t)ch * 2 * kTileBytes, kTileBytes, &afull[st]);
          if (MODE == 3)
            tc::bulk_g2s(sA + kTileBytes, atile + ((size_t)ch * 2 + 1) * kTileBytes, kTileBytes, &afull[st]);
          armed = it + 1;
        }
#pragma unroll
        for (int pass = 0; pass < kNT / 16; ++pass) {
          const int t = (pt >> 3) + 16 * pass;
          if (MODE == 3 || split == 0) {
            // full 16-byte reads only (no zero-fill operand): lanes then merge
            // into whole-sector requests; empty slots read the zero node
            const int key = sk[t];
            const size_t e0 = ((size_t)key * (KP / 8) + ch * (kKC / 8) + c8) * 16 + split * 8;
            const uint32_t d = sB + split * kTileB + (uint32_t)((c8 * (kNT / 8) + t / 8) * 128 + (t % 8) * 16);
            tc::cp_async16_full(d, Msp + e0);
          }
        }
        tc::cp_async_arrive_noinc(&full[st]);
      }
    }
    tc::cp_async_wait<0>();
    asm volatile("cp.async.wait_all;" ::: "memory");
    // the A copies issued last may not have been consumed (after a timeout):
    // wait (bounded) until each has landed, so no copy is in flight into this
    // CTA's shared memory when it exits
    if (pt == 0) {
      for (int it = armed - ST > 0 ? armed - ST : 0; it < armed; ++it)
        if (!tc::mbar_wait_bounded(&afull[it % ST], (uint32_t)(it / ST) & 1u, kWaitNs)) ok = false;
    }
    if (!ok) atomicExch(&s_err, 1);
  } else {
    // ------------------------------------------------------------ drain warps
    const int q = warp & 3;                          // TMEM lane quadrant
    const uint32_t lanebase = (uint32_t)(q * 32) << 16;
    bool ok = true;
    for (int g = 0; g < n_grp; ++g) {
      const bool got = ok && tc::mbar_wait_bounded(&pfull, (uint32_t)g & 1u, kWaitNs);
      ok = __all_sync(0xffffffffu, got);
      if (!ok) break;
      tc::fence_after_sync();
      for (int c0 = 0; c0 < kNT; c0 += 32) {
        uint32_t rp[32], rt[32];
        tc::tmem_ld32_nowait(tmem + lanebase + c0, rp);
        if (g > 0) tc::tmem_ld32_nowait(t_tot + lanebase + c0, rt);
        tc::tmem_wait_ld();
#pragma unroll
        for (int k = 0; k < 32; ++k)
          rt[k] = g == 0 ? rp[k] : __float_as_uint(__uint_as_float(rt[k]) + __uint_as_float(rp[k]));
        tc::tmem_st32(t_tot + lanebase + c0, rt);
      }
      tc::tmem_wait_st();
      tc::fence_before_sync();
      tc::mbar_arrive(&pfree);
    }
    // final: F = total
    if (ok && n_off > 0 && __all_sync(0xffffffffu, atomicAdd(&s_err, 0) == 0)) {
      const int m = q * 32 + lane;
      const int gm = mt * 128 + m;
      for (int c0 = 0; c0 < kNT; c0 += 32) {
        uint32_t rt[32];
        tc::tmem_ld32_nowait(t_tot + lanebase + c0, rt);
        tc::tmem_wait_ld();
        if (gm < 4 * P3) {
#pragma unroll
          for (int k = 0; k < 32; ++k) {
            const uint32_t t = par0 + c0 + k;
            if (t < n_par) F[(size_t)(8u * t + ctype) * 4 * P3 + gm] = __uint_as_float(rt[k]);
          }
        }
      }
    } else if (!ok) {
      atomicExch(&s_err, 1);
    }
  }
  tc::fence_before_sync();
  __syncthreads();
  if (warp == 0) tc::tmem_dealloc(tmem, kTmemCols);
  if (tid == 0 && s_err) atomicExch(err, 1);
}

// Plan time: the translation tiles A_o of every offset slot, row tile and
// stage, split into BF16 hi and lo, in the core-matrix layout the MMA reads:
// element (m, k) of a tile at byte ((k/8) 16 + m/8) 128 + (m%8) 16 + (k%8) 2.
// One thread per 16-byte core-matrix row.
template <int P>
__global__ void k_build_a(const uint4* __restrict__ tabbf, uint8_t* __restrict__ out) {
  constexpr int P3 = P * P * P, KP = ((P3 + kKC - 1) / kKC) * kKC, NCH = KP / kKC, MT = (4 * P3 + 127) / 128;
  constexpr int HW = 4 * P - 1, E = 8 * P - 1;
  const size_t rows = (size_t)kOffSlots * MT * NCH * 512;   // 512 core rows (128 m x 4 k8) per tile
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < rows; i += (size_t)gridDim.x * blockDim.x) {
    const int rowin = (int)(i % 512);
    const size_t tile = i / 512;                             // (oi, mt, ch)
    const int ch = (int)(tile % NCH);
    const int mt = (int)((tile / NCH) % MT);
    const int oi = (int)(tile / ((size_t)NCH * MT));
    const int ox = oi % 7 - 3, oy = (oi / 7) % 7 - 3, oz = oi / 49 - 3;
    const int m = rowin % 128, kc8 = rowin / 128;
    const int gm = mt * 128 + m;
    uint32_t h[4] = {0u, 0u, 0u, 0u}, l[4] = {0u, 0u, 0u, 0u};
    const bool far = ox < -1 || ox > 1 || oy < -1 || oy > 1 || oz < -1 || oz > 1;
    if (far && gm < 4 * P3) {
      const int f = gm / P3, r = gm % P3;
      const int rx = r % P, ry = (r / P) % P, rz = r / (P * P);
      for (int e = 0; e < 8; ++e) {
        const int s = ch * kKC + kc8 * 8 + e;
        uint32_t v = 0u;
        if (s < P3) {
          const int sx = s % P, sy = (s / P) % P, sz = s / (P * P);
          const int nx = ox * P + rx - sx + HW, ny = oy * P + ry - sy + HW, nz = oz * P + rz - sz + HW;
          const uint4 w = tabbf[((size_t)nz * E + ny) * E + nx];
          v = f == 0 ? w.x : (f == 1 ? w.y : (f == 2 ? w.z : w.w));
        }
        if (e & 1) {
          h[e / 2] |= v << 16;
          l[e / 2] |= v & 0xFFFF0000u;
        } else {
          h[e / 2] = v & 0xFFFFu;
          l[e / 2] = v >> 16;
        }
      }
    }
    const size_t base = tile * 2 * kTileBytes + (size_t)((kc8 * 16 + m / 8) * 128 + (m % 8) * 16);
    *reinterpret_cast<uint4*>(out + base) = make_uint4(h[0], h[1], h[2], h[3]);
    *reinterpret_cast<uint4*>(out + base + kTileBytes) = make_uint4(l[0], l[1], l[2], l[3]);
  }
}

template <int P, int MODE>
constexpr size_t smem_bytes() {
  return (size_t)TcShape<P, MODE>::SMEM;
}

template <int P, int MODE>
cudaError_t setup_one() {
  return cudaFuncSetAttribute(k_m2l_tc<P, MODE>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                              (int)smem_bytes<P, MODE>());
}

template <int P, int MODE>
cudaError_t launch_one(Plan& Pl, int level, cudaStream_t s) {
  const uint32_t n_par = 1u << (3 * (level - 1));
  // target tiles fastest: the CTAs in flight share row tile and child type,
  // hence their A tiles, which L2 then serves to all of them
  dim3 grid((n_par + kNT - 1) / kNT, TcShape<P, MODE>::MT, 8);
  const __nv_bfloat16* Msp = static_cast<const __nv_bfloat16*>(Pl.Mbf_hi[level]);
  const uint8_t* Apre = static_cast<const uint8_t*>(Pl.Apre[level]);
  k_m2l_tc<P, MODE><<<grid, kThreads, smem_bytes<P, MODE>(), s>>>(
      Msp, Apre, Pl.offsets[level], Pl.n_off[level], level, Pl.tc_group, Pl.F[level], Pl.d_err, Pl.wait_ns,
      Pl.inject_stall, Pl.iso);
  return cudaGetLastError();
}

template <int P>
cudaError_t setup_p() {
  cudaError_t e;
  if ((e = setup_one<P, 1>()) != cudaSuccess) return e;
  return setup_one<P, 3>();
}

template <int P>
cudaError_t launch_p(Plan& Pl, int level, int mode, cudaStream_t s) {
  if (mode == FMM_PREC_BF16X3) return launch_one<P, 3>(Pl, level, s);
  return launch_one<P, 1>(Pl, level, s);
}

template <int P>
cudaError_t build_a_p(Plan& Pl, int level, cudaStream_t s) {
  k_build_a<P><<<8 * Pl.num_sms, 256, 0, s>>>(Pl.tab_bf[level], static_cast<uint8_t*>(Pl.Apre[level]));
  return cudaGetLastError();
}

// Split FP32 gridlet masses into BF16 hi + lo, rows padded to KP with zeros,
// stored [node][KP/8][hi 8 | lo 8] so one stage slice of a node is contiguous.
__global__ void k_split_bf16(const float* __restrict__ M, int p3, int kp, size_t nodes, __nv_bfloat16* __restrict__ out) {
  const size_t total = nodes * kp;
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < total; i += (size_t)gridDim.x * blockDim.x) {
    const size_t node = i / kp;
    const int k = (int)(i % kp);
    const float x = k < p3 ? M[node * p3 + k] : 0.f;
    const __nv_bfloat16 h = __float2bfloat16_rn(x);
    const size_t o = (node * (kp / 8) + k / 8) * 16 + (k % 8);
    out[o] = h;
    out[o + 8] = __float2bfloat16_rn(x - __bfloat162float(h));
  }
}

}  // namespace

size_t tc_apre_bytes(int p) {
  const int p3 = p * p * p;
  const int kp = ((p3 + kKC - 1) / kKC) * kKC, nch = kp / kKC, mt = (4 * p3 + 127) / 128;
  return (size_t)kOffSlots * mt * nch * 2 * kTileBytes;
}

cudaError_t launch_build_a(Plan& P, int level, cudaStream_t s) {
  switch (P.p) {
    case 2: return build_a_p<2>(P, level, s);
    case 3: return build_a_p<3>(P, level, s);
    case 4: return build_a_p<4>(P, level, s);
    case 5: return build_a_p<5>(P, level, s);
    case 6: return build_a_p<6>(P, level, s);
    case 7: return build_a_p<7>(P, level, s);
    case 8: return build_a_p<8>(P, level, s);
    default: return cudaErrorInvalidValue;
  }
}

int tc_padded_k(int p) {
  const int p3 = p * p * p;
  return ((p3 + kKC - 1) / kKC) * kKC;
}

cudaError_t setup_m2l_tc(const Plan& P) {
  switch (P.p) {
    case 2: return setup_p<2>();
    case 3: return setup_p<3>();
    case 4: return setup_p<4>();
    case 5: return setup_p<5>();
    case 6: return setup_p<6>();
    case 7: return setup_p<7>();
    case 8: return setup_p<8>();
    default: return cudaSuccess;   // order 1 stays on CUDA cores
  }
}

cudaError_t launch_split_bf16(Plan& P, int level, cudaStream_t s) {
  const size_t nodes = (size_t)1 << (3 * level);
  const int p3 = P.p * P.p * P.p;
  k_split_bf16<<<4 * P.num_sms, 256, 0, s>>>(P.M[level], p3, tc_padded_k(P.p), nodes,
                                            static_cast<__nv_bfloat16*>(P.Mbf_hi[level]));
  return cudaGetLastError();
}

cudaError_t launch_m2l_tc(Plan& P, int level, int mode, cudaStream_t s) {
  switch (P.p) {
    case 2: return launch_p<2>(P, level, mode, s);
    case 3: return launch_p<3>(P, level, mode, s);
    case 4: return launch_p<4>(P, level, mode, s);
    case 5: return launch_p<5>(P, level, mode, s);
    case 6: return launch_p<6>(P, level, mode, s);
    case 7: return launch_p<7>(P, level, mode, s);
    case 8: return launch_p<8>(P, level, mode, s);
    default: return cudaErrorInvalidValue;
  }
}

}  // namespace fmm

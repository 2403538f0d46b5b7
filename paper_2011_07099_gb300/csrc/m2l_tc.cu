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
// memory tile layout (`k_build_a`); each pipeline stage streams its two 8 KB
// tiles with bulk asynchronous copies.
//
// The source operand B_o: a CTA's 256 targets of child type c are the
// children of an 8 x 8 x 4 box of parents, so the sources T - o of one offset
// all have the same parity class and form an 8 x 8 x 4 box in that class.
// The split multipoles are kept per parity class in spatial order with a
// 2-node halo (periodic copies, or zeros for the isolated problem), so each
// stage's B tile (256 targets x 32 reduction indices, per split) is ONE 5-D
// TMA tensor load, written in the 64-byte-swizzled K-major layout the MMA
// reads: whole lines from L2, no per-lane gathers.
//
// CTA tile: 128 rows of (f, r) x 256 targets (one M = 128, N = 256 MMA per
// 16-deep k step), or x 128 targets per the plan's tile for the level (an
// 8 x 4 x 4 box of parents; always in bf16x6).  Warp roles:
//   warp 0      issues the MMAs (one thread);
//   warp 1      one thread arms each stage's barrier with the stage's bytes
//               and issues its bulk copies (A) and tensor loads (B);
//   warps 2..5  drain TMEM (warps 2..9 in bf16x6): every G offsets
//               accumulate into a fresh TMEM partial, which the drain warps
//               add into an FP32 total kept in TMEM while the issuer waits.  A single TMEM accumulator over
//               all 189 p^3 terms drifts by ~1e-4 on the coherent, cancelling
//               far-field sums (the accumulation inside the MMA truncates);
//               per-group partials summed in FP32 with rounding to nearest
//               cost ~1e-7 (CPU emulation of the level's sums), far below the
//               bf16x3 operand error.
// A tiles: canonical no-swizzle K-major core matrices (8 rows x 16 B); B
// tiles: 64-byte swizzle, K-major.  bf16x3 mode accumulates A_hi B_hi +
// A_hi B_lo + A_lo B_hi; bf16 mode A_hi B_hi.
// TMEM: 512 columns = partial (256) | total (256).
// bf16x6 mode (the wide levels of high orders, whose local fields are FP64):
// A from the double-float table and B from the FP64 masses, each split in
// three BF16 parts; six products (hi hi, hi mid, mid hi, hi lo, mid mid,
// lo hi); 128 targets per CTA (an 8 x 4 x 4 box of parents); every stage
// accumulates into a fresh partial (two buffers, alternating), which the
// drain adds into a double-float total by TwoSum; the level's FP64 local
// field is written from hi + lo.  TMEM: partial 0 | partial 1 | hi | lo.
// (A partial over a whole group of offsets cost 2.8e-5 at order 8: the
// MMA's truncating accumulation, not the operand splits, dominated.)
// Every wait is bounded; a timeout sets the plan's error word and later work
// is skipped without leaving any barrier sequence.  Before the CTA exits the
// issuer waits (bounded) for the completion of every MMA it issued and the
// copy thread for every copy it issued, so nothing is still in flight into
// this CTA's TMEM or shared memory; then TMEM is freed and the kernel returns.
#include <cuda_bf16.h>
#include <cudaTypedefs.h>

#include <new>

#include "fmm_internal.cuh"
#include "tc_ptx.cuh"

namespace fmm {
namespace {

constexpr int kKC = 32;          // reduction indices per pipeline stage
constexpr int kBX = 8, kBZ = 4;  // the targets' parents: an 8 x BY x 4 box
constexpr int kHalo = 2;         // halo of the per-class source arrays (|(c - o - q)/2| <= 2)
constexpr int kDrainMax = 256;   // drain threads: warps 2..5 (2..9 in bf16x6)
constexpr uint32_t kTmemCols = 512;
constexpr int kTileBytes = 128 * kKC * 2;     // one 128 x 32 BF16 tile of A

// Modes: 1 = BF16 (A_hi B_hi), 3 = bf16x3 (hi hi + hi lo + lo hi); the
// wide mode of the FP64-field levels of high orders: 6 = bf16x6, both
// operands split in three BF16 parts and the six products s_i t_j with
// i + j <= 2, each stage's partial added into a double-float total (TMEM
// columns hi | lo) that is written as the level's FP64 local field.  (Four
// parts and ten products measured the same error at order 8, level 4: there
// the truncating accumulation inside each stage's MMAs, not the operands,
// limits; that level stays on the double-float CUDA-core kernel.)
// NTT: targets per CTA (MMA N), 256 or 128 (an 8 x 8 x 4 or 8 x 4 x 4 box of
// parents); the wide mode always takes 128 (TMEM room for the double-float
// total), the others 256 unless the plan's tile for the level says 128.
template <int MODE, int NTT = (MODE >= 6 ? 128 : 256)>
struct TcMode {
  static constexpr bool WIDE = MODE >= 6;
  static constexpr int NSPLIT = MODE == 6 ? 3 : (MODE == 3 ? 2 : 1);   // splits of each operand used
  static constexpr int ASPLIT = WIDE ? NSPLIT : 2;                     // A tiles stored per stage
  static constexpr int NT = NTT;                                       // targets per CTA (MMA N)
  static_assert(NT == 128 || NT == 256, "target tile");
  static_assert(!WIDE || NT == 128, "the wide mode's TMEM layout needs 128 targets");
  static constexpr int BY = NT / (kBX * kBZ);
  static constexpr int TILEB = NT * kKC * 2;                           // one NT x 32 BF16 tile of B
  // drain threads: bf16x6 adds a partial per stage into a double-float total,
  // so two warps share each TMEM lane quadrant, one half of the columns each
  static constexpr int DRAIN = WIDE ? 256 : 128;
  static constexpr int THREADS = 64 + DRAIN;
};

template <int P, int MODE, int NTT = TcMode<MODE>::NT>
struct TcShape {
  static constexpr int P3 = P * P * P;
  static constexpr int KP = ((P3 + kKC - 1) / kKC) * kKC;   // padded reduction length per offset
  static constexpr int NCH = KP / kKC;                       // stages per offset
  static constexpr int MT = (4 * P3 + 127) / 128;            // row tiles
  static constexpr int NSPLIT = TcMode<MODE, NTT>::NSPLIT;
  static constexpr int STAGE_BYTES = NSPLIT * (kTileBytes + TcMode<MODE, NTT>::TILEB);
  static constexpr int EXTRA = 64;
  static constexpr int LIMIT = 225 * 1024;                  // dynamic shared memory budget
  static constexpr int FIT = (LIMIT - EXTRA - 1024) / STAGE_BYTES;
  static constexpr int ST = FIT > 6 ? 6 : FIT;              // pipeline depth
  static_assert(FIT >= 3, "pipeline needs at least 3 stages");
  static constexpr int SMEM = ST * STAGE_BYTES + EXTRA + 1024;   // + alignment slack
};

// Offsets o with |o_i| <= 3 are indexed ((oz+3) 7 + (oy+3)) 7 + (ox+3).
__host__ __device__ constexpr int off_index(int ox, int oy, int oz) { return ((oz + 3) * 7 + (oy + 3)) * 7 + (ox + 3); }
constexpr int kOffSlots = 343;

template <int P, int MODE, int NTT>
__global__ void __launch_bounds__(64 + kDrainMax, 1)
k_m2l_tc(const __grid_constant__ CUtensorMap tmapB, const uint8_t* __restrict__ Apre,
         const int8_t* __restrict__ offs, int n_off, int level, int group,
         float* __restrict__ F, double* __restrict__ F64, int* __restrict__ err, uint64_t kWaitNs, int stall) {
  using Sh = TcShape<P, MODE, NTT>;
  using Md = TcMode<MODE, NTT>;
  constexpr int P3 = Sh::P3, NCH = Sh::NCH, MT = Sh::MT, ST = Sh::ST, NSPLIT = Sh::NSPLIT;
  constexpr int STAGE_BYTES = Sh::STAGE_BYTES;
  constexpr int kNT = Md::NT, kBY = Md::BY, kTileB = Md::TILEB, ASPLIT = Md::ASPLIT;
  static_assert(Sh::SMEM <= Sh::LIMIT, "shared-memory budget");
  static_assert(kBX * kBY * kBZ == kNT, "target box");
  constexpr uint32_t IDESC = tc::idesc_bf16_f32(128, kNT);
  constexpr uint32_t LBO_A = (128 / 8) * 128;      // next core matrix along K in an A tile
  constexpr uint32_t SBO_B = 8 * kKC * 2;          // 8 rows of 64 bytes in a B tile
  constexpr uint32_t TX = NSPLIT * (kTileBytes + kTileB);

  extern __shared__ uint8_t smem[];
  // full: the stage's copies landed (A bulk + B tensor, counted in bytes);
  // empty: the MMAs reading the stage are done; pfull / pfree: a unit's
  // partial is complete / has been added to the total.  A unit is a group of
  // `group` offsets (one partial buffer), or in bf16x6 one stage (two partial
  // buffers, alternating): the truncating accumulation inside the MMA then
  // spans only the stage's 12 products of 16 terms.
  constexpr int NB = Md::WIDE ? 2 : 1;
  __shared__ uint64_t full[ST], empty[ST], pfull[NB], pfree[NB], mdone;
  __shared__ uint32_t tmem_holder;
  __shared__ int s_err;

  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int mt = blockIdx.y, ctype = blockIdx.z;
  const int nh = 1 << (level - 1);                 // parents per dimension
  const int tiles_x = nh / kBX, tiles_y = nh / kBY;
  const int bx = (int)blockIdx.x % tiles_x, by = ((int)blockIdx.x / tiles_x) % tiles_y,
            bz = (int)blockIdx.x / (tiles_x * tiles_y);
  const int P0x = bx * kBX, P0y = by * kBY, P0z = bz * kBZ;     // the box of parents
  const int cx = ctype & 1, cy = (ctype >> 1) & 1, cz = ctype >> 2;
  const int8_t* my_offs = offs + (size_t)ctype * n_off * 3;
  const int n_units = Md::WIDE ? n_off * NCH : (n_off + group - 1) / group;
  // stages at a 1024-byte boundary (the swizzled B tiles need 512)
  const uint32_t smem_base = (tc::smem_u32(smem) + 1023u) & ~1023u;

  if (tid == 0) {
    s_err = 0;
    for (int i = 0; i < ST; ++i) {
      tc::mbar_init(&full[i], 1);              // the expect_tx arrival (+ the stage's bytes)
      tc::mbar_init(&empty[i], 1);             // one MMA completion
    }
    for (int b = 0; b < NB; ++b) {
      tc::mbar_init(&pfull[b], 1);
      tc::mbar_init(&pfree[b], Md::DRAIN);
    }
    tc::mbar_init(&mdone, 1);
    tc::mbar_fence_init();
  }
  if (warp == 0) tc::tmem_alloc(&tmem_holder, kTmemCols);
  tc::fence_before_sync();
  __syncthreads();
  tc::fence_after_sync();
  const uint32_t tmem = tmem_holder;
  // TMEM columns: partial buffer(s) | total; bf16x6: partial 0 | partial 1 | total hi | total lo
  const uint32_t t_tot = tmem + NB * kNT;
  const uint32_t t_lo = tmem + (NB + 1) * kNT;

  if (warp == 0) {
    // ------------------------------------------------------------ MMA issuer
    // (`stall` is a test hook: the issuer does nothing, so every dependent
    // bounded wait of this CTA expires and the error path runs)
    if (lane == 0) {
      bool ok = true;
      for (int io = 0; io < n_off && ok && !stall; ++io) {
        for (int ch = 0; ch < NCH; ++ch) {
          const int it = io * NCH + ch, st = it % ST;
          const int u = Md::WIDE ? it : io / group;                // the unit this stage adds to
          const bool first = Md::WIDE ? true : (io % group == 0 && ch == 0);
          const uint32_t part = tmem + (uint32_t)((u % NB) * kNT);
          // the partial buffer is reused: the drain must have added unit u - NB
          if (first && u >= NB && !tc::mbar_wait_bounded(&pfree[u % NB], (uint32_t)(u / NB - 1) & 1u, kWaitNs)) {
            ok = false;
            break;
          }
          if (!tc::mbar_wait_bounded(&full[st], (uint32_t)(it / ST) & 1u, kWaitNs)) {
            ok = false;
            break;
          }
          tc::fence_after_sync();
          const uint32_t sA = smem_base + st * STAGE_BYTES;
          const uint32_t sB = sA + NSPLIT * kTileBytes;
#pragma unroll
          for (int j = 0; j < kKC / 16; ++j) {
            if constexpr (Md::WIDE) {
              // the products s_a t_b with a + b < NSPLIT, largest first
#pragma unroll
              for (int d = 0; d < NSPLIT; ++d)
#pragma unroll
                for (int a = 0; a <= d; ++a) {
                  const uint64_t ad = tc::smem_desc(sA + a * kTileBytes + j * 2 * LBO_A, LBO_A, 128);
                  const uint64_t bd = tc::smem_desc_sw64(sB + (d - a) * kTileB + j * 32, SBO_B);
                  tc::mma_bf16(part, ad, bd, IDESC, (d == 0 && j == 0) ? 0u : 1u);
                }
            } else {
              const uint64_t ah = tc::smem_desc(sA + j * 2 * LBO_A, LBO_A, 128);
              const uint64_t bh = tc::smem_desc_sw64(sB + j * 32, SBO_B);
              tc::mma_bf16(part, ah, bh, IDESC, (!first || j > 0) ? 1u : 0u);
              if (MODE == 3) {
                const uint64_t al = tc::smem_desc(sA + kTileBytes + j * 2 * LBO_A, LBO_A, 128);
                const uint64_t bl = tc::smem_desc_sw64(sB + kTileB + j * 32, SBO_B);
                tc::mma_bf16(part, ah, bl, IDESC, 1u);
                tc::mma_bf16(part, al, bh, IDESC, 1u);
              }
            }
          }
          tc::mma_commit(&empty[st]);
          const bool last = Md::WIDE ? true : (ch == NCH - 1 && ((io % group) == group - 1 || io == n_off - 1));
          if (last) tc::mma_commit(&pfull[u % NB]);
        }
      }
      // every MMA this thread issued has finished before TMEM is released,
      // also when a wait gave up part-way
      tc::mma_commit(&mdone);
      if (!tc::mbar_wait_bounded(&mdone, 0u, kWaitNs)) ok = false;
      if (!ok || stall) atomicExch(&s_err, 1);
    }
    __syncwarp();
  } else if (warp == 1) {
    // ------------------------------------------------------- copy thread
    if (lane == 0) {
      bool ok = true;
      int armed = 0;             // stages whose copies were issued: iterations [0, armed)
      for (int io = 0; io < n_off && ok; ++io) {
        const int ox = my_offs[3 * io + 0], oy = my_offs[3 * io + 1], oz = my_offs[3 * io + 2];
        // sources T - o = 2 (P + d) + q: parity class q and class shift d
        const int qx = (cx - ox) & 1, qy = (cy - oy) & 1, qz = (cz - oz) & 1;
        const int dx = (cx - ox - qx) / 2, dy = (cy - oy - qy) / 2, dz = (cz - oz - qz) / 2;
        const int q = qx | (qy << 1) | (qz << 2);
        const uint8_t* atile = Apre + ((size_t)(off_index(ox, oy, oz) * MT + mt) * NCH) * ASPLIT * kTileBytes;
        for (int ch = 0; ch < NCH; ++ch) {
          const int it = io * NCH + ch, st = it % ST;
          if (!tc::mbar_wait_bounded(&empty[st], ((uint32_t)(it / ST) & 1u) ^ 1u, kWaitNs)) {
            ok = false;
            break;
          }
          const uint32_t sA = smem_base + st * STAGE_BYTES;
          const uint32_t sB = sA + NSPLIT * kTileBytes;
          tc::mbar_arrive_expect_tx(&full[st], TX);
          for (int sp = 0; sp < NSPLIT; ++sp)
            tc::bulk_g2s(sA + sp * kTileBytes, atile + ((size_t)ch * ASPLIT + sp) * kTileBytes, kTileBytes,
                         &full[st]);
          for (int sp = 0; sp < NSPLIT; ++sp)
            tc::tma_load_5d(sB + sp * kTileB, &tmapB, ch * kKC, P0x + dx + kHalo, P0y + dy + kHalo, P0z + dz + kHalo,
                            sp * 8 + q, &full[st]);
          armed = it + 1;
        }
      }
      // the copies issued last may not have been consumed (after a timeout):
      // wait (bounded) until each has landed, so no copy is in flight into
      // this CTA's shared memory when it exits
      for (int it = armed - ST > 0 ? armed - ST : 0; it < armed; ++it)
        if (!tc::mbar_wait_bounded(&full[it % ST], (uint32_t)(it / ST) & 1u, kWaitNs)) ok = false;
      if (!ok) atomicExch(&s_err, 1);
    }
    __syncwarp();
  } else {
    // ------------------------------------------------------------ drain warps
    const int q = warp & 3;                          // TMEM lane quadrant
    const uint32_t lanebase = (uint32_t)(q * 32) << 16;
    // columns of this warp: all, or (bf16x6) one half
    constexpr int CW = kNT * 128 / Md::DRAIN;
    const int cbeg = ((warp - 2) / 4) * CW, cend = cbeg + CW;
    bool ok = true;
    for (int g = 0; g < n_units; ++g) {
      const bool got = ok && tc::mbar_wait_bounded(&pfull[g % NB], (uint32_t)(g / NB) & 1u, kWaitNs);
      ok = __all_sync(0xffffffffu, got);
      if (!ok) break;
      tc::fence_after_sync();
      const uint32_t part = tmem + (uint32_t)((g % NB) * kNT);
      for (int c0 = cbeg; c0 < cend; c0 += 32) {
        uint32_t rp[32], rt[32], rl[32];
        tc::tmem_ld32_nowait(part + lanebase + c0, rp);
        if (g > 0) tc::tmem_ld32_nowait(t_tot + lanebase + c0, rt);
        if (Md::WIDE && g > 0) tc::tmem_ld32_nowait(t_lo + lanebase + c0, rl);
        tc::tmem_wait_ld();
        if (Md::WIDE) {
          // double-float total: (hi, lo) += partial by TwoSum, the error into lo
#pragma unroll
          for (int k = 0; k < 32; ++k) {
            if (g == 0) {
              rt[k] = rp[k];
              rl[k] = 0u;
            } else {
              const float2 t = df_two_sum(__uint_as_float(rt[k]), __uint_as_float(rp[k]));
              rt[k] = __float_as_uint(t.x);
              rl[k] = __float_as_uint(__fadd_rn(__uint_as_float(rl[k]), t.y));
            }
          }
          tc::tmem_st32(t_lo + lanebase + c0, rl);
        } else {
#pragma unroll
          for (int k = 0; k < 32; ++k)
            rt[k] = g == 0 ? rp[k] : __float_as_uint(__uint_as_float(rt[k]) + __uint_as_float(rp[k]));
        }
        tc::tmem_st32(t_tot + lanebase + c0, rt);
      }
      tc::tmem_wait_st();
      tc::fence_before_sync();
      tc::mbar_arrive(&pfree[g % NB]);
    }
    // final: F = total.  Target t of the tile is the child of parent
    // P0 + (t % 8, (t / 8) % 8, t / 64) at the CTA's child position.
    if (ok && n_off > 0 && __all_sync(0xffffffffu, atomicAdd(&s_err, 0) == 0)) {
      const int m = q * 32 + lane;
      const int gm = mt * 128 + m;
      for (int c0 = cbeg; c0 < cend; c0 += 32) {
        uint32_t rt[32], rl[32];
        tc::tmem_ld32_nowait(t_tot + lanebase + c0, rt);
        if (Md::WIDE) tc::tmem_ld32_nowait(t_lo + lanebase + c0, rl);
        tc::tmem_wait_ld();
        if (gm < 4 * P3) {
#pragma unroll
          for (int k = 0; k < 32; ++k) {
            const int t = c0 + k;
            const uint32_t tx = 2u * (uint32_t)(P0x + t % kBX) + cx, ty = 2u * (uint32_t)(P0y + (t / kBX) % kBY) + cy,
                           tz = 2u * (uint32_t)(P0z + t / (kBX * kBY)) + cz;
            const size_t o = (size_t)morton(tx, ty, tz) * 4 * P3 + gm;
            if (Md::WIDE)
              F64[o] = (double)__uint_as_float(rt[k]) + (double)__uint_as_float(rl[k]);
            else
              F[o] = __uint_as_float(rt[k]);
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

template <int P, int MODE, int NTT>
constexpr size_t smem_bytes() {
  return (size_t)TcShape<P, MODE, NTT>::SMEM;
}

template <int P, int MODE, int NTT = TcMode<MODE>::NT>
cudaError_t setup_one() {
  return cudaFuncSetAttribute(k_m2l_tc<P, MODE, NTT>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                              (int)smem_bytes<P, MODE, NTT>());
}

template <int P, int MODE, int NTT = TcMode<MODE>::NT>
cudaError_t launch_one(Plan& Pl, int level, cudaStream_t s) {
  const int nh = 1 << (level - 1);
  // target boxes fastest: the CTAs in flight share row tile and child type,
  // hence their A tiles, which L2 then serves to all of them
  dim3 grid((nh / kBX) * (nh / TcMode<MODE, NTT>::BY) * (nh / kBZ), TcShape<P, MODE, NTT>::MT, 8);
  const CUtensorMap* map = static_cast<const CUtensorMap*>(Pl.tmapB[level]);
  const uint8_t* Apre = static_cast<const uint8_t*>(Pl.Apre[level]);
  k_m2l_tc<P, MODE, NTT><<<grid, TcMode<MODE, NTT>::THREADS, smem_bytes<P, MODE, NTT>(), s>>>(
      *map, Apre, Pl.offsets[level], Pl.n_off[level], level, Pl.tc_group, Pl.F[level], Pl.F64[level], Pl.d_err,
      Pl.wait_ns, Pl.inject_stall);
  return cudaGetLastError();
}

template <int P>
cudaError_t setup_p() {
  cudaError_t e;
  if ((e = setup_one<P, 1>()) != cudaSuccess) return e;
  if ((e = setup_one<P, 1, 128>()) != cudaSuccess) return e;
  if ((e = setup_one<P, 3, 128>()) != cudaSuccess) return e;
  constexpr int PW = P >= kWideOrder ? P : kWideOrder;   // the wide modes exist at high orders only
  if (P >= kWideOrder && (e = setup_one<PW, 6>()) != cudaSuccess) return e;
  return setup_one<P, 3>();
}

template <int P>
cudaError_t launch_p(Plan& Pl, int level, int mode, cudaStream_t s) {
  if (tc_wide(Pl, level)) {
    constexpr int PW = P >= kWideOrder ? P : kWideOrder;
    if (P < kWideOrder) return cudaErrorInvalidValue;
    return launch_one<PW, 6>(Pl, level, s);
  }
  const bool t128 = tc_targets(Pl, level) == 128;
  if (mode == FMM_PREC_BF16X3) return t128 ? launch_one<P, 3, 128>(Pl, level, s) : launch_one<P, 3>(Pl, level, s);
  return t128 ? launch_one<P, 1, 128>(Pl, level, s) : launch_one<P, 1>(Pl, level, s);
}

// Plan time, wide levels: the translation tiles split in NS BF16 parts from
// the double-float table entries (G = tab + tab_lo, the wide levels keep
// both): s_0 = bf16(v), s_1 = bf16(v - s_0), ... (the differences in FP64),
// in the layout of k_build_a, NS tiles per stage.
template <int P, int NS>
__global__ void k_build_aw(const float4* __restrict__ tab, const float4* __restrict__ tab_lo,
                           uint8_t* __restrict__ out) {
  constexpr int P3 = P * P * P, KP = ((P3 + kKC - 1) / kKC) * kKC, NCH = KP / kKC, MT = (4 * P3 + 127) / 128;
  constexpr int HW = 4 * P - 1, E = 8 * P - 1;
  const size_t rows = (size_t)kOffSlots * MT * NCH * 512;
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < rows; i += (size_t)gridDim.x * blockDim.x) {
    const int rowin = (int)(i % 512);
    const size_t tile = i / 512;
    const int ch = (int)(tile % NCH);
    const int mt = (int)((tile / NCH) % MT);
    const int oi = (int)(tile / ((size_t)NCH * MT));
    const int ox = oi % 7 - 3, oy = (oi / 7) % 7 - 3, oz = oi / 49 - 3;
    const int m = rowin % 128, kc8 = rowin / 128;
    const int gm = mt * 128 + m;
    uint32_t w[NS][4] = {};
    const bool far = ox < -1 || ox > 1 || oy < -1 || oy > 1 || oz < -1 || oz > 1;
    if (far && gm < 4 * P3) {
      const int f = gm / P3, r = gm % P3;
      const int rx = r % P, ry = (r / P) % P, rz = r / (P * P);
      for (int e = 0; e < 8; ++e) {
        const int s = ch * kKC + kc8 * 8 + e;
        double v = 0.0;
        if (s < P3) {
          const int sx = s % P, sy = (s / P) % P, sz = s / (P * P);
          const int nx = ox * P + rx - sx + HW, ny = oy * P + ry - sy + HW, nz = oz * P + rz - sz + HW;
          const size_t t = ((size_t)nz * E + ny) * E + nx;
          const float4 a = tab[t], b = tab_lo[t];
          v = (double)(f == 0 ? a.x : (f == 1 ? a.y : (f == 2 ? a.z : a.w))) +
              (double)(f == 0 ? b.x : (f == 1 ? b.y : (f == 2 ? b.z : b.w)));
        }
        for (int sp = 0; sp < NS; ++sp) {
          const __nv_bfloat16 h = __float2bfloat16_rn((float)v);
          v -= (double)__bfloat162float(h);
          const uint32_t bits = (uint32_t)__bfloat16_as_ushort(h);
          w[sp][e / 2] |= (e & 1) ? bits << 16 : bits;
        }
      }
    }
    const size_t base = tile * NS * kTileBytes + (size_t)((kc8 * 16 + m / 8) * 128 + (m % 8) * 16);
    for (int sp = 0; sp < NS; ++sp)
      *reinterpret_cast<uint4*>(out + base + sp * kTileBytes) = make_uint4(w[sp][0], w[sp][1], w[sp][2], w[sp][3]);
  }
}

template <int P>
cudaError_t build_a_p(Plan& Pl, int level, cudaStream_t s) {
  if (tc_wide(Pl, level))
    k_build_aw<P, 3><<<8 * Pl.num_sms, 256, 0, s>>>(Pl.tab[level], Pl.tab_lo[level], static_cast<uint8_t*>(Pl.Apre[level]));
  else
    k_build_a<P><<<8 * Pl.num_sms, 256, 0, s>>>(Pl.tab_bf[level], static_cast<uint8_t*>(Pl.Apre[level]));
  return cudaGetLastError();
}

// Split FP32 gridlet masses into BF16 hi + lo in the layout the tensor loads
// read: [split][class q][z + halo][y + halo][x + halo][KP], q the node's
// parity class ((x & 1) | (y & 1) << 1 | (z & 1) << 2) and (x, y, z) its
// coordinates within the class (halved); the halo holds the periodic copies,
// or zeros for the isolated problem; rows padded to KP with zeros.
__global__ void k_split_bf16(const float* __restrict__ M, const double* __restrict__ M64, int nsplit, int p3, int kp,
                             int level, int iso, __nv_bfloat16* __restrict__ out) {
  const int nh = 1 << (level - 1), W = nh + 2 * kHalo;
  const size_t row = (size_t)kp, cls = (size_t)W * W * W * row, total = 8 * cls;
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < total; i += (size_t)gridDim.x * blockDim.x) {
    const int k = (int)(i % row);
    const size_t cell = i / row;
    const int xw = (int)(cell % W), yw = (int)((cell / W) % W), zw = (int)((cell / ((size_t)W * W)) % W);
    const int q = (int)(cell / ((size_t)W * W * W));
    int ux = xw - kHalo, uy = yw - kHalo, uz = zw - kHalo;
    const bool inbox = (unsigned)ux < (unsigned)nh && (unsigned)uy < (unsigned)nh && (unsigned)uz < (unsigned)nh;
    double x = 0.0;
    if (k < p3 && (inbox || !iso)) {
      ux = (ux + nh) % nh;
      uy = (uy + nh) % nh;
      uz = (uz + nh) % nh;
      const uint32_t key = morton(2u * ux + (q & 1), 2u * uy + ((q >> 1) & 1), 2u * uz + (q >> 2));
      x = M64 ? M64[(size_t)key * p3 + k] : (double)M[(size_t)key * p3 + k];
    }
    // two splits (hi, lo) from FP32 masses, or three (hi, mid, lo) from the
    // FP64 masses of a wide level
    for (int sp = 0; sp < nsplit; ++sp) {
      const __nv_bfloat16 h = __float2bfloat16_rn((float)x);
      out[sp * total + i] = h;
      x -= (double)__bfloat162float(h);
    }
  }
}

}  // namespace

size_t tc_apre_bytes(int p, int nsplit) {
  const int p3 = p * p * p;
  const int kp = ((p3 + kKC - 1) / kKC) * kKC, nch = kp / kKC, mt = (4 * p3 + 127) / 128;
  return (size_t)kOffSlots * mt * nch * nsplit * kTileBytes;
}

size_t tc_bsplit_bytes(int p, int level, int nsplit) {
  const size_t W = (size_t)(1 << (level - 1)) + 2 * kHalo;
  return (size_t)nsplit * 8 * W * W * W * (size_t)tc_padded_k(p) * sizeof(__nv_bfloat16);
}

// The 5-D tensor map of a level's split multipoles: dims (KP, W, W, W,
// 8 x splits = split x class), box (32, 8, BY, 4, 1) (BY = 8, or 4 for the
// 128-target tiles of bf16x6), 64-byte swizzle.
int make_tc_map(Plan& P, int level) {
  static PFN_cuTensorMapEncodeTiled_v12000 encode = nullptr;
  if (!encode) {
    cudaDriverEntryPointQueryResult q;
    void* fn = nullptr;
    if (cudaGetDriverEntryPoint("cuTensorMapEncodeTiled", &fn, cudaEnableDefault, &q) != cudaSuccess ||
        q != cudaDriverEntryPointSuccess || !fn)
      return FMM_ERR_CUDA;
    encode = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(fn);
  }
  if (!P.tmapB[level]) P.tmapB[level] = new (std::nothrow) CUtensorMap;
  if (!P.tmapB[level]) return FMM_ERR_ALLOC;
  const cuuint64_t kp = (cuuint64_t)tc_padded_k(P.p), W = (cuuint64_t)(1 << (level - 1)) + 2 * kHalo;
  const cuuint64_t dims[5] = {kp, W, W, W, (cuuint64_t)(8 * tc_splits(P, level))};
  const cuuint64_t strides[4] = {kp * 2, kp * 2 * W, kp * 2 * W * W, kp * 2 * W * W * W};
  const cuuint32_t box[5] = {(cuuint32_t)kKC, (cuuint32_t)kBX, (cuuint32_t)(tc_targets(P, level) / (kBX * kBZ)),
                             (cuuint32_t)kBZ, 1};
  const cuuint32_t estr[5] = {1, 1, 1, 1, 1};
  const CUresult r = encode(static_cast<CUtensorMap*>(P.tmapB[level]), CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 5,
                            P.Mbf_hi[level], dims, strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
                            CU_TENSOR_MAP_SWIZZLE_64B, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
                            CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  return r == CUDA_SUCCESS ? FMM_OK : FMM_ERR_CUDA;
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
  const int p3 = P.p * P.p * P.p;
  k_split_bf16<<<8 * P.num_sms, 256, 0, s>>>(P.M[level], tc_wide(P, level) ? P.M64[level] : nullptr,
                                            tc_splits(P, level), p3, tc_padded_k(P.p), level, P.iso,
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

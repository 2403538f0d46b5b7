// The C-ABI of libfmm: plan lifecycle, solve orchestration and errors.
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <new>
#include <set>
#include <tuple>
#include <vector>

#include <cuda.h>

#include "fmm_internal.cuh"
#include "mlp.cuh"

using fmm::Plan;

namespace {

thread_local int g_last_error = FMM_OK;

int set_err(int code) {
  g_last_error = code;
  return code;
}

bool aligned16(const void* p) { return (reinterpret_cast<uintptr_t>(p) & 15u) == 0; }

#define FMM_CUDA_TRY(expr)                  \
  do {                                      \
    cudaError_t _e = (expr);                \
    if (_e != cudaSuccess) {                \
      return set_err(FMM_ERR_CUDA);         \
    }                                       \
  } while (0)

// 1-D Lagrange basis on the gridlet points X_j = (j + 1/2)/p (node-size units)
// evaluated at the K cell-centred points y_k = (k + 1/2)/K: w[s][k] = l_s(y_k).
// This is the separable solution of the Sec. 2 Vandermonde system (the
// gridlet masses that keep every multipole Q_n, n_i < p).  Computed in double.
std::vector<double> lagrange_weights(int p, int K) {
  std::vector<double> w((size_t)p * K);
  for (int s = 0; s < p; ++s) {
    const double xs = (s + 0.5) / p;
    for (int k = 0; k < K; ++k) {
      const double y = (k + 0.5) / K;
      double v = 1.0;
      for (int j = 0; j < p; ++j) {
        if (j == s) continue;
        const double xj = (j + 0.5) / p;
        v *= (y - xj) / (xs - xj);
      }
      w[(size_t)s * K + k] = v;
    }
  }
  return w;
}

// Interaction-zone offsets o = T - S (node units, nearest periodic image) for
// the node whose position in its parent is c = cx | cy << 1 | cz << 2: the
// children of the parent's periodic neighbours minus the node's own periodic
// neighbours (Sec. 2, Fig. fmm).  Under periodic wrap every node with the same
// position in its parent has the translated list, so one list per child type.
std::vector<int8_t> interaction_offsets(int level, int c) {
  const int n = 1 << level, np = n >> 1;
  auto wrapn = [](int v, int m) { return ((v % m) + m) % m; };
  const int tx = c & 1, ty = (c >> 1) & 1, tz = (c >> 2) & 1;   // parent is (0,0,0)
  std::set<std::tuple<int, int, int>> kids, near;
  for (int a = -1; a <= 1; ++a)
    for (int b = -1; b <= 1; ++b)
      for (int d = -1; d <= 1; ++d) {
        const int qx = wrapn(a, np), qy = wrapn(b, np), qz = wrapn(d, np);
        for (int i = 0; i < 8; ++i)
          kids.insert(std::make_tuple(2 * qx + (i & 1), 2 * qy + ((i >> 1) & 1), 2 * qz + (i >> 2)));
        near.insert(std::make_tuple(wrapn(tx + a, n), wrapn(ty + b, n), wrapn(tz + d, n)));
      }
  std::vector<int8_t> out;
  for (const auto& k : kids) {
    if (near.count(k)) continue;
    int o[3] = {tx - std::get<0>(k), ty - std::get<1>(k), tz - std::get<2>(k)};
    for (int& v : o) {
      v = wrapn(v, n);
      if (v > n / 2) v -= n;          // nearest image; +n/2 kept (G_S1 is 1-periodic)
    }
    out.push_back((int8_t)o[0]);
    out.push_back((int8_t)o[1]);
    out.push_back((int8_t)o[2]);
  }
  return out;
}

// Offsets of the isolated problem's interaction zones at level 2 (Sec. 3's
// non-periodic reference, Sec. 2 zones without the wrap): the parent level 1
// has 2 nodes per dimension, all neighbours of each other, so a level-2
// node's zone is every in-box node that is not its neighbour; as offsets
// o = T - S, every o in [-3, 3]^3 with max |o_i| >= 2 (316), the in-box test
// being done by the kernels.  Levels >= 3 use the periodic lists: a periodic
// list restricted to in-box sources is the isolated list there.
std::vector<int8_t> isolated_level2_offsets() {
  std::vector<int8_t> out;
  for (int z = -3; z <= 3; ++z)
    for (int y = -3; y <= 3; ++y)
      for (int x = -3; x <= 3; ++x) {
        const int m = std::max(std::abs(x), std::max(std::abs(y), std::abs(z)));
        if (m < 2) continue;
        out.push_back((int8_t)x);
        out.push_back((int8_t)y);
        out.push_back((int8_t)z);
      }
  return out;
}

void free_plan(Plan* P) {
  if (!P) return;
  cudaFree(P->d_partials);
  cudaFree(P->m2l_part);
  cudaFree(P->d_mean);
  for (int l = 0; l <= fmm::kMaxLevel; ++l) {
    cudaFree(P->M[l]);
    cudaFree(P->F[l]);
    cudaFree(P->tab[l]);
    cudaFree(P->tab_lo[l]);
    cudaFree(P->F64[l]);
    cudaFree(P->M64[l]);
    cudaFree(P->offsets[l]);
  }
  cudaFree(P->near_tab);
  cudaFree(P->nz_K);
  cudaFree(P->nz_M);
  cudaFree(P->nz_P);
  cudaFree(P->d_err);
  cudaFree(P->corr_w);
  cudaFree(P->train_out);
  cudaFree(P->lam_cells);
  cudaFree(P->dT_all);
  cudaFree(P->grad_partials);
  cudaFree(P->grid);
  cudaFree(P->gmesh);
  fmm::free_fft(*P);
  for (int l = 0; l <= fmm::kMaxLevel; ++l) cudaFree(P->lam[l]);
  for (int l = 0; l <= fmm::kMaxLevel; ++l) {
    cudaFree(P->tab_bf[l]);
    cudaFree(P->Mbf_hi[l]);
    cudaFree(P->Apre[l]);
    delete static_cast<CUtensorMap*>(P->tmapB[l]);
  }
  cudaFree(P->w_p2m);
  cudaFree(P->w_m2m);
  cudaFree(P->stage_in);
  cudaFree(P->stage_out);
  for (auto& e : P->ev)
    if (e) cudaEventDestroy(e);
  for (auto& e : P->fev)
    if (e) cudaEventDestroy(e);
  for (auto& a : P->aux)
    if (a) cudaStreamDestroy(a);
  delete P;
}

template <typename T>
bool dev_alloc(T** ptr, size_t count) {
  return cudaMalloc(reinterpret_cast<void**>(ptr), sizeof(T) * count) == cudaSuccess;
}

// Re-tabulate every table form from G_S1 plus the plan's corrections (MLP,
// grid), synchronously.  Returns an FMM_* code.
int retabulate(Plan& P) {
  if (fmm::launch_tables(P, 0) != cudaSuccess) return FMM_ERR_CUDA;
  if (P.fft) {   // the FFT form keeps the tables' spectra: rebuild them
    fmm::free_fft(P);
    if (P.m2l_fft) {
      if (cudaDeviceSynchronize() != cudaSuccess) return FMM_ERR_CUDA;
      const int rc = fmm::prepare_fft(P);
      if (rc != FMM_OK) return rc;
    }
  }
  if (P.near_fft && fmm::launch_near_fft_kernels(P, 0) != cudaSuccess) return FMM_ERR_CUDA;
  if (P.tc_ready) {
    for (int l = fmm::kTcMinLevel; l <= P.L; ++l) {
      if (!P.Apre[l]) continue;
      if ((!fmm::tc_wide(P, l) && fmm::launch_tab_bf16(P, l, 0) != cudaSuccess) ||
          fmm::launch_build_a(P, l, 0) != cudaSuccess)
        return FMM_ERR_CUDA;
    }
  }
  return cudaDeviceSynchronize() == cudaSuccess ? FMM_OK : FMM_ERR_CUDA;
}

// Training buffers (first use) and one forward solve, cell residual and
// adjoint sweep down to the table gradients P.dT of every level; the loss is
// added to `loss`.  Returns an FMM_* code.
int table_gradient(Plan& P, const float* density, const float* target_phi, const float* target_acc, float w_phi,
                   float w_g, float* loss, void* stream) {
  const size_t n3 = (size_t)P.N * P.N * P.N;
  const size_t p3 = (size_t)P.p * P.p * P.p, E = 8 * P.p - 1;
  if (!P.train_out) {
    bool ok = dev_alloc(&P.train_out, 4 * n3) && dev_alloc(&P.lam_cells, 4 * n3) &&
              dev_alloc(&P.dT_all, (size_t)(P.L - 1) * E * E * E * 4) &&
              dev_alloc(&P.grad_partials, (size_t)fmm::mlp_backward_blocks(P) * fmm::mlp::kParams);
    for (int l = 2; l <= P.L && ok; ++l) ok = dev_alloc(&P.lam[l], ((size_t)1 << (3 * l)) * 4 * p3);
    if (!ok) return FMM_ERR_ALLOC;
    for (int l = 2; l <= P.L; ++l) P.dT[l] = P.dT_all + (size_t)(l - 2) * E * E * E * 4;
  }
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  const int rc = fmm_solve(reinterpret_cast<fmm_plan*>(&P), density, P.train_out, P.train_out + n3, stream);
  if (rc != FMM_OK) return rc;
  if (fmm::launch_residual(P.train_out, P.train_out + n3, target_phi, target_acc, n3, w_phi, w_g, P.lam_cells, loss,
                           P.num_sms, s) != cudaSuccess ||
      fmm::launch_adjoint_and_table_grad(P, P.lam_cells, s) != cudaSuccess)
    return FMM_ERR_CUDA;
  return FMM_OK;
}

}  // namespace

int fmm::set_last_error(int code) { return set_err(code); }

extern "C" {

int fmm_last_error(void) { return g_last_error; }

const char* fmm_error_string(int code) {
  switch (code) {
    case FMM_OK: return "ok";
    case FMM_ERR_ARG: return "invalid argument";
    case FMM_ERR_CUDA: return "CUDA runtime error";
    case FMM_ERR_TIMEOUT: return "bounded device wait timed out";
    case FMM_ERR_INTERNAL: return "internal consistency check failed";
    case FMM_ERR_ALLOC: return "allocation failed";
    case FMM_ERR_UNSUPPORTED: return "unsupported by this build";
    default: return "unknown error code";
  }
}

fmm_plan* fmm_plan_create(int N, int L, int order) {
  if (L < 2 || L > fmm::kMaxLevel || order < 1 || order > fmm::kMaxOrder || N <= 0) {
    set_err(FMM_ERR_ARG);
    return nullptr;
  }
  const int n = 1 << L;
  if (N % n != 0) {
    set_err(FMM_ERR_ARG);
    return nullptr;
  }
  const int S = N / n;
  if (S != 1 && S != 2 && S != 3 && S != 4 && S != 6 && S != 8 && S != 16) {
    set_err(FMM_ERR_ARG);
    return nullptr;
  }
  Plan* P = new (std::nothrow) Plan();
  if (!P) {
    set_err(FMM_ERR_ALLOC);
    return nullptr;
  }
  P->N = N;
  P->L = L;
  P->p = order;
  P->S = S;
  if (cudaGetDevice(&P->device) != cudaSuccess ||
      cudaDeviceGetAttribute(&P->num_sms, cudaDevAttrMultiProcessorCount, P->device) != cudaSuccess) {
    delete P;
    set_err(FMM_ERR_CUDA);
    return nullptr;
  }
  const int p = order, p3 = p * p * p;
  bool ok = true;
  for (auto& a : P->aux) ok = ok && cudaStreamCreateWithFlags(&a, cudaStreamNonBlocking) == cudaSuccess;
  for (auto& e : P->fev) ok = ok && cudaEventCreateWithFlags(&e, cudaEventDisableTiming) == cudaSuccess;
  if (!ok) {
    free_plan(P);
    set_err(FMM_ERR_CUDA);
    return nullptr;
  }
  P->n_partials = 4 * P->num_sms;
  ok = ok && dev_alloc(&P->d_partials, P->n_partials) && dev_alloc(&P->d_mean, 1) && dev_alloc(&P->d_err, 1) &&
       cudaMemset(P->d_err, 0, sizeof(int)) == cudaSuccess;
  for (int l = 2; l <= L && ok; ++l) {
    const size_t nodes = (size_t)1 << (3 * l);
    const size_t E = 8 * p - 1;
    ok = dev_alloc(&P->M[l], nodes * p3) && dev_alloc(&P->F[l], nodes * 4 * p3) &&
         dev_alloc(&P->tab[l], E * E * E);
    // split tables for the coarse levels, and for every wide level of the high orders
    if (ok && (l <= fmm::kExtTopLevel || (p >= fmm::kWideOrder && l < L) || S >= fmm::kWideLeaf))
      ok = dev_alloc(&P->tab_lo[l], E * E * E);
    // FP64 gridlet masses at every level at high order (the leaf copy feeds M2M:
    // the coarse far-field sums cancel ~1000-fold there, so FP32 rounding of
    // the leaf masses alone would cost ~1e-6)
    if (ok && p >= fmm::kWideOrder) ok = dev_alloc(&P->M64[l], nodes * p3);
  }
  ok = ok && dev_alloc(&P->near_tab, (size_t)8 * S * S * S) && dev_alloc(&P->w_p2m, (size_t)p * S) &&
       dev_alloc(&P->w_m2m, (size_t)p * 2 * p);
  if (!ok) {
    free_plan(P);
    set_err(FMM_ERR_ALLOC);
    return nullptr;
  }
  // host-side constants: Lagrange weights and interaction lists
  // Lagrange weights in FP64 on the host, stored as (hi, lo) FP32 pairs
  std::vector<double> wp = lagrange_weights(p, S), wm = lagrange_weights(p, 2 * p);
  auto split = [](const std::vector<double>& v) {
    std::vector<float2> o(v.size());
    for (size_t i = 0; i < v.size(); ++i) {
      const float hi = (float)v[i];
      o[i] = make_float2(hi, (float)(v[i] - (double)hi));
    }
    return o;
  };
  std::vector<float2> wp2 = split(wp), wm2 = split(wm);
  bool cok = cudaMemcpy(P->w_p2m, wp2.data(), wp2.size() * sizeof(float2), cudaMemcpyHostToDevice) == cudaSuccess &&
             cudaMemcpy(P->w_m2m, wm2.data(), wm2.size() * sizeof(float2), cudaMemcpyHostToDevice) == cudaSuccess;
  for (int l = 2; l <= L && cok; ++l) {
    std::vector<int8_t> all;
    int count = -1;
    for (int c = 0; c < 8; ++c) {
      std::vector<int8_t> o = interaction_offsets(l, c);
      const int k = (int)o.size() / 3;
      if (count >= 0 && k != count) cok = false;
      count = k;
      all.insert(all.end(), o.begin(), o.end());
    }
    P->n_off[l] = count;
    cok = cok && (l == 2 ? count == 37 : count == 189);
    cok = cok && dev_alloc(&P->offsets[l], all.size()) &&
          cudaMemcpy(P->offsets[l], all.data(), all.size(), cudaMemcpyHostToDevice) == cudaSuccess;
  }
  if (!cok) {
    free_plan(P);
    set_err(FMM_ERR_INTERNAL);
    return nullptr;
  }
  {
    // scratch for the offset-range partials of the coarse FP32 M2L levels
    size_t part = 0;
    for (int l = 2; l <= L; ++l) {
      if (!fmm::wide_level(*P, l)) continue;
      const int ns = fmm::m2l_fp32_splits(*P, l);
      const size_t need = 2 * (size_t)ns * ((size_t)1 << (3 * l)) * 4 * p3;
      if (need > part) part = need;
      if (!dev_alloc(&P->F64[l], ((size_t)1 << (3 * l)) * 4 * p3)) part = 0;
    }
    if (!part || !dev_alloc(&P->m2l_part, part)) {
      free_plan(P);
      set_err(FMM_ERR_ALLOC);
      return nullptr;
    }
  }
  if (fmm::setup_upward(*P) != cudaSuccess || fmm::setup_m2l_fp32(*P) != cudaSuccess ||
      fmm::setup_m2l_tc(*P) != cudaSuccess || fmm::setup_learn() != cudaSuccess ||
      fmm::setup_downward(*P) != cudaSuccess || fmm::setup_p2p(*P) != cudaSuccess ||
      fmm::launch_tables(*P, 0) != cudaSuccess || cudaDeviceSynchronize() != cudaSuccess) {
    free_plan(P);
    set_err(FMM_ERR_CUDA);
    return nullptr;
  }
  set_err(FMM_OK);
  return reinterpret_cast<fmm_plan*>(P);
}

void fmm_plan_destroy(fmm_plan* plan) {
  if (!plan) return;
  cudaDeviceSynchronize();
  free_plan(reinterpret_cast<Plan*>(plan));
}

int fmm_plan_get_shape(const fmm_plan* plan, int* N, int* L, int* order, int* S) {
  if (!plan) return set_err(FMM_ERR_ARG);
  const Plan* P = reinterpret_cast<const Plan*>(plan);
  if (N) *N = P->N;
  if (L) *L = P->L;
  if (order) *order = P->p;
  if (S) *S = P->S;
  return set_err(FMM_OK);
}

namespace {
// Tensor-core M2L buffers: split tables, split multipoles and the translation
// tiles of every level from the first tensor-core level down to the leaves
// (levels that already have them are kept).  Tabulated once, synchronously.
int prepare_tc(Plan& P) {
  const size_t E = 8 * P.p - 1;
  bool made = false;
  for (int l = fmm::tc_first_level(P); l <= P.L; ++l) {
    if (P.Apre[l]) continue;
    const bool wide = fmm::tc_wide(P, l);   // wide modes: tiles from tab + tab_lo, no BF16 table
    if ((!wide && !P.tab_bf[l] && !dev_alloc(&P.tab_bf[l], E * E * E)) ||
        (!P.Mbf_hi[l] && cudaMalloc(&P.Mbf_hi[l], fmm::tc_bsplit_bytes(P.p, l, fmm::tc_splits(P, l))) != cudaSuccess) ||
        cudaMalloc(&P.Apre[l], fmm::tc_apre_bytes(P.p, fmm::tc_splits(P, l))) != cudaSuccess)
      return FMM_ERR_ALLOC;
    if ((!wide && fmm::launch_tab_bf16(P, l, 0) != cudaSuccess) || fmm::launch_build_a(P, l, 0) != cudaSuccess)
      return FMM_ERR_CUDA;
    const int rc = fmm::make_tc_map(P, l);
    if (rc != FMM_OK) return rc;
    made = true;
  }
  if (made && cudaDeviceSynchronize() != cudaSuccess) return FMM_ERR_CUDA;
  P.tc_ready = 1;
  return FMM_OK;
}
}  // namespace

int fmm_plan_set_precision(fmm_plan* plan, int mode) {
  if (!plan) return set_err(FMM_ERR_ARG);
  if (mode != FMM_PREC_FP32 && mode != FMM_PREC_BF16 && mode != FMM_PREC_BF16X3) return set_err(FMM_ERR_ARG);
  Plan& P = *reinterpret_cast<Plan*>(plan);
  if (mode != FMM_PREC_FP32 && P.p >= 2) {
    const int rc = prepare_tc(P);
    if (rc != FMM_OK) return set_err(rc);
  }
  P.prec = mode;
  return set_err(FMM_OK);
}

int fmm_plan_set_boundary(fmm_plan* plan, int boundary) {
  if (!plan || (boundary != FMM_BOUNDARY_PERIODIC && boundary != FMM_BOUNDARY_ISOLATED)) return set_err(FMM_ERR_ARG);
  Plan& P = *reinterpret_cast<Plan*>(plan);
  const int iso = boundary == FMM_BOUNDARY_ISOLATED ? 1 : 0;
  if (iso == P.iso) return set_err(FMM_OK);
  FMM_CUDA_TRY(cudaDeviceSynchronize());
  // level-2 interaction lists: 37 periodic nodes, or the 316 in-box offsets
  std::vector<int8_t> all;
  int count = 0;
  for (int c = 0; c < 8; ++c) {
    std::vector<int8_t> o = iso ? isolated_level2_offsets() : interaction_offsets(2, c);
    count = (int)o.size() / 3;
    all.insert(all.end(), o.begin(), o.end());
  }
  int8_t* offs = nullptr;
  if (!dev_alloc(&offs, all.size())) return set_err(FMM_ERR_ALLOC);
  if (cudaMemcpy(offs, all.data(), all.size(), cudaMemcpyHostToDevice) != cudaSuccess) {
    cudaFree(offs);
    return set_err(FMM_ERR_CUDA);
  }
  cudaFree(P.offsets[2]);
  P.offsets[2] = offs;
  P.n_off[2] = count;
  P.iso = iso;
  // the offset-range scratch of the coarse levels follows the list length
  size_t part = 0;
  const size_t p3 = (size_t)P.p * P.p * P.p;
  for (int l = 2; l <= P.L; ++l)
    if (fmm::wide_level(P, l)) {
      const size_t need = 2 * (size_t)fmm::m2l_fp32_splits(P, l) * ((size_t)1 << (3 * l)) * 4 * p3;
      if (need > part) part = need;
    }
  cudaFree(P.m2l_part);
  P.m2l_part = nullptr;
  if (!dev_alloc(&P.m2l_part, part)) return set_err(FMM_ERR_ALLOC);
  return set_err(retabulate(P));
}

int fmm_plan_set_green(fmm_plan* plan, int kind, const double* a, int na) {
  if (!plan || (kind != FMM_GREEN_S1 && kind != FMM_GREEN_S && kind != FMM_GREEN_X)) return set_err(FMM_ERR_ARG);
  if (kind == FMM_GREEN_S && (na < 1 || na > fmm::green::kMaxAnsatz || !a)) return set_err(FMM_ERR_ARG);
  Plan& P = *reinterpret_cast<Plan*>(plan);
  fmm::green::Spec g;
  g.kind = kind == FMM_GREEN_S ? 1 : (kind == FMM_GREEN_X ? 3 : 0);
  g.na = kind == FMM_GREEN_S ? na : 0;
  for (int k = 0; k < g.na; ++k) g.a[k] = a[k];
  P.gspec = g;
  return set_err(retabulate(P));
}

int fmm_plan_set_green_mesh(fmm_plan* plan, const double* mesh, size_t n) {
  if (!plan || !mesh) return set_err(FMM_ERR_ARG);
  Plan& P = *reinterpret_cast<Plan*>(plan);
  const size_t n3 = (size_t)P.N * P.N * P.N;
  // every gridlet point of every level must sit on a mesh cell centre
  if (n != 4 * n3 || P.S % P.p != 0) return set_err(FMM_ERR_ARG);
  if (!P.gmesh && !dev_alloc(&P.gmesh, 4 * n3)) return set_err(FMM_ERR_ALLOC);
  FMM_CUDA_TRY(cudaMemcpy(P.gmesh, mesh, sizeof(double) * 4 * n3, cudaMemcpyDefault));
  fmm::green::Spec g;
  g.kind = 4;
  P.gspec = g;
  return set_err(retabulate(P));
}

int fmm_plan_set_m2l_algorithm(fmm_plan* plan, int algorithm) {
  if (!plan || (algorithm != FMM_M2L_DENSE && algorithm != FMM_M2L_FFT)) return set_err(FMM_ERR_ARG);
  Plan& P = *reinterpret_cast<Plan*>(plan);
  P.m2l_fft = algorithm == FMM_M2L_FFT ? 1 : 0;
  if (P.m2l_fft) {
    const int rc = fmm::prepare_fft(P);
    if (rc != FMM_OK) {
      fmm::free_fft(P);
      P.m2l_fft = 0;
      return set_err(rc);
    }
  }
  return set_err(FMM_OK);
}

int fmm_plan_set_near_algorithm(fmm_plan* plan, int algorithm) {
  if (!plan || (algorithm != FMM_NEAR_DIRECT && algorithm != FMM_NEAR_FFT)) return set_err(FMM_ERR_ARG);
  Plan& P = *reinterpret_cast<Plan*>(plan);
  if (algorithm == FMM_NEAR_DIRECT) {
    if (cudaDeviceSynchronize() != cudaSuccess) return set_err(FMM_ERR_CUDA);
    cudaFree(P.nz_K);
    cudaFree(P.nz_M);
    cudaFree(P.nz_P);
    P.nz_K = P.nz_M = P.nz_P = nullptr;
    P.near_fft = 0;
    return set_err(FMM_OK);
  }
  if (!fmm::near_fft_supported(P)) return set_err(FMM_ERR_UNSUPPORTED);
  if (!P.nz_K) {
    size_t nK, nM, nP;
    fmm::near_fft_counts(P, nK, nM, nP);
    if (!dev_alloc(&P.nz_K, nK) || !dev_alloc(&P.nz_M, nM) || !dev_alloc(&P.nz_P, nP)) {
      cudaFree(P.nz_K);
      cudaFree(P.nz_M);
      cudaFree(P.nz_P);
      P.nz_K = P.nz_M = P.nz_P = nullptr;
      return set_err(FMM_ERR_ALLOC);
    }
    // the all-zero spectrum of out-of-box neighbours sits after each chunk's leaves
    FMM_CUDA_TRY(cudaMemset(P.nz_M, 0, sizeof(float2) * nM));
  }
  P.near_fft = 1;
  FMM_CUDA_TRY(fmm::launch_near_fft_kernels(P, 0));
  return set_err(cudaDeviceSynchronize() == cudaSuccess ? FMM_OK : FMM_ERR_CUDA);
}

int fmm_plan_set_timeout_ms(fmm_plan* plan, int ms) {
  if (!plan || ms < 1 || ms > 600000) return set_err(FMM_ERR_ARG);
  reinterpret_cast<Plan*>(plan)->wait_ns = (uint64_t)ms * 1000000ull;
  return set_err(FMM_OK);
}

int fmm_plan_inject_fault(fmm_plan* plan, int kind) {
  if (!plan || (kind != FMM_FAULT_NONE && kind != FMM_FAULT_TC_STALL)) return set_err(FMM_ERR_ARG);
  reinterpret_cast<Plan*>(plan)->inject_stall = kind == FMM_FAULT_TC_STALL ? 1 : 0;
  return set_err(FMM_OK);
}

int fmm_plan_set_m2l_group(fmm_plan* plan, int offsets_per_partial) {
  if (!plan || offsets_per_partial < 1 || offsets_per_partial > fmm::kMaxOffsets) return set_err(FMM_ERR_ARG);
  reinterpret_cast<Plan*>(plan)->tc_group = offsets_per_partial;
  return set_err(FMM_OK);
}

int fmm_plan_set_tc_min_level(fmm_plan* plan, int level) {
  if (!plan || level < fmm::kTcMinLevel || level > fmm::kMaxLevel + 1) return set_err(FMM_ERR_ARG);
  Plan& P = *reinterpret_cast<Plan*>(plan);
  P.tc_min_level = level;
  P.tc_min_set = 1;
  if (P.tc_ready) {   // a lower first level needs its tiles now
    const int rc = prepare_tc(P);
    if (rc != FMM_OK) return set_err(rc);
  }
  return set_err(FMM_OK);
}

int fmm_plan_set_tc_tile(fmm_plan* plan, int level, int targets) {
  if (!plan || (targets != 128 && targets != 256)) return set_err(FMM_ERR_ARG);
  Plan& P = *reinterpret_cast<Plan*>(plan);
  if (level < fmm::kTcMinLevel || level > P.L) return set_err(FMM_ERR_ARG);
  P.tc_tile[level] = targets == 128 ? 128 : 0;
  if (P.tmapB[level]) {     // the tensor loads' box follows the tile
    FMM_CUDA_TRY(cudaDeviceSynchronize());
    const int rc = fmm::make_tc_map(P, level);
    if (rc != FMM_OK) return set_err(rc);
  }
  return set_err(FMM_OK);
}

int fmm_plan_autotune_tiles(fmm_plan* plan, const float* density, int* tiles, int n, void* stream) {
  if (!plan || !density || !aligned16(density) || (n > 0 && !tiles) || n < 0) return set_err(FMM_ERR_ARG);
  Plan& P = *reinterpret_cast<Plan*>(plan);
  const bool tc = P.prec != FMM_PREC_FP32 && P.tc_ready;
  const size_t n3 = (size_t)P.N * P.N * P.N;
  if (tc) {
    float* out = nullptr;
    if (cudaMalloc(&out, sizeof(float) * 4 * n3) != cudaSuccess) return set_err(FMM_ERR_ALLOC);
    const int was_timing = P.timing;
    int rc = fmm_plan_set_timing(plan, 1);
    float best[fmm::kMaxLevel + 1] = {};
    int pick[fmm::kMaxLevel + 1] = {};
    for (int c = 0; c < 2 && rc == FMM_OK; ++c) {
      const int t = c == 0 ? 256 : 128;
      for (int l = fmm::tc_first_level(P); l <= P.L && rc == FMM_OK; ++l)
        if (!fmm::tc_wide(P, l)) rc = fmm_plan_set_tc_tile(plan, l, t);
      float ms[FMM_TIME_SLOTS];
      float lev[fmm::kMaxLevel + 1];
      for (int l = 0; l <= fmm::kMaxLevel; ++l) lev[l] = 1e30f;
      for (int r = 0; r < 3 && rc == FMM_OK; ++r) {      // one warm-up, then the faster of two
        rc = fmm_solve(plan, density, out, out + n3, stream);
        if (rc == FMM_OK) rc = fmm_plan_stage_times(plan, ms, FMM_TIME_SLOTS);
        for (int l = 2; l <= P.L && r > 0 && rc == FMM_OK; ++l)
          lev[l] = ms[FMM_TIME_M2L_LEVEL0 + l] < lev[l] ? ms[FMM_TIME_M2L_LEVEL0 + l] : lev[l];
      }
      for (int l = 2; l <= P.L && rc == FMM_OK; ++l)
        if (c == 0 || lev[l] < best[l]) {
          best[l] = lev[l];
          pick[l] = t;
        }
    }
    for (int l = fmm::tc_first_level(P); l <= P.L && rc == FMM_OK; ++l)
      if (!fmm::tc_wide(P, l)) rc = fmm_plan_set_tc_tile(plan, l, pick[l]);
    fmm_plan_set_timing(plan, was_timing);
    cudaFree(out);
    if (rc != FMM_OK) return set_err(rc);
  }
  for (int l = 0; l < n; ++l)
    tiles[l] = (tc && l <= P.L && l >= fmm::tc_first_level(P)) ? fmm::tc_targets(P, l) : 0;
  return set_err(FMM_OK);
}

int fmm_plan_set_correction_inference(fmm_plan* plan, int mode) {
  if (!plan || (mode != FMM_INFER_BF16 && mode != FMM_INFER_FP32)) return set_err(FMM_ERR_ARG);
  reinterpret_cast<Plan*>(plan)->corr_fp32 = mode == FMM_INFER_FP32 ? 1 : 0;
  return set_err(FMM_OK);
}

int fmm_plan_set_correction(fmm_plan* plan, const float* weights, size_t n) {
  if (!plan) return set_err(FMM_ERR_ARG);
  Plan& P = *reinterpret_cast<Plan*>(plan);
  if (weights) {
    if (n != (size_t)fmm::mlp::kParams) return set_err(FMM_ERR_ARG);
    if (!P.corr_w && !dev_alloc(&P.corr_w, (size_t)fmm::mlp::kParams)) return set_err(FMM_ERR_ALLOC);
    FMM_CUDA_TRY(cudaMemcpy(P.corr_w, weights, n * sizeof(float), cudaMemcpyDefault));
    P.has_corr = 1;
  } else {
    P.has_corr = 0;
  }
  return set_err(retabulate(P));
}

int fmm_correction_grad(fmm_plan* plan, const float* density, const float* target_phi, const float* target_acc,
                        float w_phi, float w_g, float* grad, float* loss, void* stream) {
  if (!plan || !density || !target_phi || !target_acc || !grad || !loss) return set_err(FMM_ERR_ARG);
  Plan& P = *reinterpret_cast<Plan*>(plan);
  if (!P.has_corr) return set_err(FMM_ERR_ARG);
  const int rc = table_gradient(P, density, target_phi, target_acc, w_phi, w_g, loss, stream);
  if (rc != FMM_OK) return set_err(rc);
  FMM_CUDA_TRY(fmm::launch_mlp_backward(P, P.corr_w, grad, reinterpret_cast<cudaStream_t>(stream)));
  return set_err(FMM_OK);
}

int fmm_plan_table_grid_size(const fmm_plan* plan, size_t* n) {
  if (!plan || !n) return set_err(FMM_ERR_ARG);
  const Plan& P = *reinterpret_cast<const Plan*>(plan);
  *n = (size_t)(P.L - 1) * fmm::grid_level_size(P.p);
  return set_err(FMM_OK);
}

int fmm_plan_set_table_grid(fmm_plan* plan, const float* theta, size_t n) {
  if (!plan) return set_err(FMM_ERR_ARG);
  Plan& P = *reinterpret_cast<Plan*>(plan);
  const size_t need = (size_t)(P.L - 1) * fmm::grid_level_size(P.p);
  if (theta) {
    if (n != need) return set_err(FMM_ERR_ARG);
    if (!P.grid && !dev_alloc(&P.grid, need)) return set_err(FMM_ERR_ALLOC);
    FMM_CUDA_TRY(cudaMemcpy(P.grid, theta, need * sizeof(float), cudaMemcpyDefault));
    P.has_grid = 1;
  } else {
    P.has_grid = 0;
  }
  return set_err(retabulate(P));
}

int fmm_table_grid_grad(fmm_plan* plan, const float* density, const float* target_phi, const float* target_acc,
                        float w_phi, float w_g, float* grad, float* loss, void* stream) {
  if (!plan || !density || !target_phi || !target_acc || !grad || !loss) return set_err(FMM_ERR_ARG);
  Plan& P = *reinterpret_cast<Plan*>(plan);
  const int rc = table_gradient(P, density, target_phi, target_acc, w_phi, w_g, loss, stream);
  if (rc != FMM_OK) return set_err(rc);
  FMM_CUDA_TRY(fmm::launch_grid_grad(P, grad, reinterpret_cast<cudaStream_t>(stream)));
  return set_err(FMM_OK);
}

int fmm_adam_step(float* w, const float* g, float* m, float* v, size_t n, int step, float lr, float beta1, float beta2,
                  float eps, void* stream) {
  if (!w || !g || !m || !v || n == 0 || step < 1) return set_err(FMM_ERR_ARG);
  FMM_CUDA_TRY(fmm::launch_adam(w, g, m, v, n, step, lr, beta1, beta2, eps, reinterpret_cast<cudaStream_t>(stream)));
  return set_err(FMM_OK);
}

int fmm_mesh_green(int N, float* out, void* stream) {
  if (N < 2 || !out) return set_err(FMM_ERR_ARG);
  int dev = 0, sms = 0;
  FMM_CUDA_TRY(cudaGetDevice(&dev));
  FMM_CUDA_TRY(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
  FMM_CUDA_TRY(fmm::launch_mesh_green(N, out, sms, reinterpret_cast<cudaStream_t>(stream)));
  return set_err(FMM_OK);
}

int fmm_plan_mesh_green(const fmm_plan* plan, double* out, void* stream) {
  if (!plan || !out) return set_err(FMM_ERR_ARG);
  const Plan& P = *reinterpret_cast<const Plan*>(plan);
  FMM_CUDA_TRY(fmm::launch_mesh_green_plan(P, out, reinterpret_cast<cudaStream_t>(stream)));
  return set_err(FMM_OK);
}

int fmm_plan_check(fmm_plan* plan) {
  if (!plan) return set_err(FMM_ERR_ARG);
  Plan& P = *reinterpret_cast<Plan*>(plan);
  int h = 0;
  FMM_CUDA_TRY(cudaDeviceSynchronize());
  FMM_CUDA_TRY(cudaMemcpy(&h, P.d_err, sizeof(int), cudaMemcpyDeviceToHost));
  if (h) {
    FMM_CUDA_TRY(cudaMemset(P.d_err, 0, sizeof(int)));
    return set_err(FMM_ERR_TIMEOUT);
  }
  return set_err(FMM_OK);
}

int fmm_plan_set_timing(fmm_plan* plan, int enable) {
  if (!plan) return set_err(FMM_ERR_ARG);
  Plan& P = *reinterpret_cast<Plan*>(plan);
  if (enable && !P.ev[0]) {
    for (auto& e : P.ev) FMM_CUDA_TRY(cudaEventCreate(&e));
  }
  P.timing = enable ? 1 : 0;
  return set_err(FMM_OK);
}

int fmm_plan_stage_times(fmm_plan* plan, float* ms, int n) {
  if (!plan || !ms || n < 0) return set_err(FMM_ERR_ARG);
  Plan& P = *reinterpret_cast<Plan*>(plan);
  if (!P.timed) return set_err(FMM_ERR_ARG);
  const int k = n < FMM_TIME_SLOTS ? n : FMM_TIME_SLOTS;
  for (int i = 0; i < k; ++i) {
    ms[i] = 0.f;
    if (i == FMM_TIME_M2M && P.L <= 2) continue;
    if (i == FMM_TIME_L2L && P.L <= 2) continue;
    if (i >= FMM_TIME_M2L_LEVEL0 && (i - FMM_TIME_M2L_LEVEL0 < 2 || i - FMM_TIME_M2L_LEVEL0 > P.L)) continue;
    FMM_CUDA_TRY(cudaEventSynchronize(P.ev[2 * i + 1]));
    FMM_CUDA_TRY(cudaEventElapsedTime(&ms[i], P.ev[2 * i], P.ev[2 * i + 1]));
  }
  return set_err(FMM_OK);
}

int fmm_solve(fmm_plan* plan, const float* density, float* potential, float* accel, void* stream) {
  if (!plan || !density || !potential || !accel) return set_err(FMM_ERR_ARG);
  if (!aligned16(density) || !aligned16(potential) || !aligned16(accel)) return set_err(FMM_ERR_ARG);
  Plan& P = *reinterpret_cast<Plan*>(plan);
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  const bool t = P.timing != 0;
  auto mark = [&](int slot, int end) -> cudaError_t {
    return t ? cudaEventRecord(P.ev[2 * slot + end], s) : cudaSuccess;
  };
  FMM_CUDA_TRY(mark(FMM_TIME_MEAN, 0));
  if (P.iso)   // the isolated problem keeps every mass (m = rho / N^3)
    FMM_CUDA_TRY(cudaMemsetAsync(P.d_mean, 0, sizeof(double), s));
  else
    FMM_CUDA_TRY(fmm::launch_mean(P, density, s));
  FMM_CUDA_TRY(mark(FMM_TIME_MEAN, 1));
  const bool tc = P.prec != FMM_PREC_FP32 && P.tc_ready;
  auto on_tc = [&](int l) { return !fmm::fft_level(P, l) && tc && l >= fmm::tc_first_level(P); };
  // Untimed solves of the tensor-core forms overlap independent stages: the
  // near zone's source spectra need only the density and its mean (second
  // auxiliary stream, from the mean on); the M2L levels are independent of
  // one another until the downward pass, so the CUDA-core levels run on the
  // first auxiliary stream beside the tensor-core levels on `s` (issued
  // first).  Measured at 256^3 p = 6: 9.82 -> 9.67 ms; the two kernels
  // share few SMs (a tensor-core CTA and a CUDA-core CTA together exceed
  // one SM's shared memory or registers, and capping either cost more).
  // Timed solves stay serial, so that each stage's events bracket it alone.
  const bool overlap = !t && tc;
  const bool fwd_apart = overlap && P.near_fft;
  if (fwd_apart) {
    FMM_CUDA_TRY(cudaEventRecord(P.fev[0], s));
    FMM_CUDA_TRY(cudaStreamWaitEvent(P.aux[1], P.fev[0], 0));
    FMM_CUDA_TRY(fmm::launch_near_fft_fwd(P, density, P.aux[1]));
    FMM_CUDA_TRY(cudaEventRecord(P.fev[1], P.aux[1]));
  }
  FMM_CUDA_TRY(mark(FMM_TIME_P2M, 0));
  FMM_CUDA_TRY(fmm::launch_p2m(P, density, s));
  FMM_CUDA_TRY(mark(FMM_TIME_P2M, 1));
  FMM_CUDA_TRY(mark(FMM_TIME_M2M, 0));
  for (int l = P.L - 1; l >= 2; --l) FMM_CUDA_TRY(fmm::launch_m2m(P, l, s));
  FMM_CUDA_TRY(mark(FMM_TIME_M2M, 1));
  FMM_CUDA_TRY(mark(FMM_TIME_M2L, 0));
  if (overlap) {
    FMM_CUDA_TRY(cudaEventRecord(P.fev[2], s));
    for (int l = P.L; l >= 2; --l) {
      if (!on_tc(l)) continue;
      FMM_CUDA_TRY(fmm::launch_split_bf16(P, l, s));
      FMM_CUDA_TRY(fmm::launch_m2l_tc(P, l, P.prec, s));
    }
    FMM_CUDA_TRY(cudaStreamWaitEvent(P.aux[0], P.fev[2], 0));
    for (int l = 2; l <= P.L; ++l) {
      if (on_tc(l)) continue;
      if (fmm::fft_level(P, l))
        FMM_CUDA_TRY(fmm::launch_m2l_fft(P, l, P.aux[0]));
      else
        FMM_CUDA_TRY(fmm::launch_m2l_fp32(P, l, P.aux[0]));
    }
    FMM_CUDA_TRY(cudaEventRecord(P.fev[3], P.aux[0]));
    FMM_CUDA_TRY(cudaStreamWaitEvent(s, P.fev[3], 0));
  } else {
    for (int l = 2; l <= P.L; ++l) {
      FMM_CUDA_TRY(mark(FMM_TIME_M2L_LEVEL0 + l, 0));
      if (fmm::fft_level(P, l)) {
        FMM_CUDA_TRY(fmm::launch_m2l_fft(P, l, s));
      } else if (on_tc(l)) {
        FMM_CUDA_TRY(fmm::launch_split_bf16(P, l, s));
        FMM_CUDA_TRY(fmm::launch_m2l_tc(P, l, P.prec, s));
      } else {
        FMM_CUDA_TRY(fmm::launch_m2l_fp32(P, l, s));
      }
      FMM_CUDA_TRY(mark(FMM_TIME_M2L_LEVEL0 + l, 1));
    }
  }
  FMM_CUDA_TRY(mark(FMM_TIME_M2L, 1));
  FMM_CUDA_TRY(mark(FMM_TIME_L2L, 0));
  for (int l = 2; l < P.L; ++l) FMM_CUDA_TRY(fmm::launch_l2l(P, l, s));
  FMM_CUDA_TRY(mark(FMM_TIME_L2L, 1));
  FMM_CUDA_TRY(mark(FMM_TIME_P2P, 0));
  if (fwd_apart) FMM_CUDA_TRY(cudaStreamWaitEvent(s, P.fev[1], 0));
  FMM_CUDA_TRY(fmm::launch_p2p(P, density, potential, accel, s, fwd_apart));
  FMM_CUDA_TRY(mark(FMM_TIME_P2P, 1));
  P.solved = 1;
  if (t) P.timed = 1;
  return set_err(FMM_OK);
}

int fmm_solve_host(fmm_plan* plan, const float* density_host, float* potential_host, float* accel_host,
                   void* stream) {
  if (!plan || !density_host || !potential_host || !accel_host) return set_err(FMM_ERR_ARG);
  Plan& P = *reinterpret_cast<Plan*>(plan);
  const size_t n3 = (size_t)P.N * P.N * P.N;
  if (!P.stage_in) {
    if (!dev_alloc(&P.stage_in, n3) || !dev_alloc(&P.stage_out, 4 * n3)) return set_err(FMM_ERR_ALLOC);
  }
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  FMM_CUDA_TRY(cudaMemcpyAsync(P.stage_in, density_host, n3 * sizeof(float), cudaMemcpyHostToDevice, s));
  int rc = fmm_solve(plan, P.stage_in, P.stage_out, P.stage_out + n3, stream);
  if (rc != FMM_OK) return rc;
  FMM_CUDA_TRY(cudaMemcpyAsync(potential_host, P.stage_out, n3 * sizeof(float), cudaMemcpyDeviceToHost, s));
  FMM_CUDA_TRY(cudaMemcpyAsync(accel_host, P.stage_out + n3, 3 * n3 * sizeof(float), cudaMemcpyDeviceToHost, s));
  FMM_CUDA_TRY(cudaStreamSynchronize(s));
  return set_err(FMM_OK);
}

int fmm_plan_copy_stage(fmm_plan* plan, int stage, int level, float* dst, size_t count, void* stream) {
  if (!plan || !dst) return set_err(FMM_ERR_ARG);
  Plan& P = *reinterpret_cast<Plan*>(plan);
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  const size_t p3 = (size_t)P.p * P.p * P.p;
  if (stage == FMM_STAGE_MEAN) {
    if (count < 1) return set_err(FMM_ERR_ARG);
    // one-value conversion through the host keeps this path free of extra kernels
    double m = 0.0;
    FMM_CUDA_TRY(cudaMemcpyAsync(&m, P.d_mean, sizeof(double), cudaMemcpyDeviceToHost, s));
    FMM_CUDA_TRY(cudaStreamSynchronize(s));
    const float mf = (float)m;
    FMM_CUDA_TRY(cudaMemcpyAsync(dst, &mf, sizeof(float), cudaMemcpyHostToDevice, s));
    FMM_CUDA_TRY(cudaStreamSynchronize(s));
    return set_err(FMM_OK);
  }
  if (level < 2 || level > P.L) return set_err(FMM_ERR_ARG);
  const size_t nodes = (size_t)1 << (3 * level);
  const float* src = nullptr;
  size_t need = 0;
  if (stage == FMM_STAGE_MULTIPOLE) {
    src = P.M[level];
    need = nodes * p3;
  } else if (stage == FMM_STAGE_LOCAL) {
    src = P.F[level];
    need = nodes * 4 * p3;
  } else {
    return set_err(FMM_ERR_ARG);
  }
  if (count < need) return set_err(FMM_ERR_ARG);
  FMM_CUDA_TRY(cudaMemcpyAsync(dst, src, need * sizeof(float), cudaMemcpyDeviceToDevice, s));
  return set_err(FMM_OK);
}

int fmm_plan_error_stats(fmm_plan* plan, const float* density, const float* potential, const float* accel,
                         int samples, unsigned long long seed, double* out, void* stream) {
  if (!plan || !density || !potential || !accel || !out) return set_err(FMM_ERR_ARG);
  if (!aligned16(density) || !aligned16(potential) || !aligned16(accel)) return set_err(FMM_ERR_ARG);
  if (samples < 1 || samples > fmm::error_stats_max_samples()) return set_err(FMM_ERR_ARG);
  Plan& P = *reinterpret_cast<Plan*>(plan);
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  const unsigned long long n3 = (unsigned long long)P.N * P.N * P.N;
  std::vector<unsigned long long> targets((size_t)samples);
  for (int i = 0; i < samples; ++i) {
    // output i of splitmix64 (Steele, Lea and Flood 2014) seeded with `seed`
    unsigned long long z = seed + (unsigned long long)(i + 1) * 0x9e3779b97f4a7c15ull;
    z = (z ^ (z >> 30)) * 0xbf58476d1ce4e5b9ull;
    z = (z ^ (z >> 27)) * 0x94d049bb133111ebull;
    z ^= z >> 31;
    targets[(size_t)i] = z % n3;
  }
  struct Scratch {
    unsigned long long* targets = nullptr;
    double* partials = nullptr;
    double* sums = nullptr;
    double* mean = nullptr;
    ~Scratch() {
      cudaFree(targets);
      cudaFree(partials);
      cudaFree(sums);
      cudaFree(mean);
    }
  } d;
  const size_t np = (size_t)fmm::error_stats_grid_x(P, samples) * samples * 4;
  if (!dev_alloc(&d.targets, (size_t)samples) || !dev_alloc(&d.partials, np) || !dev_alloc(&d.sums, 4) ||
      !dev_alloc(&d.mean, (size_t)P.n_partials + 1))
    return set_err(FMM_ERR_ALLOC);
  FMM_CUDA_TRY(cudaMemcpyAsync(d.targets, targets.data(), sizeof(unsigned long long) * samples,
                               cudaMemcpyHostToDevice, s));
  FMM_CUDA_TRY(
      fmm::launch_error_stats(P, density, potential, accel, d.targets, samples, d.partials, d.sums, d.mean, s));
  double sums[4] = {0.0, 0.0, 0.0, 0.0};
  FMM_CUDA_TRY(cudaMemcpyAsync(sums, d.sums, sizeof(sums), cudaMemcpyDeviceToHost, s));
  FMM_CUDA_TRY(cudaStreamSynchronize(s));
  out[0] = sums[1] > 0.0 ? std::sqrt(sums[0] / sums[1]) : std::sqrt(sums[0]);
  out[1] = sums[3] > 0.0 ? std::sqrt(sums[2] / sums[3]) : std::sqrt(sums[2]);
  return set_err(FMM_OK);
}

}  // extern "C"

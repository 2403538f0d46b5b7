// Batched solves of many independent periodic fields of uneven size, and the
// tree-depth autotuner.
//
// A batch owns one plan per field.  fmm_batch_solve captures, once per set of
// field pointers, every field's kernel sequence into one CUDA graph: the
// fields run as parallel branches (K internal streams, largest fields first,
// round-robin), so small fields fill the SMs that large fields leave idle, and
// the whole batch is a single graph launch on the caller's stream.
//
// The autotuner picks the leaf level L of a field (it moves work between the
// tensor-core M2L and the near-zone sum) by timing candidate depths on a
// synthetic field; results are cached per GPU model in a JSON-lines file.
#include <algorithm>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <new>
#include <string>
#include <vector>

#include "fmm_internal.cuh"

struct fmm_batch {
  int n = 0;
  std::vector<fmm_plan*> plans;
  std::vector<int> N, L, p, order_by_cost;
  int branches = 0;
  cudaStream_t origin = nullptr;
  std::vector<cudaStream_t> streams;
  cudaEvent_t fork = nullptr;
  std::vector<cudaEvent_t> joins;
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t exec = nullptr;
  std::vector<const void*> sig;
};

namespace {

constexpr int kMaxBranches = 8;

// deterministic synthetic density for tuning: 1 + 0.5 * hash noise
__global__ void k_tune_density(float* rho, size_t n) {
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) {
    uint32_t h = (uint32_t)(i * 2654435761u) ^ 0x9E3779B9u;
    h ^= h >> 16;
    h *= 0x7feb352du;
    h ^= h >> 15;
    rho[i] = 1.f + 0.5f * (float)(h & 0xFFFFu) / 65535.f;
  }
}

void destroy_batch(fmm_batch* b) {
  if (!b) return;
  if (b->exec) cudaGraphExecDestroy(b->exec);
  if (b->graph) cudaGraphDestroy(b->graph);
  for (auto e : b->joins)
    if (e) cudaEventDestroy(e);
  if (b->fork) cudaEventDestroy(b->fork);
  for (auto s : b->streams)
    if (s) cudaStreamDestroy(s);
  if (b->origin) cudaStreamDestroy(b->origin);
  for (auto pl : b->plans) fmm_plan_destroy(pl);
  delete b;
}

std::string gpu_name() {
  int dev = 0;
  cudaDeviceProp prop;
  if (cudaGetDevice(&dev) != cudaSuccess || cudaGetDeviceProperties(&prop, dev) != cudaSuccess) return "unknown";
  std::string s(prop.name);
  for (auto& c : s)
    if (c == '"' || c == '\n') c = '_';
  return s;
}

bool cache_lookup(const char* path, const std::string& key, int* L, float* ms) {
  if (!path) return false;
  FILE* f = fopen(path, "r");
  if (!f) return false;
  char line[512];
  bool found = false;
  while (fgets(line, sizeof line, f)) {
    // {"key": "...", "L": x, "ms": y}
    const char* k = strstr(line, "\"key\": \"");
    if (!k) continue;
    k += 8;
    const char* e = strchr(k, '"');
    if (!e || std::string(k, e - k) != key) continue;
    const char* lp = strstr(e, "\"L\": ");
    const char* mp = strstr(e, "\"ms\": ");
    if (!lp || !mp) continue;
    *L = atoi(lp + 5);
    *ms = (float)atof(mp + 6);
    found = true;   // last entry wins
  }
  fclose(f);
  return found;
}

void cache_store(const char* path, const std::string& key, int L, float ms) {
  if (!path) return;
  FILE* f = fopen(path, "a");
  if (!f) return;
  fprintf(f, "{\"key\": \"%s\", \"L\": %d, \"ms\": %.4f}\n", key.c_str(), L, ms);
  fclose(f);
}

}  // namespace

extern "C" {

int fmm_autotune_levels(int N, int order, int precision, const char* cache_path, int* L_out, float* ms_out) {
  if (N < 4 || order < 1 || order > fmm::kMaxOrder || !L_out) return fmm::set_last_error(FMM_ERR_ARG);
  const std::string key = gpu_name() + "|N=" + std::to_string(N) + "|p=" + std::to_string(order) +
                          "|prec=" + std::to_string(precision);
  int L = 0;
  float ms = 0.f;
  if (cache_lookup(cache_path, key, &L, &ms)) {
    *L_out = L;
    if (ms_out) *ms_out = ms;
    return fmm::set_last_error(FMM_OK);
  }
  // candidates: leaf sizes S in {2, 3, 4, 6, 8}, general trees (L >= 3) first
  std::vector<int> cands;
  for (int l = 3; l <= fmm::kMaxLevel; ++l) {
    if (N % (1 << l)) continue;
    const int S = N >> l;
    if (S == 2 || S == 3 || S == 4 || S == 6 || S == 8) cands.push_back(l);
  }
  if (cands.empty()) {
    if (N % 4 == 0) {
      const int S = N / 4;
      if (S == 1 || S == 2 || S == 3 || S == 4 || S == 6 || S == 8) cands.push_back(2);
    }
    if (cands.empty()) return fmm::set_last_error(FMM_ERR_ARG);
  }
  const size_t n3 = (size_t)N * N * N;
  float *rho = nullptr, *out = nullptr;
  if (cudaMalloc(&rho, n3 * sizeof(float)) != cudaSuccess) return fmm::set_last_error(FMM_ERR_ALLOC);
  if (cudaMalloc(&out, 4 * n3 * sizeof(float)) != cudaSuccess) {
    cudaFree(rho);
    return fmm::set_last_error(FMM_ERR_ALLOC);
  }
  k_tune_density<<<256, 256>>>(rho, n3);
  cudaEvent_t e0, e1;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  int best = -1;
  float best_ms = 0.f;
  int rc = FMM_OK;
  for (int l : cands) {
    fmm_plan* pl = fmm_plan_create(N, l, order);
    if (!pl) {
      rc = fmm_last_error();
      break;
    }
    if (precision != FMM_PREC_FP32 && fmm_plan_set_precision(pl, precision) != FMM_OK) {
      rc = fmm_last_error();
      fmm_plan_destroy(pl);
      break;
    }
    float t[3];
    bool ok = fmm_solve(pl, rho, out, out + n3, nullptr) == FMM_OK;
    for (int k = 0; k < 3 && ok; ++k) {
      cudaEventRecord(e0);
      ok = fmm_solve(pl, rho, out, out + n3, nullptr) == FMM_OK;
      cudaEventRecord(e1);
      cudaEventSynchronize(e1);
      cudaEventElapsedTime(&t[k], e0, e1);
    }
    fmm_plan_destroy(pl);
    if (!ok) {
      rc = FMM_ERR_CUDA;
      break;
    }
    std::sort(t, t + 3);
    if (best < 0 || t[1] < best_ms) {
      best = l;
      best_ms = t[1];
    }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  cudaFree(rho);
  cudaFree(out);
  if (rc != FMM_OK) return fmm::set_last_error(rc);
  cache_store(cache_path, key, best, best_ms);
  *L_out = best;
  if (ms_out) *ms_out = best_ms;
  return fmm::set_last_error(FMM_OK);
}

fmm_batch* fmm_batch_create(int nfields, const int* N, const int* L, const int* order) {
  if (nfields < 1 || !N || !L || !order) {
    fmm::set_last_error(FMM_ERR_ARG);
    return nullptr;
  }
  fmm_batch* b = new (std::nothrow) fmm_batch();
  if (!b) {
    fmm::set_last_error(FMM_ERR_ALLOC);
    return nullptr;
  }
  b->n = nfields;
  const char* cache = getenv("FMM_AUTOTUNE_CACHE");
  for (int i = 0; i < nfields; ++i) {
    int l = L[i];
    if (l <= 0) {
      float ms;
      if (fmm_autotune_levels(N[i], order[i], FMM_PREC_BF16X3, cache, &l, &ms) != FMM_OK) {
        const int rc = fmm_last_error();
        destroy_batch(b);
        fmm::set_last_error(rc);
        return nullptr;
      }
    }
    fmm_plan* pl = fmm_plan_create(N[i], l, order[i]);
    if (!pl) {
      const int rc = fmm_last_error();
      destroy_batch(b);
      fmm::set_last_error(rc);
      return nullptr;
    }
    b->plans.push_back(pl);
    b->N.push_back(N[i]);
    b->L.push_back(l);
    b->p.push_back(order[i]);
  }
  // largest fields first on the branches
  b->order_by_cost.resize(nfields);
  for (int i = 0; i < nfields; ++i) b->order_by_cost[i] = i;
  std::stable_sort(b->order_by_cost.begin(), b->order_by_cost.end(), [&](int a, int c) {
    const double ca = (double)b->N[a] * b->N[a] * b->N[a] * b->p[a] * b->p[a];
    const double cc = (double)b->N[c] * b->N[c] * b->N[c] * b->p[c] * b->p[c];
    return ca > cc;
  });
  b->branches = std::min(nfields, kMaxBranches);
  bool ok = cudaStreamCreateWithFlags(&b->origin, cudaStreamNonBlocking) == cudaSuccess &&
            cudaEventCreateWithFlags(&b->fork, cudaEventDisableTiming) == cudaSuccess;
  for (int k = 0; k < b->branches && ok; ++k) {
    cudaStream_t s;
    cudaEvent_t e;
    ok = cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking) == cudaSuccess &&
         cudaEventCreateWithFlags(&e, cudaEventDisableTiming) == cudaSuccess;
    if (ok) {
      b->streams.push_back(s);
      b->joins.push_back(e);
    }
  }
  if (!ok) {
    destroy_batch(b);
    fmm::set_last_error(FMM_ERR_CUDA);
    return nullptr;
  }
  fmm::set_last_error(FMM_OK);
  return b;
}

int fmm_batch_set_precision(fmm_batch* b, int mode) {
  if (!b) return fmm::set_last_error(FMM_ERR_ARG);
  for (auto pl : b->plans) {
    const int rc = fmm_plan_set_precision(pl, mode);
    if (rc != FMM_OK) return rc;
  }
  // the captured graph holds the old kernels
  if (b->exec) cudaGraphExecDestroy(b->exec);
  if (b->graph) cudaGraphDestroy(b->graph);
  b->exec = nullptr;
  b->graph = nullptr;
  b->sig.clear();
  return fmm::set_last_error(FMM_OK);
}

int fmm_batch_set_near_algorithm(fmm_batch* b, int algorithm) {
  if (!b || (algorithm != FMM_NEAR_DIRECT && algorithm != FMM_NEAR_FFT)) return fmm::set_last_error(FMM_ERR_ARG);
  for (auto pl : b->plans) {
    // the FFT near zone needs 8-cell leaves: other fields keep the direct sum
    if (algorithm == FMM_NEAR_FFT && !fmm::near_fft_supported(*reinterpret_cast<const fmm::Plan*>(pl))) continue;
    const int rc = fmm_plan_set_near_algorithm(pl, algorithm);
    if (rc != FMM_OK) return rc;
  }
  if (b->exec) cudaGraphExecDestroy(b->exec);
  if (b->graph) cudaGraphDestroy(b->graph);
  b->exec = nullptr;
  b->graph = nullptr;
  b->sig.clear();
  return fmm::set_last_error(FMM_OK);
}

int fmm_batch_get_levels(const fmm_batch* b, int* L) {
  if (!b || !L) return fmm::set_last_error(FMM_ERR_ARG);
  for (int i = 0; i < b->n; ++i) L[i] = b->L[i];
  return fmm::set_last_error(FMM_OK);
}

int fmm_batch_solve(fmm_batch* b, const float* const* density, float* const* potential, float* const* accel,
                    void* stream) {
  if (!b || !density || !potential || !accel) return fmm::set_last_error(FMM_ERR_ARG);
  std::vector<const void*> sig;
  for (int i = 0; i < b->n; ++i) {
    if (!density[i] || !potential[i] || !accel[i]) return fmm::set_last_error(FMM_ERR_ARG);
    sig.push_back(density[i]);
    sig.push_back(potential[i]);
    sig.push_back(accel[i]);
  }
  if (!b->exec || sig != b->sig) {
    // capture every field's kernels as parallel branches of one graph
    if (b->exec) cudaGraphExecDestroy(b->exec);
    if (b->graph) cudaGraphDestroy(b->graph);
    b->exec = nullptr;
    b->graph = nullptr;
    if (cudaStreamBeginCapture(b->origin, cudaStreamCaptureModeThreadLocal) != cudaSuccess)
      return fmm::set_last_error(FMM_ERR_CUDA);
    int rc = FMM_OK;
    if (cudaEventRecord(b->fork, b->origin) != cudaSuccess) rc = FMM_ERR_CUDA;
    for (int k = 0; k < b->branches && rc == FMM_OK; ++k)
      if (cudaStreamWaitEvent(b->streams[k], b->fork, 0) != cudaSuccess) rc = FMM_ERR_CUDA;
    for (int j = 0; j < b->n && rc == FMM_OK; ++j) {
      const int i = b->order_by_cost[j];
      rc = fmm_solve(b->plans[i], density[i], potential[i], accel[i], b->streams[j % b->branches]);
    }
    for (int k = 0; k < b->branches && rc == FMM_OK; ++k) {
      if (cudaEventRecord(b->joins[k], b->streams[k]) != cudaSuccess ||
          cudaStreamWaitEvent(b->origin, b->joins[k], 0) != cudaSuccess)
        rc = FMM_ERR_CUDA;
    }
    cudaGraph_t g = nullptr;
    const cudaError_t ce = cudaStreamEndCapture(b->origin, &g);
    if (rc != FMM_OK || ce != cudaSuccess) {
      if (g) cudaGraphDestroy(g);
      return fmm::set_last_error(rc != FMM_OK ? rc : FMM_ERR_CUDA);
    }
    if (cudaGraphInstantiate(&b->exec, g, 0) != cudaSuccess) {
      cudaGraphDestroy(g);
      return fmm::set_last_error(FMM_ERR_CUDA);
    }
    b->graph = g;
    b->sig = sig;
  }
  if (cudaGraphLaunch(b->exec, reinterpret_cast<cudaStream_t>(stream)) != cudaSuccess)
    return fmm::set_last_error(FMM_ERR_CUDA);
  return fmm::set_last_error(FMM_OK);
}

int fmm_batch_check(fmm_batch* b) {
  if (!b) return fmm::set_last_error(FMM_ERR_ARG);
  int worst = FMM_OK;
  for (auto pl : b->plans) {
    const int rc = fmm_plan_check(pl);
    if (rc != FMM_OK) worst = rc;
  }
  return fmm::set_last_error(worst);
}

void fmm_batch_destroy(fmm_batch* b) {
  if (!b) return;
  cudaDeviceSynchronize();
  destroy_batch(b);
}

}  // extern "C"

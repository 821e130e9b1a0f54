// Batched evaluation of many independent periodic systems (uneven N, box and K) with one
// CUDA graph launch.  Each system owns a plan; one evaluation is captured as a graph whose
// parallel branches run the systems' pipelines (spread, SKP mode products, gather,
// reductions) on up to 16 branch streams, and the executable graph is replayed while the
// call signature repeats.  Systems with identical parameters share one SKP build.
#include "kpme_internal.cuh"

#include <algorithm>
#include <cmath>
#include <string>
#include <cstring>
#include <map>
#include <new>
#include <tuple>

struct kpme_batch_s {
  std::vector<kpme_plan_t> plans;
  cudaStream_t stream = nullptr;       // caller's stream
  cudaStream_t root = nullptr;         // capture origin
  std::vector<cudaStream_t> branches;
  cudaEvent_t fork = nullptr;
  std::vector<cudaEvent_t> joins;
  cudaGraphExec_t exec = nullptr;
  std::vector<int64_t> key;
  std::string last_error;
};

namespace {

void release(kpme_batch_t B) {
  if (!B) return;
  if (B->exec) cudaGraphExecDestroy(B->exec);
  for (auto p : B->plans) kpme_destroy(p);
  for (auto s : B->branches) cudaStreamDestroy(s);
  if (B->root) cudaStreamDestroy(B->root);
  if (B->fork) cudaEventDestroy(B->fork);
  for (auto e : B->joins) cudaEventDestroy(e);
  delete B;
}

kpme_status_t fail(kpme_batch_t B, const char* what, cudaError_t e) {
  B->last_error = std::string(what) + ": " + cudaGetErrorString(e);
  return e == cudaErrorMemoryAllocation ? KPME_ERR_OOM : KPME_ERR_CUDA;
}

}  // namespace

extern "C" {

kpme_status_t kpme_batch_create(int n_sys, const kpme_params_t* params, void* stream, kpme_batch_t* out) {
  if (!out || n_sys <= 0 || !params) return KPME_ERR_INVALID_ARG;
  *out = nullptr;
  kpme_batch_t B = new (std::nothrow) kpme_batch_s();
  if (!B) return KPME_ERR_OOM;
  B->stream = (cudaStream_t)stream;
  for (int s = 0; s < n_sys; ++s) {
    kpme_plan_t P = nullptr;
    kpme_status_t st = kpme_plan(&params[s], stream, &P);
    if (st != KPME_OK) {
      release(B);
      return st;
    }
    P->use_graphs = false;
    B->plans.push_back(P);
  }
  const int nb = std::min(n_sys, 16);
  cudaError_t e = cudaStreamCreateWithFlags(&B->root, cudaStreamNonBlocking);
  if (e == cudaSuccess) e = cudaEventCreateWithFlags(&B->fork, cudaEventDisableTiming);
  for (int i = 0; i < nb && e == cudaSuccess; ++i) {
    cudaStream_t s = nullptr;
    cudaEvent_t ev = nullptr;
    e = cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&ev, cudaEventDisableTiming);
    if (s) B->branches.push_back(s);
    if (ev) B->joins.push_back(ev);
  }
  if (e != cudaSuccess) {
    kpme_status_t st = e == cudaErrorMemoryAllocation ? KPME_ERR_OOM : KPME_ERR_CUDA;
    release(B);
    return st;
  }
  *out = B;
  return KPME_OK;
}

void kpme_batch_destroy(kpme_batch_t B) {
  if (B && B->stream) cudaStreamSynchronize(B->stream);
  release(B);
}

kpme_status_t kpme_batch_build_skp(kpme_batch_t B, int* ranks_out) {
  if (!B) return KPME_ERR_INVALID_ARG;
  using Key = std::tuple<int, int, double, double, double, int>;
  std::map<Key, int> first;
  for (size_t s = 0; s < B->plans.size(); ++s) {
    kpme_plan_t P = B->plans[s];
    const Key k{P->p.K, P->p.order, P->p.radius, P->p.beta, P->p.skp_tol, P->p.skp_method};
    auto it = first.find(k);
    kpme_status_t st;
    if (it == first.end()) {
      st = kpme_build_skp(P, nullptr, nullptr);
      first[k] = (int)s;
    } else {
      st = kpme::plan_install_skp(P, B->plans[it->second]->skp);
    }
    if (st != KPME_OK) {
      B->last_error = P->last_error;
      return st;
    }
    if (ranks_out) ranks_out[s] = P->skp.R;
  }
  if (B->exec) cudaGraphExecDestroy(B->exec);
  B->exec = nullptr;
  return KPME_OK;
}

kpme_status_t kpme_batch_energy_forces(kpme_batch_t B, const int64_t* offsets, const double* x, const double* q,
                                       double* energies, double* forces, double* dEdq, double* virials) {
  if (!B || !offsets || !energies) return KPME_ERR_INVALID_ARG;
  const int n_sys = (int)B->plans.size();
  for (int s = 0; s < n_sys; ++s) {
    const int64_t n = offsets[s + 1] - offsets[s];
    if (offsets[s] < 0 || n < 0) return KPME_ERR_INVALID_ARG;
    if (n > B->plans[s]->max_n) return KPME_ERR_CAPACITY;
    if (!B->plans[s]->skp.valid) return KPME_ERR_NOT_BUILT;
  }
  if (offsets[n_sys] > 0 && (!x || !q)) return KPME_ERR_INVALID_ARG;
  std::vector<int64_t> key(offsets, offsets + n_sys + 1);
  for (const void* p : {(const void*)x, (const void*)q, (const void*)energies, (const void*)forces,
                        (const void*)dEdq, (const void*)virials})
    key.push_back((int64_t)p);
  if (!B->exec || key != B->key) {
    if (B->exec) cudaGraphExecDestroy(B->exec);
    B->exec = nullptr;
    cudaError_t e = cudaStreamBeginCapture(B->root, cudaStreamCaptureModeRelaxed);
    if (e != cudaSuccess) return fail(B, "cudaStreamBeginCapture", e);
    cudaEventRecord(B->fork, B->root);
    for (auto s : B->branches) cudaStreamWaitEvent(s, B->fork, 0);
    kpme_status_t st = KPME_OK;
    for (int s = 0; s < n_sys && st == KPME_OK; ++s) {
      kpme_plan_t P = B->plans[s];
      const int64_t o = offsets[s], n = offsets[s + 1] - offsets[s];
      cudaStream_t keep = P->stream;
      P->stream = B->branches[s % B->branches.size()];
      st = kpme::eval_energy_forces(P, n, x ? x + 3 * o : nullptr, q ? q + o : nullptr, energies + s,
                                    forces ? forces + 3 * o : nullptr, dEdq ? dEdq + o : nullptr,
                                    virials ? virials + s : nullptr);
      if (st != KPME_OK) B->last_error = P->last_error;
      P->stream = keep;
    }
    for (size_t i = 0; i < B->branches.size(); ++i) {
      cudaEventRecord(B->joins[i], B->branches[i]);
      cudaStreamWaitEvent(B->root, B->joins[i], 0);
    }
    cudaGraph_t g = nullptr;
    e = cudaStreamEndCapture(B->root, &g);
    if (st != KPME_OK) {
      if (g) cudaGraphDestroy(g);
      return st;
    }
    if (e != cudaSuccess) return fail(B, "cudaStreamEndCapture", e);
    e = cudaGraphInstantiate(&B->exec, g, 0);
    cudaGraphDestroy(g);
    if (e != cudaSuccess) return fail(B, "cudaGraphInstantiate", e);
    B->key = key;
  }
  cudaError_t e = cudaGraphLaunch(B->exec, B->stream);
  if (e != cudaSuccess) return fail(B, "cudaGraphLaunch", e);
  return KPME_OK;
}

}  // extern "C"

namespace {

// Milliseconds of one batch evaluation (graph replay on the batch's stream; a 3-evaluation
// probe sizes the timed run to ~20 ms of work, 3 to 50 evaluations).
kpme_status_t time_batch(kpme_batch_t B, const int64_t* offsets, const double* x, const double* q, double* E,
                         double* F, double* dq, double* W, double* ms) {
  kpme_status_t st;
  for (int i = 0; i < 2; ++i)   // the first call captures the graph
    if ((st = kpme_batch_energy_forces(B, offsets, x, q, E, F, dq, W)) != KPME_OK) return st;
  cudaEvent_t e0, e1;
  if (cudaEventCreate(&e0) != cudaSuccess) return KPME_ERR_CUDA;
  if (cudaEventCreate(&e1) != cudaSuccess) {
    cudaEventDestroy(e0);
    return KPME_ERR_CUDA;
  }
  auto run = [&](int reps, double* out) {
    cudaEventRecord(e0, B->stream);
    kpme_status_t r = KPME_OK;
    for (int i = 0; i < reps && r == KPME_OK; ++i) r = kpme_batch_energy_forces(B, offsets, x, q, E, F, dq, W);
    cudaEventRecord(e1, B->stream);
    float t = 0.0f;
    if (r == KPME_OK && (cudaEventSynchronize(e1) != cudaSuccess || cudaEventElapsedTime(&t, e0, e1) != cudaSuccess))
      r = KPME_ERR_CUDA;
    *out = (double)t / reps;
    return r;
  };
  double probe = 0.0;
  st = run(3, &probe);
  if (st == KPME_OK) st = run(probe > 0.0 ? (int)std::min(50.0, std::max(3.0, std::ceil(20.0 / probe))) : 50, ms);
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  return st;
}

kpme_tune_t config_of(kpme_plan_t P) {
  kpme_tune_t t{};
  t.tile = P->tile > 0 && P->no_sort ? -1 : P->tile;
  t.fused = P->allow_fused ? 1 : 0;
  t.split = P->tune_split;
  return t;
}

}  // namespace

extern "C" {

kpme_status_t kpme_batch_autotune(kpme_batch_t B, const int64_t* offsets, const double* x, const double* q,
                                  const char* cache_path, int* n_tuned) {
  if (!B || !offsets) return KPME_ERR_INVALID_ARG;
  const int n_sys = (int)B->plans.size();
  std::vector<kpme_tune_t> before(n_sys);
  for (int s = 0; s < n_sys; ++s) before[s] = config_of(B->plans[s]);
  std::map<std::tuple<int, int, int, int>, kpme_tune_t> tuned;
  int timed = 0;
  for (size_t s = 0; s < B->plans.size(); ++s) {
    kpme_plan_t P = B->plans[s];
    const int64_t o = offsets[s], n = offsets[s + 1] - offsets[s];
    if (n < 0) return KPME_ERR_INVALID_ARG;
    const int nb = n > 0 ? (int)std::floor(std::log2((double)n)) : 0;
    const auto key = std::make_tuple(P->p.K, P->p.order, P->p.precision, nb);
    auto it = tuned.find(key);
    kpme_status_t st;
    if (it != tuned.end()) {
      st = kpme_set_tune(P, &it->second);
    } else {
      kpme_tune_t t{};
      st = kpme_autotune(P, n, x ? x + 3 * o : nullptr, q ? q + o : nullptr, cache_path, &t);
      if (st == KPME_OK) {
        tuned[key] = t;
        if (!t.from_cache) ++timed;
      }
    }
    if (st != KPME_OK) {
      B->last_error = std::string("autotune of system ") + std::to_string(s) + ": " + kpme_last_error(P);
      return st;
    }
  }
  if (B->exec) {
    cudaGraphExecDestroy(B->exec);
    B->exec = nullptr;
  }
  B->key.clear();
  // Each class was timed alone; the batch runs its systems concurrently.  Keep the tuned
  // configurations only if the whole batch is faster with them than with the ones before.
  const int64_t total = offsets[n_sys];
  if (total > 0 && x && q) {
    const size_t nn = (size_t)total;
    double *E = nullptr, *F = nullptr, *dq = nullptr, *W = nullptr;
    kpme_status_t st = KPME_OK;
    if (cudaMalloc(&E, n_sys * sizeof(double)) != cudaSuccess || cudaMalloc(&W, n_sys * sizeof(double)) != cudaSuccess ||
        cudaMalloc(&F, 3 * nn * sizeof(double)) != cudaSuccess || cudaMalloc(&dq, nn * sizeof(double)) != cudaSuccess)
      st = KPME_ERR_OOM;
    std::vector<kpme_tune_t> after(n_sys);
    for (int s = 0; s < n_sys; ++s) after[s] = config_of(B->plans[s]);
    double t_after = 0.0, t_before = 0.0;
    if (st == KPME_OK) st = time_batch(B, offsets, x, q, E, F, dq, W, &t_after);
    for (int s = 0; s < n_sys && st == KPME_OK; ++s) st = kpme_set_tune(B->plans[s], &before[s]);
    if (st == KPME_OK) st = time_batch(B, offsets, x, q, E, F, dq, W, &t_before);
    if (st == KPME_OK && t_after < t_before)
      for (int s = 0; s < n_sys && st == KPME_OK; ++s) st = kpme_set_tune(B->plans[s], &after[s]);
    cudaFree(E);
    cudaFree(F);
    cudaFree(dq);
    cudaFree(W);
    if (B->exec) {
      cudaGraphExecDestroy(B->exec);
      B->exec = nullptr;
    }
    B->key.clear();
    if (st != KPME_OK) {
      B->last_error = "batch autotune: timing the batch failed";
      return st;
    }
  }
  if (n_tuned) *n_tuned = timed;
  return KPME_OK;
}

kpme_status_t kpme_batch_set_stream(kpme_batch_t B, void* stream) {
  if (!B) return KPME_ERR_INVALID_ARG;
  B->stream = (cudaStream_t)stream;
  for (auto P : B->plans) P->stream = (cudaStream_t)stream;
  return KPME_OK;
}

const char* kpme_batch_last_error(kpme_batch_t B) { return B ? B->last_error.c_str() : ""; }

}  // extern "C"

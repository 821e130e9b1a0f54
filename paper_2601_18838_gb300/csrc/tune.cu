// Autotuner of a plan's launch configuration.
//
// The knobs are the ones whose best value depends on the workload rather than on the
// mathematics (every setting gives the same result up to summation order):
//   tile   - edge T of the cell-sort tiles of spreading and gathering (T^3 cells per CTA),
//            or -1: no cell sort (float32 atomics on the mesh, untiled gathering);
//   fused  - stages 2 and 3 of the SKP fused on the SM (K = 32, 64) or run separately;
//   split  - split-K multiplier of the term ranges (x split / 2 of the cost-model choice);
//            for the fused stages, the grid of the static schedule (x split / 2 of the SMs).
// kpme_autotune times kpme_energy_forces (graph replay, CUDA events on the plan's stream,
// after warm-ups) by coordinate descent over the knobs and keeps the fastest; the tile knob,
// which changes only the spreading and gathering steps, is judged on those steps' own event
// times (a few percent of a large evaluation, below the noise of whole evaluations).  An
// optional text cache (one line per problem key) stores the choice for later plans.
#include "kpme_internal.cuh"

#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <string>
#include <vector>

namespace {

struct Config {
  int tile, fused, split;
};

kpme_status_t apply_config(kpme_plan_t P, const Config& c) {
  kpme_status_t st;
  if (P->tile > 0 && (c.tile > 0 || c.tile == -1) && (st = kpme::set_sorted(P, c.tile > 0)) != KPME_OK) return st;
  if (c.tile > 0 && P->tile > 0 && c.tile != P->tile && (st = kpme::set_tile(P, c.tile)) != KPME_OK) return st;
  const bool reinstall = (c.fused != 0) != P->allow_fused || c.split != P->tune_split;
  P->allow_fused = c.fused != 0;
  P->tune_split = c.split;
  if (reinstall && P->skp.valid) return kpme::install_skp(P);
  return KPME_OK;
}

struct Buffers {
  double *E = nullptr, *F = nullptr, *dq = nullptr, *W = nullptr;
  ~Buffers() {
    cudaFree(E);
    cudaFree(F);
    cudaFree(dq);
    cudaFree(W);
  }
};

kpme_status_t time_config(kpme_plan_t P, int64_t n, const double* x, const double* q, const Buffers& b, double* ms) {
  kpme_status_t st;
  double* W = kpme::lagrange(P) ? nullptr : b.W;   // the per-cell form has no virial
  for (int i = 0; i < 2; ++i)   // the first call captures the evaluation graph
    if ((st = kpme_energy_forces(P, n, x, q, b.E, b.F, b.dq, W)) != KPME_OK) return st;
  cudaEvent_t e0, e1;
  if (cudaEventCreate(&e0) != cudaSuccess) return KPME_ERR_CUDA;
  if (cudaEventCreate(&e1) != cudaSuccess) {
    cudaEventDestroy(e0);
    return KPME_ERR_CUDA;
  }
  // a probe of 3 evaluations sizes the timed run to ~20 ms of work (5 to 100 evaluations),
  // so that short evaluations are not judged on a few microseconds of launch noise
  auto run = [&](int reps, double* out) {
    cudaEventRecord(e0, P->stream);
    kpme_status_t r = KPME_OK;
    for (int i = 0; i < reps && r == KPME_OK; ++i) r = kpme_energy_forces(P, n, x, q, b.E, b.F, b.dq, W);
    cudaEventRecord(e1, P->stream);
    float t = 0.0f;
    if (r == KPME_OK && (cudaEventSynchronize(e1) != cudaSuccess || cudaEventElapsedTime(&t, e0, e1) != cudaSuccess))
      r = KPME_ERR_CUDA;
    *out = (double)t / reps;
    return r;
  };
  double probe = 0.0;
  st = run(3, &probe);
  if (st == KPME_OK) {
    const int reps = probe > 0.0 ? (int)std::min(100.0, std::max(5.0, std::ceil(20.0 / probe))) : 100;
    st = run(reps, ms);
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  return st;
}

// Milliseconds of the spreading and gathering steps of one evaluation: the plan's step events
// (eager evaluations), ten evaluations after two warm-ups.
kpme_status_t time_particles(kpme_plan_t P, int64_t n, const double* x, const double* q, const Buffers& b,
                             double* ms) {
  double* W = kpme::lagrange(P) ? nullptr : b.W;
  double steps[kpme::NUM_STEPS] = {};
  int n_out = 0;
  P->profiling = true;
  kpme_status_t st = KPME_OK;
  for (int i = 0; i < 2 && st == KPME_OK; ++i) st = kpme_energy_forces(P, n, x, q, b.E, b.F, b.dq, W);
  if (st == KPME_OK) st = kpme_get_profile(P, steps, nullptr, kpme::NUM_STEPS, &n_out, 1);
  constexpr int kReps = 10;
  for (int i = 0; i < kReps && st == KPME_OK; ++i) st = kpme_energy_forces(P, n, x, q, b.E, b.F, b.dq, W);
  if (st == KPME_OK) st = kpme_get_profile(P, steps, nullptr, kpme::NUM_STEPS, &n_out, 1);
  P->profiling = false;
  *ms = (steps[kpme::STEP_SPREAD] + steps[kpme::STEP_GATHER]) / kReps;
  return st;
}

std::string key_of(kpme_plan_t P, int64_t n) {
  char buf[160];
  const int nb = n > 0 ? (int)std::floor(std::log2((double)n)) : 0;
  snprintf(buf, sizeof(buf), "K%d_order%d_prec%d_interp%d_n2^%d_sm%d_cc%d%d", P->p.K, P->p.order, P->p.precision, P->p.interp, nb,
           P->sm_count, P->cc_major, P->cc_minor);
  return buf;
}

bool cache_lookup(const char* path, const std::string& key, Config& c, double& ms) {
  FILE* f = fopen(path, "r");
  if (!f) return false;
  char k[160];
  Config t{};
  double m = 0.0;
  bool found = false;
  while (fscanf(f, "%159s %d %d %d %lf", k, &t.tile, &t.fused, &t.split, &m) == 5)
    if (key == k) {   // the last entry for a key wins
      c = t;
      ms = m;
      found = true;
    }
  fclose(f);
  return found;
}

void cache_append(const char* path, const std::string& key, const Config& c, double ms) {
  FILE* f = fopen(path, "a");
  if (!f) return;
  fprintf(f, "%s %d %d %d %.6f\n", key.c_str(), c.tile, c.fused, c.split, ms);
  fclose(f);
}

}  // namespace

extern "C" {

kpme_status_t kpme_set_tune(kpme_plan_t P, const kpme_tune_t* t) {
  if (!P || !t) return KPME_ERR_INVALID_ARG;
  if (t->tile > 0 && P->tile > 0 && !kpme::tile_ok(P->p.K, P->p.order, t->tile)) return KPME_ERR_INVALID_ARG;
  if (t->tile < -1 || (t->tile == -1 && P->tile <= 0)) return KPME_ERR_INVALID_ARG;
  if (t->split != 1 && t->split != 2 && t->split != 4) return KPME_ERR_INVALID_ARG;
  KPME_CUDA_TRY(P, cudaSetDevice(P->device));
  KPME_CUDA_TRY(P, cudaStreamSynchronize(P->stream));
  return apply_config(P, Config{t->tile, t->fused, t->split});
}

kpme_status_t kpme_autotune(kpme_plan_t P, int64_t n, const double* x, const double* q, const char* cache_path,
                            kpme_tune_t* out) {
  if (!P || !out || n < 0 || n > P->max_n || (n > 0 && (!x || !q))) return KPME_ERR_INVALID_ARG;
  if (!P->skp.valid) return KPME_ERR_NOT_BUILT;
  KPME_CUDA_TRY(P, cudaSetDevice(P->device));
  const bool prof = P->profiling;
  P->profiling = false;
  const std::string key = key_of(P, n);
  Config best{P->tile > 0 && P->no_sort ? -1 : P->tile, P->allow_fused ? 1 : 0, P->tune_split};
  double best_ms = 0.0;
  kpme_status_t st = KPME_OK;
  Config cached{};
  if (cache_path && cache_lookup(cache_path, key, cached, best_ms) &&
      (cached.tile == 0 || P->tile <= 0 || cached.tile == -1 || kpme::tile_ok(P->p.K, P->p.order, cached.tile))) {
    st = apply_config(P, cached);
    if (st == KPME_OK) *out = kpme_tune_t{cached.tile, cached.fused, cached.split, 1, best_ms};
    P->profiling = prof;
    return st;
  }
  Buffers b;
  const size_t nn = (size_t)std::max<int64_t>(n, 1);
  if (cudaMalloc(&b.E, sizeof(double)) != cudaSuccess || cudaMalloc(&b.F, 3 * nn * sizeof(double)) != cudaSuccess ||
      cudaMalloc(&b.dq, nn * sizeof(double)) != cudaSuccess || cudaMalloc(&b.W, sizeof(double)) != cudaSuccess) {
    P->profiling = prof;
    return KPME_ERR_OOM;
  }
  if ((st = apply_config(P, best)) == KPME_OK) st = time_config(P, n, x, q, b, &best_ms);
  auto trial = [&](Config c) {
    if (st != KPME_OK) return;
    double ms = 0.0;
    if ((st = apply_config(P, c)) != KPME_OK) return;
    if ((st = time_config(P, n, x, q, b, &ms)) != KPME_OK) return;
    if (ms < 0.98 * best_ms) {
      best = c;
      best_ms = ms;
    }
  };
  // knob 1: fused stages 2-3 where the kernel exists
  if (P->ozt_res && P->tc_bn == P->p.K && (P->p.K == 32 || P->p.K == 64)) trial(Config{best.tile, 1 - best.fused, best.split});
  // knob 2: spreading tile edge, or no cell sort (plans that can tile), on the particle steps
  if (P->tile > 0 && st == KPME_OK) {
    double part_ms = 0.0;
    st = time_particles(P, n, x, q, b, &part_ms);
    const int base = best.tile;
    auto trial_p = [&](Config c) {
      if (st != KPME_OK) return;
      double ms = 0.0;
      if ((st = apply_config(P, c)) != KPME_OK) return;
      if ((st = time_particles(P, n, x, q, b, &ms)) != KPME_OK) return;
      if (ms < 0.99 * part_ms) {
        best = c;
        part_ms = ms;
      }
    };
    for (int T : {4, 8, 16, 32})
      if (T != base && kpme::tile_ok(P->p.K, P->p.order, T)) trial_p(Config{T, best.fused, best.split});
    if (base != -1) trial_p(Config{-1, best.fused, best.split});
    // the evaluation time of the choice, against which the split knob is judged
    if (st == KPME_OK && (st = apply_config(P, best)) == KPME_OK) st = time_config(P, n, x, q, b, &best_ms);
  }
  // knob 3: split-K multiplier
  const int base_split = best.split;
  for (int s : {1, 2, 4})
    if (s != base_split) trial(Config{best.tile, best.fused, s});
  if (st == KPME_OK) st = apply_config(P, best);
  if (st == KPME_OK && cache_path) cache_append(cache_path, key, best, best_ms);
  if (st == KPME_OK) *out = kpme_tune_t{best.tile, best.fused, best.split, 0, best_ms};
  P->profiling = prof;
  return st;
}

}  // extern "C"

// Host side of the C ABI declared in include/kpme.h: plans, SKP installation and the
// evaluation pipeline of Algorithm 4 on one GPU (spread -> SKP mode products -> gather ->
// float64 reductions), with the mode products ordered as the three reshaped steps of
// Algorithm 2.
#include "kpme_internal.cuh"

#include <nvtx3/nvToolsExt.h>

#include <cstdio>
#include <climits>

#include <algorithm>
#include <cmath>
#include <cstdlib>
#include <cstring>
#include <new>

using namespace kpme;

namespace kpme {

PrecInfo prec_info(int precision) {
  PrecInfo pi;
  switch (precision) {
    case KPME_FP64: pi.fp64 = true; pi.elem_bytes = 8; break;
    case KPME_FP32: pi.elem_bytes = 4; break;
    case KPME_TF32: pi.tensor = pi.tf32 = true; pi.slices = 1; pi.n_products = 1; pi.elem_bytes = 4; break;
    case KPME_TF32X3: pi.tensor = pi.tf32 = true; pi.slices = 2; pi.n_products = 3; pi.elem_bytes = 4; break;
    case KPME_BF16: pi.tensor = true; pi.slices = 1; pi.n_products = 1; pi.elem_bytes = 2; break;
    case KPME_BF16X3: pi.tensor = true; pi.slices = 2; pi.n_products = 3; pi.elem_bytes = 2; break;
    case KPME_BF16X6: pi.tensor = true; pi.slices = 3; pi.n_products = 6; pi.elem_bytes = 2; break;
    case KPME_BF16X10: pi.tensor = pi.oz = true; pi.slices = 4; pi.n_products = 10; pi.elem_bytes = 2; break;
    default: break;
  }
  return pi;
}

}  // namespace kpme

namespace {

bool valid_precision(int p) { return p >= KPME_FP64 && p <= KPME_BF16X10; }

// mesh element size (meshes Q, Phi and the CUDA-core intermediates)
size_t mesh_elem(const kpme_plan_t P) { return P->prec.fp64 ? sizeof(double) : sizeof(float); }

int64_t K3(const kpme_plan_t P) { return (int64_t)P->p.K * P->p.K * P->p.K; }

template <typename T>
void dfree(T*& p) {
  if (p) cudaFree((void*)p);
  p = nullptr;
}

kpme_status_t dalloc(kpme_plan_t P, void** p, size_t bytes) {
  if (bytes == 0) bytes = 16;
  if (P->fault_alloc_at > 0 && ++P->n_allocs == P->fault_alloc_at) {   // injected (KPME_FAULT=alloc)
    *p = nullptr;
    P->last_error = "cudaMalloc: injected allocation failure";
    return KPME_ERR_OOM;
  }
  cudaError_t e = cudaMalloc(p, bytes);
  if (e != cudaSuccess) {
    P->last_error = std::string("cudaMalloc: ") + cudaGetErrorString(e);
    cudaGetLastError();
    return e == cudaErrorMemoryAllocation ? KPME_ERR_OOM : KPME_ERR_CUDA;
  }
  P->scratch_bytes += (int64_t)bytes;
  if (P->poison) {
    // a check that no kernel reads scratch it has not written: every byte starts as 0xFF, a
    // NaN in float32 and float64 and -1 in integers, so such a read spoils the results
    e = cudaMemsetAsync(*p, 0xff, bytes, P->stream);
    if (e != cudaSuccess) {
      P->last_error = std::string("cudaMemsetAsync: ") + cudaGetErrorString(e);
      return KPME_ERR_CUDA;
    }
  }
  return KPME_OK;
}

void free_joblist(JobList& j) {
  dfree(j.d_start);
  dfree(j.d_pairs);
  dfree(j.d_items);
  dfree(j.d_cta);
  j = JobList();
}

kpme_status_t upload_joblist(kpme_plan_t P, JobList& j) {
  j.n_jobs = (int)j.h_start.size() - 1;
  j.max_pairs = 0;
  for (int i = 0; i < j.n_jobs; ++i) j.max_pairs = std::max(j.max_pairs, j.h_start[i + 1] - j.h_start[i]);
  kpme_status_t st;
  if ((st = dalloc(P, (void**)&j.d_start, j.h_start.size() * sizeof(int))) != KPME_OK) return st;
  if ((st = dalloc(P, (void**)&j.d_pairs, std::max<size_t>(1, j.h_pairs.size()) * sizeof(int2))) != KPME_OK)
    return st;
  KPME_CUDA_TRY(P, cudaMemcpyAsync(j.d_start, j.h_start.data(), j.h_start.size() * sizeof(int),
                                   cudaMemcpyHostToDevice, P->stream));
  if (!j.h_pairs.empty())
    KPME_CUDA_TRY(P, cudaMemcpyAsync(j.d_pairs, j.h_pairs.data(), j.h_pairs.size() * sizeof(int2),
                                     cudaMemcpyHostToDevice, P->stream));
  if (!j.h_items.empty()) {
    if ((st = dalloc(P, (void**)&j.d_items, j.h_items.size() * sizeof(int4))) != KPME_OK) return st;
    if ((st = dalloc(P, (void**)&j.d_cta, j.h_cta.size() * sizeof(int))) != KPME_OK) return st;
    KPME_CUDA_TRY(P, cudaMemcpyAsync(j.d_items, j.h_items.data(), j.h_items.size() * sizeof(int4),
                                     cudaMemcpyHostToDevice, P->stream));
    KPME_CUDA_TRY(P, cudaMemcpyAsync(j.d_cta, j.h_cta.data(), j.h_cta.size() * sizeof(int),
                                     cudaMemcpyHostToDevice, P->stream));
  }
  return KPME_OK;
}

void release_skp_buffers(kpme_plan_t P) {
  auto drop = [&](void*& p) {
    dfree(p);
  };
  drop(P->d_fac3);
  drop(P->d_fac2);
  drop(P->d_fac1);
  drop(P->d_Qs);
  drop(P->d_Y);
  drop(P->d_Z);
  dfree(P->d_lmU);
  dfree(P->d_lmD);
  dfree(P->d_lmT);
  dfree(P->d_lmU2);
  dfree(P->d_lmD2);
  dfree(P->d_Qsl);
  dfree(P->d_Ysl);
  dfree(P->d_rmZ);
  dfree(P->d_rmQ);
  dfree(P->d_rmY);
  dfree(P->d_Qfold);
  dfree(P->d_facv_oz);
  free_joblist(P->vir_jobs);
  P->vir_tc = false;
  free_joblist(P->stage1);
  free_joblist(P->stage1_res);
  free_joblist(P->stage23);
  for (auto& g : P->groups) {
    free_joblist(g.stage2);
    free_joblist(g.stage3);
    free_joblist(g.stage2_res);
  }
  P->groups.clear();
}

void release_mesh_buffers(kpme_plan_t P) {
  dfree(P->d_Q);
  dfree(P->d_Qf);
  dfree(P->d_Phi);
  dfree(P->d_Psi);
  dfree(P->d_tmp1);
  dfree(P->d_tmp2);
  dfree(P->d_facv);
  dfree(P->d_facW);
  dfree(P->d_bmod);
  dfree(P->d_vt);
}

void drop_graph(kpme_plan_t P) {
  if (P->graph_exec) cudaGraphExecDestroy(P->graph_exec);
  P->graph_exec = nullptr;
}

// Tensor-core tile: BN output columns (<= 256, multiple of 16) and pipeline depth.
void choose_tc_tiles(kpme_plan_t P) {
  const int K = P->p.K;
  if (P->prec.oz) {
    // error-free split: four A slices (64 KB) + four B slices per stage, two stages
    P->tc_bn = K % 64 == 0 ? 64 : K == 96 ? 48 : K <= 96 ? K : 64;
    P->tc_stages = 2;
    while (P->tc_stages > 1 && oz_smem_bytes(P->tc_bn, P->tc_stages) > 227 * 1024) --P->tc_stages;
    return;
  }
  int bn = K;
  while (bn > 256 || (tc_smem_bytes(P->prec, bn, 2) > 220 * 1024 && bn % 32 == 0)) bn /= 2;
  P->tc_bn = bn;
  int stages = 4;
  while (stages > 1 && tc_smem_bytes(P->prec, bn, stages) > 220 * 1024) --stages;
  P->tc_stages = stages;
}

// Device memory for the Z planes of one term group (stages 2 and 3 run once per group).  For
// the error-free split, fewer and larger groups mean fewer launch tails and longer runs of
// terms sharing their A: by default up to 12 GiB, at most a quarter of the free device memory
// (the 10^6-charge box, R = 167 planes of 67 MB, then runs one group: 70.3 -> 77.7
// evaluations/s against 16-term groups).  The other forms keep 256 MB: their split-K sums over
// a group's terms run in float32, and longer sums cost accuracy (FP32 at 10^6 charges: phi
// 5.3e-7 with 16-term groups, 1.7e-6 with one group).  KPME_GROUP_MB overrides both.
int64_t group_budget_bytes(bool error_free) {
  const char* e = getenv("KPME_GROUP_MB");
  if (e) {
    int64_t mb = atoll(e);
    if (mb < 1) mb = 1;
    return mb << 20;
  }
  if (!error_free) return (int64_t)256 << 20;
  size_t free_b = 0, total_b = 0;
  int64_t budget = (int64_t)12 << 30;
  if (cudaMemGetInfo(&free_b, &total_b) == cudaSuccess) budget = std::min<int64_t>(budget, (int64_t)(free_b / 4));
  return std::max<int64_t>(budget, (int64_t)256 << 20);
}

kpme_status_t alloc_meshes(kpme_plan_t P) {
  release_mesh_buffers(P);
  const size_t b = (size_t)K3(P) * mesh_elem(P);
  kpme_status_t st;
  if ((st = dalloc(P, (void**)&P->d_Q, (size_t)K3(P) * sizeof(double))) != KPME_OK) return st;
  if (!P->prec.fp64 && (st = dalloc(P, (void**)&P->d_Qf, (size_t)K3(P) * sizeof(float))) != KPME_OK) return st;
  if ((st = dalloc(P, &P->d_Phi, b)) != KPME_OK) return st;
  if ((st = dalloc(P, &P->d_Psi, b)) != KPME_OK) return st;
  if ((st = dalloc(P, &P->d_tmp1, b)) != KPME_OK) return st;
  if ((st = dalloc(P, &P->d_tmp2, b)) != KPME_OK) return st;
  if (kpme::lagrange(P)) return KPME_OK;   // the virial operators are B-spline mesh operators
  // rank-one virial operator (CUDA-core format of the plan's mesh)
  double* dg = nullptr;
  if ((st = dalloc(P, (void**)&dg, P->p.K * sizeof(double))) != KPME_OK) return st;
  cudaError_t e = launch_virial_generator(P, dg);
  if (e == cudaSuccess) {
    if ((st = dalloc(P, &P->d_facv, (size_t)P->p.K * P->p.K * mesh_elem(P))) != KPME_OK) {
      cudaFree(dg);
      return st;
    }
    e = launch_materialize(P, dg, 1, P->d_facv, 1, P->prec.fp64 ? 0 : 1);
    if (e == cudaSuccess) e = cudaStreamSynchronize(P->stream);
  }
  cudaFree(dg);
  P->scratch_bytes -= P->p.K * sizeof(double);
  if (e != cudaSuccess) {
    P->last_error = std::string("virial operator: ") + cudaGetErrorString(e);
    return KPME_ERR_CUDA;
  }
  // mode-space virial tensor: real DFT matrix, B-spline moduli, float64 sums
  if ((st = dalloc(P, &P->d_facW, (size_t)P->p.K * P->p.K * mesh_elem(P))) != KPME_OK) return st;
  if ((st = dalloc(P, (void**)&P->d_bmod, (size_t)(P->p.K / 2 + 1) * sizeof(double))) != KPME_OK) return st;
  if ((st = dalloc(P, (void**)&P->d_vt, 8 * sizeof(double))) != KPME_OK) return st;
  e = launch_dft_matrix(P, P->d_facW);
  if (e == cudaSuccess) e = launch_bmod(P, P->d_bmod);
  if (e == cudaSuccess) e = cudaStreamSynchronize(P->stream);
  if (e != cudaSuccess) {
    P->last_error = std::string("virial tensor operator: ") + cudaGetErrorString(e);
    return KPME_ERR_CUDA;
  }
  return KPME_OK;
}

// Materialise the installed SKP in the plan's arithmetic: factors, intermediates, job lists
// and (tensor path) TMA descriptors.
bool getenv_flag(const char* name, bool dflt) {
  const char* e = getenv(name);
  if (!e || !*e) return dflt;
  return e[0] != '0';
}

}  // namespace

// Spreading tile edge T: divides K, covers the stencil halo (T >= n - 1) and its staged
// region (T + n - 1)^3 float32 fits in shared memory.
bool kpme::tile_ok(int K, int order, int T) {
  const int D = T + order - 1;
  return T >= 1 && K % T == 0 && T >= order - 1 && (size_t)D * D * D * sizeof(float) <= 200 * 1024;
}

// (Re)allocate the cell-sort counters for tile edge T (8 counters per tile).
kpme_status_t kpme::set_tile(kpme_plan_t P, int T) {
  if (!tile_ok(P->p.K, P->p.order, T)) return KPME_ERR_INVALID_ARG;
  if (T == P->tile && P->d_tcount) return KPME_OK;
  dfree(P->d_tcount);
  dfree(P->d_tstart);
  const int kt = P->p.K / T;
  const size_t nt = (size_t)kt * kt * kt;
  kpme_status_t st;
  if ((st = dalloc(P, (void**)&P->d_tcount, nt * kTileCounters * sizeof(int))) != KPME_OK) return st;
  if ((st = dalloc(P, (void**)&P->d_tstart, (nt * kTileCounters + 1) * sizeof(int))) != KPME_OK) return st;
  P->tile = T;
  drop_graph(P);
  return KPME_OK;
}

// Cell-sorted, tile-staged spreading and gathering (sorted) or float32 atomics on the mesh and
// untiled gathering with no sort (the autotuner's choice on every workload measured here).
kpme_status_t kpme::set_sorted(kpme_plan_t P, bool sorted) {
  if (sorted && P->tile <= 0) return KPME_ERR_INVALID_ARG;
  if (P->no_sort != !sorted) {
    P->no_sort = !sorted;
    drop_graph(P);
  }
  return KPME_OK;
}

namespace kpme {

// Jobs over runs of pairs that share their A operand: every run [a, b) is cut into pieces
// of at most J pairs, J chosen so that the persistent grid's makespan, rounds of
// ceil(items / SMs) times (J + 1) (one pair's worth for cutting A), is smallest.
template <typename PairOf>
void build_run_jobs(kpme_plan_t P, const std::vector<std::pair<int, int>>& runs, int64_t tiles, PairOf pair_of,
                    JobList& jl) {
  int maxlen = 1;
  for (const auto& r : runs) maxlen = std::max(maxlen, r.second - r.first);
  int bestJ = maxlen;
  int64_t best = INT64_MAX;
  for (int J = 1; J <= maxlen; ++J) {
    int64_t jobs = 0;
    for (const auto& r : runs) jobs += (r.second - r.first + J - 1) / J;
    const int64_t rounds = (tiles * jobs + P->sm_count - 1) / P->sm_count;
    const int64_t cost = rounds * (J + 1);
    if (cost < best) {
      best = cost;
      bestJ = J;
    }
  }
  jl.h_start.assign(1, 0);
  jl.h_pairs.clear();
  for (const auto& r : runs) {
    const int len = r.second - r.first;
    const int pieces = (len + bestJ - 1) / bestJ;
    for (int k = 0; k < pieces; ++k) {
      const int a = r.first + (int)((int64_t)len * k / pieces), b = r.first + (int)((int64_t)len * (k + 1) / pieces);
      for (int t = a; t < b; ++t) jl.h_pairs.push_back(pair_of(t));
      jl.h_start.push_back((int)jl.h_pairs.size());
    }
  }
}

kpme_status_t install_skp(kpme_plan_t P) {
  drop_graph(P);
  release_skp_buffers(P);
  const SkpHost& S = P->skp;
  if (!S.valid) return KPME_OK;
  if (lagrange_modes(P)) {   // Fourier rows, the diagonal and the transforms' scratch
    const int K = P->p.K, r = 2 * P->p.modes + 1;
    kpme_status_t s2;
    if ((s2 = dalloc(P, (void**)&P->d_lmU, S.modal_U.size() * sizeof(double))) != KPME_OK) return s2;
    if ((s2 = dalloc(P, (void**)&P->d_lmD, S.modal_D.size() * sizeof(double))) != KPME_OK) return s2;
    const size_t nt = (size_t)r * K * K + 2 * (size_t)r * r * K + (size_t)r * r * r;
    if ((s2 = dalloc(P, (void**)&P->d_lmT, nt * sizeof(double))) != KPME_OK) return s2;
    KPME_CUDA_TRY(P, cudaMemcpyAsync(P->d_lmU, S.modal_U.data(), S.modal_U.size() * sizeof(double),
                                     cudaMemcpyHostToDevice, P->stream));
    KPME_CUDA_TRY(P, cudaMemcpyAsync(P->d_lmD, S.modal_D.data(), S.modal_D.size() * sizeof(double),
                                     cudaMemcpyHostToDevice, P->stream));
    // double-float pairs (hi = float32 rounding, lo = float32 rounding of the rest)
    auto pairs = [](const std::vector<double>& v) {
      std::vector<float2> o(v.size());
      for (size_t i = 0; i < v.size(); ++i) {
        const float hi = (float)v[i];
        o[i] = make_float2(hi, (float)(v[i] - (double)hi));
      }
      return o;
    };
    const std::vector<float2> U2 = pairs(S.modal_U), D2 = pairs(S.modal_D);
    if ((s2 = dalloc(P, &P->d_lmU2, U2.size() * sizeof(float2))) != KPME_OK) return s2;
    if ((s2 = dalloc(P, &P->d_lmD2, D2.size() * sizeof(float2))) != KPME_OK) return s2;
    KPME_CUDA_TRY(P, cudaMemcpyAsync(P->d_lmU2, U2.data(), U2.size() * sizeof(float2), cudaMemcpyHostToDevice,
                                     P->stream));
    KPME_CUDA_TRY(P, cudaMemcpyAsync(P->d_lmD2, D2.data(), D2.size() * sizeof(float2), cudaMemcpyHostToDevice,
                                     P->stream));
    KPME_CUDA_TRY(P, cudaStreamSynchronize(P->stream));
    return KPME_OK;
  }
  const int K = P->p.K, r0 = S.r0, R = S.R;
  const int64_t k3 = K3(P);
  const PrecInfo& pi = P->prec;
  const int slices = pi.tensor ? pi.slices : 1;
  const size_t eb = pi.tensor ? (size_t)pi.elem_bytes : mesh_elem(P);
  const int kind = pi.oz ? 4 : pi.tensor ? (pi.tf32 ? 3 : 2) : (pi.fp64 ? 0 : 1);
  kpme_status_t st;
  // error-free split on circulant factors with K/2 a multiple of the 64-wide k chunk: the
  // factors in the reflection basis (two K/2 x K/2 blocks each), half the digit products
  P->fold = pi.oz && P->allow_fold && P->ozt_mode > 0 && !S.dense && K % 128 == 0 && ozt_supported(K, 64, true, true);
  const int kcols = P->fold ? K / 2 : K;   // stored columns of a factor row

  // factors
  auto mat = [&](const std::vector<double>& gen, int count, void** dst) -> kpme_status_t {
    kpme_status_t s2;
    if ((s2 = dalloc(P, dst, (size_t)slices * count * K * kcols * eb)) != KPME_OK) return s2;
    double* dg = nullptr;
    KPME_CUDA_TRY(P, cudaMalloc((void**)&dg, gen.size() * sizeof(double)));
    cudaError_t e = cudaMemcpyAsync(dg, gen.data(), gen.size() * sizeof(double), cudaMemcpyHostToDevice, P->stream);
    double* dmax = nullptr;
    if (S.dense) {   // dense factor matrices: one power of two per factor from its largest entry
      std::vector<double> gmax(count, 0.0);
      const size_t KK = (size_t)K * K;
      for (int t = 0; t < count; ++t)
        for (size_t i = 0; i < KK; ++i) gmax[t] = std::max(gmax[t], std::fabs(gen[(size_t)t * KK + i]));
      if (e == cudaSuccess) e = cudaMalloc((void**)&dmax, count * sizeof(double));
      if (e == cudaSuccess)
        e = cudaMemcpyAsync(dmax, gmax.data(), count * sizeof(double), cudaMemcpyHostToDevice, P->stream);
      if (e == cudaSuccess) e = launch_materialize_dense(P, dg, dmax, count, *dst, slices, kind);
      if (e == cudaSuccess) e = cudaStreamSynchronize(P->stream);
      cudaFree(dmax);
      cudaFree(dg);
      KPME_CUDA_TRY(P, e);
      return KPME_OK;
    }
    if (e == cudaSuccess) e = launch_materialize(P, dg, count, *dst, slices, kind);
    if (e == cudaSuccess) e = cudaStreamSynchronize(P->stream);
    cudaFree(dg);
    KPME_CUDA_TRY(P, e);
    return KPME_OK;
  };
  if ((st = mat(S.gen3, r0, &P->d_fac3)) != KPME_OK) return st;
  if ((st = mat(S.gen2, R, &P->d_fac2)) != KPME_OK) return st;
  if ((st = mat(S.gen1, R, &P->d_fac1)) != KPME_OK) return st;

  // intermediates (the error-free split keeps float32 values and per-row maxima)
  const int islices = pi.oz ? 1 : slices;
  const size_t ieb = pi.oz ? sizeof(float) : eb;
  // terms per group: as many as fit the budget (L2-sized by default), but at least 16 so that
  // large meshes do not degenerate into one launch pair per term
  int G = (int)std::max<int64_t>(16, group_budget_bytes(pi.oz) / std::max<int64_t>(1, (int64_t)islices * k3 * (int64_t)ieb));
  G = std::min(G, R);
  P->group_terms = G;
  if (pi.tensor && !pi.oz && (st = dalloc(P, &P->d_Qs, (size_t)slices * k3 * eb)) != KPME_OK) return st;
  if ((st = dalloc(P, &P->d_Y, (size_t)islices * r0 * k3 * ieb)) != KPME_OK) return st;
  if (pi.tensor) choose_tc_tiles(P);
  // in the reflection basis an item can cover a whole half of the output columns when the half
  // is 128 wide: N = 128 MMAs, half the MMA instructions per flop (KPME_BN128=0 keeps 64)
  if (P->fold && K / 2 == 128 && getenv_flag("KPME_BN128", true) && ozt_supported(K, 128, true, true) &&
      ozt_supported(K, 128, false, true))
    P->tc_bn = 128;
  // the tensor-memory-A kernel where K % 32 == 0; at other K % 16 == 0 (e.g. 48) it is correct
  // but the shared-memory-A kernel stays the default: a K = 48 system alone ran 3-5% faster on
  // it, the 64-system batch (26 systems at K = 48) 3% slower (5.72 against 5.56 ms)
  const bool ozt_k = P->ozt_mode >= 2 || (P->ozt_mode == 1 && K % 32 == 0);
  P->ozt_res = pi.oz && ozt_k && ozt_supported(K, P->tc_bn, true, P->fold);
  P->ozt_pp = pi.oz && ozt_k && ozt_supported(K, P->tc_bn, false, P->fold);
  if (P->fold && !(P->ozt_res && P->ozt_pp)) return KPME_ERR_UNSUPPORTED;   // excluded above
  P->ozf = P->ozt_res && ozf_supported(K) && P->tc_bn == K && P->allow_fused;
  if (pi.oz) {
    const size_t k2 = (size_t)K * K;
    if (P->ozt_res) {
      // A in tensor memory: Q and Y stay float32 and are cut by converter warps once per
      // item (shared by the item's pairs) with their row maxima
      if ((st = dalloc(P, (void**)&P->d_rmQ, k2 * sizeof(float))) != KPME_OK) return st;
      if (P->fold && (st = dalloc(P, (void**)&P->d_Qfold, (size_t)k3 * sizeof(float))) != KPME_OK) return st;
      if ((st = dalloc(P, (void**)&P->d_rmY, (size_t)r0 * k2 * sizeof(float))) != KPME_OK) return st;
    } else {
      // Q and Y are read by several jobs each: they are cut into fixed-point slices once and
      // fed by TMA
      if ((st = dalloc(P, &P->d_Qsl, (size_t)4 * k3 * sizeof(__nv_bfloat16))) != KPME_OK) return st;
      if ((st = dalloc(P, &P->d_Ysl, (size_t)4 * r0 * k3 * sizeof(__nv_bfloat16))) != KPME_OK) return st;
    }
    // Z is read once per term and is cut on the fly from float32 with its row maxima (the
    // fused kernel keeps Z on the SM)
    if (!P->ozf && (st = dalloc(P, (void**)&P->d_rmZ, (size_t)G * k2 * sizeof(float))) != KPME_OK) return st;
  }
  if (!(pi.oz && P->ozf) && (st = dalloc(P, &P->d_Z, (size_t)islices * G * k3 * ieb)) != KPME_OK) return st;

  // job lists
  P->stage1.h_start.clear();
  P->stage1.h_pairs.clear();
  for (int i = 0; i <= r0; ++i) P->stage1.h_start.push_back(i);
  for (int i = 0; i < r0; ++i) P->stage1.h_pairs.push_back(make_int2(0, i));
  if ((st = upload_joblist(P, P->stage1)) != KPME_OK) return st;

  const int m_tiles = pi.tensor ? (K * K + 127) / 128 : (K * K + 63) / 64;
  const int n_tiles = pi.tensor ? K / P->tc_bn : (K + 63) / 64;
  for (int t0 = 0; t0 < R; t0 += G) {
    TermGroup g;
    g.t0 = t0;
    g.t1 = std::min(R, t0 + G);
    const int nt = g.t1 - g.t0;
    for (int t = g.t0; t <= g.t1; ++t) g.stage2.h_start.push_back(t - g.t0);
    for (int t = g.t0; t < g.t1; ++t) g.stage2.h_pairs.push_back(make_int2(S.outer_of[t], t));
    // split-K over terms.  Floating-slice tensor forms accumulate a split's terms in the
    // tensor core's truncating float32 accumulator, so they keep many short splits.  The
    // other forms (error-free split: one drain per term; CUDA cores) take the split count
    // with the smallest makespan: ceil(items / SMs) rounds of ceil(nt / splits) terms, plus
    // about one term's worth of per-item work (the final atomic accumulation).
    int splits = (2 * P->sm_count + m_tiles * n_tiles - 1) / (m_tiles * n_tiles);
    splits = std::max(1, std::min(splits, nt));
    if (!pi.tensor || pi.oz) {
      const int64_t tiles = (int64_t)m_tiles * n_tiles;
      int64_t best = INT64_MAX;
      for (int sp = 1; sp <= nt; ++sp) {
        const int64_t rounds = (tiles * sp + P->sm_count - 1) / P->sm_count;
        const int64_t cost = rounds * ((nt + sp - 1) / sp + 1);
        if (cost < best) {
          best = cost;
          splits = sp;
        }
      }
    }
    splits = std::max(1, std::min(nt, splits * P->tune_split / 2));
    g.splits = splits;
    int pos = 0;
    g.stage3.h_start.push_back(0);
    for (int s = 0; s < splits; ++s) {
      const int a = g.t0 + (int)((int64_t)nt * s / splits), b = g.t0 + (int)((int64_t)nt * (s + 1) / splits);
      for (int t = a; t < b; ++t) g.stage3.h_pairs.push_back(make_int2(t - g.t0, t));
      pos += b - a;
      g.stage3.h_start.push_back(pos);
    }
    if (P->ozt_res) {
      // runs of consecutive terms of one outer index share Y_i: chunked for a balanced grid
      std::vector<std::pair<int, int>> runs;   // [first term, end)
      for (int t = g.t0; t < g.t1;) {
        int e = t + 1;
        while (e < g.t1 && S.outer_of[e] == S.outer_of[t]) ++e;
        runs.push_back({t, e});
        t = e;
      }
      build_run_jobs(P, runs, (int64_t)m_tiles * n_tiles, [&](int t) { return make_int2(S.outer_of[t], t); },
                     g.stage2_res);
      if ((st = upload_joblist(P, g.stage2_res)) != KPME_OK) return st;
    }
    if ((st = upload_joblist(P, g.stage2)) != KPME_OK) return st;
    if ((st = upload_joblist(P, g.stage3)) != KPME_OK) return st;
    P->groups.push_back(std::move(g));
  }
  if (P->ozt_res) {
    build_run_jobs(P, {{0, r0}}, (int64_t)m_tiles * n_tiles, [&](int i) { return make_int2(0, i); }, P->stage1_res);
    if ((st = upload_joblist(P, P->stage1_res)) != KPME_OK) return st;
  }
  if (P->ozf) {
    // fused stages 2 and 3: a static schedule.  The m_tiles x R (tile, term) steps, tile-major,
    // are cut into one contiguous range per CTA of equal cost: a step costs 1, plus 0.4 where
    // its term starts a run of a new outer index (the cut of the Y_i digits stalls step 2 for
    // about 0.4 of a term).  A range that crosses a tile boundary becomes two items.  Within
    // an item the terms run in order, so the consecutive terms of one outer index share a
    // cut of Y_i.  (The split knob scales the grid: x1/2, x1, x2 of the SM count; a batch of
    // concurrent systems may prefer fewer, longer CTAs.)
    P->stage23.h_pairs.clear();
    for (int t = 0; t < R; ++t) P->stage23.h_pairs.push_back(make_int2(S.outer_of[t], t));
    P->stage23.h_start = {0, R};
    const int64_t steps = (int64_t)m_tiles * R;
    const int grid = (int)std::min<int64_t>(std::max(1, P->sm_count * P->tune_split / 2), steps);
    constexpr double kCutCost = 0.4;
    std::vector<double> term_cost(R);
    double tile_cost = 0.0;
    for (int t = 0; t < R; ++t) {
      term_cost[t] = 1.0 + ((t == 0 || S.outer_of[t] != S.outer_of[t - 1]) ? kCutCost : 0.0);
      tile_cost += term_cost[t];
    }
    const double total = tile_cost * m_tiles;
    P->stage23.h_items.clear();
    P->stage23.h_cta.assign(1, 0);
    int64_t pos = 0;   // next step (tile-major)
    double done = 0.0;
    for (int c = 0; c < grid; ++c) {
      const double target = total * (c + 1) / grid;
      int64_t end = pos;
      double acc = done;
      // take steps while the cost stays at or below the target (the last CTA takes the rest)
      while (end < steps && (c == grid - 1 || acc + term_cost[end % R] * 0.5 <= target)) {
        acc += term_cost[end % R];
        ++end;
      }
      if (end == pos && end < steps && steps - end > grid - 1 - c) {   // every CTA gets a step if it can
        acc += term_cost[end % R];
        ++end;
      }
      int64_t a = pos;
      while (a < end) {
        const int tile = (int)(a / R), t0 = (int)(a % R);
        const int t1 = (int)std::min<int64_t>(R, t0 + (end - a));
        P->stage23.h_items.push_back(make_int4(tile, t0, t1, 0));
        a += t1 - t0;
      }
      P->stage23.h_cta.push_back((int)P->stage23.h_items.size());
      pos = end;
      done = acc;
    }
    if ((st = upload_joblist(P, P->stage23)) != KPME_OK) return st;
  }

  if (pi.tensor) {
    const bool f32 = pi.tf32;
    const uint32_t box0 = 128 / pi.elem_bytes;
    const uint64_t KK = (uint64_t)K * K;
    bool ok = (pi.oz ? (P->ozt_res || (encode_tmap(P, &P->tm_Q, P->d_Qsl, 2, false, K, KK, 4, 64, 128) &&
                                        encode_tmap(P, &P->tm_Y, P->d_Ysl, 2, false, K, KK, (uint64_t)4 * r0, 64, 128)))
                     : (encode_tmap(P, &P->tm_Q, P->d_Qs, pi.elem_bytes, f32, K, KK, (uint64_t)slices, box0, 128) &&
                encode_tmap(P, &P->tm_Y, P->d_Y, pi.elem_bytes, f32, K, KK, (uint64_t)slices * r0, box0, 128) &&
                encode_tmap(P, &P->tm_Z, P->d_Z, pi.elem_bytes, f32, K, KK, (uint64_t)slices * G, box0, 128))) &&
              encode_tmap(P, &P->tm_f3, P->d_fac3, pi.elem_bytes, f32, kcols, (uint64_t)r0 * K, slices, box0,
                          P->tc_bn) &&
              encode_tmap(P, &P->tm_f2, P->d_fac2, pi.elem_bytes, f32, kcols, (uint64_t)R * K, slices, box0,
                          P->tc_bn) &&
              encode_tmap(P, &P->tm_f1, P->d_fac1, pi.elem_bytes, f32, kcols, (uint64_t)R * K, slices, box0,
                          P->tc_bn);
    if (ok && pi.oz && (P->ozt_res || P->ozt_pp)) {
      // float32 A operands for the tensor-memory kernel: 128 rows x 32 values per box
      ok = (P->ozf || encode_tmap(P, &P->tmF_Z, P->d_Z, 4, true, K, KK, (uint64_t)G, 32, 128)) &&
           (!P->ozt_res || (encode_tmap(P, &P->tmF_Q, P->fold ? P->d_Qfold : P->d_Qf, 4, true, K, KK, 1, 32, 128) &&
                            encode_tmap(P, &P->tmF_Y, P->d_Y, 4, true, K, KK, (uint64_t)r0, 32, 128)));
    }
    if (!ok) return KPME_ERR_CUDA;
  }
  // the virial's rank-one operator V (x) V (x) V on the tensor cores where the SKP runs N = 128
  // items in the reflection basis: its circulant's digits in the basis, one pair per stage
  if (pi.oz && P->fold && P->tc_bn == 128 && !S.dense && !lagrange(P)) {
    double* dg = nullptr;
    if ((st = dalloc(P, (void**)&dg, (size_t)K * sizeof(double))) != KPME_OK) return st;
    if ((st = dalloc(P, &P->d_facv_oz, (size_t)slices * K * kcols * eb)) != KPME_OK) {
      cudaFree(dg);
      return st;
    }
    cudaError_t e = launch_virial_generator(P, dg);
    if (e == cudaSuccess) e = launch_materialize(P, dg, 1, P->d_facv_oz, slices, kind);
    if (e == cudaSuccess) e = cudaStreamSynchronize(P->stream);
    cudaFree(dg);
    P->scratch_bytes -= (int64_t)K * sizeof(double);
    KPME_CUDA_TRY(P, e);
    P->vir_jobs.h_start = {0, 1};
    P->vir_jobs.h_pairs = {make_int2(0, 0)};
    if ((st = upload_joblist(P, P->vir_jobs)) != KPME_OK) return st;
    if (!encode_tmap(P, &P->tm_v, P->d_facv_oz, pi.elem_bytes, false, kcols, (uint64_t)K, slices, 128 / pi.elem_bytes,
                     P->tc_bn))
      return KPME_ERR_CUDA;
    P->vir_tc = true;
  }
  KPME_CUDA_TRY(P, cudaStreamSynchronize(P->stream));
  return KPME_OK;
}

// ---- profiling helpers ----
cudaEvent_t take_event(kpme_plan_t P) {
  if (!P->event_pool.empty()) {
    cudaEvent_t e = P->event_pool.back();
    P->event_pool.pop_back();
    return e;
  }
  cudaEvent_t e = nullptr;
  cudaEventCreate(&e);
  return e;
}

// Every step is also an NVTX range (header-only NVTX3: without an attached tool a range costs a
// branch), so timeline tools show the steps of the eager evaluations and of graph capture.
const char* const kStepNames[kpme::NUM_STEPS] = {"kpme spread", "kpme split", "kpme SKP stage 1",
                                                 "kpme SKP stage 2", "kpme SKP stage 3", "kpme gather",
                                                 "kpme virial"};

struct StepScope {
  kpme_plan_t P;
  int step;
  cudaEvent_t a = nullptr;
  int launches;
  StepScope(kpme_plan_t p, int s, int nl) : P(p), step(s), launches(nl) {
    nvtxRangePushA(kStepNames[step]);
    if (P->profiling) {
      a = take_event(P);
      cudaEventRecord(a, P->stream);
    }
  }
  ~StepScope() {
    nvtxRangePop();
    P->launches += launches;
    if (P->profiling) {
      cudaEvent_t b = take_event(P);
      cudaEventRecord(b, P->stream);
      P->pending.push_back({step, {a, b}});
      P->prof_launch[step] += launches;
    }
  }
};

kpme_status_t check_device_status(kpme_plan_t P) {
  // the status word lives in mapped pinned host memory: readable without a synchronisation
  volatile int* h = reinterpret_cast<volatile int*>(P->d_status);
  if (h && *h >= kDevBounds) {
    static const char* const names[NUM_SITES] = {"", "no-sort spreading", "tile spreading", "tile region merge",
                                                 "gathering", "tile gathering", "cell count", "cell scatter"};
    const int site = *h - kDevBounds;
    *h = DEV_OK;
    P->last_error = std::string("device index check failed: ") + (site > 0 && site < NUM_SITES ? names[site] : "?");
    return KPME_ERR_CUDA;
  }
  if (h && *h != DEV_OK) {
    *h = DEV_OK;
    P->last_error = "a bounded device wait gave up";
    // a shortened budget (KPME_FAULT=budget) has done its work: later launches, and a graph
    // captured again, get the production budget
    if (P->wait_cycles != kWaitCycles) {
      P->wait_cycles = kWaitCycles;
      drop_graph(P);
    }
    return KPME_ERR_TIMEOUT;
  }
  return KPME_OK;
}

// The charge mesh handed to the mode products: float64 (FP64 form, untiled fallback, stage
// entry points) or float32 (cell-sorted spreading).
struct MeshRef {
  const void* p;
  bool dbl;
};

// Phi: float32 (float64 for the FP64 form).
kpme_status_t contract(kpme_plan_t P, MeshRef Q, void* Phi) {
  const int K = P->p.K;
  const int M = K * K;
  const int64_t k3 = K3(P);
  const PrecInfo& pi = P->prec;
  const SkpHost& S = P->skp;
  if (lagrange_modes(P)) {   // five transform launches in double-float, six in float64
    StepScope sc(P, STEP_SKP1, pi.fp64 ? 6 : 5);
    KPME_CUDA_TRY(P, launch_lagrange_modes(P, Q.p, Q.dbl, Phi, pi.fp64));
    return KPME_OK;
  }
  if (!pi.tensor) {
    const bool dbl = pi.fp64;
    const void* Qin = Q.p;
    if (!dbl && Q.dbl) {
      StepScope sc(P, STEP_SPLIT, 1);
      KPME_CUDA_TRY(P, launch_convert(Q.p, true, P->d_Qf, false, k3, P->stream));
      Qin = P->d_Qf;
    }
    {
      StepScope sc(P, STEP_SKP1, 1);
      KPME_CUDA_TRY(P, launch_mp_simt(dbl, Qin, 0, P->d_fac3, P->d_Y, k3, M, K, K, P->stage1, 0, P->stream));
    }
    KPME_CUDA_TRY(P, cudaMemsetAsync(Phi, 0, (size_t)k3 * mesh_elem(P), P->stream));
    for (const auto& g : P->groups) {
      {
        StepScope sc(P, STEP_SKP2, 1);
        KPME_CUDA_TRY(P, launch_mp_simt(dbl, P->d_Y, k3, P->d_fac2, P->d_Z, k3, M, K, K, g.stage2, 0, P->stream));
      }
      StepScope sc(P, STEP_SKP3, 1);
      KPME_CUDA_TRY(P, launch_mp_simt(dbl, P->d_Z, k3, P->d_fac1, Phi, 0, M, K, K, g.stage3, 1, P->stream));
    }
    (void)S;
    return KPME_OK;
  }
  if (pi.oz) {
    const int64_t k2 = (int64_t)K * K;
    const bool res = P->ozt_res;
    // N = 128 items in the reflection basis: the stage kernels take the rows' powers of two
    // from the staged rows (over the half an item contracts), so no stage publishes row maxima
    const bool self_max = P->fold && P->tc_bn == 128;
    if (res && P->fold) {
      // the charge mesh in the reflection basis of its three axes (float32; the same launch
      // clears Phi, which the following stages accumulate into) and its row maxima
      StepScope sc(P, STEP_SPLIT, self_max ? 1 : 2);
      KPME_CUDA_TRY(P, launch_fold_mesh(P, Q.p, Q.dbl, P->d_Qfold, K, (float*)Phi, k3));
      if (!self_max) KPME_CUDA_TRY(P, launch_rowmax_rows(P, P->d_Qfold, k2, K, P->d_rmQ));
    } else if (res) {
      // float32 charge mesh and its row maxima (rows of stage 1)
      StepScope sc(P, STEP_SPLIT, Q.dbl ? 2 : 1);
      if (Q.dbl) KPME_CUDA_TRY(P, launch_convert(Q.p, true, P->d_Qf, false, k3, P->stream));
      // (the same launch clears Phi, which the following stages accumulate into)
      KPME_CUDA_TRY(P, launch_rowmax_rows(P, P->d_Qf, k2, K, P->d_rmQ, (float*)Phi, k3));
    } else {
      StepScope sc(P, STEP_SPLIT, 1);
      KPME_CUDA_TRY(P, launch_slice_rows(P, Q.p, Q.dbl, k2, 1, K, P->d_Qsl));
    }
    if (res && P->ozf) {
      // stage 1, then stages 2 and 3 fused (Z stays on the SM; its rows' powers of two are
      // taken by the fused kernel itself, so stage 1 publishes no row maxima)
      {
        StepScope sc(P, STEP_SKP1, 1);
        OztArgs a{&P->tmF_Q, &P->tm_f3, P->d_rmQ, 0, (float*)P->d_Y, k3, 0, nullptr, 0, M, K, K, 2, true,
                  &P->stage1_res};
        KPME_CUDA_TRY(P, launch_mp_ozt(P, a));
      }
      StepScope sc(P, STEP_SKP2, 1);
      OzfArgs a{(const float*)P->d_Y, &P->tm_f2, &P->tm_f1, (float*)Phi, K, &P->stage23};
      KPME_CUDA_TRY(P, launch_mp_ozf(P, a));
      return KPME_OK;
    }
    if (res) {
      if (!self_max) KPME_CUDA_TRY(P, cudaMemsetAsync(P->d_rmY, 0, (size_t)S.r0 * k2 * sizeof(float), P->stream));
      StepScope sc(P, STEP_SKP1, 1);
      OztArgs a{&P->tmF_Q, &P->tm_f3, P->d_rmQ, 0, (float*)P->d_Y, k3, 0, self_max ? nullptr : P->d_rmY, k2, M, K,
                K, 2, true, &P->stage1_res};
      a.fold = P->fold;
      a.self_max = self_max;
      KPME_CUDA_TRY(P, launch_mp_ozt(P, a));
    } else {
      {
        StepScope sc(P, STEP_SKP1, 1);
        OzArgs a{&P->tm_f3, &P->tm_Q, 1, nullptr, false, 0, nullptr, 0, (float*)P->d_Y, k3, nullptr, 0, M, K, K, 0,
                 &P->stage1};
        KPME_CUDA_TRY(P, launch_mp_oz(P, a));
      }
      StepScope sc(P, STEP_SPLIT, 1);
      KPME_CUDA_TRY(P, launch_slice_rows(P, P->d_Y, false, k2, S.r0, K, P->d_Ysl));
    }
    if (!res) KPME_CUDA_TRY(P, cudaMemsetAsync(Phi, 0, (size_t)k3 * sizeof(float), P->stream));   // else cleared above
    // K = 256 in the reflection basis: a stage-3 half-row is one column of one 128 x 128 tile
    // of stage 2, which stores each tile's max |value| (plain stores, no clearing) for the
    // power of two of the rows that read it; stage 3 then needs no pass over its staged rows
    const bool tile_max = self_max && P->allow_tile_max && P->ozt_pp && P->d_rmZ && K == 256;
    const int64_t tm_bs = (int64_t)(k2 / 128) * (K / 128);   // tiles per plane
    for (const auto& g : P->groups) {
      if (!self_max)
        KPME_CUDA_TRY(P, cudaMemsetAsync(P->d_rmZ, 0, (size_t)(g.t1 - g.t0) * k2 * sizeof(float), P->stream));
      {
        StepScope sc(P, STEP_SKP2, 1);
        if (res) {
          OztArgs a{&P->tmF_Y, &P->tm_f2, P->d_rmY, k2, (float*)P->d_Z, k3, g.t0,
                    tile_max ? P->d_rmZ : (self_max ? nullptr : P->d_rmZ), tile_max ? tm_bs : k2, M, K, K, 2, true,
                    &g.stage2_res};
          a.fold = P->fold;
          a.self_max = self_max;
          a.tile_max = tile_max;
          KPME_CUDA_TRY(P, launch_mp_ozt(P, a));
        } else {
          OzArgs a{&P->tm_f2, &P->tm_Y, S.r0, nullptr, false, 0, nullptr, 0, (float*)P->d_Z, k3, P->d_rmZ, k2, M, K,
                   K, 0, &g.stage2};
          KPME_CUDA_TRY(P, launch_mp_oz(P, a));
        }
      }
      StepScope sc(P, STEP_SKP3, 1);
      if (P->ozt_pp) {
        OztArgs a{&P->tmF_Z, &P->tm_f1, P->d_rmZ, tile_max ? tm_bs : k2, (float*)Phi, 0, 0, nullptr, 0, M, K, K, 1,
                  false, &g.stage3};
        a.fold = P->fold;
        a.self_max = self_max && !tile_max;
        a.tile_max = tile_max;
        KPME_CUDA_TRY(P, launch_mp_ozt(P, a));
      } else {
        OzArgs a{&P->tm_f1, nullptr, 0, P->d_Z, false, k3, P->d_rmZ, k2, (float*)Phi, 0, nullptr, 0, M, K, K, 1,
                 &g.stage3};
        KPME_CUDA_TRY(P, launch_mp_oz(P, a));
      }
    }
    if (P->fold) {   // Phi back from the reflection basis (in place)
      StepScope sc(P, STEP_SKP3, 1);
      KPME_CUDA_TRY(P, launch_unfold_mesh(P, (float*)Phi, K));
    }
    return KPME_OK;
  }
  {
    StepScope sc(P, STEP_SPLIT, 1);
    KPME_CUDA_TRY(P, launch_split(P, Q.p, Q.dbl, P->d_Qs, k3));
  }
  {
    StepScope sc(P, STEP_SKP1, 1);
    TcArgs a{&P->tm_Q, &P->tm_f3, 1, P->d_Y, (int64_t)S.r0 * k3, M, K, K, 0, &P->stage1};
    KPME_CUDA_TRY(P, launch_mp_tc(P, a));
  }
  KPME_CUDA_TRY(P, cudaMemsetAsync(Phi, 0, (size_t)k3 * sizeof(float), P->stream));
  for (const auto& g : P->groups) {
    {
      StepScope sc(P, STEP_SKP2, 1);
      TcArgs a{&P->tm_Y, &P->tm_f2, S.r0, P->d_Z, (int64_t)P->group_terms * k3, M, K, K, 0, &g.stage2};
      KPME_CUDA_TRY(P, launch_mp_tc(P, a));
    }
    StepScope sc(P, STEP_SKP3, 1);
    TcArgs a{&P->tm_Z, &P->tm_f1, P->group_terms, Phi, 0, M, K, K, 1, &g.stage3};
    KPME_CUDA_TRY(P, launch_mp_tc(P, a));
  }
  return KPME_OK;
}

// Virial mesh part: Ψ = Q ×1 V ×2 V ×3 V with the separable kernel T' and ⟨Q, Ψ⟩ into d_qpsi.
kpme_status_t virial_mesh(kpme_plan_t P, MeshRef Q) {
  const int K = P->p.K, M = K * K;
  const int64_t k3 = K3(P);
  const bool dbl = P->prec.fp64;
  const bool conv = !dbl && Q.dbl;
  StepScope sc(P, STEP_VIRIAL, conv ? 6 : 5);
  const void* Qv = Q.p;
  if (conv) {
    KPME_CUDA_TRY(P, launch_convert(Q.p, true, P->d_Qf, false, k3, P->stream));
    Qv = P->d_Qf;
  }
  KPME_CUDA_TRY(P, launch_mp_simt(dbl, Qv, 0, P->d_facv, P->d_tmp1, 0, M, K, K, P->single, 0, P->stream));
  KPME_CUDA_TRY(P, launch_mp_simt(dbl, P->d_tmp1, 0, P->d_facv, P->d_tmp2, 0, M, K, K, P->single, 0, P->stream));
  KPME_CUDA_TRY(P, launch_mp_simt(dbl, P->d_tmp2, 0, P->d_facv, P->d_Psi, 0, M, K, K, P->single, 0, P->stream));
  KPME_CUDA_TRY(P, cudaMemsetAsync(P->d_qpsi, 0, sizeof(double), P->stream));
  KPME_CUDA_TRY(P, launch_dot(P, Qv, P->d_Psi, k3, P->d_qpsi));
  return KPME_OK;
}

// The same mesh part with Ψ = V (x) V (x) V Q applied as a one-term SKP by the tensor-core
// stage kernels (reflection basis, error-free split, the SKP's own scratch planes: it runs
// after the SKP on the plan's stream), Ψ unfolded, then ⟨Q, Ψ⟩.
kpme_status_t virial_mesh_tc(kpme_plan_t P, MeshRef Q) {
  const int K = P->p.K, M = K * K;
  const int64_t k3 = K3(P), k2 = (int64_t)K * K;
  if (Q.dbl) return KPME_ERR_UNSUPPORTED;
  StepScope sc(P, STEP_VIRIAL, 6);
  KPME_CUDA_TRY(P, cudaMemsetAsync(P->d_Psi, 0, (size_t)k3 * sizeof(float), P->stream));
  OztArgs a1{&P->tmF_Q, &P->tm_v, nullptr, 0, (float*)P->d_Y, k3, 0, nullptr, 0, M, K, K, 2, true, &P->vir_jobs};
  a1.fold = true;
  a1.self_max = true;
  KPME_CUDA_TRY(P, launch_mp_ozt(P, a1));
  OztArgs a2{&P->tmF_Y, &P->tm_v, nullptr, 0, (float*)P->d_Z, k3, 0, nullptr, 0, M, K, K, 2, true, &P->vir_jobs};
  a2.fold = true;
  a2.self_max = true;
  KPME_CUDA_TRY(P, launch_mp_ozt(P, a2));
  OztArgs a3{&P->tmF_Z, &P->tm_v, nullptr, 0, (float*)P->d_Psi, 0, 0, nullptr, 0, M, K, K, 1, false, &P->vir_jobs};
  a3.fold = true;
  a3.self_max = true;
  KPME_CUDA_TRY(P, launch_mp_ozt(P, a3));
  KPME_CUDA_TRY(P, launch_unfold_mesh(P, (float*)P->d_Psi, K));
  KPME_CUDA_TRY(P, cudaMemsetAsync(P->d_qpsi, 0, sizeof(double), P->stream));
  KPME_CUDA_TRY(P, launch_dot(P, Q.p, P->d_Psi, k3, P->d_qpsi));
  (void)k2;
  return KPME_OK;
}

// W = E − (2π²/β²)·½(⟨Q,Ψ⟩ − T'(0)(Σq)²) from the energy and the mesh part.
kpme_status_t virial_finish(kpme_plan_t P, const double* energy, double* out) {
  const double L = 2.0 * P->p.radius;
  const double t0 = 1.0 / (M_PI * L * L * L);
  const double coef = 2.0 * M_PI * M_PI / (P->p.beta * P->p.beta);
  KPME_CUDA_TRY(P, launch_virial_finalize(P, energy, P->d_qpsi, t0, coef, out));
  return KPME_OK;
}

bool tiled(kpme_plan_t P) { return !P->prec.fp64 && P->tile > 0 && !P->no_sort && !lagrange(P); }
bool lagrange(kpme_plan_t P) {
  return P->p.interp == KPME_INTERP_LAGRANGE || P->p.interp == KPME_INTERP_LAGRANGE_MODES;
}
bool lagrange_modes(kpme_plan_t P) { return P->p.interp == KPME_INTERP_LAGRANGE_MODES; }

// Charge mesh of n particles: cell sort + tile-staged float32 spreading, float32 spreading
// with no sort (lane passes, float32 atomics), or float64 atomics for the FP64 form.
// also_zero (may be NULL): a float64 accumulator of the caller cleared in the same launch.
kpme_status_t spread_mesh(kpme_plan_t P, int64_t n, const double* x, const double* q, MeshRef& out,
                          double* also_zero = nullptr) {
  const int64_t k3 = K3(P);
  if (lagrange(P)) {   // node charges Q = S_Y q of the per-cell form (every node written)
    void* Qm = P->prec.fp64 ? (void*)P->d_Q : (void*)P->d_Qf;
    KPME_CUDA_TRY(P, launch_lagrange_sort(P, n, x, P->d_sumq, also_zero));
    KPME_CUDA_TRY(P, launch_lagrange_spread(P, q, Qm, P->prec.fp64));
    out = {Qm, P->prec.fp64};
    return KPME_OK;
  }
  if (P->prec.fp64) {
    KPME_CUDA_TRY(P, cudaMemsetAsync(P->d_sumq, 0, sizeof(double), P->stream));
    if (also_zero) KPME_CUDA_TRY(P, cudaMemsetAsync(also_zero, 0, sizeof(double), P->stream));
    KPME_CUDA_TRY(P, cudaMemsetAsync(P->d_Q, 0, (size_t)k3 * sizeof(double), P->stream));
    KPME_CUDA_TRY(P, launch_spread(P, n, x, q, P->d_Q));
    out = {P->d_Q, true};
    return KPME_OK;
  }
  // the float32 mesh, the charge sum and the caller's accumulator in one launch
  KPME_CUDA_TRY(P, launch_clear(P, P->d_Qf, k3, P->d_sumq, also_zero));
  if (!tiled(P)) {
    KPME_CUDA_TRY(P, launch_spread_nosort(P, n, x, q, P->d_Qf, P->d_coords));
    out = {P->d_Qf, false};
    return KPME_OK;
  }
  KPME_CUDA_TRY(P, launch_sort(P, n, x, q, P->d_sumq));
  KPME_CUDA_TRY(P, launch_spread_tiled(P, n, q, P->d_Qf));
  out = {P->d_Qf, false};
  return KPME_OK;
}

// Potentials (and forces, energy) at n particles from the plan's potential mesh.  sorted:
// the cell sort of these positions is already in place (same call).
kpme_status_t gather_mesh(kpme_plan_t P, int64_t n, const double* x, const double* q, double* phi, double* F,
                          double* energy, bool correct, bool sorted) {
  if (lagrange(P)) {   // S_X^* of the per-cell form
    if (!correct) KPME_CUDA_TRY(P, cudaMemsetAsync(P->d_sumq, 0, sizeof(double), P->stream));
    if (!sorted) KPME_CUDA_TRY(P, launch_lagrange_sort(P, n, x, nullptr, nullptr));
    KPME_CUDA_TRY(P, launch_lagrange_gather(P, n, q, P->d_Phi, P->prec.fp64, phi, F, energy, correct));
    return KPME_OK;
  }
  if (!tiled(P)) {
    if (!correct) KPME_CUDA_TRY(P, cudaMemsetAsync(P->d_sumq, 0, sizeof(double), P->stream));
    // the same positions as the spreading of this call: its mesh coordinates are reused
    KPME_CUDA_TRY(P, launch_gather(P, n, x, q, P->d_Phi, phi, F, energy, 1.0, sorted ? P->d_coords : nullptr));
    return KPME_OK;
  }
  if (!sorted) KPME_CUDA_TRY(P, launch_sort(P, n, x, nullptr, nullptr));
  KPME_CUDA_TRY(P, launch_gather_tiled(P, n, q, (const float*)P->d_Phi, phi, F, energy, correct));
  return KPME_OK;
}

// Fault injection for the tests of the error paths, from the environment variable KPME_FAULT
// read when a plan is made (host side only; nothing is made to fault on the device):
//   alloc[:N]  the N-th device allocation of the plan (default the first) fails as out of memory;
//   plan       the plan's handle check word is spoiled before kpme_plan returns, as if the handle
//              were overwritten: every later call on it reports KPME_ERR_INVALID_ARG;
//   timeout    the device status word is raised as a bounded device wait raises it when it gives
//              up: the next call that reads it (an evaluation, kpme_build_skp) reports
//              KPME_ERR_TIMEOUT and clears it, the calls after run normally;
//   budget[:C] every bounded device wait of the plan's kernels gets a budget of C cycles
//              (default 1), so the first wait not already satisfied gives up and the kernels
//              let their copies and MMAs in flight complete, release tensor memory and return;
//              the next call reports KPME_ERR_TIMEOUT and restores the production budget.
struct FaultSpec {
  int alloc_at = 0;
  bool plan = false, timeout = false;
  long long budget = 0;
};
FaultSpec parse_fault() {
  FaultSpec f;
  const char* e = getenv("KPME_FAULT");
  if (!e || !*e) return f;
  const std::string s(e);
  const size_t colon = s.find(':');
  const std::string site = s.substr(0, colon);
  const long long arg = colon == std::string::npos ? 0 : atoll(s.c_str() + colon + 1);
  if (site == "alloc") f.alloc_at = arg > 0 ? (int)arg : 1;
  if (site == "plan") f.plan = true;
  if (site == "timeout") f.timeout = true;
  if (site == "budget") f.budget = arg > 0 ? arg : 1;
  return f;
}

bool plan_ok(kpme_plan_t P) {
  if (!P) return false;
  if (P->magic != kPlanMagic) {
    P->last_error = "corrupted plan handle";
    return false;
  }
  return true;
}

kpme_status_t common_checks(kpme_plan_t P, int64_t n) {
  if (!plan_ok(P)) return KPME_ERR_INVALID_ARG;
  if (n < 0) return KPME_ERR_INVALID_ARG;
  if (n > P->max_n) return KPME_ERR_CAPACITY;
  kpme_status_t st = check_device_status(P);
  if (st != KPME_OK) return st;
  KPME_CUDA_TRY(P, cudaSetDevice(P->device));
  return KPME_OK;
}

}  // namespace kpme

namespace kpme {
kpme_status_t plan_install_skp(kpme_plan_t P, const SkpHost& S) {
  P->skp = S;
  return install_skp(P);
}
}  // namespace kpme

extern "C" {

kpme_status_t kpme_default_params(kpme_params_t* p) {
  if (!p) return KPME_ERR_INVALID_ARG;
  memset(p, 0, sizeof(*p));
  p->radius = 1.0;
  p->beta = 0.35;
  p->order = 4;
  p->K = 32;
  p->skp_tol = 1e-8;
  p->skp_method = KPME_SKP_SVD;
  p->precision = KPME_FP32;
  p->max_n = 1 << 20;
  p->coulomb_k = 1.0;
  return KPME_OK;
}

const char* kpme_status_string(kpme_status_t s) {
  switch (s) {
    case KPME_OK: return "ok";
    case KPME_ERR_INVALID_ARG: return "invalid argument";
    case KPME_ERR_NOT_BUILT: return "SKP factors not built";
    case KPME_ERR_CUDA: return "CUDA error";
    case KPME_ERR_OOM: return "out of device memory";
    case KPME_ERR_CAPACITY: return "particle count exceeds plan capacity";
    case KPME_ERR_TIMEOUT: return "bounded device wait timed out";
    case KPME_ERR_TOLERANCE: return "tolerance not reached";
    case KPME_ERR_UNSUPPORTED: return "unsupported on this device or size";
  }
  return "unknown status";
}

const char* kpme_last_error(kpme_plan_t P) { return P ? P->last_error.c_str() : ""; }

kpme_status_t kpme_plan(const kpme_params_t* params, void* stream, kpme_plan_t* out) {
  if (!params || !out) return KPME_ERR_INVALID_ARG;
  *out = nullptr;
  const kpme_params_t& p = *params;
  const bool lag = p.interp == KPME_INTERP_LAGRANGE || p.interp == KPME_INTERP_LAGRANGE_MODES;
  const bool geometry =
      lag ? ((p.order == 4 || p.order == 6 || p.order == 8 || p.order == 12 || p.order == 16) && p.K % p.order == 0 &&
             p.K >= p.order && p.K <= 512 && p.modes >= 1 && p.modes <= 64 && p.skp_method == KPME_SKP_SINC)
          : (p.interp == KPME_INTERP_BSPLINE && (p.order == 4 || p.order == 6 || p.order == 8) && p.K % 2 == 0 &&
             p.K >= 2 * p.order && p.K <= 512 && (p.skp_method == KPME_SKP_SVD || p.skp_method == KPME_SKP_SINC));
  const bool ok = geometry && std::isfinite(p.radius) && p.radius > 0 && std::isfinite(p.beta) && p.beta > 0 &&
                  std::isfinite(p.skp_tol) && p.skp_tol >= 0 && valid_precision(p.precision) && p.max_n >= 0 &&
                  std::isfinite(p.coulomb_k) && std::isfinite(p.center[0]) && std::isfinite(p.center[1]) &&
                  std::isfinite(p.center[2]);
  if (!ok) return KPME_ERR_INVALID_ARG;
  kpme_plan_t P = new (std::nothrow) kpme_plan_s();
  if (!P) return KPME_ERR_OOM;
  P->p = p;
  P->stream = (cudaStream_t)stream;
  P->max_n = p.max_n;
  P->prec = prec_info(p.precision);
  {
    const char* g = getenv("KPME_GRAPHS");
    P->use_graphs = !(g && g[0] == '0');
  }
  P->poison = getenv_flag("KPME_POISON", false);
  auto fail = [&](kpme_status_t s) {
    kpme_destroy(P);
    return s;
  };
  if (cudaGetDevice(&P->device) != cudaSuccess) return fail(KPME_ERR_CUDA);
  cudaDeviceProp prop;
  if (cudaGetDeviceProperties(&prop, P->device) != cudaSuccess) return fail(KPME_ERR_CUDA);
  P->sm_count = prop.multiProcessorCount;
  P->cc_major = prop.major;
  P->cc_minor = prop.minor;
  if (cudaStreamCreateWithFlags(&P->side_stream, cudaStreamNonBlocking) != cudaSuccess ||
      cudaEventCreateWithFlags(&P->ev_fork, cudaEventDisableTiming) != cudaSuccess ||
      cudaEventCreateWithFlags(&P->ev_join, cudaEventDisableTiming) != cudaSuccess)
    return fail(KPME_ERR_CUDA);
  if (P->prec.tensor && (P->cc_major != 10 || p.K % 16 != 0)) {
    P->last_error = "tensor-core precisions need an sm_103 device and K divisible by 16";
    kpme_destroy(P);
    return KPME_ERR_UNSUPPORTED;
  }
  int* hs = nullptr;
  if (cudaHostAlloc((void**)&hs, sizeof(int), cudaHostAllocMapped) != cudaSuccess) return fail(KPME_ERR_CUDA);
  *hs = DEV_OK;
  P->d_status = hs;   // host pointer; its device alias is taken below
  int* ds = nullptr;
  if (cudaHostGetDevicePointer((void**)&ds, hs, 0) != cudaSuccess) return fail(KPME_ERR_CUDA);
  // keep the host pointer for polling; kernels receive the device alias
  P->d_status = ds == hs ? hs : ds;
  if (ds != hs) {
    // unified addressing makes both pointers equal on every supported system
    P->last_error = "mapped status word needs unified addressing";
    return fail(KPME_ERR_UNSUPPORTED);
  }
  double* acc = nullptr;
  kpme_status_t st = dalloc(P, (void**)&acc, 4 * sizeof(double));
  if (st != KPME_OK) return fail(st);
  P->d_sumq = acc;
  P->d_energy = acc + 1;
  P->d_qpsi = acc + 2;
  {
    const FaultSpec f = parse_fault();
    P->fault_alloc_at = f.alloc_at;
    if (f.budget > 0) P->wait_cycles = f.budget;
  }
  P->allow_fused = getenv_flag("KPME_FUSED", true);
  P->allow_fold = getenv_flag("KPME_FOLD", true);
  P->allow_tile_max = getenv_flag("KPME_TILE_MAX", true);
  {
    const char* e = getenv("KPME_OZT");
    P->ozt_mode = e ? atoi(e) : 1;
  }
  P->tile = 0;
  if (lag) {   // the cell sort of the per-cell form: counters and records
    const size_t nmax = (size_t)std::max<int64_t>(1, p.max_n);
    const int Kc = p.K / p.order;
    const size_t ncnt = (size_t)Kc * Kc * Kc * lagrange_sub(P);
    if ((st = dalloc(P, (void**)&P->d_tcount, ncnt * sizeof(int))) != KPME_OK) return fail(st);
    if ((st = dalloc(P, (void**)&P->d_tstart, (ncnt + 1) * sizeof(int))) != KPME_OK) return fail(st);
    if ((st = dalloc(P, (void**)&P->d_tslot, nmax * sizeof(int2))) != KPME_OK) return fail(st);
    if ((st = dalloc(P, (void**)&P->d_rec_in, 2 * nmax * sizeof(float4))) != KPME_OK) return fail(st);
    if ((st = dalloc(P, (void**)&P->d_rec, 2 * nmax * sizeof(float4))) != KPME_OK) return fail(st);
  } else {   // mesh coordinates shared by the no-sort spreading and gathering of one call
    const size_t nmax = (size_t)std::max<int64_t>(1, p.max_n);
    if ((st = dalloc(P, (void**)&P->d_coords, 3 * nmax * sizeof(float4))) != KPME_OK) return fail(st);
  }
  if (!lag && choose_tile(p.K, p.order) > 0) {
    const size_t nmax = (size_t)std::max<int64_t>(1, p.max_n);
    if ((st = set_tile(P, choose_tile(p.K, p.order))) != KPME_OK) return fail(st);
    if ((st = dalloc(P, (void**)&P->d_tslot, nmax * sizeof(int2))) != KPME_OK) return fail(st);
    if ((st = dalloc(P, (void**)&P->d_rec_in, 2 * nmax * sizeof(float4))) != KPME_OK) return fail(st);
    if ((st = dalloc(P, (void**)&P->d_rec, 2 * nmax * sizeof(float4))) != KPME_OK) return fail(st);
  }
  if ((st = alloc_meshes(P)) != KPME_OK) return fail(st);
  P->single.h_start = {0, 1};
  P->single.h_pairs = {make_int2(0, 0)};
  if ((st = upload_joblist(P, P->single)) != KPME_OK) return fail(st);
  if (cudaStreamSynchronize(P->stream) != cudaSuccess) return fail(KPME_ERR_CUDA);
  P->magic = kPlanMagic;
  {
    const FaultSpec f = parse_fault();
    if (f.plan) P->magic = ~kPlanMagic;
    if (f.timeout) *reinterpret_cast<volatile int*>(P->d_status) = DEV_TIMEOUT;
  }
  *out = P;
  return KPME_OK;
}

void kpme_destroy(kpme_plan_t P) {
  if (!P) return;
  cudaStreamSynchronize(P->stream);
  drop_graph(P);
  if (P->capture_stream) cudaStreamDestroy(P->capture_stream);
  if (P->side_stream) {
    cudaStreamSynchronize(P->side_stream);
    cudaStreamDestroy(P->side_stream);
  }
  if (P->ev_fork) cudaEventDestroy(P->ev_fork);
  if (P->ev_join) cudaEventDestroy(P->ev_join);
  release_skp_buffers(P);
  release_mesh_buffers(P);
  free_joblist(P->single);
  if (P->d_sumq) cudaFree(P->d_sumq);
  dfree(P->d_tcount);
  dfree(P->d_tstart);
  dfree(P->d_tslot);
  dfree(P->d_rec_in);
  dfree(P->d_rec);
  dfree(P->d_coords);
  if (P->d_status) cudaFreeHost(P->d_status);
  for (auto& pe : P->pending) {
    cudaEventDestroy(pe.second.first);
    cudaEventDestroy(pe.second.second);
  }
  for (auto e : P->event_pool) cudaEventDestroy(e);
  P->magic = 0;
  delete P;
}

kpme_status_t kpme_set_stream(kpme_plan_t P, void* stream) {
  if (!P) return KPME_ERR_INVALID_ARG;
  P->stream = (cudaStream_t)stream;
  return KPME_OK;
}

kpme_status_t kpme_set_precision(kpme_plan_t P, int precision) {
  if (!plan_ok(P) || !valid_precision(precision)) return KPME_ERR_INVALID_ARG;
  const PrecInfo pi = prec_info(precision);
  if (pi.tensor && (P->cc_major != 10 || P->p.K % 16 != 0)) {
    P->last_error = "tensor-core precisions need an sm_103 device and K divisible by 16";
    return KPME_ERR_UNSUPPORTED;
  }
  KPME_CUDA_TRY(P, cudaSetDevice(P->device));
  KPME_CUDA_TRY(P, cudaStreamSynchronize(P->stream));
  const bool mesh_change = pi.fp64 != P->prec.fp64;
  P->p.precision = precision;
  P->prec = pi;
  kpme_status_t st;
  if (mesh_change && (st = alloc_meshes(P)) != KPME_OK) return st;
  return install_skp(P);
}

kpme_status_t kpme_build_skp(kpme_plan_t P, int* rank_out, double* err_out) {
  if (!plan_ok(P)) return KPME_ERR_INVALID_ARG;
  KPME_CUDA_TRY(P, cudaSetDevice(P->device));
  SkpHost S;
  kpme_status_t st = lagrange(P) ? build_skp_lagrange(P, S)
                     : P->p.skp_method == KPME_SKP_SVD ? build_skp_svd(P, S) : build_skp_sinc(P, S);
  if (st != KPME_OK) return st;
  P->skp = S;
  if ((st = install_skp(P)) != KPME_OK) return st;
  if (rank_out) *rank_out = S.R;
  if (err_out) *err_out = S.rel_err;
  return check_device_status(P);
}

kpme_status_t kpme_set_skp(kpme_plan_t P, int r0, const int* r1, const double* gen3, const double* gen2,
                           const double* gen1, double c) {
  if (!plan_ok(P) || r0 <= 0 || !r1 || !gen3 || !gen2 || !gen1 || !std::isfinite(c)) return KPME_ERR_INVALID_ARG;
  if (lagrange(P)) return KPME_ERR_UNSUPPORTED;   // its factors are dense, built by kpme_build_skp
  KPME_CUDA_TRY(P, cudaSetDevice(P->device));
  const int K = P->p.K;
  SkpHost S;
  S.r0 = r0;
  for (int i = 0; i < r0; ++i) {
    if (r1[i] <= 0) return KPME_ERR_INVALID_ARG;
    S.r1.push_back(r1[i]);
    for (int j = 0; j < r1[i]; ++j) S.outer_of.push_back(i);
  }
  S.R = (int)S.outer_of.size();
  S.gen3.assign(gen3, gen3 + (size_t)r0 * K);
  S.gen2.assign(gen2, gen2 + (size_t)S.R * K);
  S.gen1.assign(gen1, gen1 + (size_t)S.R * K);
  S.sig_outer.assign(r0, 0.0);
  S.sig_inner.assign(S.R, 0.0);
  S.c = c;
  S.valid = true;
  P->skp = S;
  return install_skp(P);
}

kpme_status_t kpme_get_skp(kpme_plan_t P, int* r0_out, int* R_out, int* r1, double* gen3, double* gen2,
                           double* gen1, double* so, double* si, double* c_out) {
  if (!P) return KPME_ERR_INVALID_ARG;
  const SkpHost& S = P->skp;
  if (!S.valid) return KPME_ERR_NOT_BUILT;
  if (S.dense && (gen3 || gen2 || gen1)) return KPME_ERR_UNSUPPORTED;   // dense factors: sizes and c only
  if (r0_out) *r0_out = S.r0;
  if (R_out) *R_out = S.R;
  if (r1) std::copy(S.r1.begin(), S.r1.end(), r1);
  if (gen3) std::copy(S.gen3.begin(), S.gen3.end(), gen3);
  if (gen2) std::copy(S.gen2.begin(), S.gen2.end(), gen2);
  if (gen1) std::copy(S.gen1.begin(), S.gen1.end(), gen1);
  if (so) std::copy(S.sig_outer.begin(), S.sig_outer.end(), so);
  if (si) std::copy(S.sig_inner.begin(), S.sig_inner.end(), si);
  if (c_out) *c_out = S.c;
  return KPME_OK;
}

// SKP file: 8-byte tag, int32 K, order, r0, R, float64 radius, beta, tolerance, c, int32 r1[r0],
// float64 gen3[r0 K], gen2[R K], gen1[R K] (host byte order)
static const char kSkpTag[8] = {'K', 'P', 'M', 'E', 'S', 'K', 'P', '1'};

kpme_status_t kpme_save_skp(kpme_plan_t P, const char* path) {
  if (!plan_ok(P) || !path) return KPME_ERR_INVALID_ARG;
  const SkpHost& S = P->skp;
  if (!S.valid) return KPME_ERR_NOT_BUILT;
  if (S.dense || lagrange(P)) return KPME_ERR_UNSUPPORTED;
  FILE* f = fopen(path, "wb");
  if (!f) {
    P->last_error = std::string("kpme_save_skp: cannot open ") + path;
    return KPME_ERR_INVALID_ARG;
  }
  const int32_t hdr[4] = {P->p.K, P->p.order, S.r0, S.R};
  const double geo[4] = {P->p.radius, P->p.beta, P->p.skp_tol, S.c};
  std::vector<int32_t> r1(S.r1.begin(), S.r1.end());
  bool ok = fwrite(kSkpTag, 1, 8, f) == 8 && fwrite(hdr, sizeof(int32_t), 4, f) == 4 &&
            fwrite(geo, sizeof(double), 4, f) == 4 && fwrite(r1.data(), sizeof(int32_t), r1.size(), f) == r1.size() &&
            fwrite(S.gen3.data(), sizeof(double), S.gen3.size(), f) == S.gen3.size() &&
            fwrite(S.gen2.data(), sizeof(double), S.gen2.size(), f) == S.gen2.size() &&
            fwrite(S.gen1.data(), sizeof(double), S.gen1.size(), f) == S.gen1.size();
  ok = (fclose(f) == 0) && ok;
  if (!ok) {
    P->last_error = std::string("kpme_save_skp: write failed: ") + path;
    return KPME_ERR_INVALID_ARG;
  }
  return KPME_OK;
}

kpme_status_t kpme_load_skp(kpme_plan_t P, const char* path) {
  if (!plan_ok(P) || !path) return KPME_ERR_INVALID_ARG;
  if (lagrange(P)) return KPME_ERR_UNSUPPORTED;
  FILE* f = fopen(path, "rb");
  if (!f) {
    P->last_error = std::string("kpme_load_skp: cannot open ") + path;
    return KPME_ERR_INVALID_ARG;
  }
  char tag[8];
  int32_t hdr[4];
  double geo[4];
  bool ok = fread(tag, 1, 8, f) == 8 && memcmp(tag, kSkpTag, 8) == 0 && fread(hdr, sizeof(int32_t), 4, f) == 4 &&
            fread(geo, sizeof(double), 4, f) == 4;
  const int K = P->p.K;
  std::string why = ok ? "" : "not an SKP file";
  if (ok && (hdr[0] != K || hdr[1] != P->p.order)) why = "K or order differs from the plan's";
  else if (ok && (geo[0] != P->p.radius || geo[1] != P->p.beta)) why = "box radius or beta differs from the plan's";
  else if (ok && (hdr[2] <= 0 || hdr[3] < hdr[2] || hdr[3] > (1 << 20))) why = "bad sizes";
  std::vector<int32_t> r1;
  std::vector<double> g3, g2, g1;
  if (why.empty()) {
    r1.resize(hdr[2]);
    g3.resize((size_t)hdr[2] * K);
    g2.resize((size_t)hdr[3] * K);
    g1.resize((size_t)hdr[3] * K);
    ok = fread(r1.data(), sizeof(int32_t), r1.size(), f) == r1.size() &&
         fread(g3.data(), sizeof(double), g3.size(), f) == g3.size() &&
         fread(g2.data(), sizeof(double), g2.size(), f) == g2.size() &&
         fread(g1.data(), sizeof(double), g1.size(), f) == g1.size();
    int64_t sum = 0;
    for (int32_t v : r1) sum += v;
    bool finite = std::isfinite(geo[3]);
    for (const auto* g : {&g3, &g2, &g1})
      for (double v : *g) finite = finite && std::isfinite(v);
    if (!ok) why = "file is short";
    else if (sum != hdr[3]) why = "inner counts do not add up to R";
    else if (!finite) why = "non-finite generator values";
  }
  fclose(f);
  if (!why.empty()) {
    P->last_error = std::string("kpme_load_skp: ") + path + ": " + why;
    return KPME_ERR_INVALID_ARG;
  }
  std::vector<int> r1i(r1.begin(), r1.end());
  return kpme_set_skp(P, hdr[2], r1i.data(), g3.data(), g2.data(), g1.data(), geo[3]);
}

kpme_status_t kpme_spread(kpme_plan_t P, int64_t n, const double* x, const double* q, double* Q) {
  kpme_status_t st = common_checks(P, n);
  if (st != KPME_OK) return st;
  if (!Q || (n > 0 && (!x || !q))) return KPME_ERR_INVALID_ARG;
  const int64_t k3 = K3(P);
  MeshRef m;
  if ((st = spread_mesh(P, n, x, q, m)) != KPME_OK) return st;
  KPME_CUDA_TRY(P, launch_convert(m.p, m.dbl, Q, true, k3, P->stream));
  return KPME_OK;
}

kpme_status_t kpme_apply(kpme_plan_t P, const double* Q, double* Phi) {
  kpme_status_t st = common_checks(P, 0);
  if (st != KPME_OK) return st;
  if (!Q || !Phi) return KPME_ERR_INVALID_ARG;
  if (!P->skp.valid) return KPME_ERR_NOT_BUILT;
  const int64_t k3 = K3(P);
  MeshRef m{P->d_Q, true};
  if (tiled(P)) {
    KPME_CUDA_TRY(P, launch_convert(Q, true, P->d_Qf, false, k3, P->stream));
    m = {P->d_Qf, false};
  } else {
    KPME_CUDA_TRY(P, cudaMemcpyAsync(P->d_Q, Q, (size_t)k3 * sizeof(double), cudaMemcpyDeviceToDevice, P->stream));
  }
  if ((st = contract(P, m, P->d_Phi)) != KPME_OK) return st;
  KPME_CUDA_TRY(P, launch_convert(P->d_Phi, P->prec.fp64, Phi, true, k3, P->stream));
  if (P->skp.c != 0.0) KPME_CUDA_TRY(P, launch_mesh_correction(P, Q, Phi, k3, P->skp.c, P->d_qpsi));
  return KPME_OK;
}

kpme_status_t kpme_gather(kpme_plan_t P, int64_t n, const double* x, const double* q, const double* Phi,
                          double* phi, double* F) {
  kpme_status_t st = common_checks(P, n);
  if (st != KPME_OK) return st;
  if (!Phi || (n > 0 && (!x || !phi || (F && !q)))) return KPME_ERR_INVALID_ARG;
  KPME_CUDA_TRY(P, launch_convert(Phi, true, P->d_Phi, P->prec.fp64, K3(P), P->stream));
  return gather_mesh(P, n, x, F ? q : nullptr, phi, F, nullptr, false, false);
}

}  // extern "C"

kpme_status_t kpme::eval_energy_forces(kpme_plan_t P, int64_t n, const double* x, const double* q, double* energy,
                                       double* forces, double* dEdq, double* vir) {
  kpme_status_t st;
  if (vir && lagrange(P)) return KPME_ERR_UNSUPPORTED;   // the virial is a B-spline mesh operator here
  P->launches = 0;
  const int64_t k3 = K3(P);
  (void)k3;
  MeshRef m;
  {
    // per-cell form: clear, count, scan, scatter, per-cell spreading (count and scatter skipped
    // when empty)
    const int spread_launches = lagrange(P) ? (n > 0 ? 5 : 3)
                                : P->prec.fp64 ? (n > 0 ? 1 : 0) : (n > 0 ? (tiled(P) ? 5 : 2) : 1);
    StepScope sc(P, STEP_SPREAD, spread_launches);
    if ((st = spread_mesh(P, n, x, q, m, energy)) != KPME_OK) return st;   // also clears energy
  }
  // the virial's mesh part only reads Q: outside profiling it runs on a forked branch,
  // concurrently with the SKP stages, and joins before the finalisation
  const bool fork = vir && n > 0 && !P->profiling && P->side_stream && !P->vir_tc;
  if (fork) {
    KPME_CUDA_TRY(P, cudaEventRecord(P->ev_fork, P->stream));
    KPME_CUDA_TRY(P, cudaStreamWaitEvent(P->side_stream, P->ev_fork, 0));
    cudaStream_t main_stream = P->stream;
    P->stream = P->side_stream;
    st = virial_mesh(P, m);
    P->stream = main_stream;
    if (st != KPME_OK) return st;
    KPME_CUDA_TRY(P, cudaEventRecord(P->ev_join, P->side_stream));
  }
  if (n > 0) {
    if ((st = contract(P, m, P->d_Phi)) != KPME_OK) return st;
    StepScope sc(P, STEP_GATHER, 1);
    if ((st = gather_mesh(P, n, x, q, dEdq, forces, energy, true, true)) != KPME_OK) return st;
  }
  if (vir) {
    if (n > 0) {
      if (fork)
        KPME_CUDA_TRY(P, cudaStreamWaitEvent(P->stream, P->ev_join, 0));
      else if ((st = P->vir_tc ? virial_mesh_tc(P, m) : virial_mesh(P, m)) != KPME_OK)
        return st;
      if ((st = virial_finish(P, energy, vir)) != KPME_OK) return st;
    } else {
      KPME_CUDA_TRY(P, cudaMemsetAsync(vir, 0, sizeof(double), P->stream));
    }
  }
  return KPME_OK;
}

extern "C" {

kpme_status_t kpme_energy_forces(kpme_plan_t P, int64_t n, const double* x, const double* q, double* energy,
                                 double* forces, double* dEdq, double* vir) {
  kpme_status_t st = common_checks(P, n);
  if (st != KPME_OK) return st;
  if (!energy || (n > 0 && (!x || !q))) return KPME_ERR_INVALID_ARG;
  if (!P->skp.valid) return KPME_ERR_NOT_BUILT;
  if (P->profiling || !P->use_graphs) return eval_energy_forces(P, n, x, q, energy, forces, dEdq, vir);
  // Replay a captured graph when the call signature repeats (the usual MD / benchmark loop).
  const int64_t key[8] = {n, (int64_t)x, (int64_t)q, (int64_t)energy, (int64_t)forces, (int64_t)dEdq,
                          (int64_t)vir, (int64_t)P->p.precision};
  if (!P->graph_exec || memcmp(key, P->graph_key, sizeof(key)) != 0) {
    drop_graph(P);
    if (!P->capture_stream) KPME_CUDA_TRY(P, cudaStreamCreateWithFlags(&P->capture_stream, cudaStreamNonBlocking));
    cudaStream_t user = P->stream;
    P->stream = P->capture_stream;
    KPME_CUDA_TRY(P, cudaStreamBeginCapture(P->capture_stream, cudaStreamCaptureModeRelaxed));
    st = eval_energy_forces(P, n, x, q, energy, forces, dEdq, vir);
    cudaGraph_t g = nullptr;
    cudaError_t e = cudaStreamEndCapture(P->capture_stream, &g);
    P->stream = user;
    if (st != KPME_OK) {
      if (g) cudaGraphDestroy(g);
      return st;
    }
    KPME_CUDA_TRY(P, e);
    e = cudaGraphInstantiate(&P->graph_exec, g, 0);
    cudaGraphDestroy(g);
    KPME_CUDA_TRY(P, e);
    memcpy(P->graph_key, key, sizeof(key));
  }
  KPME_CUDA_TRY(P, cudaGraphLaunch(P->graph_exec, P->stream));
  return KPME_OK;
}

kpme_status_t kpme_virial_tensor(kpme_plan_t P, int64_t n, const double* x, const double* q, double* tensor,
                                 double* energy) {
  kpme_status_t st = common_checks(P, n);
  if (st != KPME_OK) return st;
  if (!tensor || (n > 0 && (!x || !q))) return KPME_ERR_INVALID_ARG;
  if (lagrange(P)) return KPME_ERR_UNSUPPORTED;
  MeshRef m;
  if ((st = spread_mesh(P, n, x, q, m)) != KPME_OK) return st;
  const bool dbl = P->prec.fp64;
  const int K = P->p.K, M = K * K;
  const void* in = m.p;
  if (!dbl && m.dbl) {
    KPME_CUDA_TRY(P, launch_convert(m.p, true, P->d_Qf, false, K3(P), P->stream));
    in = P->d_Qf;
  }
  // Q^ = Q x1 W x2 W x3 W (the mode products rotate the axes back to [m1][m2][m3])
  KPME_CUDA_TRY(P, launch_mp_simt(dbl, in, 0, P->d_facW, P->d_tmp1, 0, M, K, K, P->single, 0, P->stream));
  KPME_CUDA_TRY(P, launch_mp_simt(dbl, P->d_tmp1, 0, P->d_facW, P->d_tmp2, 0, M, K, K, P->single, 0, P->stream));
  KPME_CUDA_TRY(P, launch_mp_simt(dbl, P->d_tmp2, 0, P->d_facW, P->d_Psi, 0, M, K, K, P->single, 0, P->stream));
  KPME_CUDA_TRY(P, launch_virial_tensor(P, P->d_Psi, P->d_vt, tensor, energy));
  return KPME_OK;
}

kpme_status_t kpme_potential(kpme_plan_t P, int64_t n_y, const double* y, const double* q, int64_t n_x,
                             const double* x, double* p) {
  kpme_status_t st = common_checks(P, std::max(n_y, n_x));
  if (st != KPME_OK) return st;
  if ((n_y > 0 && (!y || !q)) || (n_x > 0 && (!x || !p)) || n_y < 0 || n_x < 0) return KPME_ERR_INVALID_ARG;
  if (!P->skp.valid) return KPME_ERR_NOT_BUILT;
  MeshRef m;
  if ((st = spread_mesh(P, n_y, y, q, m)) != KPME_OK) return st;
  if ((st = contract(P, m, P->d_Phi)) != KPME_OK) return st;
  return gather_mesh(P, n_x, x, nullptr, p, nullptr, nullptr, true, false);
}

kpme_status_t kpme_set_profiling(kpme_plan_t P, int enable) {
  if (!P) return KPME_ERR_INVALID_ARG;
  P->profiling = enable != 0;
  return KPME_OK;
}

kpme_status_t kpme_get_profile(kpme_plan_t P, double* ms, int64_t* launches, int n_steps, int* n_out, int reset) {
  if (!P) return KPME_ERR_INVALID_ARG;
  KPME_CUDA_TRY(P, cudaStreamSynchronize(P->stream));
  for (auto& pe : P->pending) {
    float t = 0.f;
    if (cudaEventElapsedTime(&t, pe.second.first, pe.second.second) == cudaSuccess) P->prof_ms[pe.first] += t;
    P->event_pool.push_back(pe.second.first);
    P->event_pool.push_back(pe.second.second);
  }
  P->pending.clear();
  for (int i = 0; i < NUM_STEPS && i < n_steps; ++i) {
    if (ms) ms[i] = P->prof_ms[i];
    if (launches) launches[i] = P->prof_launch[i];
  }
  if (n_out) *n_out = NUM_STEPS;
  if (reset) {
    for (int i = 0; i < NUM_STEPS; ++i) {
      P->prof_ms[i] = 0.0;
      P->prof_launch[i] = 0;
    }
  }
  return check_device_status(P);
}

kpme_status_t kpme_get_info(kpme_plan_t P, kpme_info_t* info) {
  if (!P || !info) return KPME_ERR_INVALID_ARG;
  memset(info, 0, sizeof(*info));
  const double K = P->p.K;
  info->K = P->p.K;
  info->order = P->p.order;
  info->precision = P->p.precision;
  info->r0 = P->skp.valid ? P->skp.r0 : 0;
  info->R = P->skp.valid ? P->skp.R : 0;
  info->skp_rel_err = P->skp.rel_err;
  info->max_n = P->max_n;
  info->scratch_bytes = P->scratch_bytes;
  info->flops_useful = 6.0 * info->R * K * K * K * K;
  const double mp = 2.0 * K * K * K * K;   // one mode product of one term
  // (folded factors: every product contracts K/2 values)
  const double per_eval = (info->r0 + 2.0 * info->R) * mp * (P->fold ? 0.5 : 1.0);
  info->flops_executed = per_eval * (P->prec.tensor ? P->prec.n_products : 1);
  if (lagrange_modes(P) && P->skp.valid) {   // three forward and three backward transforms
    const double r = 2.0 * P->p.modes + 1.0;
    info->flops_useful = info->flops_executed = 4.0 * (r * K * K * K + r * r * K * K + r * r * r * K) + r * r * r;
  }
  int kernels = 1 /*spread*/ + 1 /*gather*/ + 1 /*stage 1*/ + 2 * (int)P->groups.size();
  if (P->prec.tensor) kernels += 1;
  if (P->fold) kernels += 2;   // fold of Q (with the row maxima launch), unfold of Phi
  info->kernels_per_eval = kernels;
  return KPME_OK;
}

}  // extern "C"

// Internal declarations shared by the translation units of libkpme.
#pragma once

#include <cuda.h>
#include <cuda_runtime.h>
#include <cuda_bf16.h>
#include <cudaTypedefs.h>

#include <cstdint>
#include <cstdio>
#include <string>
#include <vector>

#include "kpme.h"

namespace kpme {

// Device status word values (written by bounded waits that give up, and by the index checks of
// the checked build: kDevBounds + the first failing site).
enum DeviceStatus : int { DEV_OK = 0, DEV_TIMEOUT = 1 };
enum BoundsSite : int {
  SITE_SPREAD_NOSORT = 1, SITE_SPREAD_TILE, SITE_TILE_MERGE, SITE_GATHER, SITE_GATHER_TILE, SITE_TILE_COUNT,
  SITE_TILE_SCATTER, NUM_SITES
};
constexpr int kDevBounds = 16;

// Checked build (compiled with -DKPME_DEBUG: `build(debug=True)`, libkpme_debug.so): the particle
// and mesh kernels check every computed index against its buffer; a failed check records the
// first failing site in the status word (the next call on the plan reports it) and the access
// is skipped.  The release build compiles the checks away.
__device__ __forceinline__ bool in_bounds(int* status, bool ok, int site) {
#ifdef KPME_DEBUG
  if (!ok && status) atomicCAS(status, 0, kDevBounds + site);
  return ok;
#else
  (void)status;
  (void)ok;
  (void)site;
  return true;
#endif
}

// Bounded spin budget for every device-side wait (~1 s at 2 GHz).
constexpr long long kWaitCycles = 2000000000LL;
// Handle check word of a live plan.
constexpr uint32_t kPlanMagic = 0x454d504bu;

// The cap on a kernel's dynamic shared memory (cudaFuncAttributeMaxDynamicSharedMemorySize) is
// a property of the function, not of one launch: a kernel launched several times in one
// captured graph with different sizes must carry a cap that covers every launch, since a node
// launched on its own (a replayed or profiled node) is checked against the function's current
// cap.  Every such kernel is given the device's opt-in maximum once; each launch still passes
// its own size.  (The cap counts dynamic memory only: the opt-in maximum less the function's
// static shared memory.)
inline cudaError_t raise_smem_cap(const void* func) {
  int dev = 0, cap = 0;
  cudaFuncAttributes fa{};
  cudaError_t e = cudaGetDevice(&dev);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&cap, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
  if (e == cudaSuccess) e = cudaFuncGetAttributes(&fa, func);
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(func, cudaFuncAttributeMaxDynamicSharedMemorySize, cap - (int)fa.sharedSizeBytes);
  return e;
}

// Steps reported by kpme_get_profile.
enum Step : int {
  STEP_SPREAD = 0, STEP_SPLIT, STEP_SKP1, STEP_SKP2, STEP_SKP3, STEP_GATHER, STEP_VIRIAL, NUM_STEPS
};

// Mode-product job list: job j accumulates pairs [start[j], start[j+1]) of (a_batch, factor).
struct JobList {
  int n_jobs = 0;
  int* d_start = nullptr;   // n_jobs + 1
  int2* d_pairs = nullptr;  // (a_batch, factor)
  std::vector<int> h_start;
  std::vector<int2> h_pairs;
  int max_pairs = 0;
  // optional static schedule (fused stages): items (m tile, first pair, end pair, 0) and
  // for every CTA c its items [cta[c], cta[c + 1])
  std::vector<int4> h_items;
  std::vector<int> h_cta;
  int4* d_items = nullptr;
  int* d_cta = nullptr;
};

// One group of consecutive Kronecker terms processed by stages 2 and 3 together.
struct TermGroup {
  int t0 = 0, t1 = 0;       // terms [t0, t1)
  JobList stage2;           // one job per term: (outer index of the term, term)
  JobList stage3;           // split-K jobs: (term - t0, term)
  JobList stage2_res;       // A-resident jobs: runs of terms of one outer index, (outer, term)
  int splits = 1;
};

struct SkpHost {
  int r0 = 0, R = 0;
  std::vector<int> r1;
  std::vector<int> outer_of;               // term -> outer index
  std::vector<double> gen3, gen2, gen1;    // r0 x K, R x K, R x K (dense: r0, R, R x K x K)
  bool dense = false;                      // full factor matrices instead of circulant generators
  // mode-space form of the per-cell operator: real Fourier rows U ((2M+1) x K: 1, then cos and
  // sin of 2 pi m y per m) and the diagonal on the (2M+1)^3 real modes
  std::vector<double> modal_U, modal_D;
  std::vector<double> sig_outer, sig_inner;
  double c = 0.0;
  double rel_err = 0.0;
  bool valid = false;
};

// Precision traits of a plan.
struct PrecInfo {
  bool tensor = false;    // tcgen05 path
  bool fp64 = false;      // SIMT DFMA
  bool tf32 = false;      // kind::tf32 (else kind::f16 with bf16)
  int slices = 1;         // operand slices per value
  int n_products = 1;     // MMAs per k-step
  int elem_bytes = 4;     // bytes per stored slice element
  bool oz = false;        // error-free fixed-point split (float32 intermediates + row maxima)
};
PrecInfo prec_info(int precision);

}  // namespace kpme

struct kpme_plan_s {
  kpme_params_t p{};
  cudaStream_t stream = nullptr;
  int device = 0;
  int sm_count = 0;
  int cc_major = 0, cc_minor = 0;
  std::string last_error;
  kpme::PrecInfo prec;

  // particle-side scratch
  int64_t max_n = 0;
  double* d_sumq = nullptr;        // sum of charges of the last spread
  double* d_energy = nullptr;      // accumulators (float64)
  double* d_qpsi = nullptr;        // <Q, Psi> for the virial
  int* d_status = nullptr;         // device status word

  // cell sort (float32-mesh arithmetics): tiles of tile^3 cells
  int tile = 0;
  int* d_tcount = nullptr;         // particles per tile
  int* d_tstart = nullptr;         // exclusive prefix (tiles + 1)
  int2* d_tslot = nullptr;         // (tile, slot) per particle
  float4* d_rec_in = nullptr;      // per-particle records (cell, index, offsets), input order
  float4* d_rec = nullptr;         // the same records sorted by tile
  float4* d_coords = nullptr;      // per particle and axis: mesh index and the double-float
                                   // fraction (g, f hi, f lo) of the last no-sort spreading,
                                   // reused by the gathering of the same call
  // meshes, K^3 each: Q float64 (FP64 form, or untiled fallback) / Qf float32, Phi float32
  // (float64 for FP64)
  double* d_Q = nullptr;
  float* d_Qf = nullptr;           // float32 copy of Q for the CUDA-core float32 consumers
  void* d_Phi = nullptr;
  void* d_Psi = nullptr;           // virial contraction output
  void* d_tmp1 = nullptr;          // K^3 scratch for the rank-one virial contraction
  void* d_tmp2 = nullptr;

  // SKP
  kpme::SkpHost skp;
  void* d_fac3 = nullptr;          // factors in the plan's format
  void* d_fac2 = nullptr;
  void* d_fac1 = nullptr;
  void* d_facv = nullptr;          // virial circulant (float/double), K x K
  void* d_facW = nullptr;          // real DFT matrix (cosine / sine rows), K x K, plan's mesh format
  double* d_bmod = nullptr;        // B-spline moduli |b(m)|^2, m = 0..K/2
  double* d_vt = nullptr;          // virial-tensor sums (E and six components)
  double* d_lmU = nullptr;         // mode-space per-cell form: Fourier rows, diagonal,
  double* d_lmD = nullptr;         //   and the transforms' intermediates (r n^2, r^2 n, r^3,
  double* d_lmT = nullptr;         //   r^2 n; r = 2M + 1) in one allocation
  void* d_lmU2 = nullptr;          // the rows and the diagonal as double-float pairs (float2)
  void* d_lmD2 = nullptr;
  void* d_Qs = nullptr;            // tensor path: sliced Q
  void* d_Y = nullptr;             // stage-1 output (r0 tensors)
  void* d_Z = nullptr;             // stage-2 output (one term group)
  void* d_Qsl = nullptr;           // error-free split: fixed-point slices of Q [4][K^2][K]
  void* d_Ysl = nullptr;           // error-free split: fixed-point slices of Y [4][r0][K^2][K]
  float* d_rmZ = nullptr;          // error-free split: row maxima of Z (rows of stage 3)
  float* d_rmQ = nullptr;          // row maxima of the float32 charge mesh (rows of stage 1)
  float* d_rmY = nullptr;          // row maxima of Y (rows of stage 2)
  bool ozt_res = false;            // stages 1 and 2 by the A-in-tensor-memory kernel, A resident
  bool ozt_pp = false;             // stage 3 by the A-in-tensor-memory kernel, A per pair
  bool ozf = false;                // stages 2 and 3 fused on the SM (K = 32, 64)
  bool fold = false;               // error-free split on the reflection basis of every axis
                                   // (K % 128 == 0): block-diagonal factors, K/2 contraction
  bool allow_fold = true;          // KPME_FOLD=0 keeps the dense factors
  bool allow_tile_max = true;      // KPME_TILE_MAX=0: stage 3 rows take their own row maxima
  bool poison = false;             // KPME_POISON=1: every plan allocation starts as 0xFF bytes (NaN)
  int ozt_mode = 1;                // KPME_OZT: 0 the shared-memory-A kernel for every stage, 1 the
                                   // tensor-memory-A kernel where K % 32 == 0, 2 also K % 16 == 0
  float* d_Qfold = nullptr;        // the charge mesh in the reflection basis (float32)
  // the virial's rank-one mesh operator on the tensor cores (reflection basis, N = 128 items):
  // digits of its circulant in the basis, its tensor map and the three one-pair job lists
  bool vir_tc = false;
  void* d_facv_oz = nullptr;
  CUtensorMap tm_v{};
  kpme::JobList vir_jobs;
  bool allow_fused = true;         // tuning knob: may the fused kernel be used
  int tune_split = 2;              // tuning knob: split-K counts x tune_split / 2
  bool no_sort = false;            // tuning knob: float64-atomic spreading, untiled gathering
  kpme::JobList stage23;           // fused jobs: term ranges, pairs (outer index, term)
  kpme::JobList stage1_res;        // A-resident stage-1 jobs: runs of outer factors, (0, i)
  CUtensorMap tmF_Q{}, tmF_Y{}, tmF_Z{};   // float32 A operands, 128 x 32 boxes
  int group_terms = 0;             // capacity of d_Z in terms
  kpme::JobList stage1;
  std::vector<kpme::TermGroup> groups;
  kpme::JobList single;            // one job, one pair (0,0): rank-one contractions

  // tensor maps (tcgen05 path)
  CUtensorMap tm_Q{}, tm_Y{}, tm_Z{}, tm_f3{}, tm_f2{}, tm_f1{};
  int tc_bn = 0, tc_stages = 0;

  // profiling
  bool profiling = false;
  cudaEvent_t ev[2 * kpme::NUM_STEPS] = {};
  double prof_ms[kpme::NUM_STEPS] = {};
  int64_t prof_launch[kpme::NUM_STEPS] = {};
  std::vector<std::pair<int, std::pair<cudaEvent_t, cudaEvent_t>>> pending;
  std::vector<cudaEvent_t> event_pool;
  int64_t launches = 0;            // kernels launched by the last evaluation

  int64_t scratch_bytes = 0;

  // handle check word (kPlanMagic while the plan is valid) and host-side fault injection
  // (KPME_FAULT, read by kpme_plan; see parse_fault in api.cu)
  uint32_t magic = 0;
  int fault_alloc_at = 0;          // the n-th device allocation of the plan fails (0: never)
  int n_allocs = 0;
  long long wait_cycles = kpme::kWaitCycles;   // budget of every bounded device wait

  // CUDA graph of kpme_energy_forces, keyed by its arguments; replayed on the caller's stream
  cudaStream_t capture_stream = nullptr;
  // the virial's mesh part runs on a branch forked after spreading (it only reads Q)
  cudaStream_t side_stream = nullptr;
  cudaEvent_t ev_fork = nullptr, ev_join = nullptr;
  cudaGraphExec_t graph_exec = nullptr;
  int64_t graph_key[8] = {};
  bool use_graphs = true;
};

namespace kpme {

// ---- launchers implemented in the .cu files -------------------------------------------------

// particles.cu
cudaError_t launch_spread(kpme_plan_t P, int64_t n, const double* x, const double* q, double* Q);
// coords (may be NULL): the mesh coordinates of these positions from launch_spread_nosort
cudaError_t launch_gather(kpme_plan_t P, int64_t n, const double* x, const double* q, const void* Phi,
                          double* phi, double* F, double* energy, double scale_phi_extra,
                          const float4* coords = nullptr);
cudaError_t launch_dot(kpme_plan_t P, const void* a, const void* b, int64_t count, double* out);
cudaError_t launch_virial_finalize(kpme_plan_t P, const double* energy, const double* qpsi,
                                   double t0, double coef, double* virial);
cudaError_t launch_convert(const void* src, bool src_double, void* dst, bool dst_double, int64_t count,
                           cudaStream_t s);
cudaError_t launch_spread_raw(const kpme_params_t& p, int sm_count, cudaStream_t s, int64_t n, const double* x,
                              const double* q, float* Q, double* sumq);
int choose_tile(int K, int order);
bool tile_ok(int K, int order, int T);
kpme_status_t set_tile(kpme_plan_t P, int T);
kpme_status_t set_sorted(kpme_plan_t P, bool sorted);
kpme_status_t install_skp(kpme_plan_t P);
constexpr int kTileCounters = 8;   // counters per tile of the cell sort (sub-ranges per tile)
cudaError_t launch_sort(kpme_plan_t P, int64_t n, const double* x, const double* q, double* sumq);
cudaError_t launch_spread_tiled(kpme_plan_t P, int64_t n, const double* q, float* Q);
// coords (may be NULL): receives each particle's mesh coordinates (3 float4 per particle)
cudaError_t launch_spread_nosort(kpme_plan_t P, int64_t n, const double* x, const double* q, float* Q,
                                 float4* coords = nullptr);
cudaError_t launch_gather_tiled(kpme_plan_t P, int64_t n, const double* q, const float* Phi, double* phi, double* F,
                                double* energy, bool correct);

// skp_build.cu
kpme_status_t build_skp_svd(kpme_plan_t P, SkpHost& out);
kpme_status_t build_skp_sinc(kpme_plan_t P, SkpHost& out);
kpme_status_t build_skp_lagrange(kpme_plan_t P, SkpHost& out);
kpme_status_t sinc_search(kpme_plan_t P, const std::vector<double>& args, double tol, int& nq, double& h,
                          double& best);
cudaError_t launch_materialize_dense(kpme_plan_t P, const double* d_dense, const double* d_gmax, int count, void* dst,
                                     int slices, int kind);
bool lagrange(kpme_plan_t P);         // per-cell Lagrange interpolation (either form)
bool lagrange_modes(kpme_plan_t P);   // its node operator applied in mode space
// Phi = U^T (x) U^T (x) U^T diag(D) U (x) U (x) U Q in float64 (lagrange_modes.cu); Q and Phi
// are float64 when dbl, else float32
cudaError_t launch_lagrange_modes(kpme_plan_t P, const void* Q, bool qdbl, void* Phi, bool pdbl);
// per-cell form: counting sort of n particles by cell into the plan's records (also clears the
// float64 accumulators zero0 and zero1 when given), then the per-cell spreading (node charges and
// their sum into sumq) and gathering over the sorted records
int lagrange_sub(kpme_plan_t P);   // counters per cell of the sort
cudaError_t launch_lagrange_sort(kpme_plan_t P, int64_t n, const double* x, double* zero0, double* zero1);
cudaError_t launch_lagrange_spread(kpme_plan_t P, const double* q, void* Q, bool dbl);
cudaError_t launch_lagrange_gather(kpme_plan_t P, int64_t n, const double* q, const void* Phi, bool dbl, double* phi,
                                   double* F, double* energy, bool correct);
cudaError_t launch_materialize(kpme_plan_t P, const double* d_gen, int count, void* dst, int fmt_slices,
                               int fmt_kind);
cudaError_t launch_virial_generator(kpme_plan_t P, double* d_gen);
cudaError_t launch_bmod(kpme_plan_t P, double* d_out);   // K/2 + 1 moduli
cudaError_t launch_dft_matrix(kpme_plan_t P, void* W);
cudaError_t launch_virial_tensor(kpme_plan_t P, const void* Qhat, double* acc, double* out9, double* energy);

// gemm_simt.cu: out[job][n][m] (+)= sum_pairs sum_k fac[f][n][k] in[a][m][k]
cudaError_t launch_mp_simt(bool dbl, const void* in, int64_t in_bs, const void* fac, void* out,
                           int64_t out_bs, int M, int N, int Kr, const JobList& jobs, int mode,
                           cudaStream_t s);

// gemm_tc.cu
struct TcArgs {
  const CUtensorMap* tmA;
  const CUtensorMap* tmB;
  int nbatchA;              // batches per slice plane of A
  void* out;                // slices [S][nbatch_out][N][M] or float Phi [N][M]
  int64_t out_plane;        // elements per output slice plane (nbatch_out * N * M)
  int M, N, Kr;
  int mode;                 // 0 store slices, 1 atomic-add float
  const JobList* jobs;
};
cudaError_t launch_mp_tc(kpme_plan_t P, const TcArgs& a);
cudaError_t launch_split(kpme_plan_t P, const void* src, bool src_double, void* dst, int64_t count);

// gemm_oz.cu: error-free fixed-point split (KPME_BF16X10)
struct OzArgs {
  const CUtensorMap* tmB;
  const CUtensorMap* tmA;          // pre-sliced A by TMA (nullptr: slice float32 rows on the fly)
  int nbatch_a;
  const void* in;                  // float32, or float2 hi/lo pairs when in_double
  bool in_double;
  int64_t in_bs;
  const float* rowmax_in;
  int64_t rm_in_bs;
  float* out;
  int64_t out_bs;
  float* rowmax_out;
  int64_t rm_out_bs;
  int M, N, Kr, mode;
  const JobList* jobs;
};
struct OztArgs {
  const CUtensorMap* tmF;    // float32 A rows (planes x K^2 rows x K)
  const CUtensorMap* tmB;    // factor digits
  const float* rowmax_in;
  int64_t rm_in_bs;
  float* out;
  int64_t out_bs;
  int out_base;
  float* rowmax_out;
  int64_t rm_out_bs;
  int M, N, Kr;
  int mode;                  // 1: sum of the item's pairs (atomics), 2: one plane per pair
  bool a_res;
  const JobList* jobs;
  bool fold = false;         // block-diagonal factors: an item contracts the K/2 values of its
                             // output column's half (A columns [K/2, K) for columns n >= K/2)
  bool self_max = false;     // the kernel takes the rows' powers of two from the staged rows
                             // (rowmax_in unused; needs BN = 128 and the unit's chunks staged)
  bool tile_max = false;     // mode 2: rowmax_out gets one max |value| per (plane, 128 x 128
                             // tile); A per pair: rowmax_in holds them (K = 256 folded, BN = 128)
};
struct OzfArgs {
  const float* Y;            // float32 Y (r0 planes x K^2 rows x K), device
  const CUtensorMap* tmB2;   // digits of the axis-1 factors B_t
  const CUtensorMap* tmB1;   // digits of the axis-0 factors A_t
  float* phi;
  int K;
  const JobList* jobs;       // items: runs of terms, pairs (outer index, term)
};
bool ozf_supported(int K);
cudaError_t launch_mp_ozf(kpme_plan_t P, const OzfArgs& a);
bool ozt_supported(int K, int bn, bool a_res, bool fold = false);
// the K^3 mesh in the reflection basis of its three axes (pairs a <-> K - 1 - a: the sum at
// a, the difference at K - 1 - a) as float32; zero (may be NULL): nz floats cleared alike
cudaError_t launch_fold_mesh(kpme_plan_t P, const void* in, bool in_double, float* out, int K, float* zero,
                             int64_t nz);
// back from the reflection basis, in place (each octet of mirror points is its own inverse
// butterfly, scaled by 1/8)
cudaError_t launch_unfold_mesh(kpme_plan_t P, float* mesh, int K);
cudaError_t launch_mp_ozt(kpme_plan_t P, const OztArgs& a);
cudaError_t launch_mesh_correction(kpme_plan_t P, const double* Q, double* Phi, int64_t count, double c,
                                   double* scratch);
cudaError_t launch_rowmax_rows(kpme_plan_t P, const float* in, int64_t rows, int K, float* out,
                               float* zero = nullptr, int64_t nz = 0);
cudaError_t launch_clear(kpme_plan_t P, float* a, int64_t n, double* s0, double* s1);
cudaError_t launch_mp_oz(kpme_plan_t P, const OzArgs& a);
cudaError_t launch_slice_rows(kpme_plan_t P, const void* in, bool in_double, int64_t rows_per_batch, int nbatch,
                              int K, void* out);
int oz_smem_bytes(int bn, int stages);
bool encode_tmap(kpme_plan_t P, CUtensorMap* map, const void* base, int elem_bytes, bool is_f32,
                 uint64_t dim0, uint64_t dim1, uint64_t dim2, uint32_t box0, uint32_t box1);
int tc_smem_bytes(const PrecInfo& pi, int bn, int stages);

}  // namespace kpme

namespace kpme {
// api.cu: the uncaptured evaluation of kpme_energy_forces on P->stream, and SKP installation
kpme_status_t eval_energy_forces(kpme_plan_t P, int64_t n, const double* x, const double* q, double* energy,
                                 double* forces, double* dEdq, double* vir);
kpme_status_t plan_install_skp(kpme_plan_t P, const SkpHost& S);
}  // namespace kpme

#define KPME_CUDA_TRY(P, expr)                                                   \
  do {                                                                           \
    cudaError_t _e = (expr);                                                     \
    if (_e != cudaSuccess) {                                                     \
      (P)->last_error = std::string(#expr) + ": " + cudaGetErrorString(_e);      \
      return _e == cudaErrorMemoryAllocation ? KPME_ERR_OOM : KPME_ERR_CUDA;     \
    }                                                                            \
  } while (0)

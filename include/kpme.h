/*
 * kpme.h — C ABI of the GB300 reciprocal-space Kroneckerised PME library.
 *
 * The library evaluates the reciprocal (long-range) part of the Ewald
 * splitting of the periodic Coulomb problem
 *
 *     p(x) = sum_{t in 2 r_B Z^3} sum_{y in Y} G(|x - y + t|) q(y),  G(R) = 1/R,
 *
 * (§1.1, Eq. qmutheta_coulomb; splitting §1.2, Eqs. tau and hexpr) for point
 * clouds X (targets) and Y (sources) in a cubic box B of radius r_B centred at
 * c_B.  The reciprocal kernel is applied on a K^3 periodic mesh as a Sum of
 * Kronecker Products (Thm. 1; Eq. VtV; Algorithm 4):
 *
 *     Phi = sum_r  Q x_1 A_r x_2 B_r x_3 C_r  -  c (sum q)
 *
 * where Q is the charge mesh built by cardinal B-spline spreading (the
 * interpolation option named in §2.2), A_r, B_r, C_r are real symmetric
 * circulant K x K factors (§2.3, Eq. kronw), and c is the m = 0 correction
 * of Eq. termbonsum (zero for the SVD-built SKP).  Potentials and forces are
 * gathered back with the same B-splines and their derivatives.
 *
 * Conventions
 *   - box side L = 2 r_B, volume V = L^3, fractional s = (x - c_B)/L + 1/2,
 *     mesh coordinate u = K s wrapped into [0, K); k = m / L.
 *   - reciprocal potential phi(x) = (1/(pi V)) sum_{m != 0}
 *       exp(-pi^2 |k|^2 / beta^2)/|k|^2 ... (§1.2, Eq. hexpr with the
 *     dimensionless xi = beta L), times coulomb_k.
 *   - energy E = 1/2 sum_i q_i phi_i (X = Y), forces F_i = -dE/dx_i,
 *     dE/dq_i = phi_i; virial trace W = sum_m E(m)(1 - 2 pi^2 |k|^2 / beta^2).
 *
 * Memory and ownership
 *   - Every particle array is a DEVICE pointer owned by the caller: positions
 *     are n x 3 row-major float64 (x0 y0 z0 x1 ...), charges and outputs are
 *     float64.  Meshes passed to the stage entry points are K^3 float64 device
 *     arrays in [k1][k2][k3] order (k3 fastest; k1 along x).
 *   - The plan owns its scratch (sorted particles, meshes, SKP factors,
 *     intermediates); it is allocated by kpme_plan / kpme_build_skp /
 *     kpme_set_skp and freed by kpme_destroy.
 *   - All work is enqueued on the plan's CUDA stream; calls return once the
 *     work is enqueued (kpme_build_skp, kpme_set_skp, kpme_get_skp and
 *     kpme_get_profile synchronise the stream).
 *
 * Errors
 *   - Every entry point returns a kpme_status_t; nothing aborts, traps or
 *     throws across the ABI.  KPME_ERR_CUDA leaves the text of the CUDA error in
 *     kpme_last_error(plan).  Device-side waits are bounded; a wait that runs
 *     out sets a device status word that the next call reports as
 *     KPME_ERR_TIMEOUT.
 *   - A call with n == 0 particles succeeds and writes zero energy.
 *
 * Not thread-safe per plan: one host thread at a time may use a given plan.
 */
#ifndef KPME_H
#define KPME_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct kpme_plan_s* kpme_plan_t;

typedef enum {
  KPME_OK = 0,
  KPME_ERR_INVALID_ARG = 1,   /* bad pointer, size or parameter                       */
  KPME_ERR_NOT_BUILT = 2,     /* evaluation requested before the SKP exists           */
  KPME_ERR_CUDA = 3,          /* a CUDA runtime/driver call failed                    */
  KPME_ERR_OOM = 4,           /* device allocation failed                             */
  KPME_ERR_CAPACITY = 5,      /* n exceeds the plan's max_n                           */
  KPME_ERR_TIMEOUT = 6,       /* a bounded device wait gave up                        */
  KPME_ERR_TOLERANCE = 7,     /* SVD did not converge / tolerance unreachable         */
  KPME_ERR_UNSUPPORTED = 8    /* precision or size not supported on this device       */
} kpme_status_t;

/* Arithmetic of the SKP mode products (the dominant step).  In every mode the
 * mesh coordinates are float64, the charge mesh is accumulated in float64, and
 * energy and virial are reduced in float64; the potential mesh and the gather
 * are float32 except for KPME_FP64. */
typedef enum {
  KPME_FP64 = 0,    /* CUDA-core DFMA mode products                                 */
  KPME_FP32 = 1,    /* CUDA-core FFMA mode products                                 */
  KPME_TF32 = 2,    /* tcgen05 kind::tf32, one product, FP32 accumulate             */
  KPME_TF32X3 = 3,  /* tcgen05 kind::tf32, hi+lo split, three products              */
  KPME_BF16 = 4,    /* tcgen05 kind::f16 (bf16), one product                        */
  KPME_BF16X3 = 5,  /* bf16 hi+lo split, three products                             */
  KPME_BF16X6 = 6,  /* bf16 hi+mid+lo split, six products (all with slice sum <= 2) */
  KPME_BF16X10 = 7  /* error-free split: four fixed-point bf16 slices per row with a common
                       exponent, ten products; the leading products sum exactly in FP32
                       (Ozaki et al. splitting); float32 intermediates                  */
} kpme_precision_t;

typedef enum {
  KPME_SKP_SVD = 0,   /* two-level truncated SVD, §2.1.1 (NKPA)                      */
  KPME_SKP_SINC = 1   /* sinc quadrature of 1/|m|^2, §2.1.2 (m = 0 correction c)     */
} kpme_skp_method_t;

/* Particle <-> node interpolation. */
typedef enum {
  KPME_INTERP_BSPLINE = 0,    /* cardinal B-splines of order `order` on one periodic K^3 mesh
                                 (smooth PME; the path of the benchmarks)                    */
  KPME_INTERP_LAGRANGE = 1,   /* the paper's per-cell form (§2.2, §4.1, Algorithm 4):
                                 K / order cells per axis, `order` equispaced Lagrange nodes
                                 per cell and axis (K nodes per axis), modes |m|_inf <= modes,
                                 quadrature SKP of alpha_M with dense axis factors applied
                                 term by term (the mode-product kernels of the precision)    */
  KPME_INTERP_LAGRANGE_MODES = 2  /* the same form and quadrature, the node operator applied
                                 in mode space: the terms share their Fourier factors
                                 (Eq. VtV, V[lambda] = omega^(1/3) sqrt(alpha_lambda) W), so
                                 the sum over lambda is one diagonal on the (2M+1)^3 real
                                 modes between three forward and three backward transforms
                                 of the node tensor (double-float arithmetic on the float32
                                 pipe for float32 meshes, float64 for KPME_FP64); the m = 0
                                 correction is inside the diagonal (kpme_get_skp reports
                                 c = 0)                                                      */
} kpme_interp_t;

typedef struct {
  double center[3];   /* c_B                                                          */
  double radius;      /* r_B > 0; the box side is 2 r_B                               */
  double beta;        /* Ewald parameter (1/length), > 0                              */
  int order;          /* B-spline order n: even, 4 <= n <= 8                          */
  int K;              /* mesh points per axis: even, 2n <= K <= 512                   */
  double skp_tol;     /* SKP compression tolerance (relative, see kpme_build_skp)    */
  int skp_method;     /* kpme_skp_method_t                                            */
  int precision;      /* kpme_precision_t                                             */
  int64_t max_n;      /* largest particle count of any call (scratch capacity)        */
  double coulomb_k;   /* scale of potentials, energies and forces (1 = Gaussian)      */
  int interp;         /* interpolation, a kpme_interp_t; 0 = B-spline                 */
  int modes;          /* per-cell forms: largest mode M per axis (|m|_inf <= M)       */
} kpme_params_t;

/* Fill *p with defaults (centre 0, radius 1, beta 0.35, order 4, K 32, tol 1e-8,
 * SVD, KPME_FP32, max_n 1<<20, coulomb_k 1, B-spline interpolation).  Never fails for
 * p != NULL.
 *
 * KPME_INTERP_LAGRANGE(_MODES) plans: order = Ln nodes per cell (4, 6, 8, 12 or 16), K = Kc Ln with
 * Kc >= 1 cells per axis, 1 <= modes <= 64, skp_method = KPME_SKP_SINC (the quadrature SKP of
 * Eq. quaddecompalpham over the mode cube, built by kpme_build_skp; kpme_set_skp / kpme_get_skp,
 * the virial and kpme_virial_tensor are not available for them).  The potential is
 * (1/(pi L)) sum_{0 != m, |m|_inf <= M} alpha(|m|) ... interpolated per cell (Thm. 3 bounds the
 * interpolation error by (pi M r / Ln)^Ln (2 Ln)! / Ln!^2 with the cell radius r = 1/(2 Kc) in
 * fractional coordinates). */
kpme_status_t kpme_default_params(kpme_params_t* p);

/* Create a plan on the current CUDA device.  stream: a cudaStream_t (NULL =
 * legacy default stream).  Validates the parameters (INVALID_ARG), allocates the
 * particle and mesh scratch for max_n particles (OOM), and returns the plan in
 * *out.  The SKP factors are not built yet. */
kpme_status_t kpme_plan(const kpme_params_t* params, void* stream, kpme_plan_t* out);

/* Release everything the plan owns.  NULL is ignored. */
void kpme_destroy(kpme_plan_t plan);

/* Change the stream later work is enqueued on. */
kpme_status_t kpme_set_stream(kpme_plan_t plan, void* stream);

/* Switch the mode-product arithmetic; the factors are re-materialised in the
 * new format if they exist.  May allocate (OOM). */
kpme_status_t kpme_set_precision(kpme_plan_t plan, int precision);

/* Build the SKP factors on the GPU in float64 (§2.1; §2.3, Eq. VtV).
 * SVD method: the influence tensor T(m) = B(m) C(m) on the half range
 * m in [0, K/2]^3, weighted by sqrt(w_m) per axis (w = 1 at m = 0 and m = K/2,
 * else 2) which makes its SVDs those of the full mode grid, is compressed by the
 * two-level truncated SVD of §2.1.1 (one-sided Jacobi), with ranks chosen so that
 * the right-hand side of Eq. estimate_svd is <= skp_tol * ||T||_F.  Sinc method:
 * the quadrature rule of §2.1.2 with the smallest N_quad whose max relative error
 * on 1/|m|^2 over the mesh modes is <= skp_tol.  The real circulant factors are
 * then synthesised from the mode factors.  Synchronises the stream.
 * rank_out (may be NULL): number of Kronecker terms R.  rel_err_out (may be NULL):
 * achieved relative error (Frobenius for SVD, max-norm for sinc). */
kpme_status_t kpme_build_skp(kpme_plan_t plan, int* rank_out, double* rel_err_out);

/* Install SKP factors given on the HOST instead of building them.
 * r0: number of outer terms; r1[i]: inner terms of outer term i (R = sum r1).
 * gen3: r0 x K, gen2: R x K, gen1: R x K circulant generators g(d), d = 0..K-1,
 * so that the axis-a factor of term r is the matrix A(k,k') = g_r((k-k') mod K)
 * (axis 3 uses gen3 of the term's outer index).  Each generator already carries
 * its share of the term weight.  c: m = 0 correction constant (potential shift
 * -c sum q).  Copies the data; synchronises the stream. */
kpme_status_t kpme_set_skp(kpme_plan_t plan, int r0, const int* r1, const double* gen3,
                           const double* gen2, const double* gen1, double c);

/* Store the plan's SKP in a binary file at path, so that another plan of the same mesh and
 * box can install it without building it (the SKP build is the plan-time cost of §2.1, the
 * two-level truncated SVD of the influence function of Eq. VtV and Theorem 1).  The file holds
 * the generator form of kpme_get_skp (sizes, inner counts, the three sets of circulant
 * generators, the correction constant c) with the plan's K, order, box radius, beta and SKP
 * tolerance, in the host's byte order.  Synchronises nothing; KPME_ERR_NOT_BUILT before an SKP
 * exists, KPME_ERR_UNSUPPORTED for the per-cell form (dense factors), KPME_ERR_INVALID_ARG for a
 * NULL argument or a file that cannot be written. */
kpme_status_t kpme_save_skp(kpme_plan_t plan, const char* path);

/* Install an SKP stored by kpme_save_skp (as kpme_set_skp does).  The file's K, order, box
 * radius and beta must equal the plan's (KPME_ERR_INVALID_ARG otherwise, and for a missing,
 * short or foreign file); kpme_last_error says which.  Synchronises the stream. */
kpme_status_t kpme_load_skp(kpme_plan_t plan, const char* path);

/* Copy the plan's SKP to HOST arrays.  Any output pointer may be NULL.
 * *r0_out, *R_out: sizes; r1 (capacity r0): inner counts; gen3 (r0 x K),
 * gen2 (R x K), gen1 (R x K): generators as in kpme_set_skp; sigma_outer (r0),
 * sigma_inner (R): singular values of the two SVD levels (zeros if the SKP was
 * installed or built by quadrature); c_out: correction constant.  Call once with
 * NULL arrays to learn the sizes.  Synchronises the stream. */
kpme_status_t kpme_get_skp(kpme_plan_t plan, int* r0_out, int* R_out, int* r1, double* gen3,
                           double* gen2, double* gen1, double* sigma_outer,
                           double* sigma_inner, double* c_out);

/* Full reciprocal virial tensor of smooth PME for the n charges x, q (DEVICE, as in
 * kpme_energy_forces).  The paper gives no virial; the standard analytic strain derivative
 * of the mesh energy is used:
 *   Pi_ab = sum_{m != 0} E(m) [delta_ab - 2 (1 + pi^2 |k|^2/beta^2) k_a k_b / |k|^2],
 *   E(m) = 1/2 coulomb_k T(m) |S(m)|^2,  T(m) = B(m) exp(-pi^2 |k|^2/beta^2) / (pi V |k|^2),
 * k = m / L, S the discrete Fourier transform of the charge mesh, so Pi_ab = -dE/d eps_ab
 * under the affine strain x -> (1 + eps) x of positions and box.  It is evaluated in mode
 * space (three real-DFT mode products of the mesh and one float64 reduction), with the exact
 * mesh kernel T rather than its SKP, so its trace equals the scalar virial of
 * kpme_energy_forces up to the SKP approximation.  tensor: DEVICE, 9 doubles, row-major,
 * symmetric (overwritten).  energy (DEVICE, 1 double, may be NULL): sum_m E(m), the mesh
 * energy.  The plan's arithmetic (FP64 form or float32) is used for the mode products. */
kpme_status_t kpme_virial_tensor(kpme_plan_t plan, int64_t n, const double* x, const double* q, double* tensor,
                                 double* energy);

/* Reciprocal potentials at the targets X from the charges on the sources Y
 * (Algorithm 4: spread, SKP products, gather, correction).  y: n_y x 3,
 * q: n_y, x: n_x x 3, p: n_x (output, overwritten).  n_y, n_x <= max_n. */
kpme_status_t kpme_potential(kpme_plan_t plan, int64_t n_y, const double* y, const double* q,
                             int64_t n_x, const double* x, double* p);

/* Energy and its derivatives for X = Y.  x: n x 3, q: n.  Outputs (device, any may
 * be NULL except energy): energy (1 value), forces (n x 3, -dE/dx), dEdq (n,
 * = phi), virial (1 value, trace of the reciprocal virial). */
kpme_status_t kpme_energy_forces(kpme_plan_t plan, int64_t n, const double* x, const double* q,
                                 double* energy, double* forces, double* dEdq, double* virial);

/* Stage entry points (each one step of the path, for composition and testing). */

/* Charge mesh Q (K^3 float64, device) from n charges (B-spline spreading). */
kpme_status_t kpme_spread(kpme_plan_t plan, int64_t n, const double* x, const double* q, double* Q);

/* Phi = SKP(Q) - c sum(Q): the mode products in the plan's precision, float64 I/O. */
kpme_status_t kpme_apply(kpme_plan_t plan, const double* Q, double* Phi);

/* phi_i = sum_k W_i(k) Phi(k) and F_i = -q_i grad_i (F may be NULL). */
kpme_status_t kpme_gather(kpme_plan_t plan, int64_t n, const double* x, const double* q,
                          const double* Phi, double* phi, double* F);

/* Per-step device timing of the evaluation entry points.  While enabled, every
 * call records CUDA events on the plan's stream around each step; read the
 * accumulated milliseconds and launch counts with kpme_get_profile (which
 * synchronises).  Steps: 0 frac+spread, 1 split/convert, 2 SKP stage 1 (axis 3),
 * 3 SKP stage 2 (axis 2), 4 SKP stage 3 (axis 1), 5 gather+reduce, 6 virial.
 * n_steps: capacity of ms/launches; returns the number of steps in *n_out. */
kpme_status_t kpme_set_profiling(kpme_plan_t plan, int enable);
kpme_status_t kpme_get_profile(kpme_plan_t plan, double* ms, int64_t* launches, int n_steps,
                               int* n_out, int reset);

/* Charge spreading without any device allocation (the paper has no counterpart: this
 * serves callers that may not call cudaMalloc — code running during CUDA-graph stream
 * capture, engines whose device memory belongs to their own pool allocator, loops that
 * cannot afford an allocation's device synchronisation).  Same result as kpme_spread
 * with a float32 mesh, but without a plan: params describes the box, order and K
 * (the other fields are ignored), stream is a cudaStream_t, x (n x 3), q (n) and Q
 * (K^3, float64) are device pointers owned by the caller.
 * Scratch: a static device array of 256 B + KPME_NOALLOC_MAX_K^3 float32 (1 MiB for
 * K <= 64) that every GPU loading the library keeps until process exit.  K above
 * KPME_NOALLOC_MAX_K returns KPME_ERR_CAPACITY; bad arguments KPME_ERR_INVALID_ARG.
 * The first call on a device looks up the array's device address (with that device
 * current); make that first call before any stream capture begins.  All calls share the
 * array and each clears it first: calls whose GPU work overlaps race and must be
 * serialised by the caller.  Allocates nothing (no cudaMalloc, cudaFree or allocating
 * library call). */
#define KPME_NOALLOC_MAX_K 64
kpme_status_t kpme_spread_noalloc(const kpme_params_t* params, void* stream, int64_t n, const double* x,
                                  const double* q, double* Q);

/* ---- Batches of independent systems --------------------------------------------
 * Many independent periodic systems (uneven particle counts, boxes and meshes) evaluated
 * by ONE CUDA graph launch per call: every system's pipeline (Algorithm 4 on its own box)
 * is a parallel branch of the captured graph, replayed while the call signature repeats.
 * Each system is described by its own kpme_params_t; systems with identical box, order,
 * K, beta, tolerance and method share one SKP build. */
typedef struct kpme_batch_s* kpme_batch_t;

/* Create plans for n_sys systems (params[n_sys]) on one stream. */
kpme_status_t kpme_batch_create(int n_sys, const kpme_params_t* params, void* stream, kpme_batch_t* out);
void kpme_batch_destroy(kpme_batch_t batch);
kpme_status_t kpme_batch_set_stream(kpme_batch_t batch, void* stream);

/* Build (or share) the SKP of every system; ranks_out[n_sys] (may be NULL) gets each R. */
kpme_status_t kpme_batch_build_skp(kpme_batch_t batch, int* ranks_out);

/* Evaluate all systems.  offsets (HOST, n_sys + 1 entries, non-decreasing) delimit each
 * system's particles in the concatenated DEVICE arrays x (total x 3), q (total), forces
 * (total x 3, may be NULL) and dEdq (total, may be NULL); energies and virials (may be NULL)
 * are DEVICE arrays of n_sys values.  A system with zero particles gets zero energy. */
kpme_status_t kpme_batch_energy_forces(kpme_batch_t batch, const int64_t* offsets, const double* x, const double* q,
                                       double* energies, double* forces, double* dEdq, double* virials);

const char* kpme_batch_last_error(kpme_batch_t batch);

/* ---- autotuning of the launch configuration ----
 * The knobs change only the schedule (every setting gives the same result up to the
 * order of floating-point sums):
 *   tile     - edge T of the cell-sort tiles of spreading and gathering (T divides K,
 *              T >= order - 1, the staged region (T + order - 1)^3 float32 <= 200 KB);
 *              -1 = no cell sort (float64 atomics on the mesh, untiled gathering: fewer
 *              launches, faster for few particles per mesh point), where T could be set;
 *              0 = untiled path (float64 meshes) of a plan the tiling does not fit, not
 *              tunable;
 *   fused    - 1: SKP stages 2 and 3 fused on the SM where the kernel exists (error-free
 *              split, K = 32 or 64), 0: separate stages;
 *   split    - split-K multiplier of the term ranges: 1 (half), 2 (the cost model's
 *              choice), 4 (double); for the fused stages the number of CTAs of their
 *              static schedule: half, one or two per SM. */
typedef struct {
  int tile, fused, split;
  int from_cache;        /* 1: taken from the cache file, not timed                   */
  double ms_per_eval;    /* measured (or cached) time of one kpme_energy_forces        */
} kpme_tune_t;

/* Time kpme_energy_forces for the n particles x, q (DEVICE, as in kpme_energy_forces) by
 * coordinate descent over the knobs (each candidate: 2 warm-up evaluations, a 3-evaluation
 * probe, then 5 to 100 timed evaluations, about 20 ms of work; CUDA events on the plan's
 * stream), leave the plan configured with the fastest and
 * report it in *out.  cache_path (may be NULL): a text file with one line per problem key
 * (K, order, precision, log2 n, SM count, compute capability); a matching entry is applied
 * without timing, a new result is appended.  Needs a built SKP (else KPME_ERR_NOT_BUILT).
 * Allocates scratch for the outputs; synchronises the stream. */
kpme_status_t kpme_autotune(kpme_plan_t plan, int64_t n, const double* x, const double* q, const char* cache_path,
                            kpme_tune_t* out);

/* Apply a configuration (tile, fused, split of *t) to a plan. */
kpme_status_t kpme_set_tune(kpme_plan_t plan, const kpme_tune_t* t);

/* Autotune a batch: the first system of each class (K, order, precision, log2 n) is tuned
 * with kpme_autotune on its own particles (offsets, x, q as in kpme_batch_energy_forces);
 * the others of the class take its configuration.  The whole batch (graph replay, forces,
 * dE/dq and virials) is then timed with the tuned configurations and with those it had
 * before, and the faster set is kept (systems timed alone do not see the concurrency of
 * the batch).  n_tuned (may be NULL): number of systems timed.  The batch's graph is
 * captured again at the next evaluation. */
kpme_status_t kpme_batch_autotune(kpme_batch_t batch, const int64_t* offsets, const double* x, const double* q,
                                  const char* cache_path, int* n_tuned);

typedef struct {
  int K, order, precision, r0, R;
  double skp_rel_err;
  int64_t max_n;
  int64_t scratch_bytes;      /* device bytes owned by the plan                 */
  double flops_useful;        /* 6 R K^4 per evaluation (mode-space per-cell
                                 form: its transforms, as flops_executed)       */
  double flops_executed;      /* mode-product flops actually issued per eval    */
  int kernels_per_eval;       /* kernel launches of one kpme_energy_forces      */
} kpme_info_t;

kpme_status_t kpme_get_info(kpme_plan_t plan, kpme_info_t* info);

/* Measurement helper (no counterpart in the paper): the device's float32 atomic-add rate in
 * the access pattern of B-spline spreading (§2.2, Eq. interpkrons: every particle adds its
 * order^3 stencil, rows of `order` consecutive points along the last axis, order lanes per
 * row) for n_particles hashed cells of a K^3 mesh, into (a) a float32 mesh in device memory
 * (global atomics, as the spreading with no cell sort) and (b) a (15 + order)^3-point
 * shared-memory region per CTA (shared atomics, as the tile-staged spreading), and (c) the
 * read rate of the gathering's pattern (one thread per particle reads its order^3 stencil
 * values of the float32 mesh).  Allocates and frees a K^3 float32 scratch mesh, synchronises
 * the device, and writes the best of three timed runs of each as updates (reads) per second,
 * n_particles * order^3 / seconds, to *global_rate, *shared_rate and *read_rate (any may be
 * NULL).  order: 4, 6 or 8; K >= 16 and a multiple of 4; n_particles >= 1 (else
 * KPME_ERR_INVALID_ARG). */
kpme_status_t kpme_measure_update_rate(int K, int order, int64_t n_particles, double* global_rate,
                                       double* shared_rate, double* read_rate);

const char* kpme_status_string(kpme_status_t status);

/* Text of the last CUDA error seen by this plan ("" if none). */
const char* kpme_last_error(kpme_plan_t plan);

#ifdef __cplusplus
}
#endif

#endif /* KPME_H */

// Mode-space form of the per-cell node operator (KPME_INTERP_LAGRANGE_MODES).
//
// The quadrature SKP of the per-cell form applies, per term lambda, the Kronecker product of
// the axis factors A(lambda) = V[lambda]^* V[lambda] with V[lambda] = omega^(1/3)
// sqrt(alpha_lambda) W (Eq. VtV): every term uses the same Fourier rows W of the node positions
// and differs only by a diagonal on the modes.  On one GPU the sum over lambda therefore
// collapses into one diagonal D(m) = (1/(pi L)) sum_lambda omega_lambda prod_j alpha_lambda(m_j)
// on the mode cube, whose m = 0 entry is exactly the c_Lambda of the correction term and is
// set to zero (Eq. formfinale's - c_Lambda 1 1^T).  With the real rows of one axis,
// U = [1; cos 2 pi m y; sin 2 pi m y]_{m = 1..M} ((2M + 1) x K, kappa = 1, 2, 2 the weights
// of the folded +-m pairs, taken into D), the operator is
//     Phi = (U^T (x) U^T (x) U^T) diag(D) (U (x) U (x) U) Q,
// three forward transforms (node axis -> modes, K -> 2M + 1), the diagonal, three backward
// ones.  The float forms run them in double-float arithmetic on the float32 pipe (about 44
// significant bits, so the float32 node charges and potentials stay the only rounding that
// matters); the FP64 form runs them in float64.
#include "kpme_internal.cuh"
#include "df.cuh"

namespace kpme {
namespace {

constexpr int kThreads = 256;

// out[a][o][b] = sum_{i < n_in} W(o, i) in[a][i][b], times diag[a][o][b] when given, with
// W(o, i) = U[o][i] (forward: nodes -> modes) or U[i][o] (backward: modes -> nodes); U is
// (2M + 1) x K, row-major.
template <typename Tin, typename Tout>
__global__ void __launch_bounds__(kThreads)
    modes_axis_kernel(const Tin* __restrict__ in, Tout* __restrict__ out, const double* __restrict__ U, int K,
                      int64_t A, int n_in, int n_out, int64_t B, bool backward, const double* __restrict__ diag) {
  const int64_t total = A * n_out * B;
  for (int64_t idx = blockIdx.x * (int64_t)kThreads + threadIdx.x; idx < total; idx += (int64_t)gridDim.x * kThreads) {
    const int64_t b = idx % B, ao = idx / B;
    const int o = (int)(ao % n_out);
    const int64_t a = ao / n_out;
    const Tin* src = in + a * n_in * B + b;
    double s = 0.0;
    // unrolled so that the loads of several steps are in flight (the sum keeps its order)
    if (backward) {
#pragma unroll 8
      for (int i = 0; i < n_in; ++i) s = fma(U[(int64_t)i * K + o], (double)src[(int64_t)i * B], s);
    } else {
      const double* u = U + (int64_t)o * K;
#pragma unroll 8
      for (int i = 0; i < n_in; ++i) s = fma(u[i], (double)src[(int64_t)i * B], s);
    }
    if (diag) s *= diag[idx];
    out[idx] = (Tout)s;
  }
}

int blocks_for(kpme_plan_t P, int64_t threads) {
  int64_t b = (threads + kThreads - 1) / kThreads;
  const int64_t cap = (int64_t)P->sm_count * 16;
  if (b > cap) b = cap;
  return (int)(b < 1 ? 1 : b);
}

// ---- float32 meshes: double-float transforms on the float32 pipe ----
__device__ __forceinline__ df ld(const float* p) { return {*p, 0.0f}; }
__device__ __forceinline__ df ld(const float2* p) {
  const float2 v = *p;
  return {v.x, v.y};
}
__device__ __forceinline__ void st(float* p, df v) { *p = v.hi + v.lo; }
__device__ __forceinline__ void st(float2* p, df v) { *p = make_float2(v.hi, v.lo); }

// As modes_axis_kernel with U (and the input, the partial sums and the output) in double-float.
template <typename Tin, typename Tout>
__global__ void __launch_bounds__(kThreads)
    modes_axis_df_kernel(const Tin* __restrict__ in, Tout* __restrict__ out, const float2* __restrict__ U, int K,
                         int64_t A, int n_in, int n_out, int64_t B, bool backward) {
  const int64_t total = A * n_out * B;
  for (int64_t idx = blockIdx.x * (int64_t)kThreads + threadIdx.x; idx < total; idx += (int64_t)gridDim.x * kThreads) {
    const int64_t b = idx % B, ao = idx / B;
    const int o = (int)(ao % n_out);
    const int64_t a = ao / n_out;
    const Tin* src = in + a * n_in * B + b;
    df s = {0.0f, 0.0f};
#pragma unroll 8
    for (int i = 0; i < n_in; ++i) {   // unrolled: the loads of several steps in flight
      const df u = ld(U + (backward ? (int64_t)i * K + o : (int64_t)o * K + i));
      s = df_fma(s, u, ld(src + (int64_t)i * B));
    }
    st(out + idx, s);
  }
}

// The last forward transform, the diagonal and the first backward one, fused: one CTA per
// (mu0, mu1) row a of T2: t[mu2] = D[a][mu2] sum_i U[mu2][i] T2[a][i] (thread mu2), then
// S2[a][g] = sum_mu2 U[mu2][g] t[mu2] (thread g).
__global__ void __launch_bounds__(kThreads)
    modes_mid_df_kernel(const float2* __restrict__ T2, float2* __restrict__ S2, const float2* __restrict__ U,
                        const float2* __restrict__ D, int K, int r) {
  extern __shared__ float2 t_sm[];
  const int a = blockIdx.x;
  for (int mu = threadIdx.x; mu < r; mu += blockDim.x) {
    df s = {0.0f, 0.0f};
#pragma unroll 8
    for (int i = 0; i < K; ++i) s = df_fma(s, ld(U + (int64_t)mu * K + i), ld(T2 + (int64_t)a * K + i));
    s = df_mul(s, ld(D + (int64_t)a * r + mu));
    t_sm[mu] = make_float2(s.hi, s.lo);
  }
  __syncthreads();
  for (int g = threadIdx.x; g < K; g += blockDim.x) {
    df s = {0.0f, 0.0f};
#pragma unroll 8
    for (int mu = 0; mu < r; ++mu) s = df_fma(s, ld(U + (int64_t)mu * K + g), ld(t_sm + mu));
    st(S2 + (int64_t)a * K + g, s);
  }
}

template <typename Tin, typename Tout>
cudaError_t axis_df(kpme_plan_t P, const Tin* in, Tout* out, int64_t A, int n_in, int n_out, int64_t B,
                    bool backward) {
  modes_axis_df_kernel<Tin, Tout><<<blocks_for(P, A * n_out * B), kThreads, 0, P->stream>>>(
      in, out, reinterpret_cast<const float2*>(P->d_lmU2), P->p.K, A, n_in, n_out, B, backward);
  return cudaGetLastError();
}

cudaError_t apply_df(kpme_plan_t P, const float* Q, float* Phi) {
  const int K = P->p.K, r = 2 * P->p.modes + 1;
  const int64_t K2 = (int64_t)K * K;
  float2* T1 = reinterpret_cast<float2*>(P->d_lmT);   // [mu0][g1][g2], later S1
  float2* T2 = T1 + (int64_t)r * K2;                  // [mu0][mu1][g2]
  float2* S2 = T2 + (int64_t)r * r * K;               // [mu0][mu1][g2], after the diagonal
  cudaError_t e;
  if ((e = axis_df<float, float2>(P, Q, T1, 1, K, r, K2, false)) != cudaSuccess) return e;
  if ((e = axis_df<float2, float2>(P, T1, T2, r, K, r, K, false)) != cudaSuccess) return e;
  int nt = 32;
  while (nt < K && nt < kThreads) nt *= 2;
  modes_mid_df_kernel<<<r * r, nt, (size_t)r * sizeof(float2), P->stream>>>(
      T2, S2, reinterpret_cast<const float2*>(P->d_lmU2), reinterpret_cast<const float2*>(P->d_lmD2), K, r);
  if ((e = cudaGetLastError()) != cudaSuccess) return e;
  if ((e = axis_df<float2, float2>(P, S2, T1, r, r, K, K, true)) != cudaSuccess) return e;
  return axis_df<float2, float>(P, T1, Phi, 1, r, K, K2, true);
}

// ---- float64 meshes (the FP64 form): the same transforms in float64 ----
template <typename Tin, typename Tout>
cudaError_t axis(kpme_plan_t P, const Tin* in, Tout* out, int64_t A, int n_in, int n_out, int64_t B, bool backward,
                 const double* diag) {
  modes_axis_kernel<Tin, Tout><<<blocks_for(P, A * n_out * B), kThreads, 0, P->stream>>>(
      in, out, P->d_lmU, P->p.K, A, n_in, n_out, B, backward, diag);
  return cudaGetLastError();
}

cudaError_t apply_fp64(kpme_plan_t P, const double* Q, double* Phi) {
  const int K = P->p.K, r = 2 * P->p.modes + 1;
  const int64_t K2 = (int64_t)K * K;
  double* T1 = P->d_lmT;                     // [mu0][g1][g2]
  double* T2 = T1 + (int64_t)r * K2;         // [mu0][mu1][g2]
  double* T3 = T2 + (int64_t)r * r * K;      // [mu0][mu1][mu2]
  cudaError_t e;
  if ((e = axis<double, double>(P, Q, T1, 1, K, r, K2, false, nullptr)) != cudaSuccess) return e;
  if ((e = axis<double, double>(P, T1, T2, r, K, r, K, false, nullptr)) != cudaSuccess) return e;
  if ((e = axis<double, double>(P, T2, T3, (int64_t)r * r, K, r, 1, false, P->d_lmD)) != cudaSuccess) return e;
  if ((e = axis<double, double>(P, T3, T2, (int64_t)r * r, r, K, 1, true, nullptr)) != cudaSuccess) return e;
  if ((e = axis<double, double>(P, T2, T1, r, r, K, K, true, nullptr)) != cudaSuccess) return e;
  return axis<double, double>(P, T1, Phi, 1, r, K, K2, true, nullptr);
}

}  // namespace

cudaError_t launch_lagrange_modes(kpme_plan_t P, const void* Q, bool qdbl, void* Phi, bool pdbl) {
  if (qdbl != pdbl) return cudaErrorInvalidValue;
  return pdbl ? apply_fp64(P, (const double*)Q, (double*)Phi) : apply_df(P, (const float*)Q, (float*)Phi);
}

}  // namespace kpme

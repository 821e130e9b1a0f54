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
// ones.  The arithmetic is float64 at every precision: it is a few million fused
// multiply-adds per evaluation, and the float32 node charges and potentials are the only
// rounding of the float forms.
#include "kpme_internal.cuh"

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
    if (backward) {
      for (int i = 0; i < n_in; ++i) s = fma(U[(int64_t)i * K + o], (double)src[(int64_t)i * B], s);
    } else {
      const double* u = U + (int64_t)o * K;
      for (int i = 0; i < n_in; ++i) s = fma(u[i], (double)src[(int64_t)i * B], s);
    }
    if (diag) s *= diag[idx];
    out[idx] = (Tout)s;
  }
}

template <typename Tin, typename Tout>
cudaError_t axis(kpme_plan_t P, const Tin* in, Tout* out, int64_t A, int n_in, int n_out, int64_t B, bool backward,
                 const double* diag) {
  const int64_t total = A * n_out * B;
  int64_t blocks = (total + kThreads - 1) / kThreads;
  const int64_t cap = (int64_t)P->sm_count * 16;
  if (blocks > cap) blocks = cap;
  if (blocks < 1) blocks = 1;
  modes_axis_kernel<Tin, Tout><<<(unsigned)blocks, kThreads, 0, P->stream>>>(in, out, P->d_lmU, P->p.K, A, n_in,
                                                                             n_out, B, backward, diag);
  return cudaGetLastError();
}

template <typename T>
cudaError_t apply(kpme_plan_t P, const T* Q, T* Phi) {
  const int K = P->p.K, r = 2 * P->p.modes + 1;
  const int64_t K2 = (int64_t)K * K;
  double* T1 = P->d_lmT;                     // [mu0][g1][g2]
  double* T2 = T1 + (int64_t)r * K2;         // [mu0][mu1][g2]
  double* T3 = T2 + (int64_t)r * r * K;      // [mu0][mu1][mu2]
  cudaError_t e;
  if ((e = axis<T, double>(P, Q, T1, 1, K, r, K2, false, nullptr)) != cudaSuccess) return e;
  if ((e = axis<double, double>(P, T1, T2, r, K, r, K, false, nullptr)) != cudaSuccess) return e;
  if ((e = axis<double, double>(P, T2, T3, (int64_t)r * r, K, r, 1, false, P->d_lmD)) != cudaSuccess) return e;
  if ((e = axis<double, double>(P, T3, T2, (int64_t)r * r, r, K, 1, true, nullptr)) != cudaSuccess) return e;
  if ((e = axis<double, double>(P, T2, T1, r, r, K, K, true, nullptr)) != cudaSuccess) return e;
  return axis<double, T>(P, T1, Phi, 1, r, K, K2, true, nullptr);
}

}  // namespace

cudaError_t launch_lagrange_modes(kpme_plan_t P, const void* Q, bool qdbl, void* Phi, bool pdbl) {
  if (qdbl != pdbl) return cudaErrorInvalidValue;
  return pdbl ? apply<double>(P, (const double*)Q, (double*)Phi) : apply<float>(P, (const float*)Q, (float*)Phi);
}

}  // namespace kpme

// Full reciprocal virial tensor of SPME, evaluated in mode space.
//
// The paper gives no virial (reading R8: the standard analytic strain derivative of the mesh
// energy is used):
//   Pi_ab = sum_{m != 0} E(m) [delta_ab - 2 (1 + pi^2 |k|^2/beta^2) k_a k_b / |k|^2],
//   E(m) = 1/2 T(m) |S(m)|^2,  T(m) = B(m) exp(-pi^2 |k|^2/beta^2) / (pi V |k|^2),  k = m / L,
// with S the discrete Fourier transform of the charge mesh.  Three mode products of the mesh
// with one real K x K DFT matrix (cosine rows for m = 0..K/2, sine rows for the others) give
// the cosine / sine parts of S for m in [0, K/2]^3; one reduction expands them into the signed
// modes and sums E(m) and the six tensor components in float64.  The cost is that of the
// scalar virial (three mode products and a reduction), and the kernel is exact (no SKP).
#include "kpme_internal.cuh"

namespace kpme {
namespace {

// W (K x K): row m (0 <= m <= K/2) = cos(2 pi m k / K); row K/2 + m (1 <= m <= K - K/2 - 1)
// = sin(2 pi m k / K).  The sine rows of m = 0 and of the Nyquist mode vanish and are left out.
template <typename T>
__global__ void dft_matrix_kernel(int K, T* __restrict__ W) {
  const int idx = blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= K * K) return;
  const int row = idx / K, k = idx % K, Kh = K / 2;
  const bool is_sin = row > Kh;
  const int m = is_sin ? row - Kh : row;
  const long long num = (2LL * m * k) % (2LL * K);   // angle 2 pi m k / K = pi num / K
  double s, c;
  sincospi((double)num / (double)K, &s, &c);
  W[idx] = (T)(is_sin ? s : c);
}

// One thread per (m0, m1, m2) in [0, K/2]^3 and its signed modes (+-m_j where the sine row
// exists).  With xyz the transformed mesh at (cos|sin) rows per axis and sigma_j = sign(m_j),
// S(m) = sum_k Q(k) prod_j (cos_j + i sigma_j sin_j):
//   Re S = ccc - s0 s1 ssc - s0 s2 scs - s1 s2 css,  Im S = s0 scc + s1 csc + s2 ccs - s0 s1 s2 sss.
template <typename T>
__global__ void __launch_bounds__(256) virial_tensor_kernel(const T* __restrict__ Qh, int K, double L, double beta,
                                                           const double* __restrict__ bmod,
                                                           double* __restrict__ acc) {
  const int Kh = K / 2, n1 = Kh + 1;
  const int64_t total = (int64_t)n1 * n1 * n1;
  const double V = L * L * L, pb = M_PI * M_PI / (beta * beta);
  double r[7] = {0.0, 0.0, 0.0, 0.0, 0.0, 0.0, 0.0};   // E, S00, S11, S22, S01, S02, S12
  for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < total; t += (int64_t)gridDim.x * blockDim.x) {
    const int mm[3] = {(int)(t / ((int64_t)n1 * n1)), (int)((t / n1) % n1), (int)(t % n1)};
    if (mm[0] == 0 && mm[1] == 0 && mm[2] == 0) continue;
    bool hs[3];
#pragma unroll
    for (int j = 0; j < 3; ++j) hs[j] = mm[j] >= 1 && mm[j] <= K - Kh - 1;
    double v[8];
#pragma unroll
    for (int b = 0; b < 8; ++b) {   // bit j of b: the sine row on axis j
      bool ok = true;
      int row[3];
#pragma unroll
      for (int j = 0; j < 3; ++j) {
        const bool sn = (b >> j) & 1;
        ok = ok && (!sn || hs[j]);
        row[j] = sn ? Kh + mm[j] : mm[j];
      }
      v[b] = ok ? (double)Qh[((int64_t)row[0] * K + row[1]) * K + row[2]] : 0.0;
    }
    const double k[3] = {mm[0] / L, mm[1] / L, mm[2] / L};
    const double ksq = k[0] * k[0] + k[1] * k[1] + k[2] * k[2];
    const double Tm = bmod[mm[0]] * bmod[mm[1]] * bmod[mm[2]] * exp(-pb * ksq) / (M_PI * V * ksq);
    const double f = 2.0 * (1.0 + pb * ksq) / ksq;
    for (int g0 = 0; g0 < (hs[0] ? 2 : 1); ++g0)
      for (int g1 = 0; g1 < (hs[1] ? 2 : 1); ++g1)
        for (int g2 = 0; g2 < (hs[2] ? 2 : 1); ++g2) {
          const double s0 = g0 ? -1.0 : 1.0, s1 = g1 ? -1.0 : 1.0, s2 = g2 ? -1.0 : 1.0;
          const double re = v[0] - s0 * s1 * v[3] - s0 * s2 * v[5] - s1 * s2 * v[6];
          const double im = s0 * v[1] + s1 * v[2] + s2 * v[4] - s0 * s1 * s2 * v[7];
          const double Em = 0.5 * Tm * (re * re + im * im);
          const double w = Em * f;
          r[0] += Em;
          r[1] += w * k[0] * k[0];
          r[2] += w * k[1] * k[1];
          r[3] += w * k[2] * k[2];
          r[4] += w * s0 * s1 * k[0] * k[1];
          r[5] += w * s0 * s2 * k[0] * k[2];
          r[6] += w * s1 * s2 * k[1] * k[2];
        }
  }
  __shared__ double red[7][8];
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
#pragma unroll
  for (int i = 0; i < 7; ++i) {
    double x = r[i];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) x += __shfl_down_sync(0xffffffffu, x, o);
    if (lane == 0) red[i][wid] = x;
  }
  __syncthreads();
  if (threadIdx.x < 7) {
    double x = 0.0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) x += red[threadIdx.x][w];
    if (x != 0.0) atomicAdd(acc + threadIdx.x, x);
  }
}

__global__ void virial_tensor_finish_kernel(const double* __restrict__ acc, double ke, double* __restrict__ out,
                                            double* __restrict__ energy) {
  const double E = acc[0];
  out[0] = ke * (E - acc[1]);
  out[4] = ke * (E - acc[2]);
  out[8] = ke * (E - acc[3]);
  out[1] = out[3] = -ke * acc[4];
  out[2] = out[6] = -ke * acc[5];
  out[5] = out[7] = -ke * acc[6];
  if (energy) *energy = ke * E;
}

}  // namespace

cudaError_t launch_dft_matrix(kpme_plan_t P, void* W) {
  const int K = P->p.K;
  const int blocks = (K * K + 255) / 256;
  if (P->prec.fp64)
    dft_matrix_kernel<double><<<blocks, 256, 0, P->stream>>>(K, (double*)W);
  else
    dft_matrix_kernel<float><<<blocks, 256, 0, P->stream>>>(K, (float*)W);
  return cudaGetLastError();
}

cudaError_t launch_virial_tensor(kpme_plan_t P, const void* Qhat, double* acc, double* out9, double* energy) {
  const int K = P->p.K, n1 = K / 2 + 1;
  const int64_t total = (int64_t)n1 * n1 * n1;
  int64_t blocks = (total + 255) / 256;
  if (blocks > (int64_t)P->sm_count * 8) blocks = (int64_t)P->sm_count * 8;
  cudaError_t e = cudaMemsetAsync(acc, 0, 7 * sizeof(double), P->stream);
  if (e != cudaSuccess) return e;
  const double L = 2.0 * P->p.radius;
  if (P->prec.fp64)
    virial_tensor_kernel<double><<<(unsigned)blocks, 256, 0, P->stream>>>((const double*)Qhat, K, L, P->p.beta,
                                                                            P->d_bmod, acc);
  else
    virial_tensor_kernel<float><<<(unsigned)blocks, 256, 0, P->stream>>>((const float*)Qhat, K, L, P->p.beta,
                                                                           P->d_bmod, acc);
  virial_tensor_finish_kernel<<<1, 1, 0, P->stream>>>(acc, P->p.coulomb_k, out9, energy);
  return cudaGetLastError();
}

}  // namespace kpme

// Building the SKP factors on the GPU in float64 (§2.1.1 NKPA; §2.3 real factors; Eq. VtV).
//
// The influence tensor T(m) = B(m) C(m) is even in every mode index, so its SVDs on the full
// mode grid [-K/2, K/2)^3 equal those of the half range [0, K/2]^3 weighted by sqrt(w_m) per
// axis (w_m = number of grid modes with |m| = m: 1 for m = 0 and m = K/2, else 2).  We
// therefore decompose  T~(m) = T(m) sqrt(w_m1 w_m2 w_m3)  on the half range:
//   1. one-sided Jacobi SVD of I_2(T~) (rows m_3, columns (m_1, m_2)), i.e. of its transpose
//      X = I_2(T~)^T whose K_h columns are orthogonalised pairwise in a round-robin order;
//   2. truncation by the right-hand side of Eq. estimate_svd;
//   3. a batched one-sided Jacobi SVD of every kept I_1(v_i) (rows m_2, columns m_1);
//   4. synthesis of the real circulant generators
//        g(d) = sum_{m=0}^{K/2} sqrt(w_m) u~(m) cos(2 pi m d / K)
//      which is sum over the full grid of the unweighted factor u(m) = u~(m)/sqrt(w_m).
#include "kpme_internal.cuh"
#include <cstring>

#include <algorithm>
#include <cmath>
#include <numeric>

namespace kpme {
namespace {

constexpr int kT = 256;

__device__ double bspline_at_int(int n, int u) {
  // M_n at the integer u by the order recursion (n <= 8); M_1(i) = 1 only for i = 0
  double cur[10], nxt[10];
  for (int i = 0; i < 10; ++i) cur[i] = (i == 0) ? 1.0 : 0.0;   // M_1(i)
  for (int k = 2; k <= n; ++k) {
    for (int i = 0; i < 10; ++i) {
      const double a = cur[i];
      const double b = (i >= 1) ? cur[i - 1] : 0.0;
      nxt[i] = ((double)i * a + (double)(k - i) * b) / (double)(k - 1);
    }
    for (int i = 0; i < 10; ++i) cur[i] = nxt[i];
  }
  return (u >= 0 && u < 10) ? cur[u] : 0.0;
}

// |b(m)|^2 = 1 / |sum_{j=0}^{n-2} M_n(j+1) exp(2 pi i m j / K)|^2, m = 0..Kh-1
__global__ void bmod_kernel(int K, int n, int Kh, double* __restrict__ out) {
  const int m = blockIdx.x * blockDim.x + threadIdx.x;
  if (m >= Kh) return;
  double re = 0.0, im = 0.0;
  for (int j = 0; j <= n - 2; ++j) {
    const double Mv = bspline_at_int(n, j + 1);
    const long long num = (2LL * m * j) % (2LL * K);   // angle 2 pi m j / K = pi * num / K
    double s, c;
    sincospi((double)num / (double)K, &s, &c);
    re += Mv * c;
    im += Mv * s;
  }
  out[m] = 1.0 / (re * re + im * im);
}

__device__ __forceinline__ double sqrtw(int m, int K) { return (m == 0 || 2 * m == K) ? 1.0 : 1.4142135623730951; }

// T~ in layout [m3][m1][m2] (column m3 of X = I_2(T~)^T is contiguous)
__global__ void build_T_kernel(int K, int Kh, double L, double beta, const double* __restrict__ bmod,
                               double* __restrict__ X) {
  const int64_t total = (int64_t)Kh * Kh * Kh;
  const double xi2 = (beta * L) * (beta * L);
  const double pre = L * L / (M_PI * L * L * L);   // L^2 / (pi V)
  for (int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; idx < total;
       idx += (int64_t)gridDim.x * blockDim.x) {
    const int m2 = (int)(idx % Kh);
    const int m1 = (int)((idx / Kh) % Kh);
    const int m3 = (int)(idx / ((int64_t)Kh * Kh));
    const double msq = (double)m1 * m1 + (double)m2 * m2 + (double)m3 * m3;
    double v = 0.0;
    if (msq > 0.0) {
      v = pre * bmod[m1] * bmod[m2] * bmod[m3] * exp(-M_PI * M_PI * msq / xi2) / msq;
      v *= sqrtw(m1, K) * sqrtw(m2, K) * sqrtw(m3, K);
    }
    X[idx] = v;
  }
}

// round-robin ("circle") pairing of nplayers (even) columns at a given step
__device__ __forceinline__ void rr_pair(int nplayers, int step, int i, int& p, int& q) {
  const int m = nplayers - 1;
  if (i == 0) {
    p = m;
    q = step;
  } else {
    p = (step + i) % m;
    q = (step - i + m) % m;
  }
}

template <int NT>
__device__ __forceinline__ void block_sum3(double& a, double& b, double& c) {
  __shared__ double s[3][NT / 32];
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    a += __shfl_down_sync(0xffffffffu, a, o);
    b += __shfl_down_sync(0xffffffffu, b, o);
    c += __shfl_down_sync(0xffffffffu, c, o);
  }
  const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
  if (l == 0) {
    s[0][w] = a;
    s[1][w] = b;
    s[2][w] = c;
  }
  __syncthreads();
  if (threadIdx.x < 32) {
    a = (l < NT / 32) ? s[0][l] : 0.0;
    b = (l < NT / 32) ? s[1][l] : 0.0;
    c = (l < NT / 32) ? s[2][l] : 0.0;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      a += __shfl_down_sync(0xffffffffu, a, o);
      b += __shfl_down_sync(0xffffffffu, b, o);
      c += __shfl_down_sync(0xffffffffu, c, o);
    }
    if (l == 0) {
      s[0][0] = a;
      s[1][0] = b;
      s[2][0] = c;
    }
  }
  __syncthreads();
  a = s[0][0];
  b = s[1][0];
  c = s[2][0];
}

// One parallel Jacobi step: block (pair i, batch b) orthogonalises columns p, q of X_b
// (nrows x ncols, column-major) and applies the same rotation to V_b (ncols x ncols).
__global__ void __launch_bounds__(kT) jacobi_step_kernel(double* __restrict__ X, double* __restrict__ V, int nrows,
                                                         int ncols, int nplayers, int step, int64_t xs, int64_t vs,
                                                         double tol, int* __restrict__ rotated) {
  int p, q;
  rr_pair(nplayers, step, blockIdx.x, p, q);
  if (p >= ncols || q >= ncols) return;
  if (p > q) {
    const int t = p;
    p = q;
    q = t;
  }
  double* xp = X + blockIdx.y * xs + (int64_t)p * nrows;
  double* xq = X + blockIdx.y * xs + (int64_t)q * nrows;
  double a = 0.0, b = 0.0, c = 0.0;
  for (int r = threadIdx.x; r < nrows; r += kT) {
    const double u = xp[r], v = xq[r];
    a += u * u;
    b += v * v;
    c += u * v;
  }
  block_sum3<kT>(a, b, c);
  if (c == 0.0 || !(fabs(c) > tol * sqrt(a) * sqrt(b))) return;
  const double zeta = (b - a) / (2.0 * c);
  double t;
  if (fabs(zeta) > 1e150)
    t = 0.5 / zeta;
  else
    t = (zeta >= 0.0 ? 1.0 : -1.0) / (fabs(zeta) + sqrt(1.0 + zeta * zeta));
  const double cs = 1.0 / sqrt(1.0 + t * t), sn = cs * t;
  for (int r = threadIdx.x; r < nrows; r += kT) {
    const double u = xp[r], v = xq[r];
    xp[r] = cs * u - sn * v;
    xq[r] = sn * u + cs * v;
  }
  double* vp = V + blockIdx.y * vs + (int64_t)p * ncols;
  double* vq = V + blockIdx.y * vs + (int64_t)q * ncols;
  for (int r = threadIdx.x; r < ncols; r += kT) {
    const double u = vp[r], v = vq[r];
    vp[r] = cs * u - sn * v;
    vq[r] = sn * u + cs * v;
  }
  if (threadIdx.x == 0) atomicOr(rotated, 1);
}

__global__ void __launch_bounds__(kT) col_norm_kernel(const double* __restrict__ X, int nrows, int ncols, int64_t xs,
                                                      double* __restrict__ out) {
  const double* x = X + blockIdx.y * xs + (int64_t)blockIdx.x * nrows;
  double a = 0.0, b = 0.0, c = 0.0;
  for (int r = threadIdx.x; r < nrows; r += kT) a += x[r] * x[r];
  block_sum3<kT>(a, b, c);
  if (threadIdx.x == 0) out[blockIdx.y * ncols + blockIdx.x] = sqrt(a);
}

__global__ void identity_kernel(double* __restrict__ V, int n, int batch) {
  const int64_t total = (int64_t)n * n * batch;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < total; i += (int64_t)gridDim.x * blockDim.x) {
    const int64_t r = i % ((int64_t)n * n);
    V[i] = (r / n == r % n) ? 1.0 : 0.0;
  }
}

// Xin[i][c][r] = X[col_i][r * Kh + c] / sigma_i  (I_1 of v_i, transposed for column access)
__global__ void inner_setup_kernel(const double* __restrict__ X, const int* __restrict__ cols,
                                   const double* __restrict__ sig, int Kh, double* __restrict__ Xin) {
  const int i = blockIdx.y;
  const double* v = X + (int64_t)cols[i] * Kh * Kh;
  const double inv = 1.0 / sig[i];
  for (int idx = blockIdx.x * blockDim.x + threadIdx.x; idx < Kh * Kh; idx += gridDim.x * blockDim.x) {
    const int c = idx / Kh, r = idx % Kh;
    Xin[(int64_t)i * Kh * Kh + idx] = v[(int64_t)r * Kh + c] * inv;
  }
}

// g_t(d) = scale_t * sum_{m=0}^{Kh-1} sqrt(w_m) vec_t(m) cos(2 pi m d / K)
__global__ void generator_kernel(const double* __restrict__ vecs, int64_t vstride, const double* __restrict__ scale,
                                 int count, int K, int Kh, double* __restrict__ gen) {
  const int t = blockIdx.y;
  if (t >= count) return;
  const double* v = vecs + (int64_t)t * vstride;
  for (int d = blockIdx.x * blockDim.x + threadIdx.x; d < K; d += gridDim.x * blockDim.x) {
    double acc = 0.0;
    for (int m = 0; m < Kh; ++m) {
      const long long num = (2LL * m * d) % (2LL * K);
      acc += sqrtw(m, K) * v[m] * cospi((double)num / (double)K);
    }
    gen[(int64_t)t * K + d] = acc * scale[t];
  }
}

// virial generator: (1/(pi V))^(1/3) sum_m w_m |b(m)|^2 exp(-pi^2 m^2 / (beta L)^2) cos(2 pi m d / K)
__global__ void virial_gen_kernel(const double* __restrict__ bmod, int K, int Kh, double L, double beta,
                                  double* __restrict__ gen) {
  const int d = blockIdx.x * blockDim.x + threadIdx.x;
  if (d >= K) return;
  const double xi2 = (beta * L) * (beta * L);
  double acc = 0.0;
  for (int m = 0; m < Kh; ++m) {
    const double w = (m == 0 || 2 * m == K) ? 1.0 : 2.0;
    const long long num = (2LL * m * d) % (2LL * K);
    acc += w * bmod[m] * exp(-M_PI * M_PI * (double)m * m / xi2) * cospi((double)num / (double)K);
  }
  gen[d] = acc * cbrt(1.0 / (M_PI * L * L * L));
}

__device__ __forceinline__ float tf32_rn(float x) {
  uint32_t u = __float_as_uint(x);
  if ((u & 0x7f800000u) == 0x7f800000u) return x;
  u += 0xfffu + ((u >> 13) & 1u);
  u &= 0xffffe000u;
  return __uint_as_float(u);
}

// Circulant matrices F[s][t][n][k] = slice s of g_t((n - k) mod K) in the requested format.
// kind: 0 float64, 1 float32, 2 bf16 slices (round-to-nearest cascade), 3 tf32 hi/lo in float32,
// 4 fixed-point bf16 slices with one exponent per factor (every circulant row holds the same
// values): v = 2^(e-7) sum_s d_s 2^(-8s), d_s integers in [-128, 128], 2^e >= max |g|.
//
// fold != 0 (kind 4 only): the two diagonal blocks of the circulant in the reflection basis of
// the mesh axis (pairs a <-> K - 1 - a, see fold_mesh_kernel), K rows x K/2 columns: row n < K/2
// holds C+(n, k) = g(n - k) + g(n + k + 1); row n >= K/2 is the odd block at a' = K - 1 - n,
// column k at a = K/2 - 1 - k: C-(a', a) = g(a' - a) - g(a' + a + 1) (indices mod K).  Their
// entries are bounded by 2 max |g|, which sets the exponent.
__device__ __forceinline__ double folded_entry(const double* g, int K, int n, int k) {
  const int h = K / 2;
  if (n < h) return g[((n - k) % K + K) % K] + g[(n + k + 1) % K];
  const int ap = K - 1 - n, a = h - 1 - k;
  return g[((ap - a) % K + K) % K] - g[(ap + a + 1) % K];
}

__global__ void materialize_kernel(const double* __restrict__ gen, int count, int K, int slices, int kind,
                                   int fold, void* __restrict__ dst) {
  const int kc = fold ? K / 2 : K;   // stored columns per row
  const int64_t per = (int64_t)K * kc;
  const int64_t total = per * count;
  for (int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; idx < total;
       idx += (int64_t)gridDim.x * blockDim.x) {
    const int t = (int)(idx / per);
    const int n = (int)((idx % per) / kc), k = (int)(idx % kc);
    int d = n - k;
    d += (d < 0) ? K : 0;
    const double v = fold ? folded_entry(gen + (int64_t)t * K, K, n, k) : gen[(int64_t)t * K + d];
    if (kind == 0) {
      ((double*)dst)[idx] = v;
    } else if (kind == 1) {
      ((float*)dst)[idx] = (float)v;
    } else if (kind == 2) {
      double r = v;
      for (int s = 0; s < slices; ++s) {
        const __nv_bfloat16 h = __double2bfloat16(r);
        ((__nv_bfloat16*)dst)[s * total + idx] = h;
        r -= (double)__bfloat162float(h);
      }
    } else if (kind == 4) {
      double gmax = 0.0;
      for (int j = 0; j < K; ++j) gmax = fmax(gmax, fabs(gen[(int64_t)t * K + j]));
      if (fold) gmax *= 2.0;
      int e = 0;
      frexp(gmax, &e);
      double u = ldexp(v, 7 - e);
      for (int s = 0; s < slices; ++s) {
        const double dg = rint(u);
        u = (u - dg) * 256.0;
        ((__nv_bfloat16*)dst)[s * total + idx] = __double2bfloat16(ldexp(dg, e - 7 - 8 * s));
      }
    } else {
      const float hi = tf32_rn((float)v);
      ((float*)dst)[idx] = hi;
      if (slices > 1) ((float*)dst)[total + idx] = tf32_rn((float)(v - (double)hi));   // exact tf32 for the MMA
    }
  }
}

std::vector<double> to_host(const double* d, size_t n, cudaStream_t s, cudaError_t& err) {
  std::vector<double> h(n);
  if (n) {
    err = cudaMemcpyAsync(h.data(), d, n * sizeof(double), cudaMemcpyDeviceToHost, s);
    if (err == cudaSuccess) err = cudaStreamSynchronize(s);
  }
  return h;
}

// Batched one-sided Jacobi: X (batch x [ncols][nrows]), V (batch x [ncols][ncols]) initialised to I.
kpme_status_t jacobi_svd(kpme_plan_t P, double* X, double* V, int nrows, int ncols, int batch, int* d_flag) {
  const int nplayers = ncols + (ncols & 1);
  const int64_t xs = (int64_t)nrows * ncols, vs = (int64_t)ncols * ncols;
  KPME_CUDA_TRY(P, cudaGetLastError());
  identity_kernel<<<256, kT, 0, P->stream>>>(V, ncols, batch);
  const double tol = 1e-15;
  for (int sweep = 0; sweep < 60; ++sweep) {
    KPME_CUDA_TRY(P, cudaMemsetAsync(d_flag, 0, sizeof(int), P->stream));
    for (int step = 0; step < nplayers - 1; ++step)
      jacobi_step_kernel<<<dim3(nplayers / 2, batch), kT, 0, P->stream>>>(X, V, nrows, ncols, nplayers, step, xs, vs,
                                                                         tol, d_flag);
    KPME_CUDA_TRY(P, cudaGetLastError());
    int flag = 0;
    KPME_CUDA_TRY(P, cudaMemcpyAsync(&flag, d_flag, sizeof(int), cudaMemcpyDeviceToHost, P->stream));
    KPME_CUDA_TRY(P, cudaStreamSynchronize(P->stream));
    if (!flag) return KPME_OK;
  }
  P->last_error = "one-sided Jacobi SVD did not converge in 60 sweeps";
  return KPME_ERR_TOLERANCE;
}

std::vector<double> tail_norms(const std::vector<double>& s) {
  // tail[r] = sqrt(sum_{k >= r} s_k^2), tail[size] = 0
  std::vector<double> t(s.size() + 1, 0.0);
  for (int r = (int)s.size() - 1; r >= 0; --r) t[r] = std::sqrt(t[r + 1] * t[r + 1] + s[r] * s[r]);
  return t;
}

struct DevBuf {
  void* p = nullptr;
  ~DevBuf() {
    if (p) cudaFree(p);
  }
};

}  // namespace

kpme_status_t build_skp_svd(kpme_plan_t P, SkpHost& out) {
  const int K = P->p.K, Kh = K / 2 + 1, n = P->p.order;
  const double L = 2.0 * P->p.radius, beta = P->p.beta, tol = P->p.skp_tol;
  cudaStream_t s = P->stream;
  DevBuf bmod, X, V, flag, Xin, Vin, sig, cols, vecs, scales, gen;
  KPME_CUDA_TRY(P, cudaMalloc(&bmod.p, Kh * sizeof(double)));
  KPME_CUDA_TRY(P, cudaMalloc(&X.p, (size_t)Kh * Kh * Kh * sizeof(double)));
  KPME_CUDA_TRY(P, cudaMalloc(&V.p, (size_t)Kh * Kh * sizeof(double)));
  KPME_CUDA_TRY(P, cudaMalloc(&flag.p, sizeof(int)));
  bmod_kernel<<<(Kh + 127) / 128, 128, 0, s>>>(K, n, Kh, (double*)bmod.p);
  build_T_kernel<<<512, kT, 0, s>>>(K, Kh, L, beta, (const double*)bmod.p, (double*)X.p);
  KPME_CUDA_TRY(P, cudaGetLastError());

  // 1. outer SVD of I_2(T~): X is Kh^2 x Kh (column m3 = slice [m3][m1][m2])
  kpme_status_t st = jacobi_svd(P, (double*)X.p, (double*)V.p, Kh * Kh, Kh, 1, (int*)flag.p);
  if (st != KPME_OK) return st;
  KPME_CUDA_TRY(P, cudaMalloc(&sig.p, (size_t)Kh * Kh * sizeof(double)));
  col_norm_kernel<<<dim3(Kh, 1), kT, 0, s>>>((const double*)X.p, Kh * Kh, Kh, 0, (double*)sig.p);
  KPME_CUDA_TRY(P, cudaGetLastError());
  cudaError_t err = cudaSuccess;
  std::vector<double> so = to_host((const double*)sig.p, Kh, s, err);
  KPME_CUDA_TRY(P, err);
  std::vector<int> ord(Kh);
  std::iota(ord.begin(), ord.end(), 0);
  std::stable_sort(ord.begin(), ord.end(), [&](int a, int b) { return so[a] > so[b]; });
  std::vector<double> sigma(Kh);
  for (int i = 0; i < Kh; ++i) sigma[i] = so[ord[i]];
  double norm2 = 0.0;
  for (double v : sigma) norm2 += v * v;
  const double norm = std::sqrt(norm2);
  if (!(norm > 0.0)) {
    P->last_error = "influence tensor is zero";
    return KPME_ERR_INVALID_ARG;
  }

  // 2. outer truncation: outer tail <= tol/2 ||T||
  const std::vector<double> otail = tail_norms(sigma);
  int r0 = Kh;
  if (tol > 0.0) {
    for (int r = 0; r <= Kh; ++r)
      if (otail[r] <= 0.5 * tol * norm) {
        r0 = r;
        break;
      }
  }
  if (r0 == 0) r0 = 1;
  const double inner_budget = tol * norm - otail[r0];

  // 3. inner SVDs of I_1(v_i), batched over i < r0
  std::vector<int> hcols(ord.begin(), ord.begin() + r0);
  std::vector<double> hsig(sigma.begin(), sigma.begin() + r0);
  DevBuf dsig_o;
  KPME_CUDA_TRY(P, cudaMalloc(&cols.p, r0 * sizeof(int)));
  KPME_CUDA_TRY(P, cudaMalloc(&dsig_o.p, r0 * sizeof(double)));
  KPME_CUDA_TRY(P, cudaMemcpyAsync(cols.p, hcols.data(), r0 * sizeof(int), cudaMemcpyHostToDevice, s));
  KPME_CUDA_TRY(P, cudaMemcpyAsync(dsig_o.p, hsig.data(), r0 * sizeof(double), cudaMemcpyHostToDevice, s));
  KPME_CUDA_TRY(P, cudaMalloc(&Xin.p, (size_t)r0 * Kh * Kh * sizeof(double)));
  KPME_CUDA_TRY(P, cudaMalloc(&Vin.p, (size_t)r0 * Kh * Kh * sizeof(double)));
  inner_setup_kernel<<<dim3(32, r0), kT, 0, s>>>((const double*)X.p, (const int*)cols.p,
                                                 (const double*)dsig_o.p, Kh, (double*)Xin.p);
  KPME_CUDA_TRY(P, cudaGetLastError());
  st = jacobi_svd(P, (double*)Xin.p, (double*)Vin.p, Kh, Kh, r0, (int*)flag.p);
  if (st != KPME_OK) return st;
  col_norm_kernel<<<dim3(Kh, r0), kT, 0, s>>>((const double*)Xin.p, Kh, Kh, (int64_t)Kh * Kh, (double*)sig.p);
  KPME_CUDA_TRY(P, cudaGetLastError());
  std::vector<double> si = to_host((const double*)sig.p, (size_t)r0 * Kh, s, err);
  KPME_CUDA_TRY(P, err);

  std::vector<double> hX = to_host((const double*)Xin.p, (size_t)r0 * Kh * Kh, s, err);
  KPME_CUDA_TRY(P, err);
  std::vector<double> hVin = to_host((const double*)Vin.p, (size_t)r0 * Kh * Kh, s, err);
  KPME_CUDA_TRY(P, err);
  std::vector<double> hV = to_host((const double*)V.p, (size_t)Kh * Kh, s, err);
  KPME_CUDA_TRY(P, err);

  out = SkpHost();
  out.r0 = r0;
  double err2 = 0.0;
  for (int i = r0; i < Kh; ++i) err2 += sigma[i] * sigma[i];
  // mode vectors: axis 3 (outer), axis 2 (inner left), axis 1 (inner right); weights sigma_i, sigma_ij
  std::vector<double> v3, v2, v1, w3, w2, w1;
  for (int i = 0; i < r0; ++i) {
    std::vector<int> o2(Kh);
    std::iota(o2.begin(), o2.end(), 0);
    const double* sii = &si[(size_t)i * Kh];
    std::stable_sort(o2.begin(), o2.end(), [&](int a, int b) { return sii[a] > sii[b]; });
    std::vector<double> ss(Kh);
    for (int j = 0; j < Kh; ++j) ss[j] = sii[o2[j]];
    const std::vector<double> itail = tail_norms(ss);
    int r1 = Kh;
    if (tol > 0.0) {
      const double thr = sigma[i] > 0.0 ? inner_budget / (r0 * sigma[i]) : 1e300;
      for (int r = 0; r <= Kh; ++r)
        if (itail[r] <= thr) {
          r1 = r;
          break;
        }
    }
    if (r1 == 0) r1 = 1;
    err2 += sigma[i] * sigma[i] * itail[r1] * itail[r1];
    out.r1.push_back(r1);
    out.sig_outer.push_back(sigma[i]);
    for (int k = 0; k < Kh; ++k) v3.push_back(hV[(size_t)ord[i] * Kh + k]);
    w3.push_back(sigma[i]);
    for (int j = 0; j < r1; ++j) {
      const int c = o2[j];
      out.sig_inner.push_back(ss[j]);
      out.outer_of.push_back(i);
      for (int k = 0; k < Kh; ++k) v2.push_back(hVin[(size_t)i * Kh * Kh + (size_t)c * Kh + k]);
      for (int k = 0; k < Kh; ++k) v1.push_back(hX[(size_t)i * Kh * Kh + (size_t)c * Kh + k] / ss[j]);
      w2.push_back(ss[j]);
      w1.push_back(1.0);
    }
  }
  out.R = (int)out.outer_of.size();
  out.rel_err = std::sqrt(err2) / norm;

  // 4. generators on the GPU (float64)
  auto synth = [&](const std::vector<double>& vec, const std::vector<double>& w, std::vector<double>& g) -> kpme_status_t {
    const int count = (int)w.size();
    DevBuf dv, dw, dg;
    KPME_CUDA_TRY(P, cudaMalloc(&dv.p, vec.size() * sizeof(double)));
    KPME_CUDA_TRY(P, cudaMalloc(&dw.p, w.size() * sizeof(double)));
    KPME_CUDA_TRY(P, cudaMalloc(&dg.p, (size_t)count * K * sizeof(double)));
    KPME_CUDA_TRY(P, cudaMemcpyAsync(dv.p, vec.data(), vec.size() * sizeof(double), cudaMemcpyHostToDevice, s));
    KPME_CUDA_TRY(P, cudaMemcpyAsync(dw.p, w.data(), w.size() * sizeof(double), cudaMemcpyHostToDevice, s));
    generator_kernel<<<dim3((K + 127) / 128, count), 128, 0, s>>>((const double*)dv.p, Kh, (const double*)dw.p,
                                                                  count, K, Kh, (double*)dg.p);
    KPME_CUDA_TRY(P, cudaGetLastError());
    cudaError_t e2 = cudaSuccess;
    g = to_host((const double*)dg.p, (size_t)count * K, s, e2);
    KPME_CUDA_TRY(P, e2);
    return KPME_OK;
  };
  if ((st = synth(v3, w3, out.gen3)) != KPME_OK) return st;
  if ((st = synth(v2, w2, out.gen2)) != KPME_OK) return st;
  if ((st = synth(v1, w1, out.gen1)) != KPME_OK) return st;
  out.c = 0.0;
  out.valid = true;
  return KPME_OK;
}

// Cardinal-sine quadrature of 1/R = int_0^inf exp(-t R) dt (§2.1.2): nodes l = -nq..nq,
// w_l = h / (1 + exp(-l h)), lambda_l = log(1 + exp(l h)).  One CTA per candidate h evaluates
// max over the arguments R of |R sum_l w_l exp(-lambda_l R) - 1|.
constexpr int kMaxSincNodes = 801;   // nq <= 400

__global__ void sinc_err_kernel(const double* __restrict__ args, int nargs, const double* __restrict__ hs, int nq,
                                unsigned long long* __restrict__ maxerr) {
  __shared__ double sw[kMaxSincNodes], slam[kMaxSincNodes];
  const double h = hs[blockIdx.x];
  for (int l = threadIdx.x; l <= 2 * nq; l += blockDim.x) {
    const double lh = (double)(l - nq) * h;
    sw[l] = h / (1.0 + exp(-lh));
    slam[l] = log1p(exp(lh));
  }
  __syncthreads();
  double mx = 0.0;
  for (int a = threadIdx.x; a < nargs; a += blockDim.x) {
    const double R = args[a];
    double acc = 0.0;
    for (int l = 0; l <= 2 * nq; ++l) acc += sw[l] * exp(-slam[l] * R);
    mx = fmax(mx, fabs(acc * R - 1.0));
  }
  __shared__ double red[kT];
  red[threadIdx.x] = mx;
  __syncthreads();
  for (int o = kT / 2; o > 0; o >>= 1) {
    if (threadIdx.x < o) red[threadIdx.x] = fmax(red[threadIdx.x], red[threadIdx.x + o]);
    __syncthreads();
  }
  // non-negative doubles order like their bit patterns
  if (threadIdx.x == 0) maxerr[blockIdx.x] = __double_as_longlong(red[0]);
}

// Smallest node count per side N (<= 400) whose cardinal-sine rule of 1/R has a max relative
// error <= tol over the arguments, with its best step h among 64 candidates around
// pi / sqrt(2N + 1) (the brute-force search of §2.1.2); the errors are evaluated on the GPU.
kpme_status_t sinc_search(kpme_plan_t P, const std::vector<double>& args, double tol, int& nq, double& h,
                          double& best) {
  cudaStream_t s = P->stream;
  constexpr int kH = 64;
  DevBuf dargs, dhs, derr;
  KPME_CUDA_TRY(P, cudaMalloc(&dargs.p, args.size() * sizeof(double)));
  KPME_CUDA_TRY(P, cudaMalloc(&dhs.p, kH * sizeof(double)));
  KPME_CUDA_TRY(P, cudaMalloc(&derr.p, kH * sizeof(unsigned long long)));
  KPME_CUDA_TRY(P, cudaMemcpyAsync(dargs.p, args.data(), args.size() * sizeof(double), cudaMemcpyHostToDevice, s));
  nq = 0;
  h = 0.0;
  best = 0.0;
  for (int q = 1; q <= 400 && nq == 0; ++q) {
    const double h0 = M_PI / std::sqrt(2.0 * q + 1.0);
    std::vector<double> hs(kH);
    for (int i = 0; i < kH; ++i) hs[i] = h0 * (0.5 + 1.5 * i / (kH - 1));
    KPME_CUDA_TRY(P, cudaMemcpyAsync(dhs.p, hs.data(), kH * sizeof(double), cudaMemcpyHostToDevice, s));
    sinc_err_kernel<<<kH, kT, 0, s>>>((const double*)dargs.p, (int)args.size(), (const double*)dhs.p, q,
                                      (unsigned long long*)derr.p);
    KPME_CUDA_TRY(P, cudaGetLastError());
    std::vector<unsigned long long> bits(kH);
    KPME_CUDA_TRY(P, cudaMemcpyAsync(bits.data(), derr.p, kH * sizeof(unsigned long long), cudaMemcpyDeviceToHost, s));
    KPME_CUDA_TRY(P, cudaStreamSynchronize(s));
    int bi = 0;
    double be = 0.0;
    for (int i = 0; i < kH; ++i) {
      double e;
      std::memcpy(&e, &bits[i], sizeof(double));
      if (i == 0 || e < be) {
        be = e;
        bi = i;
      }
    }
    if (be <= tol) {
      nq = q;
      h = hs[bi];
      best = be;
    }
  }
  if (nq == 0) {
    P->last_error = "sinc quadrature did not reach the tolerance with 400 nodes per side";
    return KPME_ERR_TOLERANCE;
  }
  return KPME_OK;
}

// Quadrature-based SKP (§2.1.2, Eq. quaddecompalpham) with the B-spline factor:
// T(m) = (1/(pi L)) B(m) exp(-pi^2 |m|^2 / (beta L)^2) / |m|^2, and 1/|m|^2 ~ sum_l w_l exp(-lambda_l |m|^2)
// gives rank-one terms with the same factor a_l(m) = |b(m)|^2 exp(-(lambda_l + pi^2/(beta L)^2) m^2) on
// every axis, weight w_l / (pi L), minus c delta_0 with c = |b(0)|^6 sum_l w_l / (pi L).  The node
// count is the smallest whose best h (64 candidates in [0.5, 2] pi / sqrt(2 nq + 1)) keeps the
// max relative error of the 1/R rule over the actual arguments R = |m|^2 > 0 within tol; that
// error is returned as rel_err.  Terms are laid out in the two-level form with one inner term per
// outer term.
kpme_status_t build_skp_sinc(kpme_plan_t P, SkpHost& out) {
  const int K = P->p.K, n = P->p.order, Kh = K / 2 + 1;
  const double L = 2.0 * P->p.radius, beta = P->p.beta, tol = P->p.skp_tol;
  if (!(tol > 0.0)) {
    P->last_error = "the sinc-quadrature SKP needs a positive tolerance";
    return KPME_ERR_INVALID_ARG;
  }
  cudaStream_t s = P->stream;
  cudaError_t err = cudaSuccess;
  // arguments: distinct m1^2 + m2^2 + m3^2 > 0 over the wrapped modes (|m| <= K/2)
  const int h2 = (K / 2) * (K / 2);
  std::vector<char> seen(3 * h2 + 1, 0);
  for (int a = 0; a <= K / 2; ++a)
    for (int b = a; b <= K / 2; ++b)
      for (int c = b; c <= K / 2; ++c) seen[a * a + b * b + c * c] = 1;
  std::vector<double> args;
  for (int r = 1; r <= 3 * h2; ++r)
    if (seen[r]) args.push_back((double)r);
  int nq = 0;
  double h = 0.0, best = 0.0;
  {
    const kpme_status_t sst = sinc_search(P, args, tol, nq, h, best);
    if (sst != KPME_OK) return sst;
  }
  DevBuf bmod, vecs, scales, gen;
  // factors
  KPME_CUDA_TRY(P, cudaMalloc(&bmod.p, Kh * sizeof(double)));
  bmod_kernel<<<(Kh + 127) / 128, 128, 0, s>>>(K, n, Kh, (double*)bmod.p);
  KPME_CUDA_TRY(P, cudaGetLastError());
  std::vector<double> bm = to_host((const double*)bmod.p, Kh, s, err);
  KPME_CUDA_TRY(P, err);
  const double pre = 1.0 / (M_PI * L);
  const double xi2 = (beta * L) * (beta * L);
  const int R = 2 * nq + 1;
  std::vector<double> v((size_t)R * Kh), w3(R), ones(R, 1.0);
  double wsum = 0.0;
  for (int t = 0; t < R; ++t) {
    const int l = t - nq;
    const double wl = h / (1.0 + std::exp(-l * h));
    const double lam = std::log1p(std::exp(l * h));
    wsum += wl;
    w3[t] = pre * wl;
    for (int m = 0; m < Kh; ++m) {
      const double sw = (m == 0 || 2 * m == K) ? 1.0 : std::sqrt(2.0);
      v[(size_t)t * Kh + m] = sw * bm[m] * std::exp(-(lam + M_PI * M_PI / xi2) * (double)m * m);
    }
  }
  KPME_CUDA_TRY(P, cudaMalloc(&vecs.p, v.size() * sizeof(double)));
  KPME_CUDA_TRY(P, cudaMalloc(&scales.p, 2 * R * sizeof(double)));
  KPME_CUDA_TRY(P, cudaMalloc(&gen.p, (size_t)R * K * sizeof(double)));
  KPME_CUDA_TRY(P, cudaMemcpyAsync(vecs.p, v.data(), v.size() * sizeof(double), cudaMemcpyHostToDevice, s));
  KPME_CUDA_TRY(P, cudaMemcpyAsync(scales.p, w3.data(), R * sizeof(double), cudaMemcpyHostToDevice, s));
  KPME_CUDA_TRY(P, cudaMemcpyAsync((double*)scales.p + R, ones.data(), R * sizeof(double), cudaMemcpyHostToDevice, s));
  out = SkpHost();
  for (int pass = 0; pass < 2; ++pass) {
    generator_kernel<<<dim3((K + 127) / 128, R), 128, 0, s>>>((const double*)vecs.p, Kh, (const double*)scales.p + pass * R,
                                                              R, K, Kh, (double*)gen.p);
    KPME_CUDA_TRY(P, cudaGetLastError());
    std::vector<double> g = to_host((const double*)gen.p, (size_t)R * K, s, err);
    KPME_CUDA_TRY(P, err);
    if (pass == 0)
      out.gen3 = g;
    else
      out.gen2 = out.gen1 = g;
  }
  out.r0 = R;
  out.R = R;
  out.r1.assign(R, 1);
  out.outer_of.resize(R);
  std::iota(out.outer_of.begin(), out.outer_of.end(), 0);
  out.sig_outer = w3;
  out.sig_inner.assign(R, 1.0);
  out.c = pre * bm[0] * bm[0] * bm[0] * wsum;
  out.rel_err = best;
  out.valid = true;
  return KPME_OK;
}

// Quadrature SKP of the per-cell Lagrange form (§2.1.2, §2.2, §4.1): alpha_M on the mode cube
// |m|_inf <= M by the sinc rule of 1/|m|^2 searched over the cube's arguments, and dense axis
// factors on the K node positions y (cell i, node l at (i + (1 + t_l)/2) / Kc, t_l = -1 + 2l/(Ln-1)):
//   A_l(g, h) = sum_{m=-M}^{M} exp(-(lambda_l + pi^2/xi^2) m^2) cos(2 pi m (y_g - y_h)),
// the real cosine form of §2.3 summed over the modes.  Term l is (w_l/(pi L)) A_l x A_l x A_l (its
// weight on the axis-3 factor) and the m = 0 correction is c = sum_l w_l / (pi L).  The factors
// are formed here, at plan time, in float64.
kpme_status_t build_skp_lagrange(kpme_plan_t P, SkpHost& out) {
  const int K = P->p.K, Ln = P->p.order, Kc = K / Ln, M = P->p.modes;
  const double L = 2.0 * P->p.radius, beta = P->p.beta, tol = P->p.skp_tol;
  if (!(tol > 0.0)) {
    P->last_error = "the sinc-quadrature SKP needs a positive tolerance";
    return KPME_ERR_INVALID_ARG;
  }
  std::vector<char> seen(3 * M * M + 1, 0);
  for (int a = 0; a <= M; ++a)
    for (int b = a; b <= M; ++b)
      for (int c = b; c <= M; ++c) seen[a * a + b * b + c * c] = 1;
  std::vector<double> args;
  for (int r = 1; r <= 3 * M * M; ++r)
    if (seen[r]) args.push_back((double)r);
  int nq = 0;
  double h = 0.0, best = 0.0;
  {
    const kpme_status_t sst = sinc_search(P, args, tol, nq, h, best);
    if (sst != KPME_OK) return sst;
  }
  const int R = 2 * nq + 1;
  const double pre = 1.0 / (M_PI * L), xi2 = (beta * L) * (beta * L);
  std::vector<double> y(K);
  for (int i = 0; i < Kc; ++i)
    for (int l = 0; l < Ln; ++l) {
      const double t = -1.0 + 2.0 * l / (Ln - 1);
      y[i * Ln + l] = (i + 0.5 * (1.0 + t)) / Kc;
    }
  if (lagrange_modes(P)) {   // the sum over the terms as one diagonal on the real modes
    const int r = 2 * M + 1;
    out = SkpHost();
    out.dense = true;
    out.modal_U.assign((size_t)r * K, 0.0);
    for (int g = 0; g < K; ++g) {
      out.modal_U[g] = 1.0;
      for (int m = 1; m <= M; ++m) {
        out.modal_U[(size_t)(2 * m - 1) * K + g] = std::cos(2.0 * M_PI * m * y[g]);
        out.modal_U[(size_t)(2 * m) * K + g] = std::sin(2.0 * M_PI * m * y[g]);
      }
    }
    std::vector<double> wl(R), lam(R), dsq(3 * M * M + 1, 0.0);
    for (int t = 0; t < R; ++t) {
      const int l = t - nq;
      wl[t] = h / (1.0 + std::exp(-l * h));
      lam[t] = std::log1p(std::exp(l * h));
    }
    for (int s2 = 1; s2 <= 3 * M * M; ++s2) {   // pre sum_l w_l prod_j a_l(m_j), by |m|^2
      double acc = 0.0;
      for (int t = 0; t < R; ++t) acc += wl[t] * std::exp(-(lam[t] + M_PI * M_PI / xi2) * s2);
      dsq[s2] = pre * acc;
    }
    // real mode mu: 0 -> m = 0; 2m - 1, 2m -> cos, sin of mode m, the +-m pair folded (kappa 2)
    auto mo = [](int mu) { return (mu + 1) / 2; };
    auto kap = [](int mu) { return mu == 0 ? 1.0 : 2.0; };
    out.modal_D.resize((size_t)r * r * r);
    for (int a = 0; a < r; ++a)
      for (int b = 0; b < r; ++b)
        for (int c = 0; c < r; ++c) {
          const int s2 = mo(a) * mo(a) + mo(b) * mo(b) + mo(c) * mo(c);
          out.modal_D[((size_t)a * r + b) * r + c] = s2 == 0 ? 0.0 : dsq[s2] * kap(a) * kap(b) * kap(c);
        }
    out.r0 = R;
    out.R = R;
    out.r1.assign(R, 1);
    out.outer_of.resize(R);
    std::iota(out.outer_of.begin(), out.outer_of.end(), 0);
    out.sig_outer.resize(R);
    for (int t = 0; t < R; ++t) out.sig_outer[t] = pre * wl[t];
    out.sig_inner.assign(R, 1.0);
    out.c = 0.0;   // the diagonal has no m = 0 entry: the correction term is inside it
    out.rel_err = best;
    out.valid = true;
    return KPME_OK;
  }
  const size_t KK = (size_t)K * K;
  std::vector<double> cs((size_t)M * KK);   // cos(2 pi m (y_g - y_h)), m = 1..M
  for (int m = 1; m <= M; ++m)
    for (int g = 0; g < K; ++g)
      for (int hh = 0; hh < K; ++hh) cs[(m - 1) * KK + (size_t)g * K + hh] = std::cos(2.0 * M_PI * m * (y[g] - y[hh]));
  out = SkpHost();
  out.dense = true;
  out.gen3.resize((size_t)R * KK);
  out.gen2.resize((size_t)R * KK);
  double wsum = 0.0;
  std::vector<double> am(M + 1), w3(R);
  for (int t = 0; t < R; ++t) {
    const int l = t - nq;
    const double wl = h / (1.0 + std::exp(-l * h));
    const double lam = std::log1p(std::exp(l * h));
    wsum += wl;
    w3[t] = pre * wl;
    for (int m = 0; m <= M; ++m) am[m] = std::exp(-(lam + M_PI * M_PI / xi2) * (double)m * m);
    for (size_t gh = 0; gh < KK; ++gh) {
      double A = am[0];
      for (int m = 1; m <= M; ++m) A += 2.0 * am[m] * cs[(m - 1) * KK + gh];
      out.gen2[(size_t)t * KK + gh] = A;
      out.gen3[(size_t)t * KK + gh] = w3[t] * A;
    }
  }
  out.gen1 = out.gen2;
  out.r0 = R;
  out.R = R;
  out.r1.assign(R, 1);
  out.outer_of.resize(R);
  std::iota(out.outer_of.begin(), out.outer_of.end(), 0);
  out.sig_outer = w3;
  out.sig_inner.assign(R, 1.0);
  out.c = pre * wsum;
  out.rel_err = best;
  out.valid = true;
  return KPME_OK;
}

// Dense factors F[s][t][n][k] = slice s of D_t[n][k] in the requested format (the formats of
// materialize_kernel; the fixed-point digits use one power of two per factor, gmax[t]).
__global__ void materialize_dense_kernel(const double* __restrict__ D, const double* __restrict__ gmax, int count,
                                         int K, int slices, int kind, void* __restrict__ dst) {
  const int64_t per = (int64_t)K * K;
  const int64_t total = per * count;
  for (int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; idx < total;
       idx += (int64_t)gridDim.x * blockDim.x) {
    const double v = D[idx];
    if (kind == 0) {
      ((double*)dst)[idx] = v;
    } else if (kind == 1) {
      ((float*)dst)[idx] = (float)v;
    } else if (kind == 2) {
      double r = v;
      for (int s = 0; s < slices; ++s) {
        const __nv_bfloat16 h = __double2bfloat16(r);
        ((__nv_bfloat16*)dst)[s * total + idx] = h;
        r -= (double)__bfloat162float(h);
      }
    } else if (kind == 4) {
      int e = 0;
      frexp(gmax[idx / per], &e);
      double u = ldexp(v, 7 - e);
      for (int s = 0; s < slices; ++s) {
        const double dg = rint(u);
        u = (u - dg) * 256.0;
        ((__nv_bfloat16*)dst)[s * total + idx] = __double2bfloat16(ldexp(dg, e - 7 - 8 * s));
      }
    } else {
      const float hi = tf32_rn((float)v);
      ((float*)dst)[idx] = hi;
      if (slices > 1) ((float*)dst)[total + idx] = tf32_rn((float)(v - (double)hi));   // exact tf32 for the MMA
    }
  }
}

cudaError_t launch_materialize_dense(kpme_plan_t P, const double* d_dense, const double* d_gmax, int count, void* dst,
                                     int slices, int kind) {
  materialize_dense_kernel<<<1024, kT, 0, P->stream>>>(d_dense, d_gmax, count, P->p.K, slices, kind, dst);
  return cudaGetLastError();
}

cudaError_t launch_materialize(kpme_plan_t P, const double* d_gen, int count, void* dst, int slices, int kind) {
  const int fold = (kind == 4 && P->fold) ? 1 : 0;
  materialize_kernel<<<1024, kT, 0, P->stream>>>(d_gen, count, P->p.K, slices, kind, fold, dst);
  return cudaGetLastError();
}

cudaError_t launch_bmod(kpme_plan_t P, double* d_out) {
  const int Kh = P->p.K / 2 + 1;
  bmod_kernel<<<(Kh + 127) / 128, 128, 0, P->stream>>>(P->p.K, P->p.order, Kh, d_out);
  return cudaGetLastError();
}

cudaError_t launch_virial_generator(kpme_plan_t P, double* d_gen) {
  const int K = P->p.K, Kh = K / 2 + 1;
  double* bm = nullptr;
  cudaError_t e = cudaMalloc(&bm, Kh * sizeof(double));
  if (e != cudaSuccess) return e;
  bmod_kernel<<<(Kh + 127) / 128, 128, 0, P->stream>>>(K, P->p.order, Kh, bm);
  virial_gen_kernel<<<(K + 127) / 128, 128, 0, P->stream>>>(bm, K, Kh, 2.0 * P->p.radius, P->p.beta, d_gen);
  e = cudaGetLastError();
  cudaError_t e2 = cudaStreamSynchronize(P->stream);
  cudaFree(bm);
  return e != cudaSuccess ? e : e2;
}

}  // namespace kpme

// Particle <-> mesh transfer: cardinal B-spline spreading of charges and gathering of
// potentials / forces (the B-spline form of the interpolation matrices S_Y and S_X^* of
// §2.2, Eq. interpkrons, applied as in Algorithm 4), plus the float64 reductions.
#include "kpme_internal.cuh"

namespace kpme {
namespace {

constexpr int kThreads = 256;

struct MeshGeom {
  double c0, c1, c2, L;
  int K;
};

// Mesh coordinate of one component: u = K ((x - c)/L + 1/2) wrapped into [0, K), split
// into g = floor(u) and f = u - g.  Every operation is an explicitly rounded float64
// operation so that the integer g is decided exactly as the float64 reference decides it.
__device__ __forceinline__ void mesh_coord(double x, double c, double L, int K, int& g, double& f) {
  double s = __dadd_rn(__ddiv_rn(__dsub_rn(x, c), L), 0.5);
  double u = __dmul_rn((double)K, s);
  double m = fmod(u, (double)K);
  if (m != 0.0 && m < 0.0) m = __dadd_rn(m, (double)K);
  if (m >= (double)K) m = __dsub_rn(m, (double)K);
  double fl = floor(m);
  g = (int)fl;
  f = __dsub_rn(m, fl);
}

// Weights M_n(f + j), j = 0..n-1, by the order recursion, and their derivatives
// dM_n/du (f + j) = M_{n-1}(f + j) - M_{n-1}(f + j - 1).
template <typename T, int N>
__device__ __forceinline__ void bspline(T f, T* w, T* dw) {
  w[0] = f;
  w[1] = T(1) - f;
#pragma unroll
  for (int j = 2; j < N; ++j) w[j] = T(0);
#pragma unroll
  for (int k = 3; k <= N; ++k) {
    if (k == N) {
#pragma unroll
      for (int j = 0; j < N; ++j) dw[j] = (j < N - 1 ? w[j] : T(0)) - (j > 0 ? w[j - 1] : T(0));
    }
    const T inv = T(1) / T(k - 1);
    w[k - 1] = (T(1) - f) * w[k - 2] * inv;
#pragma unroll
    for (int j = k - 2; j >= 1; --j) w[j] = ((f + T(j)) * w[j] + (T(k) - f - T(j)) * w[j - 1]) * inv;
    w[0] = f * w[0] * inv;
  }
}

template <typename T>
__device__ __forceinline__ T block_sum_to_thread0(T v) {
  __shared__ T red[kThreads / 32];
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
  const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
  if (l == 0) red[w] = v;
  __syncthreads();
  T s = T(0);
  if (threadIdx.x == 0)
    for (int i = 0; i < kThreads / 32; ++i) s += red[i];
  return s;
}

template <typename T, int N>
__global__ void __launch_bounds__(kThreads) spread_kernel(MeshGeom G, int64_t n, const double* __restrict__ x,
                                                          const double* __restrict__ q, T* __restrict__ Q,
                                                          double* __restrict__ sumq) {
  const int K = G.K;
  double qsum = 0.0;
  for (int64_t i = blockIdx.x * (int64_t)kThreads + threadIdx.x; i < n; i += (int64_t)gridDim.x * kThreads) {
    int g[3];
    T w[3][N], dw[N];
#pragma unroll
    for (int a = 0; a < 3; ++a) {
      double f;
      mesh_coord(x[3 * i + a], a == 0 ? G.c0 : (a == 1 ? G.c1 : G.c2), G.L, K, g[a], f);
      bspline<T, N>((T)f, w[a], dw);
    }
    const double qi = q[i];
    qsum += qi;
    const T qt = (T)qi;
#pragma unroll
    for (int j0 = 0; j0 < N; ++j0) {
      int k0 = g[0] - j0;
      k0 += (k0 < 0) ? K : 0;
      const T w0 = qt * w[0][j0];
#pragma unroll
      for (int j1 = 0; j1 < N; ++j1) {
        int k1 = g[1] - j1;
        k1 += (k1 < 0) ? K : 0;
        const T w01 = w0 * w[1][j1];
        T* row = Q + ((int64_t)k0 * K + k1) * K;
#pragma unroll
        for (int j2 = 0; j2 < N; ++j2) {
          int k2 = g[2] - j2;
          k2 += (k2 < 0) ? K : 0;
          atomicAdd(row + k2, w01 * w[2][j2]);
        }
      }
    }
  }
  double s = block_sum_to_thread0<double>(qsum);
  if (threadIdx.x == 0 && s != 0.0) atomicAdd(sumq, s);
}

template <typename T, int N>
__global__ void __launch_bounds__(kThreads) gather_kernel(MeshGeom G, int64_t n, const double* __restrict__ x,
                                                          const double* __restrict__ q, const T* __restrict__ Phi,
                                                          double* __restrict__ phi_out, double* __restrict__ F_out,
                                                          double* __restrict__ energy, const double* __restrict__ sumq,
                                                          double corr_c, double ke) {
  const int K = G.K;
  const double shift = corr_c * (sumq ? *sumq : 0.0);
  const T gscale = (T)((double)K / G.L);
  double e = 0.0;
  for (int64_t i = blockIdx.x * (int64_t)kThreads + threadIdx.x; i < n; i += (int64_t)gridDim.x * kThreads) {
    int g[3];
    T w[3][N], dw[3][N];
#pragma unroll
    for (int a = 0; a < 3; ++a) {
      double f;
      mesh_coord(x[3 * i + a], a == 0 ? G.c0 : (a == 1 ? G.c1 : G.c2), G.L, K, g[a], f);
      bspline<T, N>((T)f, w[a], dw[a]);
    }
    T p = 0, g0 = 0, g1 = 0, g2 = 0;
#pragma unroll
    for (int j0 = 0; j0 < N; ++j0) {
      int k0 = g[0] - j0;
      k0 += (k0 < 0) ? K : 0;
      T s_p = 0, s_1 = 0, s_2 = 0;   // partial sums over j1, j2 for fixed j0
#pragma unroll
      for (int j1 = 0; j1 < N; ++j1) {
        int k1 = g[1] - j1;
        k1 += (k1 < 0) ? K : 0;
        const T* row = Phi + ((int64_t)k0 * K + k1) * K;
        T t = 0, td = 0;
#pragma unroll
        for (int j2 = 0; j2 < N; ++j2) {
          int k2 = g[2] - j2;
          k2 += (k2 < 0) ? K : 0;
          const T v = row[k2];
          t += w[2][j2] * v;
          td += dw[2][j2] * v;
        }
        s_p += w[1][j1] * t;
        s_1 += dw[1][j1] * t;
        s_2 += w[1][j1] * td;
      }
      p += w[0][j0] * s_p;
      g0 += dw[0][j0] * s_p;
      g1 += w[0][j0] * s_1;
      g2 += w[0][j0] * s_2;
    }
    const double phi = ((double)p - shift) * ke;
    const double qi = q ? q[i] : 0.0;
    if (phi_out) phi_out[i] = phi;
    if (F_out) {
      const double s = -qi * ke * (double)gscale;
      F_out[3 * i + 0] = s * (double)g0;
      F_out[3 * i + 1] = s * (double)g1;
      F_out[3 * i + 2] = s * (double)g2;
    }
    e += 0.5 * qi * phi;
  }
  if (energy) {
    double s = block_sum_to_thread0<double>(e);
    if (threadIdx.x == 0) atomicAdd(energy, s);
  }
}

template <typename T>
__global__ void __launch_bounds__(kThreads) dot_kernel(const T* __restrict__ a, const T* __restrict__ b,
                                                       int64_t count, double* __restrict__ out) {
  double acc = 0.0;
  for (int64_t i = blockIdx.x * (int64_t)kThreads + threadIdx.x; i < count; i += (int64_t)gridDim.x * kThreads)
    acc += (double)a[i] * (double)b[i];
  double s = block_sum_to_thread0<double>(acc);
  if (threadIdx.x == 0) atomicAdd(out, s);
}

__global__ void virial_finalize_kernel(const double* energy, const double* qpsi, const double* sumq, double t0,
                                       double coef, double ke, double* virial) {
  const double sq = sumq ? *sumq : 0.0;
  virial[0] = energy[0] - ke * coef * 0.5 * (qpsi[0] - t0 * sq * sq);
}

template <typename S, typename D>
__global__ void convert_kernel(const S* __restrict__ src, D* __restrict__ dst, int64_t count) {
  for (int64_t i = blockIdx.x * (int64_t)kThreads + threadIdx.x; i < count; i += (int64_t)gridDim.x * kThreads)
    dst[i] = (D)src[i];
}

int grid_for(kpme_plan_t P, int64_t n) {
  int64_t want = (n + kThreads - 1) / kThreads;
  int64_t cap = (int64_t)P->sm_count * 8;
  if (want > cap) want = cap;
  return (int)(want < 1 ? 1 : want);
}

MeshGeom geom(kpme_plan_t P) {
  MeshGeom G;
  G.c0 = P->p.center[0];
  G.c1 = P->p.center[1];
  G.c2 = P->p.center[2];
  G.L = 2.0 * P->p.radius;
  G.K = P->p.K;
  return G;
}

template <typename T>
cudaError_t spread_t(kpme_plan_t P, int64_t n, const double* x, const double* q, T* Q) {
  const int grid = grid_for(P, n);
  const MeshGeom G = geom(P);
  switch (P->p.order) {
    case 4: spread_kernel<T, 4><<<grid, kThreads, 0, P->stream>>>(G, n, x, q, Q, P->d_sumq); break;
    case 6: spread_kernel<T, 6><<<grid, kThreads, 0, P->stream>>>(G, n, x, q, Q, P->d_sumq); break;
    case 8: spread_kernel<T, 8><<<grid, kThreads, 0, P->stream>>>(G, n, x, q, Q, P->d_sumq); break;
    default: return cudaErrorInvalidValue;
  }
  return cudaGetLastError();
}

template <typename T>
cudaError_t gather_t(kpme_plan_t P, int64_t n, const double* x, const double* q, const T* Phi, double* phi,
                     double* F, double* energy, double ke) {
  const int grid = grid_for(P, n);
  const MeshGeom G = geom(P);
  const double c = P->skp.c;
  switch (P->p.order) {
    case 4: gather_kernel<T, 4><<<grid, kThreads, 0, P->stream>>>(G, n, x, q, Phi, phi, F, energy, P->d_sumq, c, ke); break;
    case 6: gather_kernel<T, 6><<<grid, kThreads, 0, P->stream>>>(G, n, x, q, Phi, phi, F, energy, P->d_sumq, c, ke); break;
    case 8: gather_kernel<T, 8><<<grid, kThreads, 0, P->stream>>>(G, n, x, q, Phi, phi, F, energy, P->d_sumq, c, ke); break;
    default: return cudaErrorInvalidValue;
  }
  return cudaGetLastError();
}

}  // namespace

cudaError_t launch_spread(kpme_plan_t P, int64_t n, const double* x, const double* q, double* Q) {
  // The charge mesh is accumulated in float64 for every arithmetic: each mesh value is a sum
  // of many contributions of both signs (neutral molecules), and float32 accumulation of it
  // dominates the potential error of the float32-class paths.
  if (n <= 0) return cudaSuccess;
  return spread_t<double>(P, n, x, q, Q);
}

cudaError_t launch_gather(kpme_plan_t P, int64_t n, const double* x, const double* q, const void* Phi,
                          double* phi, double* F, double* energy, double scale) {
  if (n <= 0) return cudaSuccess;
  const double ke = P->p.coulomb_k * scale;
  if (P->prec.fp64) return gather_t<double>(P, n, x, q, (const double*)Phi, phi, F, energy, ke);
  return gather_t<float>(P, n, x, q, (const float*)Phi, phi, F, energy, ke);
}

cudaError_t launch_dot(kpme_plan_t P, const void* a, const void* b, int64_t count, double* out) {
  const int grid = grid_for(P, count);
  if (P->prec.fp64)
    dot_kernel<double><<<grid, kThreads, 0, P->stream>>>((const double*)a, (const double*)b, count, out);
  else
    dot_kernel<float><<<grid, kThreads, 0, P->stream>>>((const float*)a, (const float*)b, count, out);
  return cudaGetLastError();
}

cudaError_t launch_virial_finalize(kpme_plan_t P, const double* energy, const double* qpsi, double t0, double coef,
                                   double* virial) {
  virial_finalize_kernel<<<1, 1, 0, P->stream>>>(energy, qpsi, P->d_sumq, t0, coef, P->p.coulomb_k, virial);
  return cudaGetLastError();
}

cudaError_t launch_convert(const void* src, bool src_double, void* dst, bool dst_double, int64_t count,
                           cudaStream_t s) {
  int grid = (int)((count + kThreads - 1) / kThreads);
  if (grid > 4096) grid = 4096;
  if (grid < 1) grid = 1;
  if (src_double && dst_double)
    convert_kernel<double, double><<<grid, kThreads, 0, s>>>((const double*)src, (double*)dst, count);
  else if (src_double)
    convert_kernel<double, float><<<grid, kThreads, 0, s>>>((const double*)src, (float*)dst, count);
  else if (dst_double)
    convert_kernel<float, double><<<grid, kThreads, 0, s>>>((const float*)src, (double*)dst, count);
  else
    convert_kernel<float, float><<<grid, kThreads, 0, s>>>((const float*)src, (float*)dst, count);
  return cudaGetLastError();
}

}  // namespace kpme

namespace kpme {

// Spread into caller-provided float32 mesh / float64 charge-sum buffers, without a plan.
cudaError_t launch_spread_raw(const kpme_params_t& p, int sm_count, cudaStream_t s, int64_t n, const double* x,
                              const double* q, float* Q, double* sumq) {
  if (n <= 0) return cudaSuccess;
  MeshGeom G;
  G.c0 = p.center[0];
  G.c1 = p.center[1];
  G.c2 = p.center[2];
  G.L = 2.0 * p.radius;
  G.K = p.K;
  int64_t want = (n + kThreads - 1) / kThreads;
  const int64_t cap = (int64_t)sm_count * 8;
  const int grid = (int)(want > cap ? cap : (want < 1 ? 1 : want));
  switch (p.order) {
    case 4: spread_kernel<float, 4><<<grid, kThreads, 0, s>>>(G, n, x, q, Q, sumq); break;
    case 6: spread_kernel<float, 6><<<grid, kThreads, 0, s>>>(G, n, x, q, Q, sumq); break;
    case 8: spread_kernel<float, 8><<<grid, kThreads, 0, s>>>(G, n, x, q, Q, sumq); break;
    default: return cudaErrorInvalidValue;
  }
  return cudaGetLastError();
}

}  // namespace kpme
